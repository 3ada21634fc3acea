"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers only: generating vectors, row sets, sparse
signals and noise.  It holds none of the method's arithmetic (no products with
the sensing matrix, no thresholds, no FFTs); measurements y = A x* are formed
by whichever side consumes the inputs.  Both the oracle's tests and the GPU
tests / bench draw from here, so they see identical numbers.

Workloads (Sec. 6 shapes, with the readings recorded in the design notes):

* ``small_instance``: n=4096, m=1024 rows without replacement, c ~ N(0, 1/m),
  x* with exactly k=64 nonzeros on a uniform support, N(0,1) amplitudes,
  noiseless;
* ``large_instance``: n=2^22, m=n/4, c ~ N(0, 1/m), x* Bernoulli(1/200)
  support with N(0,1) amplitudes, noise N(0, 1e-4^2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SMALL_SEED = 1707000
LARGE_SEED = 1707001


@dataclass
class Instance:
    n: int
    m: int
    c: np.ndarray        # float64 [n]: first row of the circulant C
    rows: np.ndarray     # int64 [m]: distinct rows of C kept by P, in draw order
    x_true: np.ndarray   # float64 [n]: sparse signal x*
    noise: np.ndarray    # float64 [m]: additive measurement noise (may be zeros)
    seed: int


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def draw_rows(g: np.random.Generator, n: int, m: int) -> np.ndarray:
    """m distinct rows of {0..n-1}, uniformly without replacement, in draw
    order (not sorted)."""
    return g.choice(n, size=m, replace=False).astype(np.int64)


def gaussian_c(g: np.random.Generator, n: int, m: int) -> np.ndarray:
    """Generating vector with i.i.d. N(0, 1/m) entries."""
    return g.standard_normal(n) / np.sqrt(m)


def k_sparse(g: np.random.Generator, n: int, k: int) -> np.ndarray:
    """Exactly k nonzeros on a uniform random support, N(0,1) amplitudes."""
    x = np.zeros(n)
    supp = g.choice(n, size=k, replace=False)
    x[supp] = g.standard_normal(k)
    return x


def bernoulli_gaussian(g: np.random.Generator, n: int, p: float) -> np.ndarray:
    """Each entry nonzero with probability p, N(0,1) amplitude."""
    on = g.random(n) < p
    return np.where(on, g.standard_normal(n), 0.0)


def instance(n: int, m: int, *, k: int | None = None, p: float | None = None,
             noise_std: float = 0.0, seed: int = 0) -> Instance:
    """Generic seeded instance: c ~ N(0,1/m), rows, x* (k-sparse or
    Bernoulli(p)-Gaussian), noise N(0, noise_std^2)."""
    g = rng(seed)
    c = gaussian_c(g, n, m)
    rows = draw_rows(g, n, m)
    if k is not None:
        x = k_sparse(g, n, k)
    elif p is not None:
        x = bernoulli_gaussian(g, n, p)
    else:
        x = np.zeros(n)
    noise = g.standard_normal(m) * noise_std if noise_std > 0 else np.zeros(m)
    return Instance(n, m, c, rows, x, noise, seed)


def small_instance(seed: int = SMALL_SEED) -> Instance:
    """n=4096, m=1024, k=64, noiseless (lambda=1e-3, 500 iterations)."""
    return instance(4096, 1024, k=64, seed=seed)


def large_instance(seed: int = LARGE_SEED, n: int = 1 << 22) -> Instance:
    """n=2^22, m=n/4, Bernoulli(1/200)-Gaussian x*, noise N(0,1e-4^2)
    (lambda=5e-3, rho=1, stop at NMSE<=1e-4 or 2000 iterations)."""
    return instance(n, n // 4, p=1.0 / 200.0, noise_std=1e-4, seed=seed)


BATCH_SEED = 1707003


def smooth_numbers(hi: int) -> np.ndarray:
    """All 7-smooth integers 2^a 3^b 5^c 7^d <= hi, ascending."""
    out = []
    p2 = 1
    while p2 <= hi:
        p3 = p2
        while p3 <= hi:
            p5 = p3
            while p5 <= hi:
                p7 = p5
                while p7 <= hi:
                    out.append(p7)
                    p7 *= 7
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return np.array(sorted(out), dtype=np.int64)


def batch_sizes(count: int, lg_lo: float, lg_hi: float, seed: int,
                snap: str = "pow2") -> tuple[np.ndarray, np.ndarray]:
    """Sizes of a batch of independent instances: n log-uniform in
    [2^lg_lo, 2^lg_hi], snapped to the nearest power of two (log2 rounded,
    snap="pow2") or to the nearest 7-smooth integer (snap="smooth", the
    smaller on a tie), m/n uniform in [0.2, 0.5]."""
    g = rng(seed)
    u = g.uniform(lg_lo, lg_hi, size=count)
    if snap == "pow2":
        n = np.left_shift(np.int64(1), np.rint(u).astype(np.int64))
    elif snap == "smooth":
        target = np.exp2(u)
        cand = smooth_numbers(int(np.ceil(2.0 ** lg_hi)) * 2)
        j = np.clip(np.searchsorted(cand, target), 1, len(cand) - 1)
        lo, hi = cand[j - 1], cand[j]
        n = np.where(target - lo <= hi - target, lo, hi).astype(np.int64)
    else:
        raise ValueError(snap)
    m = np.maximum(1, np.rint(g.uniform(0.2, 0.5, size=count) * n)).astype(np.int64)
    return n, m


def batch_instances(n, m, *, k_frac: float = 0.01, noise_std: float = 1e-3, seed: int = BATCH_SEED) -> list:
    """One instance per (n_i, m_i), each with its own c, rows and
    max(1, k_frac * n_i)-sparse x*; instance i is seeded with seed + i."""
    return [instance(int(ni), int(mi), k=max(1, int(round(k_frac * ni))), noise_std=noise_std, seed=seed + i)
            for i, (ni, mi) in enumerate(zip(n, m))]


STAR_SEED = 1707002


def box_blur_c(n: int, L: int = 5) -> np.ndarray:
    """First row of the order-L box blur (its first L entries 1/L)."""
    b = np.zeros(n)
    b[:L] = 1.0 / L
    return b


def composite_c(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """First row of C(a) C(b) for first-row circulants (C[i][j] = a[(j - i)
    mod n]): entry s is sum_d a[d] b[(s - d) mod n], summed over the nonzeros
    of b (a short filter)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.zeros_like(a)
    for e in np.flatnonzero(b):
        out += b[e] * np.roll(a, e)
    return out


def gaussian_psf(sigma: float = 2.5, support: int = 15) -> np.ndarray:
    """support x support Gaussian point-spread function, normalised to sum 1."""
    h = support // 2
    d = np.arange(-h, h + 1, dtype=np.float64)
    g = np.exp(-0.5 * (d / sigma) ** 2)
    psf = np.outer(g, g)
    return psf / psf.sum()


def psf_generator(psf: np.ndarray, n0: int, n1: int) -> np.ndarray:
    """Generating array c2 (n0 x n1) of the periodic convolution with psf
    (centred): c2[d] = psf[-d], indices mod (n0, n1)."""
    c2 = np.zeros((n0, n1))
    h0, h1 = psf.shape[0] // 2, psf.shape[1] // 2
    for u in range(psf.shape[0]):
        for v in range(psf.shape[1]):
            c2[(h0 - u) % n0, (h1 - v) % n1] += psf[u, v]
    return c2


class Image2D:
    """A 2D instance: image x (flattened row-major), generating array c2,
    kept pixels pix (flattened indices, draw order), noise on y."""

    def __init__(self, n0, n1, c2, pix, x_true, noise, seed):
        self.n0, self.n1, self.c2, self.pix, self.x_true, self.noise, self.seed = n0, n1, c2, pix, x_true, noise, seed
        self.n = n0 * n1
        self.m = len(pix)


def star_field(n0: int = 4096, n1: int = 4096, k: int = 20000, m_frac: float = 1.0 / 3.0,
               noise_std: float = 1e-3, sigma_psf: float = 2.5, seed: int = STAR_SEED) -> Image2D:
    """Sparse star field: k point sources at distinct uniform pixels with
    log-normal(0, 1) fluxes, blurred periodically by a 15 x 15 Gaussian PSF
    (sigma_psf), m = floor(m_frac n) pixels kept, noise N(0, noise_std^2)."""
    g = rng(seed)
    n = n0 * n1
    x = np.zeros(n)
    pos = g.choice(n, size=k, replace=False)
    x[pos] = g.lognormal(0.0, 1.0, size=k)
    c2 = psf_generator(gaussian_psf(sigma_psf), n0, n1)
    m = int(np.floor(m_frac * n))
    pix = draw_rows(g, n, m)
    noise = g.standard_normal(m) * noise_std
    return Image2D(n0, n1, c2, pix, x, noise, seed)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Dense N(0,1) vector (operator tests)."""
    return rng(seed).standard_normal(n)


def unit_modulus_c(n: int, seed: int) -> np.ndarray:
    """Random phases for a real generating vector whose circulant is
    orthogonal: returns the spectrum samples (complex, Hermitian, |.|=1)
    as an array of length n.  The consumer turns it into c by an inverse DFT.
    """
    g = rng(seed)
    ph = g.uniform(0.0, 2.0 * np.pi, size=n)
    spec = np.exp(1j * ph)
    spec[0] = 1.0 if g.random() < 0.5 else -1.0
    if n % 2 == 0:
        spec[n // 2] = 1.0 if g.random() < 0.5 else -1.0
    k = np.arange(1, (n + 1) // 2)
    spec[n - k] = np.conj(spec[k])
    return spec
