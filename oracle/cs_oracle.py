"""FP64 CPU oracle for circulant LASSO recovery (arXiv 1707.02244).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
this module.  The product path (the CUDA library and its Python binding) never
does, and this module never imports the product package: the two share no
code.  Inputs arrive as plain arrays (the seeded generators live in ``synth``).

Everything here is plain numpy in float64.  Each function follows one passage
of the paper, cited as section / equation / algorithm:

* dense oracle: the sensing matrix is built explicitly and every product is a
  dense mat-vec; ADMM's x-update solve uses a dense Cholesky factor;
* FFT oracle: the same algorithms with the circulant products taken through
  numpy's FFT (a library primitive used as one step), for sizes where dense
  matrices do not fit.  It is pinned against the dense oracle by the tests.

Conventions (readings of the paper, all listed in the design notes):

* circulant index (Sec. 4.2): ``C[i, j] = c[(j - i) mod n]``; ``c`` is the
  first row of C;
* A = P C (Sec. 4.3): P keeps the rows ``rows`` of C; ``y[i]`` pairs with row
  ``rows[i]``; ``P^T y`` is y zero-filled onto those rows;
* LASSO (Eq. 3) is minimised in the equivalent form
  ``0.5 ||y - A x||^2 + lam ||x||_1`` (lam plays the role of alpha);
* ISTA (Algorithm 1) thresholds at ``tau * lam`` (proximal-gradient reading);
* soft threshold (Eq. 4): ``|x| == gamma`` maps to 0.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "circulant_matrix", "sensing_matrix", "soft_threshold", "lasso_objective",
    "kkt_violation", "forward_dense", "adjoint_dense", "spectrum",
    "forward_fft", "adjoint_fft", "circulant_apply_fft", "forward_sampled",
    "adjoint_sampled", "zero_fill", "ista_dense",
    "ista_fft", "admm_dense", "admm_fft", "admm_standard_dense",
    "admm_d_diagonal", "opnorm2_dense", "opnorm2_power_fft",
    "lasso_bruteforce", "l0_bruteforce", "nmse", "naive_dft",
    "ista_unrolled_grad_dense", "ista_unrolled_grad_fft", "ista_unrolled_loss",
    "circulant2d_matrix", "sensing2d_matrix", "spectrum2d", "circulant2d_apply_fft", "forward2d_fft",
    "adjoint2d_fft", "ista_dense2d", "ista_fft2d", "admm_dense2d", "admm_fft2d", "naive_dft2",
    "set_fft_threads", "admm_unrolled_grad_dense", "admm_unrolled_grad_fft", "admm_unrolled_loss",
]


# --------------------------------------------------------------------------
# FFT library step
# --------------------------------------------------------------------------

class _FFT:
    """The FFT used as a library step by the FFT forms below: numpy's (one
    thread) by default; scipy's with a worker pool after set_fft_threads(k),
    k > 1 (used to time the oracle on all host cores).  Both compute the same
    DFT; they may differ in the last bits of rounding."""
    threads = 1

    @classmethod
    def _lib(cls):
        if cls.threads > 1:
            import scipy.fft as sf
            return sf, {"workers": cls.threads}
        return np.fft, {}

    @classmethod
    def call(cls, name, *a, **kw):
        lib, extra = cls._lib()
        return getattr(lib, name)(*a, **kw, **extra)


def set_fft_threads(k: int) -> int:
    """Threads for the FFT library step (1 = numpy); returns the old value."""
    old = _FFT.threads
    _FFT.threads = max(1, int(k))
    return old


def _fft(a): return _FFT.call("fft", a)
def _rfft(a): return _FFT.call("rfft", a)
def _irfft(a, n): return _FFT.call("irfft", a, n)
def _fft2(a): return _FFT.call("fft2", a)
def _rfft2(a): return _FFT.call("rfft2", a)
def _irfft2(a, s): return _FFT.call("irfft2", a, s)


# --------------------------------------------------------------------------
# Sensing operator (Sec. 4.2, Sec. 4.3)
# --------------------------------------------------------------------------

def circulant_matrix(c: np.ndarray) -> np.ndarray:
    """Dense circulant C with ``C[i, j] = c[(j - i) mod n]`` (Sec. 4.2).

    Each row is the previous row shifted circularly one place to the right.
    """
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return c[(j - i) % n]


def sensing_matrix(c: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Partial circulant A = P C: the rows ``rows`` of C, in the given order
    (Sec. 4.3, P selects the rows in Omega)."""
    return circulant_matrix(c)[np.asarray(rows, dtype=np.int64), :]


def forward_dense(c, rows, x):
    """A x by dense mat-vec (Algorithm 1, residual step)."""
    return sensing_matrix(c, rows) @ np.asarray(x, dtype=np.float64)


def adjoint_dense(c, rows, r):
    """A^T r by dense mat-vec (Algorithm 1, gradient step)."""
    return sensing_matrix(c, rows).T @ np.asarray(r, dtype=np.float64)


def naive_dft(v: np.ndarray) -> np.ndarray:
    """O(n^2) DFT ``V_k = sum_j v_j exp(-2 pi i j k / n)`` (no FFT library)."""
    v = np.asarray(v, dtype=np.complex128)
    n = v.shape[0]
    jk = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(-2j * np.pi * jk / n) @ v


def spectrum(c: np.ndarray) -> np.ndarray:
    """DFT of the generating vector, ``chat = FFT(c)`` (Sec. 4.2: circulant
    matrices are diagonalised by the Fourier matrix)."""
    return _fft(np.asarray(c, dtype=np.float64))


def circulant_apply_fft(chat: np.ndarray, x: np.ndarray, transpose: bool = False):
    """C x (or C^T x) through the convolution theorem.

    With ``C[i, j] = c[(j - i) mod n]`` and real c, ``FFT(C x) = conj(chat) *
    FFT(x)`` and ``FFT(C^T x) = chat * FFT(x)``.  x and the result are real,
    so only bins 0..n/2 are formed (real-input FFT).
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    xh = _rfft(x)                         # bins 0..n/2 of the real input
    h = chat[: n // 2 + 1]
    h = h if transpose else np.conj(h)
    return _irfft(h * xh, n)


def forward_fft(chat, rows, x):
    """A x = (C x)[rows] (Sec. 4.3) with C x taken by FFT."""
    return circulant_apply_fft(chat, x)[np.asarray(rows, dtype=np.int64)]


def forward_sampled(c, rows, x, idx):
    """Entries ``idx`` of A x, each by its own O(n) dot product with the
    shifted generating vector: ``(A x)_i = sum_j c[(j - rows[i]) mod n] x_j``
    (Sec. 4.2 index rule).  For full-size checks where A cannot be formed."""
    c = np.asarray(c, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    return np.array([float(np.roll(c, int(rows[i])) @ x) for i in idx])


def adjoint_sampled(c, rows, r, idx):
    """Entries ``idx`` of A^T r, each by its own O(m) sum:
    ``(A^T r)_j = sum_i c[(j - rows[i]) mod n] r_i``."""
    c = np.asarray(c, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    n = c.shape[0]
    return np.array([float(c[(int(j) - rows) % n] @ r) for j in idx])


def zero_fill(n: int, rows, r):
    """P^T r: r scattered onto the rows of Omega, zero elsewhere (Sec. 4.3)."""
    out = np.zeros(n, dtype=np.float64)
    out[np.asarray(rows, dtype=np.int64)] = np.asarray(r, dtype=np.float64)
    return out


def adjoint_fft(chat, rows, r):
    """A^T r = C^T P^T r (Sec. 4.3) with C^T taken by FFT."""
    n = chat.shape[0]
    return circulant_apply_fft(chat, zero_fill(n, rows, r), transpose=True)


# --------------------------------------------------------------------------
# LASSO pieces (Eq. 3, Eq. 4)
# --------------------------------------------------------------------------

def soft_threshold(x, gamma):
    """Eq. 4: ``sgn(x)(|x| - gamma)`` where ``|x| > gamma``, else 0."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) > gamma, np.sign(x) * (np.abs(x) - gamma), 0.0)


def lasso_objective(A, y, x, lam):
    """``0.5 ||y - A x||^2 + lam ||x||_1`` -- Eq. 3 divided by 2 (same
    minimiser, lam = alpha; the split form of Sec. 4.3 uses this scaling)."""
    r = y - A @ x
    return 0.5 * float(r @ r) + lam * float(np.abs(x).sum())


def kkt_violation(A, y, x, lam):
    """Largest violation of the LASSO optimality conditions at x.

    With ``g = A^T (y - A x)``: on the support ``g_i = lam sgn(x_i)``; off the
    support ``|g_i| <= lam``.  Returns the max violation (0 at a minimiser).
    """
    g = A.T @ (y - A @ x)
    on = x != 0
    v_on = np.abs(g[on] - lam * np.sign(x[on])).max(initial=0.0)
    v_off = np.maximum(np.abs(g[~on]) - lam, 0.0).max(initial=0.0)
    return max(v_on, v_off)


def nmse(x, x_true):
    """Normalised MSE ``||x - x*||^2 / ||x*||^2`` (the MSE of Sec. 6 divided
    by the signal energy per sample)."""
    x = np.asarray(x, dtype=np.float64)
    x_true = np.asarray(x_true, dtype=np.float64)
    d = x - x_true
    return float(d @ d) / float(x_true @ x_true)


# --------------------------------------------------------------------------
# ISTA (Algorithm 1)
# --------------------------------------------------------------------------

def _ista(apply_A, apply_At, y, lam, tau, iters, x0, n, history):
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    hist = [x.copy()] if history else None
    for _ in range(iters):
        r = y - apply_A(x)                  # residual r(t) = y - A x(t-1)
        delta = tau * apply_At(r)           # gradient step tau A^T r(t)
        x = soft_threshold(x + delta, tau * lam)   # x(t) = eta[x(t-1) + delta]
        if history:
            hist.append(x.copy())
    return (x, hist) if history else x


def ista_dense(c, rows, y, lam, tau, iters, x0=None, history=False):
    """Algorithm 1 with a dense A = P C.  Threshold ``tau * lam``."""
    A = sensing_matrix(c, rows)
    y = np.asarray(y, dtype=np.float64)
    return _ista(lambda v: A @ v, lambda r: A.T @ r, y, lam, tau, iters, x0,
                 A.shape[1], history)


def ista_fft(c, rows, y, lam, tau, iters, x0=None, history=False):
    """Algorithm 1 with A x and A^T r taken by FFT (same steps as ista_dense)."""
    chat = spectrum(c)
    y = np.asarray(y, dtype=np.float64)
    return _ista(lambda v: forward_fft(chat, rows, v),
                 lambda r: adjoint_fft(chat, rows, r), y, lam, tau, iters, x0,
                 chat.shape[0], history)


# --------------------------------------------------------------------------
# Circulant ADMM (Algorithm 3)
# --------------------------------------------------------------------------

def admm_d_diagonal(n, rows, rho):
    """Diagonal of D = (P^T P + rho I)^(-1) (Algorithm 3, initial inversion).

    P^T P is diagonal with 1 on Omega and 0 elsewhere, so D is ``1/(1+rho)``
    on Omega and ``1/rho`` elsewhere (Sec. 4.3)."""
    d = np.full(n, 1.0 / rho)
    d[np.asarray(rows, dtype=np.int64)] = 1.0 / (1.0 + rho)
    return d


def _admm(C_apply, Ct_apply, B_apply, n, rows, y, lam, sigma, rho, tau1, tau2,
          iters, state, history):
    d = admm_d_diagonal(n, rows, rho)
    pty = zero_fill(n, rows, y)
    if state is None:
        v = np.zeros(n); z = np.zeros(n); mu = np.zeros(n); nu = np.zeros(n)
    else:
        v, z, mu, nu = (np.asarray(s, dtype=np.float64).copy() for s in state)
    x = np.zeros(n)
    hist = [] if history else None
    for _ in range(iters):
        # primal update (Algorithm 3): x then v
        x = B_apply(rho * Ct_apply(v) + sigma * (z - nu))
        cx = C_apply(x)
        v = d * (rho * cx - rho * mu + pty)
        # soft-thresholding step
        z = soft_threshold(x + nu, lam / sigma)
        # dual update, then v <- v + mu
        mu = mu + tau1 * (v - cx)
        nu = nu + tau2 * (x - z)
        v = v + mu
        if history:
            hist.append((x.copy(), z.copy()))
    out = {"x": x, "z": z, "mu": mu, "nu": nu, "v": v}
    if history:
        out["history"] = hist
    return out


def admm_dense(c, rows, y, lam, sigma, rho, tau1=1.0, tau2=1.0, iters=100,
               state=None, history=False):
    """Algorithm 3 with dense C; B = (rho C^T C + sigma I)^(-1) applied by a
    dense Cholesky factor computed once (the "initial inversion").

    ``state`` = (v, z, mu, nu) to warm-start (v is the folded v + mu of the
    last line of the loop); ``None`` is the paper's zero start.
    Returns dict with x, z, mu, nu, v after ``iters`` iterations.
    """
    C = circulant_matrix(c)
    n = C.shape[0]
    M = rho * (C.T @ C) + sigma * np.eye(n)
    L = np.linalg.cholesky(M)

    def B_apply(b):
        return np.linalg.solve(L.T, np.linalg.solve(L, b))

    return _admm(lambda v: C @ v, lambda v: C.T @ v, B_apply, n, rows,
                 np.asarray(y, dtype=np.float64), lam, sigma, rho, tau1, tau2,
                 iters, state, history)


def admm_fft(c, rows, y, lam, sigma, rho, tau1=1.0, tau2=1.0, iters=100,
             state=None, history=False):
    """Algorithm 3 with the circulant inverse taken by FFT (Sec. 4.3: rho C^T C
    + sigma I is circulant with eigenvalues ``rho |chat|^2 + sigma``)."""
    chat = spectrum(c)
    n = chat.shape[0]
    bhat = 1.0 / (rho * np.abs(chat) ** 2 + sigma)

    def B_apply(b):
        return _irfft(bhat[: n // 2 + 1] * _rfft(b), n)

    return _admm(lambda v: circulant_apply_fft(chat, v),
                 lambda v: circulant_apply_fft(chat, v, transpose=True),
                 B_apply, n, rows, np.asarray(y, dtype=np.float64), lam, sigma,
                 rho, tau1, tau2, iters, state, history)


def admm_standard_dense(A, y, lam, rho, iters):
    """Algorithm 2 (standard ADMM) with B = (A^T A + rho I)^(-1) by Cholesky.

    Cross-check only: it minimises the same LASSO as Algorithm 3 with the
    threshold ``lam / rho``.  Returns (x, z, u)."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = A.shape[1]
    L = np.linalg.cholesky(A.T @ A + rho * np.eye(n))
    aty = A.T @ y
    x = np.zeros(n); z = np.zeros(n); u = np.zeros(n)
    for _ in range(iters):
        b = aty + rho * (z - u)
        x = np.linalg.solve(L.T, np.linalg.solve(L, b))
        z = soft_threshold(x + u, lam / rho)
        u = u + x - z
    return x, z, u


# --------------------------------------------------------------------------
# Step size (Algorithm 1 initialisation: tau in (0, ||A||^-2))
# --------------------------------------------------------------------------

def opnorm2_dense(c, rows):
    """||A||_2^2 from the SVD of the dense A."""
    s = np.linalg.svd(sensing_matrix(c, rows), compute_uv=False)
    return float(s[0] ** 2)


def opnorm2_power_fft(c, rows, iters=200, seed=0, tol=1e-12):
    """||A||_2^2 by power iteration on A^T A with FFT products."""
    chat = spectrum(c)
    n = chat.shape[0]
    u = np.random.default_rng(seed).standard_normal(n)
    u /= np.linalg.norm(u)
    lam_prev = 0.0
    lam_est = 0.0
    for _ in range(iters):
        w = adjoint_fft(chat, rows, forward_fft(chat, rows, u))
        lam_est = float(u @ w)
        u = w / np.linalg.norm(w)
        if abs(lam_est - lam_prev) <= tol * abs(lam_est):
            break
        lam_prev = lam_est
    return lam_est


# --------------------------------------------------------------------------
# Brute force on tiny instances (Eq. 2, Eq. 3)
# --------------------------------------------------------------------------

def lasso_bruteforce(A, y, lam):
    """Exact LASSO minimiser by enumerating sign patterns (n <= ~10).

    For a sign pattern s with support S the optimality conditions give
    ``x_S = (A_S^T A_S)^(-1) (A_S^T y - lam s_S)``; the pattern is accepted when
    sgn(x_S) = s_S and ``|A_j^T (y - A x)| <= lam`` off S.  Among accepted
    patterns the one with the smallest objective is returned.
    """
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = A.shape[1]
    best = None
    best_f = np.inf
    for s in itertools.product((-1, 0, 1), repeat=n):
        s = np.array(s, dtype=np.float64)
        S = np.flatnonzero(s)
        x = np.zeros(n)
        if S.size:
            As = A[:, S]
            G = As.T @ As
            if np.linalg.matrix_rank(G) < S.size:
                continue
            xs = np.linalg.solve(G, As.T @ y - lam * s[S])
            if np.any(np.sign(xs) != s[S]):
                continue
            x[S] = xs
        g = A.T @ (y - A @ x)
        off = np.setdiff1d(np.arange(n), S)
        if off.size and np.any(np.abs(g[off]) > lam * (1 + 1e-12)):
            continue
        f = lasso_objective(A, y, x, lam)
        if f < best_f:
            best_f = f
            best = x
    return best


def l0_bruteforce(A, y, kmax, tol=1e-9):
    """Sparsest x with A x = y among supports of size <= kmax (Eq. 2).

    Returns (x, list_of_supports_of_that_size_that_fit)."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = A.shape[1]
    scale = max(1.0, float(np.linalg.norm(y)))
    if np.linalg.norm(y) <= tol:
        return np.zeros(n), [()]
    for k in range(1, kmax + 1):
        fits = []
        xbest = None
        for S in itertools.combinations(range(n), k):
            As = A[:, S]
            xs, *_ = np.linalg.lstsq(As, y, rcond=None)
            if np.linalg.norm(As @ xs - y) <= tol * scale:
                fits.append(S)
                if xbest is None:
                    xbest = np.zeros(n)
                    xbest[list(S)] = xs
        if fits:
            return xbest, fits
    return None, []


# --------------------------------------------------------------------------
# Reverse mode of unrolled ISTA (no counterpart in the paper: the derivative of
# T steps of Algorithm 1, from x(0) = 0, with respect to c, lambda and y)
# --------------------------------------------------------------------------
#
# One step is u = x + tau C^T M (P^T y - C x), x' = eta_theta(u), theta =
# tau * lam (Eq. 4 with the threshold reading of Algorithm 1).  Given g =
# dL/dx', the step's contributions are, with w = g on {|u| > theta} and 0
# elsewhere (the soft threshold's derivative; |u| == theta counts as 0):
#   dL/dx      = w - tau C^T M C w
#   dL/dtheta += -sum(sign(u) w)            (dL/dlam = tau dL/dtheta)
#   dL/dy     += tau P C w
#   dL/dc_k   += tau (sum_i r_i w_{i+k} - sum_i q_i x_{i+k}),
#                r = M (P^T y - C x),  q = M C w  (indices mod n),
# the last from dC/dc_k = Pi_k, (Pi_k)_{ij} = 1 if (j - i) mod n == k, so that
# w^T du/dc_k = tau ((Pi_k w)^T r - (M C w)^T (Pi_k x)).

def _ista_grad(C_apply, Ct_apply, corr, n, rows, y, lam, tau, T, gx_T, active=None):
    rows = np.asarray(rows, dtype=np.int64)
    y = np.asarray(y, dtype=np.float64)
    theta = tau * lam
    mask = np.zeros(n)
    mask[rows] = 1.0
    pty = zero_fill(n, rows, y)
    xs = [np.zeros(n)]
    us = []
    for _ in range(T):
        x = xs[-1]
        u = x + tau * Ct_apply(mask * (pty - C_apply(x)))
        us.append(u)
        xs.append(soft_threshold(u, theta))
    g = np.asarray(gx_T, dtype=np.float64).copy()
    dc = np.zeros(n)
    dtheta = 0.0
    dy = np.zeros(len(rows))
    for t in range(T - 1, -1, -1):
        x, u = xs[t], us[t]
        on = np.abs(u) > theta if active is None else np.asarray(active(t), dtype=bool)
        w = np.where(on, g, 0.0)
        dtheta -= float(np.sum(np.sign(u) * w))
        cw = C_apply(w)
        q = mask * cw
        dy += tau * cw[rows]
        r = mask * (pty - C_apply(x))
        dc += tau * (corr(r, w) - corr(q, x))
        g = w - tau * Ct_apply(q)
    return {"x_T": xs[-1], "dc": dc, "dlam": tau * dtheta, "dy": dy, "dx0": g}


def ista_unrolled_grad_dense(c, rows, y, lam, tau, T, gx_T):
    """Gradient of L(x(T)) for T ISTA steps from x(0) = 0 with respect to c,
    lam and y, given gx_T = dL/dx(T).  Dense C; the correlation
    sum_i b_i a_{(i+k) mod n} is formed for every k by rolling a."""
    C = circulant_matrix(c)
    n = C.shape[0]

    def corr(b, a):
        return np.array([np.dot(b, np.roll(a, -k)) for k in range(n)])

    return _ista_grad(lambda v: C @ v, lambda v: C.T @ v, corr, n, rows, y, lam, tau, T, gx_T)


def ista_unrolled_grad_fft(c, rows, y, lam, tau, T, gx_T, active=None):
    """As ista_unrolled_grad_dense with the products and correlations taken
    by FFT: DFT(sum_i b_i a_{i+k}) = conj(DFT b) DFT a for real a, b.

    ``active``: optional callable, active(t) = the boolean set on which step
    t's soft threshold passes its input (x(t+1) != 0) of some other forward
    trajectory, used in place of this trajectory's {|u(t)| > theta}.  The
    reverse pass is then the derivative along that trajectory's supports (an
    analysis aid: it separates the effect of support differences between two
    forward passes from the rest)."""
    chat = spectrum(c)
    n = chat.shape[0]

    def corr(b, a):
        return _irfft(np.conj(_rfft(b)) * _rfft(a), n)

    return _ista_grad(lambda v: circulant_apply_fft(chat, v), lambda v: circulant_apply_fft(chat, v, True),
                      corr, n, rows, y, lam, tau, T, gx_T, active)


def ista_unrolled_loss(c, rows, y, lam, tau, T, x_star, dense=True):
    """L = ||x(T) - x*||^2 after T ISTA steps from x(0) = 0, and dL/dx(T)."""
    run = ista_dense if dense else ista_fft
    xT = run(c, rows, y, lam, tau, T)
    d = xT - np.asarray(x_star, dtype=np.float64)
    return float(np.dot(d, d)), 2.0 * d


# --------------------------------------------------------------------------
# Reverse mode of unrolled circulant ADMM (no counterpart in the paper: the
# derivative of T iterations of Algorithm 3, from the zero state, with
# respect to c, lambda and y)
# --------------------------------------------------------------------------
#
# One iteration maps the state (v, z, mu, nu) -- v the folded v + mu of the
# loop's last line -- to (v2, z1, mu1, nu1):
#   b  = rho C^T v + sigma (z - nu),   x = B b,   B = (rho C^T C + sigma I)^-1
#   p  = C x,   v1 = D (rho p - rho mu + P^T y)
#   s  = x + nu,   z1 = eta_theta(s),   theta = lam / sigma
#   mu1 = mu + tau1 (v1 - p),   nu1 = nu + tau2 (x - z1),   v2 = v1 + mu1.
# Given the adjoints (v2', z1', mu1', nu1') of the new state (primes denote
# dL/d.), the chain rule gives, in this order,
#   mu1' += v2';  v1' = v2' + tau1 mu1';  p' = -tau1 mu1'
#   x' = tau2 nu1';  z1' -= tau2 nu1';  nu' = nu1'
#   s' = z1' on {|s| > theta} (0 elsewhere, |s| == theta included);
#   lam' += -(1/sigma) sum sign(s) s';  x' += s';  nu' += s'
#   a' = D v1';  p' += rho a';  mu' = mu1' - rho a';  y' += P a'
#   x' += C^T p';  c'_k += sum_i p'_i x_{i+k}
#   b' = B x';  c'_k -= rho (sum_i p_i b'_{i+k} + sum_i (C b')_i x_{i+k})
#   v' = rho C b';  c'_k += rho sum_i v_i b'_{i+k};  z' = sigma b';  nu' -= sigma b'
# (indices mod n).  The c-terms come from dC/dc_k = Pi_k, (Pi_k u)_i =
# u_{i+k}: p = C x gives p'^T Pi_k x; C^T v gives b'^T Pi_k^T v; and
# dB = -B dM B with dM = rho (dC^T C + C^T dC) gives -b'^T dM x.  D depends on
# rho alone.  The loss may depend on z(T) and x(T) of the last iteration.

def _admm_grad(C_apply, Ct_apply, B_apply, corr, n, rows, y, lam, sigma, rho, tau1, tau2, T, gz_T,
               gx_T=None):
    rows = np.asarray(rows, dtype=np.int64)
    y = np.asarray(y, dtype=np.float64)
    theta = lam / sigma
    d = admm_d_diagonal(n, rows, rho)
    pty = zero_fill(n, rows, y)
    v = np.zeros(n); z = np.zeros(n); mu = np.zeros(n); nu = np.zeros(n)
    steps = []
    for _ in range(T):
        x = B_apply(rho * Ct_apply(v) + sigma * (z - nu))
        p = C_apply(x)
        v1 = d * (rho * p - rho * mu + pty)
        s = x + nu
        z1 = soft_threshold(s, theta)
        mu1 = mu + tau1 * (v1 - p)
        nu1 = nu + tau2 * (x - z1)
        steps.append((v, x, p, s))
        v, z, mu, nu = v1 + mu1, z1, mu1, nu1
    out = {"x_T": steps[-1][1], "z_T": z}
    vb = np.zeros(n)
    zb = np.asarray(gz_T, dtype=np.float64).copy()
    mub = np.zeros(n)
    nub = np.zeros(n)
    dc = np.zeros(n)
    dlam = 0.0
    dy = np.zeros(len(rows))
    for t in range(T - 1, -1, -1):
        v0, x, p, s = steps[t]
        mub = mub + vb
        v1b = vb + tau1 * mub
        pb = -tau1 * mub
        xb = tau2 * nub
        if t == T - 1 and gx_T is not None:
            xb = xb + np.asarray(gx_T, dtype=np.float64)
        zb = zb - tau2 * nub
        sb = np.where(np.abs(s) > theta, zb, 0.0)
        dlam -= float(np.sum(np.sign(s) * sb)) / sigma
        xb = xb + sb
        nub = nub + sb
        ab = d * v1b
        pb = pb + rho * ab
        mub = mub - rho * ab
        dy += ab[rows]
        xb = xb + Ct_apply(pb)
        dc += corr(pb, x)
        bb = B_apply(xb)
        cbb = C_apply(bb)
        dc -= rho * (corr(p, bb) + corr(cbb, x))
        dc += rho * corr(v0, bb)
        vb = rho * cbb
        zb = sigma * bb
        nub = nub - sigma * bb
    out.update({"dc": dc, "dlam": dlam, "dy": dy})
    return out


def admm_unrolled_grad_dense(c, rows, y, lam, sigma, rho, tau1, tau2, T, gz_T, gx_T=None):
    """Gradient of a loss L(z(T), x(T)) of T iterations of Algorithm 3 from
    the zero state with respect to c, lam and y, given gz_T = dL/dz(T) (and
    gx_T = dL/dx(T), optional).  Dense C, B by a dense Cholesky factor; the
    correlation sum_i b_i a_{(i+k) mod n} is formed for every k by rolling a."""
    C = circulant_matrix(c)
    n = C.shape[0]
    L = np.linalg.cholesky(rho * (C.T @ C) + sigma * np.eye(n))

    def B_apply(b):
        return np.linalg.solve(L.T, np.linalg.solve(L, b))

    def corr(b, a):
        return np.array([np.dot(b, np.roll(a, -k)) for k in range(n)])

    return _admm_grad(lambda v: C @ v, lambda v: C.T @ v, B_apply, corr, n, rows, y, lam, sigma, rho, tau1, tau2,
                      T, gz_T, gx_T)


def admm_unrolled_grad_fft(c, rows, y, lam, sigma, rho, tau1, tau2, T, gz_T, gx_T=None):
    """As admm_unrolled_grad_dense with products, the circulant inverse B and
    the correlations taken by FFT."""
    chat = spectrum(c)
    n = chat.shape[0]
    bhat = 1.0 / (rho * np.abs(chat) ** 2 + sigma)

    def B_apply(b):
        return _irfft(bhat[: n // 2 + 1] * _rfft(b), n)

    def corr(b, a):
        return _irfft(np.conj(_rfft(b)) * _rfft(a), n)

    return _admm_grad(lambda v: circulant_apply_fft(chat, v), lambda v: circulant_apply_fft(chat, v, True),
                      B_apply, corr, n, rows, y, lam, sigma, rho, tau1, tau2, T, gz_T, gx_T)


def admm_unrolled_loss(c, rows, y, lam, sigma, rho, tau1, tau2, T, x_star, dense=True):
    """L = ||z(T) - x*||^2 after T iterations of Algorithm 3 from the zero
    state, and dL/dz(T)."""
    run = admm_dense if dense else admm_fft
    zT = run(c, rows, y, lam, sigma=sigma, rho=rho, tau1=tau1, tau2=tau2, iters=T)["z"]
    dz = zT - np.asarray(x_star, dtype=np.float64)
    return float(np.dot(dz, dz)), 2.0 * dz


# --------------------------------------------------------------------------
# Two-dimensional operator (Sec. 7, compressed deblurring: A = P H with H the
# periodic blur of an n0 x n1 image, a product of a sampling and a circulant
# -- here block-circulant with circulant blocks -- matrix)
# --------------------------------------------------------------------------
#
# Images are flattened row-major (pixel (a, b) is entry a n1 + b).  The blur
# follows Sec. 4.2's index rule in both axes:
#   (H x)[i0, i1] = sum_{j0, j1} c2[(j0 - i0) mod n0, (j1 - i1) mod n1] x[j0, j1]
# so that, for real c2, DFT2(H x) = conj(DFT2 c2) DFT2 x and
# DFT2(H^T x) = DFT2(c2) DFT2 x.  A convolution with a point-spread function
# psf is H with c2[d] = psf[-d].

def circulant2d_matrix(c2: np.ndarray) -> np.ndarray:
    """Dense (n0 n1) x (n0 n1) matrix H of the 2D index rule above."""
    c2 = np.asarray(c2, dtype=np.float64)
    n0, n1 = c2.shape
    a = np.arange(n0 * n1) // n1
    b = np.arange(n0 * n1) % n1
    return c2[(a[None, :] - a[:, None]) % n0, (b[None, :] - b[:, None]) % n1]


def sensing2d_matrix(c2, pix) -> np.ndarray:
    """A = P H: the rows ``pix`` (flattened pixel indices) of H."""
    return circulant2d_matrix(c2)[np.asarray(pix, dtype=np.int64), :]


def naive_dft2(v: np.ndarray) -> np.ndarray:
    """O(n^2) 2D DFT by the 1D definition along each axis (no FFT library)."""
    v = np.asarray(v, dtype=np.complex128)
    rows = np.array([naive_dft(r) for r in v])
    return np.array([naive_dft(col) for col in rows.T]).T


def spectrum2d(c2: np.ndarray) -> np.ndarray:
    """2D DFT of the generating array: the eigenvalues of H (conjugated)."""
    return _fft2(np.asarray(c2, dtype=np.float64))


def circulant2d_apply_fft(chat2, x, transpose=False):
    """H x (or H^T x) of a flattened image by the 2D convolution theorem."""
    n0, n1 = chat2.shape
    xh = _rfft2(np.asarray(x, dtype=np.float64).reshape(n0, n1))
    h = chat2[:, : n1 // 2 + 1]
    h = h if transpose else np.conj(h)
    return _irfft2(h * xh, (n0, n1)).ravel()


def forward2d_fft(chat2, pix, x):
    """A x = (H x)[pix]."""
    return circulant2d_apply_fft(chat2, x)[np.asarray(pix, dtype=np.int64)]


def adjoint2d_fft(chat2, pix, r):
    """A^T r = H^T P^T r."""
    n = chat2.size
    return circulant2d_apply_fft(chat2, zero_fill(n, pix, r), transpose=True)


def ista_dense2d(c2, pix, y, lam, tau, iters, x0=None, history=False):
    """Algorithm 1 with the dense 2D sensing matrix (tiny images)."""
    A = sensing2d_matrix(c2, pix)
    y = np.asarray(y, dtype=np.float64)
    return _ista(lambda v: A @ v, lambda r: A.T @ r, y, lam, tau, iters, x0, A.shape[1], history)


def ista_fft2d(c2, pix, y, lam, tau, iters, x0=None, history=False):
    """Algorithm 1 with the 2D products taken by FFT."""
    chat2 = spectrum2d(c2)
    y = np.asarray(y, dtype=np.float64)
    return _ista(lambda v: forward2d_fft(chat2, pix, v), lambda r: adjoint2d_fft(chat2, pix, r), y, lam, tau,
                 iters, x0, chat2.size, history)


def admm_dense2d(c2, pix, y, lam, sigma, rho, tau1=1.0, tau2=1.0, iters=100, state=None, history=False):
    """Algorithm 3 with the dense 2D blur H; B = (rho H^T H + sigma I)^-1 by
    a dense Cholesky factor (tiny images)."""
    H = circulant2d_matrix(c2)
    n = H.shape[0]
    L = np.linalg.cholesky(rho * (H.T @ H) + sigma * np.eye(n))

    def B_apply(b):
        return np.linalg.solve(L.T, np.linalg.solve(L, b))

    return _admm(lambda v: H @ v, lambda v: H.T @ v, B_apply, n, pix, np.asarray(y, dtype=np.float64), lam,
                 sigma, rho, tau1, tau2, iters, state, history)


def admm_fft2d(c2, pix, y, lam, sigma, rho, tau1=1.0, tau2=1.0, iters=100, state=None, history=False):
    """Algorithm 3 with the 2D blur: rho H^T H + sigma I is diagonalised by
    the 2D DFT with eigenvalues rho |chat2|^2 + sigma."""
    chat2 = spectrum2d(c2)
    n0, n1 = chat2.shape
    bhat = 1.0 / (rho * np.abs(chat2) ** 2 + sigma)

    def B_apply(b):
        return _irfft2(bhat[:, : n1 // 2 + 1] * _rfft2(b.reshape(n0, n1)), (n0, n1)).ravel()

    return _admm(lambda v: circulant2d_apply_fft(chat2, v), lambda v: circulant2d_apply_fft(chat2, v, True),
                 B_apply, n0 * n1, pix, np.asarray(y, dtype=np.float64), lam, sigma, rho, tau1, tau2, iters,
                 state, history)
