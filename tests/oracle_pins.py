"""Pins for the FP64 oracle: checks against what the paper and mathematics fix.

Each ``check_*`` takes the oracle module and raises AssertionError when the
oracle disagrees with an independent fact: a worked example of a definition,
a closed form, an invariant, or brute force on a tiny instance.  None of them
re-types the formula under test.  ``test_oracle_pins`` runs them on the real
oracle; ``test_oracle_mutants`` plants mistakes in the oracle and checks that
at least one pin fails for each.
"""
from __future__ import annotations

import json
import pathlib

import numpy as np

import synth

GOLDEN = pathlib.Path(__file__).parent / "golden"


def _paper_constants():
    return json.loads((GOLDEN / "paper_constants.json").read_text())


# ---------------------------------------------------------------- operator

def check_circulant_worked_example(O):
    """Sec. 4.2: C[i, j] = c[(j - i) mod n], c the first row; each row is the
    previous one shifted circularly right by one (Sec. 1).  Matrix written out
    by hand for c = (1, 2, 3, 4)."""
    g = json.loads((GOLDEN / "circulant_n4.json").read_text())
    C = O.circulant_matrix(np.array(g["c"], dtype=float))
    assert np.array_equal(C, np.array(g["C"], dtype=float)), C
    A = O.sensing_matrix(np.array(g["c"], dtype=float), np.array(g["rows"]))
    assert np.array_equal(A, np.array(g["A"], dtype=float)), A


def check_eigenvalues_are_dft(O):
    """Circulant matrices are diagonalised by the Fourier basis (Sec. 4.2):
    C f_k = conj(chat_k) f_k with f_k = exp(2 pi i j k / n) and chat the DFT of
    c computed by the O(n^2) definition (no FFT library)."""
    for n, seed in ((5, 1), (8, 2), (16, 3), (33, 4)):
        c = synth.random_vector(n, seed)
        C = O.circulant_matrix(c)
        chat = O.naive_dft(c)
        j = np.arange(n)
        for k in range(n):
            f = np.exp(2j * np.pi * j * k / n)
            assert np.allclose(C @ f, np.conj(chat[k]) * f, atol=1e-12), (n, k)
        ev = np.sort_complex(np.round(np.linalg.eigvals(C), 9))
        dv = np.sort_complex(np.round(chat, 9))
        assert np.allclose(ev, dv, atol=1e-7), n
        # spectrum() (library FFT) equals the definition
        assert np.allclose(O.spectrum(c), chat, atol=1e-11), n


def check_fft_products_match_dense(O):
    """FFT-oracle A x and A^T r equal the dense mat-vecs (exact up to
    rounding), at power-of-two and odd sizes, rows in draw order."""
    for n, m, seed in ((16, 5, 11), (100, 37, 12), (257, 64, 13), (1024, 256, 14)):
        g = synth.rng(seed)
        c = g.standard_normal(n)
        rows = synth.draw_rows(g, n, m)
        x = g.standard_normal(n)
        r = g.standard_normal(m)
        chat = O.spectrum(c)
        A = O.sensing_matrix(c, rows)
        assert np.allclose(O.forward_fft(chat, rows, x), A @ x, rtol=0, atol=1e-11 * n)
        assert np.allclose(O.adjoint_fft(chat, rows, r), A.T @ r, rtol=0, atol=1e-11 * n)
        assert np.allclose(O.forward_dense(c, rows, x), A @ x, atol=1e-12)
        idx = np.arange(0, m, 3)
        assert np.allclose(O.forward_sampled(c, rows, x, idx), (A @ x)[idx], atol=1e-12)
        jdx = np.arange(0, n, 5)
        assert np.allclose(O.adjoint_sampled(c, rows, r, jdx), (A.T @ r)[jdx], atol=1e-12)


def check_adjoint_identity(O):
    """<A x, r> = <x, A^T r> for the FFT products (dot-product test)."""
    for n, m, seed in ((64, 16, 21), (4096, 1024, 22)):
        g = synth.rng(seed)
        c = g.standard_normal(n) / np.sqrt(m)
        rows = synth.draw_rows(g, n, m)
        x = g.standard_normal(n)
        r = g.standard_normal(m)
        chat = O.spectrum(c)
        lhs = float(O.forward_fft(chat, rows, x) @ r)
        rhs = float(x @ O.adjoint_fft(chat, rows, r))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)) * np.sqrt(n), (lhs, rhs)


def check_soft_threshold_values(O):
    """Eq. 4 evaluated by hand, including the tie |x| = gamma -> 0."""
    x = np.array([3.0, -3.0, 1.0, -1.0, 0.5, 0.0, 2.5])
    want = np.array([2.0, -2.0, 0.0, 0.0, 0.0, 0.0, 1.5])
    assert np.array_equal(O.soft_threshold(x, 1.0), want)


def check_d_diagonal(O):
    """Sec. 4.3: D = (P^T P + rho I)^-1 has 1/(1+rho) on Omega, 1/rho off it
    (the text's diagonal values; the sign in the printed matrix is a typo)."""
    k = _paper_constants()["D_diagonal"]
    rho = 0.25
    d = O.admm_d_diagonal(6, np.array([4, 1]), rho)
    on = 1.0 / eval(k["on_omega"], {"rho": rho})
    off = 1.0 / eval(k["off_omega"], {"rho": rho})
    assert np.allclose(d, [off, on, off, off, on, off], rtol=0, atol=0)


# ---------------------------------------------------------------- closed forms

def check_identity_sensing_closed_form(O):
    """c = delta and all rows kept: A = I, so the LASSO minimiser is
    eta_lam(y) exactly; ISTA with tau = 1 reaches it in one step and ADMM
    converges to it (dense and FFT forms)."""
    n = 32
    c = np.zeros(n); c[0] = 1.0
    rows = np.arange(n)[::-1].copy()
    y = synth.random_vector(n, 31)
    lam = 0.3
    # y is indexed like rows: y[i] pairs with row rows[i]
    xhat = np.zeros(n)
    for i, rw in enumerate(rows):
        v = y[i]
        xhat[rw] = np.sign(v) * max(abs(v) - lam, 0.0)
    for ista in (O.ista_dense, O.ista_fft):
        x1 = ista(c, rows, y, lam, 1.0, 1)
        assert np.allclose(x1, xhat, atol=1e-13), ista.__name__
    for admm in (O.admm_dense, O.admm_fft):
        out = admm(c, rows, y, lam, sigma=1.0, rho=1.0, iters=400)
        assert np.allclose(out["z"], xhat, atol=1e-9), admm.__name__


def _orthogonal_c(O, n, seed):
    spec = synth.unit_modulus_c(n, seed)
    # inverse DFT by definition (Hermitian spectrum -> real c)
    j = np.arange(n)
    c = (np.exp(2j * np.pi * np.outer(j, j) / n) @ spec).real / n
    return c


def check_orthogonal_circulant_closed_form(O):
    """|chat_k| = 1 makes C orthogonal; with every row kept the LASSO
    minimiser is eta_lam(C^T y) in closed form (C^T y computed here by the
    dense transpose)."""
    n = 64
    c = _orthogonal_c(O, n, 41)
    C = O.circulant_matrix(c)
    assert np.allclose(C.T @ C, np.eye(n), atol=1e-12)
    rows = np.arange(n)
    y = synth.random_vector(n, 42)
    lam = 0.2
    u = C.T @ y
    xhat = np.sign(u) * np.maximum(np.abs(u) - lam, 0.0)
    for ista in (O.ista_dense, O.ista_fft):
        assert np.allclose(ista(c, rows, y, lam, 1.0, 1), xhat, atol=1e-12)
        assert np.allclose(ista(c, rows, y, lam, 0.5, 200), xhat, atol=1e-10)
    for admm in (O.admm_dense, O.admm_fft):
        out = admm(c, rows, y, lam, sigma=1.0, rho=1.0, iters=300)
        assert np.allclose(out["z"], xhat, atol=1e-8), admm.__name__
        assert np.allclose(out["x"], xhat, atol=1e-8), admm.__name__


# ---------------------------------------------------------------- invariants

def _tiny(seed, n=24, m=12, k=3):
    inst = synth.instance(n, m, k=k, seed=seed)
    return inst


def check_ista_monotone(O):
    """With tau <= 1/||A||^2 the objective never increases along ISTA
    (descent lemma for proximal gradient; Algorithm 1's step range)."""
    inst = _tiny(51, n=64, m=32, k=4)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true + 0.01 * synth.random_vector(inst.m, 52)
    L = np.linalg.norm(A, 2) ** 2
    lam = 0.02
    _, hist = O.ista_dense(inst.c, inst.rows, y, lam, 1.0 / L, 200, history=True)
    f = [O.lasso_objective(A, y, x, lam) for x in hist]
    assert all(f[t + 1] <= f[t] + 1e-13 for t in range(len(f) - 1))
    assert f[-1] < f[0]


def check_kkt_at_convergence(O):
    """Converged ISTA and ADMM (Algorithm 3) satisfy the LASSO optimality
    conditions; Algorithm 2 reaches the same point."""
    inst = _tiny(61, n=48, m=24, k=3)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true + 0.01 * synth.random_vector(inst.m, 62)
    lam = 0.01
    L = np.linalg.norm(A, 2) ** 2
    xi = O.ista_dense(inst.c, inst.rows, y, lam, 1.0 / L, 20000)
    assert O.kkt_violation(A, y, xi, lam) < 1e-9
    out = O.admm_dense(inst.c, inst.rows, y, lam, sigma=0.6, rho=1.5, iters=4000)
    assert O.kkt_violation(A, y, out["z"], lam) < 1e-8
    assert np.allclose(out["z"], xi, atol=1e-8)
    _, z2, _ = O.admm_standard_dense(A, y, lam, 1.0, 4000)
    assert np.allclose(z2, xi, atol=1e-8)


def check_admm_fixed_point_relations(O):
    """At the fixed point of Algorithm 3: z = x; the unfolded v equals C x;
    sigma nu = A^T (y - A x) and rho mu = P^T (y - P C x) (stationarity of the
    augmented Lagrangian of Sec. 4.3 in x and v)."""
    inst = _tiny(71, n=32, m=16, k=2)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true
    lam, sigma, rho = 0.01, 0.7, 1.3
    out = O.admm_dense(inst.c, inst.rows, y, lam, sigma=sigma, rho=rho, iters=6000)
    C = O.circulant_matrix(inst.c)
    x, z, mu, nu, v = out["x"], out["z"], out["mu"], out["nu"], out["v"]
    assert np.allclose(x, z, atol=1e-9)
    assert np.allclose(v - mu, C @ x, atol=1e-9)
    assert np.allclose(sigma * nu, A.T @ (y - A @ x), atol=1e-9)
    pty = np.zeros(32); pty[inst.rows] = y - A @ x
    assert np.allclose(rho * mu, pty, atol=1e-9)


def check_bruteforce_lasso(O):
    """Exact LASSO minimiser by sign-pattern enumeration (n = 8) against
    converged ISTA, Algorithm 3 ADMM (dense and FFT) and Algorithm 2 ADMM."""
    inst = synth.instance(8, 5, k=2, seed=81)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true + 0.05 * synth.random_vector(inst.m, 82)
    lam = 0.02
    xb = O.lasso_bruteforce(A, y, lam)
    assert xb is not None
    assert O.kkt_violation(A, y, xb, lam) < 1e-10
    L = np.linalg.norm(A, 2) ** 2
    xi = O.ista_dense(inst.c, inst.rows, y, lam, 1.0 / L, 40000)
    assert np.allclose(xi, xb, atol=1e-8), (xi, xb)
    for admm in (O.admm_dense, O.admm_fft):
        out = admm(inst.c, inst.rows, y, lam, sigma=0.5, rho=0.8, iters=20000)
        assert np.allclose(out["z"], xb, atol=1e-7), admm.__name__
    _, z2, _ = O.admm_standard_dense(A, y, lam, 0.5, 20000)
    assert np.allclose(z2, xb, atol=1e-7)


def check_exact_recovery_tiny(O):
    """Noiseless k-sparse signal: the l0 problem (Eq. 2) has x* as its unique
    sparsest solution (brute force over supports); LASSO with a small lam
    (ISTA) finds exactly that support with error O(lam sqrt(k))."""
    inst = synth.instance(40, 20, k=3, seed=91)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true
    x0, fits = O.l0_bruteforce(A, y, 3)
    assert len(fits) == 1
    assert set(fits[0]) == set(np.flatnonzero(inst.x_true))
    assert np.allclose(x0, inst.x_true, atol=1e-9)
    lam = 1e-4
    L = np.linalg.norm(A, 2) ** 2
    xi = O.ista_dense(inst.c, inst.rows, y, lam, 1.0 / L, 60000)
    assert set(np.flatnonzero(np.abs(xi) > 1e-6)) == set(fits[0])
    assert np.linalg.norm(xi - inst.x_true) <= 50 * lam * np.sqrt(3)


def check_admm_inverse(O):
    """B = (rho C^T C + sigma I)^-1 (Algorithm 3): the FFT spectrum
    1/(rho |chat|^2 + sigma) applied to b solves the dense system."""
    n = 48
    c = synth.random_vector(n, 101)
    rho, sigma = 0.8, 0.3
    C = O.circulant_matrix(c)
    b = synth.random_vector(n, 102)
    chat = O.naive_dft(c)
    x = np.fft.ifft(np.fft.fft(b) / (rho * np.abs(chat) ** 2 + sigma)).real
    assert np.linalg.norm((rho * C.T @ C + sigma * np.eye(n)) @ x - b) < 1e-10
    # one ADMM iteration from a chosen state reproduces that solve
    v = synth.random_vector(n, 103); z = synth.random_vector(n, 104)
    nu = synth.random_vector(n, 105); mu = np.zeros(n)
    rows = np.arange(0, n, 3)
    y = np.zeros(rows.size)
    for admm in (O.admm_dense, O.admm_fft):
        out = admm(c, rows, y, 0.0, sigma=sigma, rho=rho, iters=1,
                   state=(v, z, mu, nu))
        rhs = rho * C.T @ v + sigma * (z - nu)
        assert np.linalg.norm((rho * C.T @ C + sigma * np.eye(n)) @ out["x"] - rhs) < 1e-10


def check_dense_fft_agree(O):
    """Dense and FFT oracles produce the same iterates (1e-12 relative)."""
    inst = synth.instance(256, 64, k=8, seed=111)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true
    L = np.linalg.norm(A, 2) ** 2
    xd = O.ista_dense(inst.c, inst.rows, y, 1e-3, 1.0 / L, 50)
    xf = O.ista_fft(inst.c, inst.rows, y, 1e-3, 1.0 / L, 50)
    assert np.linalg.norm(xd - xf) <= 1e-12 * np.linalg.norm(xd)
    od = O.admm_dense(inst.c, inst.rows, y, 1e-3, sigma=1.0, rho=1.0, iters=50)
    of = O.admm_fft(inst.c, inst.rows, y, 1e-3, sigma=1.0, rho=1.0, iters=50)
    for key in ("x", "z", "mu", "nu", "v"):
        assert np.linalg.norm(od[key] - of[key]) <= 1e-11 * max(1.0, np.linalg.norm(od[key])), key


def check_opnorm(O):
    """Power iteration with FFT products matches the largest singular value."""
    inst = synth.instance(128, 40, k=4, seed=121)
    L1 = O.opnorm2_dense(inst.c, inst.rows)
    A = O.sensing_matrix(inst.c, inst.rows)
    sv = np.linalg.eigvalsh(A @ A.T).max()
    assert abs(L1 - sv) <= 1e-10 * sv
    L2 = O.opnorm2_power_fft(inst.c, inst.rows, iters=5000, tol=1e-15)
    assert abs(L2 - sv) <= 1e-6 * sv


# ---------------------------------------------------------------- unrolled ISTA gradient

def _smooth_grad_instance(O, n, m, k, T, seed0, margin=1e-4):
    """A seeded instance whose T ISTA iterates keep every |u| at least
    `margin` away from the threshold (so that central differences with a
    much smaller step never cross a kink of the soft threshold)."""
    for seed in range(seed0, seed0 + 50):
        inst = synth.instance(n, m, k=k, noise_std=1e-2, seed=seed)
        A = O.sensing_matrix(inst.c, inst.rows)
        y = A @ inst.x_true + inst.noise
        tau = 0.9 / O.opnorm2_dense(inst.c, inst.rows)
        lam = 0.05 * float(np.max(np.abs(A.T @ y)))
        x = np.zeros(n)
        gap = np.inf
        for _ in range(T):
            u = x + tau * (A.T @ (y - A @ x))
            gap = min(gap, float(np.min(np.abs(np.abs(u) - tau * lam))))
            x = O.soft_threshold(u, tau * lam)
        if gap > margin and np.count_nonzero(x) > 0:
            return inst, y, lam, tau
    raise AssertionError("no smooth instance found")


def check_unrolled_grad_finite_differences(O):
    """The reverse-mode gradient of L = ||x(T) - x*||^2 (T ISTA steps from
    x(0) = 0) equals central finite differences of the forward iteration
    (ista_dense, itself pinned above) along random directions in c, y and
    for lambda."""
    n, m, T = 32, 14, 15
    inst, y, lam, tau = _smooth_grad_instance(O, n, m, 3, T, 131)
    L0, gx = O.ista_unrolled_loss(inst.c, inst.rows, y, lam, tau, T, inst.x_true)
    gr = O.ista_unrolled_grad_dense(inst.c, inst.rows, y, lam, tau, T, gx)
    h = 1e-6
    g = synth.rng(132)

    def loss(c, yy, ll):
        return O.ista_unrolled_loss(c, inst.rows, yy, ll, tau, T, inst.x_true)[0]

    dcdir = g.standard_normal(n)
    fd = (loss(inst.c + h * dcdir, y, lam) - loss(inst.c - h * dcdir, y, lam)) / (2 * h)
    an = float(np.dot(gr["dc"], dcdir))
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), ("dc", fd, an)
    dydir = g.standard_normal(m)
    fd = (loss(inst.c, y + h * dydir, lam) - loss(inst.c, y - h * dydir, lam)) / (2 * h)
    an = float(np.dot(gr["dy"], dydir))
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), ("dy", fd, an)
    fd = (loss(inst.c, y, lam + h) - loss(inst.c, y, lam - h)) / (2 * h)
    assert abs(fd - gr["dlam"]) <= 1e-6 * max(1.0, abs(fd)), ("dlam", fd, gr["dlam"])
    assert np.allclose(gr["x_T"], O.ista_dense(inst.c, inst.rows, y, lam, tau, T), atol=1e-14)


def check_unrolled_grad_active_override(O):
    """Handing the reverse mode the forward pass's own supports (x(t+1) != 0)
    reproduces the default result exactly; handing it the supports with one
    entry removed changes dy (so the override is really used)."""
    inst = synth.instance(256, 96, k=6, noise_std=1e-3, seed=8123)
    chat = O.spectrum(inst.c)
    y = O.forward_fft(chat, inst.rows, inst.x_true) + inst.noise
    tau = 0.9 / float(np.max(np.abs(chat) ** 2))
    lam, T = 2e-3, 12
    xs = [np.zeros(inst.n)]
    for _ in range(T):
        xs.append(O.ista_fft(inst.c, inst.rows, y, lam, tau, 1, x0=xs[-1]))
    gx = 2.0 * (xs[-1] - inst.x_true)
    base = O.ista_unrolled_grad_fft(inst.c, inst.rows, y, lam, tau, T, gx)
    same = O.ista_unrolled_grad_fft(inst.c, inst.rows, y, lam, tau, T, gx, active=lambda t: xs[t + 1] != 0)
    for key in ("dc", "dy", "dx0"):
        assert np.array_equal(base[key], same[key]), key
    assert base["dlam"] == same["dlam"]
    t0 = T - 1
    on = np.flatnonzero(xs[t0 + 1])
    assert on.size > 0

    def fewer(t):
        a = xs[t + 1] != 0
        if t == t0:
            a = a.copy()
            a[on[0]] = False
        return a

    other = O.ista_unrolled_grad_fft(inst.c, inst.rows, y, lam, tau, T, gx, active=fewer)
    assert not np.allclose(other["dy"], base["dy"], rtol=1e-9, atol=0.0)


def check_unrolled_grad_dense_fft_agree(O):
    """Dense and FFT forms of the gradient agree to rounding, and the FFT
    form also matches central differences at a larger size."""
    n, m, T = 128, 50, 12
    inst, y, lam, tau = _smooth_grad_instance(O, n, m, 5, T, 141)
    _, gx = O.ista_unrolled_loss(inst.c, inst.rows, y, lam, tau, T, inst.x_true)
    gd = O.ista_unrolled_grad_dense(inst.c, inst.rows, y, lam, tau, T, gx)
    gf = O.ista_unrolled_grad_fft(inst.c, inst.rows, y, lam, tau, T, gx)
    for key in ("dc", "dy", "dx0", "x_T"):
        scale = max(1.0, float(np.max(np.abs(gd[key]))))
        assert np.max(np.abs(gd[key] - gf[key])) <= 1e-10 * scale, key
    assert abs(gd["dlam"] - gf["dlam"]) <= 1e-10 * max(1.0, abs(gd["dlam"]))
    h = 1e-6
    d = synth.rng(142).standard_normal(n)
    lp = O.ista_unrolled_loss(inst.c + h * d, inst.rows, y, lam, tau, T, inst.x_true, dense=False)[0]
    lm = O.ista_unrolled_loss(inst.c - h * d, inst.rows, y, lam, tau, T, inst.x_true, dense=False)[0]
    fd = (lp - lm) / (2 * h)
    assert abs(fd - float(np.dot(gf["dc"], d))) <= 1e-6 * max(1.0, abs(fd))


def _smooth_admm_instance(O, n, m, k, T, sigma, rho, tau1, tau2, seed0, margin=1e-4):
    """A seeded instance whose T ADMM iterations keep every |x + nu| at least
    `margin` away from the threshold lam / sigma (central differences with a
    much smaller step then never cross a kink of the soft threshold)."""
    for seed in range(seed0, seed0 + 50):
        inst = synth.instance(n, m, k=k, noise_std=1e-2, seed=seed)
        A = O.sensing_matrix(inst.c, inst.rows)
        y = A @ inst.x_true + inst.noise
        lam = 0.05 * float(np.max(np.abs(A.T @ y)))
        gap, nz = np.inf, 0
        for t in range(1, T + 1):
            st = O.admm_dense(inst.c, inst.rows, y, lam, sigma, rho, tau1, tau2, iters=t)
            prev = O.admm_dense(inst.c, inst.rows, y, lam, sigma, rho, tau1, tau2, iters=t - 1) if t > 1 else None
            nu_in = prev["nu"] if prev is not None else np.zeros(n)
            s = st["x"] + nu_in
            gap = min(gap, float(np.min(np.abs(np.abs(s) - lam / sigma))))
            nz = np.count_nonzero(st["z"])
        if gap > margin and nz > 0:
            return inst, y, lam
    raise AssertionError("no smooth instance found")


def check_admm_grad_finite_differences(O):
    """The reverse-mode gradient of L = ||z(T) - x*||^2 + 0.5 ||x(T)||^2 over
    T iterations of Algorithm 3 (general sigma, rho, tau1, tau2) equals
    central finite differences of the forward iteration (admm_dense, pinned
    above) along random directions in c, y and for lambda."""
    n, m, T = 32, 14, 10
    sg, rh, t1, t2 = 0.8, 1.3, 1.1, 0.9
    inst, y, lam = _smooth_admm_instance(O, n, m, 3, T, sg, rh, t1, t2, 311)

    def loss(c, yy, ll):
        st = O.admm_dense(c, inst.rows, yy, ll, sg, rh, t1, t2, iters=T)
        dz = st["z"] - inst.x_true
        return float(dz @ dz) + 0.5 * float(st["x"] @ st["x"]), 2.0 * dz, st["x"]

    _, gz, xT = loss(inst.c, y, lam)
    gr = O.admm_unrolled_grad_dense(inst.c, inst.rows, y, lam, sg, rh, t1, t2, T, gz, gx_T=xT)
    h = 1e-6
    g = synth.rng(312)
    d = g.standard_normal(n)
    fd = (loss(inst.c + h * d, y, lam)[0] - loss(inst.c - h * d, y, lam)[0]) / (2 * h)
    assert abs(fd - float(gr["dc"] @ d)) <= 1e-6 * max(1.0, abs(fd)), ("dc", fd, float(gr["dc"] @ d))
    d = g.standard_normal(m)
    fd = (loss(inst.c, y + h * d, lam)[0] - loss(inst.c, y - h * d, lam)[0]) / (2 * h)
    assert abs(fd - float(gr["dy"] @ d)) <= 1e-6 * max(1.0, abs(fd)), ("dy", fd, float(gr["dy"] @ d))
    fd = (loss(inst.c, y, lam + h)[0] - loss(inst.c, y, lam - h)[0]) / (2 * h)
    assert abs(fd - gr["dlam"]) <= 1e-6 * max(1.0, abs(fd)), ("dlam", fd, gr["dlam"])
    assert np.allclose(gr["z_T"], O.admm_dense(inst.c, inst.rows, y, lam, sg, rh, t1, t2, iters=T)["z"],
                       atol=1e-14)


def check_admm_grad_dense_fft_agree(O):
    """The FFT form of the ADMM reverse mode equals the dense form."""
    inst = synth.instance(128, 50, k=5, noise_std=1e-3, seed=321)
    A = O.sensing_matrix(inst.c, inst.rows)
    y = A @ inst.x_true + inst.noise
    lam, T = 0.02 * float(np.max(np.abs(A.T @ y))), 15
    _, gz = O.admm_unrolled_loss(inst.c, inst.rows, y, lam, 1.0, 0.7, 1.0, 1.2, T, inst.x_true)
    a = O.admm_unrolled_grad_dense(inst.c, inst.rows, y, lam, 1.0, 0.7, 1.0, 1.2, T, gz)
    b = O.admm_unrolled_grad_fft(inst.c, inst.rows, y, lam, 1.0, 0.7, 1.0, 1.2, T, gz)
    for key in ("dc", "dy", "z_T"):
        assert np.linalg.norm(a[key] - b[key]) <= 1e-11 * max(1.0, np.linalg.norm(a[key])), key
    assert abs(a["dlam"] - b["dlam"]) <= 1e-11 * max(1.0, abs(a["dlam"]))


def check_product_of_circulants(O):
    """Sec. 7: the product of circulant matrices is circulant (A = C B for a
    circulant sensing C and blur B).  C(a) C(b), formed densely, equals the
    circulant of the generating vector the input generator builds for it,
    for a box blur of order 5 and for a random short filter."""
    g = synth.rng(161)
    for n, b in ((16, synth.box_blur_c(16, 5)), (12, np.r_[g.standard_normal(3), np.zeros(9)])):
        a = g.standard_normal(n)
        prod = O.circulant_matrix(a) @ O.circulant_matrix(b)
        assert np.allclose(prod, O.circulant_matrix(synth.composite_c(a, b)), atol=1e-12), n
    # the box blur averages L consecutive entries (its definition)
    x = g.standard_normal(16)
    bx = O.circulant_matrix(synth.box_blur_c(16, 5)) @ x
    assert np.allclose(bx, [np.mean(x[np.arange(i, i + 5) % 16]) for i in range(16)], atol=1e-14)


# ---------------------------------------------------------------- 2D operator

def check_2d_separable_is_kronecker(O):
    """A separable generating array c2 = c0 c1^T blurs rows and columns
    independently: H = C(c0) kron C(c1), built from the pinned 1D circulant."""
    g = synth.rng(151)
    for n0, n1 in ((4, 8), (3, 5), (8, 4)):
        c0, c1 = g.standard_normal(n0), g.standard_normal(n1)
        H = O.circulant2d_matrix(np.outer(c0, c1))
        K = np.kron(O.circulant_matrix(c0), O.circulant_matrix(c1))
        assert np.allclose(H, K, atol=1e-13), (n0, n1)


def check_2d_eigenvectors(O):
    """H f = conj(chat2[k0, k1]) f for the 2D Fourier vectors
    f = exp(2 pi i (j0 k0 / n0 + j1 k1 / n1)), chat2 by the O(n^2) definition
    along both axes (no FFT library); spectrum2d equals it."""
    g = synth.rng(152)
    n0, n1 = 4, 6
    c2 = g.standard_normal((n0, n1))
    H = O.circulant2d_matrix(c2)
    ch = O.naive_dft2(c2)
    j0 = np.arange(n0 * n1) // n1
    j1 = np.arange(n0 * n1) % n1
    for k0 in range(n0):
        for k1 in range(n1):
            f = np.exp(2j * np.pi * (j0 * k0 / n0 + j1 * k1 / n1))
            assert np.allclose(H @ f, np.conj(ch[k0, k1]) * f, atol=1e-12), (k0, k1)
    assert np.allclose(O.spectrum2d(c2), ch, atol=1e-12)


def check_2d_point_source_is_psf(O):
    """Blurring a single bright pixel reproduces the point-spread function
    around it (periodic), for the generating array of a non-symmetric PSF."""
    n0, n1 = 16, 32
    psf = synth.rng(153).random((5, 3))
    psf /= psf.sum()
    c2 = synth.psf_generator(psf, n0, n1)
    a, b = 14, 1                      # near two edges: wrap-around
    x = np.zeros(n0 * n1)
    x[a * n1 + b] = 1.0
    img = O.circulant2d_apply_fft(O.spectrum2d(c2), x).reshape(n0, n1)
    want = np.zeros((n0, n1))
    for u in range(5):
        for v in range(3):
            want[(a + u - 2) % n0, (b + v - 1) % n1] += psf[u, v]
    assert np.allclose(img, want, atol=1e-14)


def check_2d_fft_matches_dense(O):
    """2D FFT products and both solvers equal their dense forms."""
    g = synth.rng(154)
    n0, n1 = 8, 16
    c2 = g.standard_normal((n0, n1)) / 8
    pix = synth.draw_rows(g, n0 * n1, 50)
    A = O.sensing2d_matrix(c2, pix)
    ch = O.spectrum2d(c2)
    x = g.standard_normal(n0 * n1)
    r = g.standard_normal(50)
    assert np.allclose(O.forward2d_fft(ch, pix, x), A @ x, atol=1e-12)
    assert np.allclose(O.adjoint2d_fft(ch, pix, r), A.T @ r, atol=1e-12)
    xs = np.zeros(n0 * n1)
    xs[g.choice(n0 * n1, 4, replace=False)] = g.standard_normal(4)
    y = A @ xs
    tau = 1.0 / np.linalg.norm(A, 2) ** 2
    a = O.ista_dense2d(c2, pix, y, 1e-3, tau, 60)
    b = O.ista_fft2d(c2, pix, y, 1e-3, tau, 60)
    assert np.allclose(a, b, atol=1e-11)
    a = O.admm_dense2d(c2, pix, y, 1e-3, 0.7, 1.3, iters=60)
    b = O.admm_fft2d(c2, pix, y, 1e-3, 0.7, 1.3, iters=60)
    for key in ("x", "z", "mu", "nu", "v"):
        assert np.allclose(a[key], b[key], atol=1e-10), key


ALL_CHECKS = [
    check_circulant_worked_example, check_eigenvalues_are_dft,
    check_fft_products_match_dense, check_adjoint_identity,
    check_soft_threshold_values, check_d_diagonal,
    check_identity_sensing_closed_form, check_orthogonal_circulant_closed_form,
    check_ista_monotone, check_kkt_at_convergence,
    check_admm_fixed_point_relations, check_bruteforce_lasso,
    check_exact_recovery_tiny, check_admm_inverse, check_dense_fft_agree,
    check_opnorm, check_unrolled_grad_finite_differences, check_unrolled_grad_dense_fft_agree,
    check_unrolled_grad_active_override, check_admm_grad_finite_differences, check_admm_grad_dense_fft_agree,
    check_2d_separable_is_kronecker, check_2d_eigenvectors, check_2d_point_source_is_psf,
    check_2d_fft_matches_dense, check_product_of_circulants,
]
