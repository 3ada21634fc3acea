"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins catch every one of them: a transposed operand, a wrong index, a dropped
term, a flipped sign, a wrong threshold."""
import numpy as np
import pytest

import oracle.cs_oracle as O
from oracle_pins import ALL_CHECKS


def _mut_transposed_circulant(c):
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return c[(i - j) % n]


def _mut_reverse_circulant(c):
    # the i + j indexing of the ISTA kernels printed in Sec. 5.2
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return c[(i + j) % n]


def _mut_conj_fft(chat, x, transpose=False):
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    h = chat[: n // 2 + 1]
    h = np.conj(h) if transpose else h
    return np.fft.irfft(h * np.fft.rfft(x), n)


def _mut_threshold_hard(x, gamma):
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) > gamma, x, 0.0)


def _mut_d_minus(n, rows, rho):
    d = np.full(n, 1.0 / rho)
    d[np.asarray(rows, dtype=np.int64)] = 1.0 / (1.0 - rho) if rho != 1.0 else 0.5
    return d


def _mut_ista_threshold_lam(apply_A, apply_At, y, lam, tau, iters, x0, n, history):
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    hist = [x.copy()] if history else None
    for _ in range(iters):
        r = y - apply_A(x)
        x = O.soft_threshold(x + tau * apply_At(r), lam)
        if history:
            hist.append(x.copy())
    return (x, hist) if history else x


def _mut_ista_residual_sign(apply_A, apply_At, y, lam, tau, iters, x0, n, history):
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    hist = [x.copy()] if history else None
    for _ in range(iters):
        r = apply_A(x) - y
        x = O.soft_threshold(x + tau * apply_At(r), tau * lam)
        if history:
            hist.append(x.copy())
    return (x, hist) if history else x


def _admm_variant(drop_sigma=False, no_fold=False, nu_sign=+1, z_thr_rho=False):
    def _admm(C_apply, Ct_apply, B_apply, n, rows, y, lam, sigma, rho, tau1,
              tau2, iters, state, history):
        d = O.admm_d_diagonal(n, rows, rho)
        pty = O.zero_fill(n, rows, y)
        if state is None:
            v = np.zeros(n); z = np.zeros(n); mu = np.zeros(n); nu = np.zeros(n)
        else:
            v, z, mu, nu = (np.asarray(s, dtype=np.float64).copy() for s in state)
        x = np.zeros(n)
        for _ in range(iters):
            s = 1.0 if drop_sigma else sigma
            x = B_apply(rho * Ct_apply(v) + s * (z - nu))
            cx = C_apply(x)
            v = d * (rho * cx - rho * mu + pty)
            z = O.soft_threshold(x + nu, lam / (rho if z_thr_rho else sigma))
            mu = mu + tau1 * (v - cx)
            nu = nu + nu_sign * tau2 * (x - z)
            if not no_fold:
                v = v + mu
        return {"x": x, "z": z, "mu": mu, "nu": nu, "v": v}
    return _admm


def _grad_variant(drop_q=False, active_from_x=False, dy_no_tau=False, dlam_sign=-1.0, corr_swap=False):
    """_ista_grad with one planted mistake."""
    def _g(C_apply, Ct_apply, corr, n, rows, y, lam, tau, T, gx_T, active=None):
        rows = np.asarray(rows, dtype=np.int64)
        y = np.asarray(y, dtype=np.float64)
        theta = tau * lam
        mask = np.zeros(n)
        mask[rows] = 1.0
        pty = O.zero_fill(n, rows, y)
        xs = [np.zeros(n)]
        us = []
        for _ in range(T):
            x = xs[-1]
            u = x + tau * Ct_apply(mask * (pty - C_apply(x)))
            us.append(u)
            xs.append(O.soft_threshold(u, theta))
        g = np.asarray(gx_T, dtype=np.float64).copy()
        dc = np.zeros(n)
        dtheta = 0.0
        dy = np.zeros(len(rows))
        for t in range(T - 1, -1, -1):
            x, u = xs[t], us[t]
            act = (np.abs(x) > 0) if active_from_x else (np.abs(u) > theta)
            if active is not None:
                act = np.asarray(active(t), dtype=bool)
            w = np.where(act, g, 0.0)
            dtheta += dlam_sign * float(np.sum(np.sign(u) * w))
            cw = C_apply(w)
            q = mask * cw
            dy += (1.0 if dy_no_tau else tau) * cw[rows]
            r = mask * (pty - C_apply(x))
            term = corr(w, r) if corr_swap else corr(r, w)
            dc += tau * (term - (0.0 if drop_q else corr(q, x)))
            g = w - tau * Ct_apply(q)
        return {"x_T": xs[-1], "dc": dc, "dlam": tau * dtheta, "dy": dy, "dx0": g}
    return _g


def _admm_grad_variant(drop_b_term=False, drop_ctv_term=False, no_d=False, mu_sign=-1.0, drop_nu_sigma=False,
                       no_fold=False):
    """_admm_grad with one planted mistake."""
    def _g(C_apply, Ct_apply, B_apply, corr, n, rows, y, lam, sigma, rho, tau1, tau2, T, gz_T, gx_T=None):
        rows = np.asarray(rows, dtype=np.int64)
        y = np.asarray(y, dtype=np.float64)
        theta = lam / sigma
        d = O.admm_d_diagonal(n, rows, rho)
        pty = O.zero_fill(n, rows, y)
        v = np.zeros(n); z = np.zeros(n); mu = np.zeros(n); nu = np.zeros(n)
        steps = []
        for _ in range(T):
            x = B_apply(rho * Ct_apply(v) + sigma * (z - nu))
            p = C_apply(x)
            v1 = d * (rho * p - rho * mu + pty)
            s = x + nu
            z1 = O.soft_threshold(s, theta)
            mu1 = mu + tau1 * (v1 - p)
            nu1 = nu + tau2 * (x - z1)
            steps.append((v, x, p, s))
            v, z, mu, nu = v1 + mu1, z1, mu1, nu1
        vb = np.zeros(n); zb = np.asarray(gz_T, dtype=np.float64).copy(); mub = np.zeros(n); nub = np.zeros(n)
        dc = np.zeros(n); dlam = 0.0; dy = np.zeros(len(rows))
        for t in range(T - 1, -1, -1):
            v0, x, p, s = steps[t]
            if not no_fold:
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
            ab = v1b if no_d else d * v1b
            pb = pb + rho * ab
            mub = mub + mu_sign * rho * ab
            dy += ab[rows]
            xb = xb + Ct_apply(pb)
            dc += corr(pb, x)
            bb = B_apply(xb)
            cbb = C_apply(bb)
            if not drop_b_term:
                dc -= rho * (corr(p, bb) + corr(cbb, x))
            if not drop_ctv_term:
                dc += rho * corr(v0, bb)
            vb = rho * cbb
            zb = sigma * bb
            if not drop_nu_sigma:
                nub = nub - sigma * bb
        return {"x_T": steps[-1][1], "z_T": z, "dc": dc, "dlam": dlam, "dy": dy}
    return _g


def _mut_circulant2d_transposed(c2):
    c2 = np.asarray(c2, dtype=np.float64)
    n0, n1 = c2.shape
    a = np.arange(n0 * n1) // n1
    b = np.arange(n0 * n1) % n1
    return c2[(a[:, None] - a[None, :]) % n0, (b[:, None] - b[None, :]) % n1]


def _mut_circulant2d_axes_mixed(c2):
    c2 = np.asarray(c2, dtype=np.float64)
    n0, n1 = c2.shape
    a = np.arange(n0 * n1) // n1
    b = np.arange(n0 * n1) % n1
    return c2[(a[None, :] - a[:, None]) % n0, (b[:, None] - b[None, :]) % n1]


def _mut_c2d_apply_conj(chat2, x, transpose=False):
    n0, n1 = chat2.shape
    xh = np.fft.rfft2(np.asarray(x, dtype=np.float64).reshape(n0, n1))
    h = chat2[:, : n1 // 2 + 1]
    h = np.conj(h) if transpose else h
    return np.fft.irfft2(h * xh, (n0, n1)).ravel()


MUTANTS = {
    "transposed_circulant": ("circulant_matrix", _mut_transposed_circulant),
    "reverse_circulant": ("circulant_matrix", _mut_reverse_circulant),
    "fft_conj_swapped": ("circulant_apply_fft", _mut_conj_fft),
    "hard_threshold": ("soft_threshold", _mut_threshold_hard),
    "d_minus_rho": ("admm_d_diagonal", _mut_d_minus),
    "ista_threshold_lam": ("_ista", _mut_ista_threshold_lam),
    "ista_residual_sign": ("_ista", _mut_ista_residual_sign),
    "admm_drop_sigma": ("_admm", _admm_variant(drop_sigma=True)),
    "admm_no_fold": ("_admm", _admm_variant(no_fold=True)),
    "admm_nu_sign": ("_admm", _admm_variant(nu_sign=-1)),
    "admm_threshold_rho": ("_admm", _admm_variant(z_thr_rho=True)),
    "grad_drop_q_term": ("_ista_grad", _grad_variant(drop_q=True)),
    "grad_active_from_x": ("_ista_grad", _grad_variant(active_from_x=True)),
    "grad_dy_no_tau": ("_ista_grad", _grad_variant(dy_no_tau=True)),
    "grad_dlam_sign": ("_ista_grad", _grad_variant(dlam_sign=+1.0)),
    "grad_corr_swapped": ("_ista_grad", _grad_variant(corr_swap=True)),
    "admm_grad_drop_inverse_term": ("_admm_grad", _admm_grad_variant(drop_b_term=True)),
    "admm_grad_drop_ctv_term": ("_admm_grad", _admm_grad_variant(drop_ctv_term=True)),
    "admm_grad_no_d": ("_admm_grad", _admm_grad_variant(no_d=True)),
    "admm_grad_mu_sign": ("_admm_grad", _admm_grad_variant(mu_sign=+1.0)),
    "admm_grad_drop_nu_sigma": ("_admm_grad", _admm_grad_variant(drop_nu_sigma=True)),
    "admm_grad_no_fold": ("_admm_grad", _admm_grad_variant(no_fold=True)),
    "c2d_transposed": ("circulant2d_matrix", _mut_circulant2d_transposed),
    "c2d_axes_mixed": ("circulant2d_matrix", _mut_circulant2d_axes_mixed),
    "c2d_fft_conj_swapped": ("circulant2d_apply_fft", _mut_c2d_apply_conj),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = []
    for check in ALL_CHECKS:
        try:
            with np.errstate(all="ignore"):
                check(O)
        except (AssertionError, np.linalg.LinAlgError, ValueError, ZeroDivisionError):
            caught.append(check.__name__)
    assert caught, f"mutant {name} passed every pin"
