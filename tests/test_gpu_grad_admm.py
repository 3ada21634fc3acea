"""GPU parity of cs_grad_admm (reverse mode of unrolled circulant ADMM,
Algorithm 3) against the FP64 oracle gradient and against central finite
differences of the GPU forward.

Both sides get the same dL/dz(T) (and dL/dx(T) where the loss uses it),
formed from the oracle's last iterate, so the comparison isolates the
reverse pass.  As for the ISTA gradient, the fp32 forward may keep or drop
an entry of z that the FP64 forward does not where |x + nu| is within
rounding of lambda / sigma; the bar is relative l2 <= 1e-3 (measured errors
are printed by the assertion messages).
"""
import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import f32, host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def cs():
    import paper_1707_02244_gb300 as cs
    return cs


def _setup(n, m, k, seed, lam_scale=0.05):
    inst = synth.instance(n, m, k=k, noise_std=1e-3, seed=seed)
    chat = O.spectrum(inst.c)
    y32 = (O.forward_fft(chat, inst.rows, inst.x_true) + inst.noise).astype(np.float32)
    lam = f32(lam_scale * np.max(np.abs(O.adjoint_fft(chat, inst.rows, y32.astype(np.float64)))))
    return inst, y32, lam


def _gpu_grad(cs, inst, y32, lam, prm, T, K, gz, gx=None):
    torch, dev = torch_dev()
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        dc = torch.empty(inst.n, dtype=torch.float32, device=dev)
        dl = torch.empty(1, dtype=torch.float32, device=dev)
        dy = torch.empty(inst.m, dtype=torch.float32, device=dev)
        cs.cs_grad_admm(plan, to_dev(y32), lam, *prm, T, K, to_dev(gz), dc, dl, dy,
                        gx_T=None if gx is None else to_dev(gx))
        assert cs.cs_status_sync(plan) == cs.CS_OK
        return host(dc), float(host(dl)[0]), host(dy)
    finally:
        plan.close()


def _oracle(inst, y32, lam, prm, T, with_x):
    """dL/dz(T) (and dL/dx(T)) of L = ||z(T) - x*||^2 (+ 0.5 ||x(T)||^2) from
    the oracle's forward, and the oracle's gradient."""
    sg, rh, t1, t2 = prm
    y64 = y32.astype(np.float64)
    st = O.admm_fft(inst.c, inst.rows, y64, lam, sigma=sg, rho=rh, tau1=t1, tau2=t2, iters=T)
    gz = (2.0 * (st["z"] - inst.x_true)).astype(np.float32)
    gx = st["x"].astype(np.float32) if with_x else None
    o = O.admm_unrolled_grad_fft(inst.c, inst.rows, y64, lam, sg, rh, t1, t2, T, gz.astype(np.float64),
                                 None if gx is None else gx.astype(np.float64))
    return gz, gx, o


@pytest.mark.parametrize("n,m,k,T,K,prm,with_x", [
    (256, 100, 4, 1, 1, (1.0, 1.0, 1.0, 1.0), False),
    (4096, 1024, 40, 30, 7, (0.8, 1.3, 1.1, 0.9), True),
    (1 << 14, 4000, 150, 40, 40, (1.0, 1.0, 1.0, 1.0), False),
    (1 << 16, 1 << 14, 600, 60, 25, (1.0, 0.7, 1.2, 1.0), True),
    (1 << 20, 1 << 18, 10000, 50, 25, (1.0, 1.0, 1.0, 1.0), False),
])
def test_admm_grad_matches_oracle(cs, n, m, k, T, K, prm, with_x):
    inst, y32, lam = _setup(n, m, k, 9000 + n + T)
    gz, gx, o = _oracle(inst, y32, lam, prm, T, with_x)
    dc, dl, dy = _gpu_grad(cs, inst, y32, lam, prm, T, K, gz, gx)
    print(f"n={n} T={T} K={K}: rel l2 dc {rel_l2(dc, o['dc']):.2e}, dy {rel_l2(dy, o['dy']):.2e}, "
          f"dlam {abs(dl - o['dlam']) / max(abs(o['dlam']), 1e-12):.2e}")
    assert rel_l2(dc, o["dc"]) <= GRAD_TOL, ("dc", rel_l2(dc, o["dc"]))
    assert rel_l2(dy, o["dy"]) <= GRAD_TOL, ("dy", rel_l2(dy, o["dy"]))
    assert abs(dl - o["dlam"]) <= GRAD_TOL * max(abs(o["dlam"]), 1e-12), ("dlam", dl, o["dlam"])


def test_admm_grad_is_deterministic_and_checkpoint_independent(cs):
    """Same gradient for K = 4 and K = T (replay from the start), bit for bit
    across repeated calls."""
    inst, y32, lam = _setup(2048, 700, 20, 9100)
    prm = (1.0, 1.0, 1.0, 1.0)
    gz, _, _ = _oracle(inst, y32, lam, prm, 20, False)
    a = _gpu_grad(cs, inst, y32, lam, prm, 20, 4, gz)
    b = _gpu_grad(cs, inst, y32, lam, prm, 20, 4, gz)
    c = _gpu_grad(cs, inst, y32, lam, prm, 20, 20, gz)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], c[0]) and a[1] == c[1] and np.array_equal(a[2], c[2])


def test_admm_grad_finite_differences(cs):
    """Directional derivatives of L = ||z(T) - x*||^2 (GPU forward through
    cs_admm_ex, loss in FP64) by central differences with eps = 1e-3 against
    cs_grad_admm."""
    torch, dev = torch_dev()
    n, m, T, eps = 4096, 1024, 30, 1e-3
    prm = (0.9, 1.1, 1.0, 1.0)
    inst, y32, lam = _setup(n, m, 40, 9200)
    g = synth.rng(9201)

    def loss(c, y, lm):
        plan = cs.cs_plan(n, m, inst.rows, c, torch.cuda.current_stream(dev))
        try:
            vs = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(5)]
            x, z, mu, nu, v = vs
            cs.cs_admm_ex(plan, to_dev(y), f32(lm), prm[0], prm[1], prm[2], prm[3], T, False, x, z, mu, nu, v)
            d = host(z) - inst.x_true
            return float(d @ d), d
        finally:
            plan.close()

    L0, d0 = loss(inst.c, y32, lam)
    dc, dl, dy = _gpu_grad(cs, inst, y32, lam, prm, T, 8, (2.0 * d0).astype(np.float32))
    u = g.standard_normal(n) * np.linalg.norm(inst.c) / np.sqrt(n)
    fd = (loss(inst.c + eps * u, y32, lam)[0] - loss(inst.c - eps * u, y32, lam)[0]) / (2 * eps)
    assert abs(fd - dc @ u) <= 2e-2 * abs(fd) + 1e-6, ("c", fd, dc @ u)
    v = (g.standard_normal(m) * np.linalg.norm(y32) / np.sqrt(m)).astype(np.float32)
    fd = (loss(inst.c, y32 + np.float32(eps) * v, lam)[0] - loss(inst.c, y32 - np.float32(eps) * v, lam)[0]) / (2 * eps)
    assert abs(fd - dy @ v) <= 2e-2 * abs(fd) + 1e-6, ("y", fd, dy @ v)
    h = eps * lam
    fd = (loss(inst.c, y32, lam + h)[0] - loss(inst.c, y32, lam - h)[0]) / (2 * h)
    assert abs(fd - dl) <= 2e-2 * abs(fd) + 1e-6, ("lambda", fd, dl)


def test_admm_grad_rejects_2d_plans_and_bad_arguments(cs):
    torch, dev = torch_dev()
    img = synth.star_field(16, 32, k=5, seed=91)
    p2 = cs.cs_plan_2d(img.n0, img.n1, img.m, img.pix, img.c2, torch.cuda.current_stream(dev))
    try:
        buf = torch.zeros(img.n, dtype=torch.float32, device=dev)
        yb = torch.zeros(img.m, dtype=torch.float32, device=dev)
        one = torch.zeros(1, dtype=torch.float32, device=dev)
        with pytest.raises(cs.CsError) as e:
            cs.cs_grad_admm(p2, yb, 1e-3, 1.0, 1.0, 1.0, 1.0, 4, 2, buf, buf, one, yb)
        assert e.value.code == cs.CS_ERR_UNSUPPORTED
    finally:
        p2.close()
    inst, y32, lam = _setup(256, 100, 4, 93)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        buf = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        yb = to_dev(y32)
        one = torch.zeros(1, dtype=torch.float32, device=dev)
        for args in [(lam, 1.0, 1.0, 1.0, 1.0, 4, 5), (lam, 0.0, 1.0, 1.0, 1.0, 4, 2), (lam, 1.0, -1.0, 1.0, 1.0, 4, 2)]:
            with pytest.raises(cs.CsError) as e:
                cs.cs_grad_admm(plan, yb, *args, buf, buf, one, yb)
            assert e.value.code == cs.CS_ERR_ARG
    finally:
        plan.close()
