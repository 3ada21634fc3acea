"""GPU parity of ISTA (Algorithm 1) and circulant ADMM (Algorithm 3) against
the FP64 oracle on identical inputs: c in fp64, y / lambda / tau / rho rounded
once to fp32 and promoted to fp64 for the oracle.

Bars: the fp32 iterates match the oracle's to relative l2 <= 1e-5 after 100
iterations, and the final solution to NMSE(gpu, oracle) <= 1e-6.
"""
import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import f32, host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5
FINAL_NMSE = 1e-6


@pytest.fixture(scope="module")
def cs():
    import paper_1707_02244_gb300 as cs
    return cs


def _plan(cs, inst):
    torch, dev = torch_dev()
    return cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))


def _y32(inst, dense):
    if dense:
        y = O.forward_dense(inst.c, inst.rows, inst.x_true)
    else:
        y = O.forward_fft(O.spectrum(inst.c), inst.rows, inst.x_true)
    return (y + inst.noise).astype(np.float32)


# ------------------------------------------------------------------ ISTA

def test_ista_small_instance(cs):
    """n=4096, m=1024, k=64, lambda=1e-3, tau=1/||A||^2, 500 iterations
    (run as 100 + 400 through the x(0) input)."""
    torch, dev = torch_dev()
    inst = synth.small_instance()
    y32 = _y32(inst, dense=True)
    lam = f32(1e-3)
    tau = f32(1.0 / O.opnorm2_dense(inst.c, inst.rows))
    plan = _plan(cs, inst)
    try:
        x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        yd = to_dev(y32)
        xt = to_dev(inst.x_true)      # the plan reads it: keep it alive
        cs.cs_set_monitor(plan, xt, 0.0, 10)
        st1 = cs.cs_ista(plan, yd, lam, tau, 100, x)
        x100 = host(x)
        st2 = cs.cs_ista(plan, yd, lam, tau, 400, x)
        x500 = host(x)
    finally:
        plan.close()
    y64 = y32.astype(np.float64)
    xo100, hist = O.ista_dense(inst.c, inst.rows, y64, lam, tau, 100, history=True)
    xo500 = O.ista_dense(inst.c, inst.rows, y64, lam, tau, 400, x0=xo100)
    assert rel_l2(x100, xo100) <= ITER_TOL, rel_l2(x100, xo100)
    assert O.nmse(x500, xo500) <= FINAL_NMSE, O.nmse(x500, xo500)
    # the device-side statistics agree with the oracle's view of the iterate
    assert st1["iters_run"] == 100 and st2["iters_run"] == 400
    assert abs(st2["nmse"] - O.nmse(x500, inst.x_true)) <= 1e-4 * O.nmse(x500, inst.x_true) + 1e-12
    A = O.sensing_matrix(inst.c, inst.rows)
    f99 = O.lasso_objective(A, y64, hist[99], lam)
    assert abs(st1["objective"] - f99) <= 1e-4 * f99
    rel = np.linalg.norm(x100 - hist[99]) / np.linalg.norm(x100)
    assert abs(st1["rel_change"] - rel) <= 1e-3 * rel + 1e-9


@pytest.mark.parametrize("n,m,k", [(64, 32, 3), (256, 64, 5), (1 << 14, 1 << 12, 40), (1 << 16, 1 << 14, 160),
                                   (1 << 18, 1 << 16, 600)])
def test_ista_sizes(cs, n, m, k):
    torch, dev = torch_dev()
    inst = synth.instance(n, m, k=k, noise_std=1e-3, seed=3000 + n)
    dense = n <= 4096
    y32 = _y32(inst, dense)
    lam = f32(2e-3)
    chat = O.spectrum(inst.c)
    tau = f32(1.0 / np.max(np.abs(chat) ** 2))   # 1/||C||^2 <= 1/||A||^2
    plan = _plan(cs, inst)
    try:
        x = torch.zeros(n, dtype=torch.float32, device=dev)
        cs.cs_ista(plan, to_dev(y32), lam, tau, 100, x)
        xg = host(x)
    finally:
        plan.close()
    ista = O.ista_dense if dense else O.ista_fft
    xo = ista(inst.c, inst.rows, y32.astype(np.float64), lam, tau, 100)
    assert rel_l2(xg, xo) <= ITER_TOL, rel_l2(xg, xo)


def test_ista_full_size(cs):
    """The timed workload: n=2^22, m=n/4, Bernoulli(1/200) x*, noise 1e-4,
    lambda=5e-3; 100 iterations against the FFT oracle."""
    torch, dev = torch_dev()
    inst = synth.large_instance()
    y32 = _y32(inst, dense=False)
    lam = f32(5e-3)
    chat = O.spectrum(inst.c)
    tau = f32(1.0 / np.max(np.abs(chat) ** 2))
    plan = _plan(cs, inst)
    try:
        x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        cs.cs_ista(plan, to_dev(y32), lam, tau, 100, x)
        xg = host(x)
    finally:
        plan.close()
    xo = O.ista_fft(inst.c, inst.rows, y32.astype(np.float64), lam, tau, 100)
    assert rel_l2(xg, xo) <= ITER_TOL, rel_l2(xg, xo)


def test_ista_all_rows_and_lambda_zero(cs):
    """m = n (A = C) and lambda = 0 (plain Landweber steps)."""
    torch, dev = torch_dev()
    n = 2048
    inst = synth.instance(n, n, k=20, seed=41)
    y32 = _y32(inst, dense=True)
    tau = f32(1.0 / O.opnorm2_dense(inst.c, inst.rows))
    plan = _plan(cs, inst)
    try:
        for lam in (0.0, f32(1e-2)):
            x = torch.zeros(n, dtype=torch.float32, device=dev)
            cs.cs_ista(plan, to_dev(y32), lam, tau, 100, x)
            xo = O.ista_dense(inst.c, inst.rows, y32.astype(np.float64), lam, tau, 100)
            assert rel_l2(host(x), xo) <= ITER_TOL, (lam, rel_l2(host(x), xo))
    finally:
        plan.close()


def test_ista_zero_iterations_and_warm_start(cs):
    torch, dev = torch_dev()
    inst = synth.instance(1024, 300, k=10, seed=43)
    y32 = _y32(inst, dense=True)
    x0 = synth.random_vector(1024, 44).astype(np.float32)
    lam, tau = f32(1e-2), f32(0.5 / O.opnorm2_dense(inst.c, inst.rows))
    plan = _plan(cs, inst)
    try:
        x = to_dev(x0)
        st = cs.cs_ista(plan, to_dev(y32), lam, tau, 0, x)
        assert st["iters_run"] == 0
        assert np.array_equal(host(x), x0.astype(np.float64))
        cs.cs_ista(plan, to_dev(y32), lam, tau, 37, x)
        xo = O.ista_dense(inst.c, inst.rows, y32.astype(np.float64), lam, tau, 37, x0=x0.astype(np.float64))
        assert rel_l2(host(x), xo) <= ITER_TOL
    finally:
        plan.close()


def test_ista_monitor_stops_early(cs):
    torch, dev = torch_dev()
    inst = synth.small_instance()
    y32 = _y32(inst, dense=True)
    lam = f32(1e-3)
    tau = f32(1.0 / O.opnorm2_dense(inst.c, inst.rows))
    plan = _plan(cs, inst)
    try:
        xt = to_dev(inst.x_true)      # the plan reads it: keep it alive
        cs.cs_set_monitor(plan, xt, 0.5, 5)   # this instance needs ~800 iterations
        x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        st = cs.cs_ista(plan, to_dev(y32), lam, tau, 5000, x)
    finally:
        plan.close()
    assert st["converged"] == 1
    assert st["iters_run"] % 5 == 0 and st["iters_run"] < 5000
    assert st["nmse"] <= 0.5
    # one check point earlier the oracle is still above the tolerance
    xo_prev = O.ista_dense(inst.c, inst.rows, y32.astype(np.float64), lam, tau, st["iters_run"] - 5)
    assert O.nmse(xo_prev, inst.x_true) > 0.5 * 0.999
    assert abs(O.nmse(host(x), inst.x_true) - st["nmse"]) <= 1e-4 * st["nmse"]


def test_ista_deterministic(cs):
    torch, dev = torch_dev()
    inst = synth.instance(1 << 16, 1 << 14, k=100, seed=47)
    y32 = _y32(inst, dense=False)
    plan = _plan(cs, inst)
    try:
        outs = []
        for _ in range(2):
            x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
            cs.cs_ista(plan, to_dev(y32), f32(1e-3), f32(0.01), 50, x)
            outs.append(host(x))
    finally:
        plan.close()
    assert np.array_equal(outs[0], outs[1])


# ------------------------------------------------------------------ ADMM

def _admm_gpu(cs, plan, n, y32, lam, sigma, rho, tau1, tau2, iters, state=None):
    torch, dev = torch_dev()
    if state is None:
        vs = [torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(4)]
        warm = False
    else:
        vs = [to_dev(s) for s in state]
        warm = True
    v, z, mu, nu = vs
    x = torch.zeros(n, dtype=torch.float32, device=dev)
    st = cs.cs_admm_ex(plan, to_dev(y32), lam, sigma, rho, tau1, tau2, iters, warm, x, z, mu, nu, v)
    return {"x": host(x), "z": host(z), "mu": host(mu), "nu": host(nu), "v": host(v)}, st


def test_admm_small_instance(cs):
    """Config-1 data, sigma = rho = 1, tau1 = tau2 = 1 through cs_admm (z) and
    cs_admm_ex (x, z); 100 and 500 iterations."""
    torch, dev = torch_dev()
    inst = synth.small_instance()
    y32 = _y32(inst, dense=True)
    lam = f32(1e-3)
    plan = _plan(cs, inst)
    try:
        z = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        cs.cs_admm(plan, to_dev(y32), lam, 1.0, 100, z)
        z100 = host(z)
        g100, _ = _admm_gpu(cs, plan, inst.n, y32, lam, 1.0, 1.0, 1.0, 1.0, 100)
        g500, _ = _admm_gpu(cs, plan, inst.n, y32, lam, 1.0, 1.0, 1.0, 1.0, 500)
    finally:
        plan.close()
    y64 = y32.astype(np.float64)
    o100 = O.admm_dense(inst.c, inst.rows, y64, lam, sigma=1.0, rho=1.0, iters=100)
    o500 = O.admm_dense(inst.c, inst.rows, y64, lam, sigma=1.0, rho=1.0, iters=500)
    assert rel_l2(z100, o100["z"]) <= ITER_TOL, rel_l2(z100, o100["z"])
    for key in ("x", "z"):
        assert rel_l2(g100[key], o100[key]) <= ITER_TOL, (key, rel_l2(g100[key], o100[key]))
        assert O.nmse(g500[key], o500[key]) <= FINAL_NMSE, (key, O.nmse(g500[key], o500[key]))


def test_admm_general_parameters_and_warm_start(cs):
    """sigma != rho, tau1 = tau2 = 1.2 (inside (0, 1.618)); 60 + 40 iterations
    through the state in/out equal 100 straight iterations bit for bit, and
    match the oracle."""
    inst = synth.instance(2048, 700, k=25, noise_std=1e-3, seed=51)
    y32 = _y32(inst, dense=True)
    lam, sigma, rho, t = f32(2e-3), 0.7, 1.3, 1.2
    plan = _plan(cs, inst)
    try:
        full, _ = _admm_gpu(cs, plan, inst.n, y32, lam, sigma, rho, t, t, 100)
        half, _ = _admm_gpu(cs, plan, inst.n, y32, lam, sigma, rho, t, t, 60)
        rest, _ = _admm_gpu(cs, plan, inst.n, y32, lam, sigma, rho, t, t, 40,
                            state=(half["v"], half["z"], half["mu"], half["nu"]))
    finally:
        plan.close()
    for key in ("z", "mu", "nu", "v"):
        assert np.array_equal(full[key], rest[key]), key
    o = O.admm_dense(inst.c, inst.rows, y32.astype(np.float64), lam, sigma=sigma, rho=rho, tau1=t, tau2=t,
                     iters=100)
    for key in ("x", "z", "v"):
        assert rel_l2(full[key], o[key]) <= ITER_TOL, (key, rel_l2(full[key], o[key]))
    # mu = running sum of v - C x and nu of x - z: differences of O(|v|) and
    # O(|x|) quantities, so their fp32 error floor is eps32 * |v| (|x|), not
    # eps32 * |mu| (|nu|); the bar is taken relative to those magnitudes.
    assert np.linalg.norm(full["mu"] - o["mu"]) <= ITER_TOL * np.linalg.norm(o["v"])
    assert np.linalg.norm(full["nu"] - o["nu"]) <= ITER_TOL * np.linalg.norm(o["x"])


@pytest.mark.parametrize("n,m,k", [(64, 20, 2), (1 << 14, 1 << 12, 40), (1 << 18, 1 << 16, 600)])
def test_admm_sizes(cs, n, m, k):
    inst = synth.instance(n, m, k=k, noise_std=1e-3, seed=5000 + n)
    dense = n <= 4096
    y32 = _y32(inst, dense)
    lam = f32(2e-3)
    plan = _plan(cs, inst)
    try:
        g, _ = _admm_gpu(cs, plan, n, y32, lam, 1.0, 1.0, 1.0, 1.0, 100)
    finally:
        plan.close()
    admm = O.admm_dense if dense else O.admm_fft
    o = admm(inst.c, inst.rows, y32.astype(np.float64), lam, sigma=1.0, rho=1.0, iters=100)
    for key in ("x", "z"):
        assert rel_l2(g[key], o[key]) <= ITER_TOL, (key, rel_l2(g[key], o[key]))


def test_admm_full_size(cs):
    """The timed workload at n=2^22: 100 iterations, rho=1, against the FFT
    oracle."""
    inst = synth.large_instance()
    y32 = _y32(inst, dense=False)
    lam = f32(5e-3)
    plan = _plan(cs, inst)
    try:
        g, _ = _admm_gpu(cs, plan, inst.n, y32, lam, 1.0, 1.0, 1.0, 1.0, 100)
    finally:
        plan.close()
    o = O.admm_fft(inst.c, inst.rows, y32.astype(np.float64), lam, sigma=1.0, rho=1.0, iters=100)
    for key in ("x", "z"):
        assert rel_l2(g[key], o[key]) <= ITER_TOL, (key, rel_l2(g[key], o[key]))


def test_ista_and_admm_reach_the_same_minimiser(cs):
    """Both solvers minimise the same LASSO (small, well-conditioned case)."""
    torch, dev = torch_dev()
    inst = synth.instance(256, 128, k=6, noise_std=1e-2, seed=61)
    y32 = _y32(inst, dense=True)
    lam = f32(1e-2)
    tau = f32(1.0 / O.opnorm2_dense(inst.c, inst.rows))
    plan = _plan(cs, inst)
    try:
        x = torch.zeros(256, dtype=torch.float32, device=dev)
        cs.cs_ista(plan, to_dev(y32), lam, tau, 20000, x)
        g, _ = _admm_gpu(cs, plan, 256, y32, lam, 1.0, 1.0, 1.0, 1.0, 3000)
    finally:
        plan.close()
    A = O.sensing_matrix(inst.c, inst.rows)
    assert O.kkt_violation(A, y32.astype(np.float64), host(x), lam) <= 1e-5
    assert rel_l2(g["z"], host(x)) <= 1e-4


def test_graphs_match_direct_launches(cs, monkeypatch):
    """The captured-graph chunks (default) and direct launches (CS_GRAPHS=0)
    run the same kernels in the same order: results are bit-identical, for
    iteration counts that are not multiples of the chunk length."""
    torch, dev = torch_dev()
    inst = synth.instance(1 << 14, 1 << 12, k=40, noise_std=1e-3, seed=71)
    y32 = _y32(inst, dense=False)
    outs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("CS_GRAPHS", mode)
        plan = _plan(cs, inst)
        try:
            x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
            cs.cs_ista(plan, to_dev(y32), f32(2e-3), f32(0.05), 37, x)
            z = torch.zeros(inst.n, dtype=torch.float32, device=dev)
            cs.cs_admm(plan, to_dev(y32), f32(2e-3), 1.0, 23, z)
            outs[mode] = (host(x), host(z))
        finally:
            plan.close()
    assert np.array_equal(outs["1"][0], outs["0"][0])
    assert np.array_equal(outs["1"][1], outs["0"][1])


def test_compressed_deblurring_1d(cs):
    """Sec. 7's setting in one dimension: A = P C B, C a random circulant,
    B the order-5 box blur, m = n/2; the plan takes the generating vector of
    the product C B.  A x matches C applied to B x (two oracle products), and
    ISTA matches the oracle on the composite operator."""
    torch, dev = torch_dev()
    n, m = 1 << 16, 1 << 15
    inst = synth.instance(n, m, k=n // 10, noise_std=1e-3, seed=73)
    cB = synth.composite_c(inst.c, synth.box_blur_c(n, 5))
    chB = O.spectrum(cB)
    ch, hb = O.spectrum(inst.c), O.spectrum(synth.box_blur_c(n, 5))
    x = inst.x_true
    want = O.circulant_apply_fft(ch, O.circulant_apply_fft(hb, x))[inst.rows]
    y32 = (want + inst.noise).astype(np.float32)
    lam = f32(1e-2)
    tau = f32(1.0 / np.max(np.abs(chB) ** 2))
    plan = cs.cs_plan(n, m, inst.rows, cB, torch.cuda.current_stream(dev))
    try:
        yg = torch.empty(m, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, to_dev(x), yg)
        xg = torch.zeros(n, dtype=torch.float32, device=dev)
        cs.cs_ista(plan, to_dev(y32), lam, tau, 100, xg)
        torch.cuda.synchronize()
        got_y, got_x = host(yg), host(xg)
    finally:
        plan.close()
    assert rel_l2(got_y, want) <= 2e-6, rel_l2(got_y, want)
    xo = O.ista_fft(cB, inst.rows, y32.astype(np.float64), lam, tau, 100)
    assert rel_l2(got_x, xo) <= ITER_TOL, rel_l2(got_x, xo)
