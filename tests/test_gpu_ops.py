"""GPU parity of the sensing products A x and A^T r against the FP64 oracle.

Tolerance.  The fp32 FFT path has a relative rms error of about
c * eps32 * log2(N) per transform (c < 1), i.e. below 1e-6 for N <= 2^22;
a product is two transforms and a spectrum multiply.  The tests bound the
relative l2 error by 2e-6 and every element by 2e-5 * rms(oracle) (a
Gaussian-like error stays within ~6 sigma over 4M samples).
"""
import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu

REL = 2e-6
ELEM = 2e-5


@pytest.fixture(scope="module")
def cs():
    import paper_1707_02244_gb300 as cs
    return cs


def _products(cs, n, m, seed, dense):
    torch, dev = torch_dev()
    g = synth.rng(seed)
    c = synth.gaussian_c(g, n, m)
    rows = synth.draw_rows(g, n, m)
    x = g.standard_normal(n).astype(np.float32)
    r = g.standard_normal(m).astype(np.float32)
    plan = cs.cs_plan(n, m, rows, c, torch.cuda.current_stream(dev))
    try:
        y_d = torch.empty(m, dtype=torch.float32, device=dev)
        xa_d = torch.empty(n, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, to_dev(x), y_d)
        cs.cs_adjoint(plan, to_dev(r), xa_d)
        torch.cuda.synchronize()
        yg, xg = host(y_d), host(xa_d)
    finally:
        plan.close()
    x64, r64 = x.astype(np.float64), r.astype(np.float64)
    if dense:
        yo, xo = O.forward_dense(c, rows, x64), O.adjoint_dense(c, rows, r64)
    else:
        chat = O.spectrum(c)
        yo, xo = O.forward_fft(chat, rows, x64), O.adjoint_fft(chat, rows, r64)
    return yg, yo, xg, xo


def _check(got, want):
    assert rel_l2(got, want) <= REL, rel_l2(got, want)
    rms = np.sqrt(np.mean(want ** 2))
    assert np.max(np.abs(got - want)) <= ELEM * rms


@pytest.mark.parametrize("n,m", [(64, 1), (64, 64), (128, 37), (256, 100), (1024, 1024),
                                 (4096, 1024), (8192, 2731)])
def test_products_vs_dense(cs, n, m):
    yg, yo, xg, xo = _products(cs, n, m, seed=1000 + n + m, dense=True)
    _check(yg, yo)
    _check(xg, xo)


@pytest.mark.parametrize("n,m", [(1 << 14, 5000), (1 << 16, 1 << 14), (1 << 18, 1 << 16), (1 << 20, 1 << 18)])
def test_products_vs_fft_oracle(cs, n, m):
    yg, yo, xg, xo = _products(cs, n, m, seed=2000 + m, dense=False)
    _check(yg, yo)
    _check(xg, xo)


def test_products_full_size_sampled(cs):
    """n = 2^22, m = n/4 (the timed workload): 256 outputs of A x and A^T r,
    each computed by the oracle as its own dot product."""
    torch, dev = torch_dev()
    inst = synth.large_instance()
    n, m = inst.n, inst.m
    g = synth.rng(77)
    x = g.standard_normal(n).astype(np.float32)
    r = g.standard_normal(m).astype(np.float32)
    plan = cs.cs_plan(n, m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        y_d = torch.empty(m, dtype=torch.float32, device=dev)
        xa_d = torch.empty(n, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, to_dev(x), y_d)
        cs.cs_adjoint(plan, to_dev(r), xa_d)
        torch.cuda.synchronize()
        yg, xg = host(y_d), host(xa_d)
    finally:
        plan.close()
    idx = g.choice(m, 256, replace=False)
    jdx = g.choice(n, 256, replace=False)
    yo = O.forward_sampled(inst.c, inst.rows, x, idx)
    xo = O.adjoint_sampled(inst.c, inst.rows, r, jdx)
    # the sampled entries against the typical size of an entry
    rms_y = np.sqrt(np.mean(yg ** 2))
    rms_x = np.sqrt(np.mean(xg ** 2))
    assert np.max(np.abs(yg[idx] - yo)) <= ELEM * rms_y
    assert np.max(np.abs(xg[jdx] - xo)) <= ELEM * rms_x
    # adjoint identity over the whole vectors: <A x, r> = <x, A^T r>
    lhs = float(yg @ r.astype(np.float64))
    rhs = float(x.astype(np.float64) @ xg)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(yg) * np.linalg.norm(r)


def test_adjoint_identity_gpu(cs):
    torch, dev = torch_dev()
    n, m = 1 << 16, 3 << 12
    g = synth.rng(5)
    c = synth.gaussian_c(g, n, m)
    rows = synth.draw_rows(g, n, m)
    x = g.standard_normal(n).astype(np.float32)
    r = g.standard_normal(m).astype(np.float32)
    plan = cs.cs_plan(n, m, rows, c, torch.cuda.current_stream(dev))
    try:
        y_d = torch.empty(m, dtype=torch.float32, device=dev)
        xa_d = torch.empty(n, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, to_dev(x), y_d)
        cs.cs_adjoint(plan, to_dev(r), xa_d)
        torch.cuda.synchronize()
        yg = host(y_d)
        lhs = float(yg @ r.astype(np.float64))
        rhs = float(x.astype(np.float64) @ host(xa_d))
    finally:
        plan.close()
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(yg) * np.linalg.norm(r)


def test_identity_circulant_products(cs):
    """c = delta: A x is x restricted to the rows, exactly representable."""
    torch, dev = torch_dev()
    n, m = 4096, 999
    c = np.zeros(n); c[0] = 1.0
    rows = synth.draw_rows(synth.rng(3), n, m)
    x = synth.random_vector(n, 4).astype(np.float32)
    plan = cs.cs_plan(n, m, rows, c, torch.cuda.current_stream(dev))
    try:
        y_d = torch.empty(m, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, to_dev(x), y_d)
        torch.cuda.synchronize()
        yg = host(y_d)
    finally:
        plan.close()
    assert np.max(np.abs(yg - x[rows])) <= 1e-5 * np.max(np.abs(x))


def test_opnorm2(cs):
    """Power iteration on the GPU against the dense SVD (config-1 shape).
    The estimate is a Rayleigh quotient: never above ||A||^2."""
    torch, dev = torch_dev()
    inst = synth.small_instance()
    L = O.opnorm2_dense(inst.c, inst.rows)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        Lg = cs.cs_opnorm2(plan, 1000)
    finally:
        plan.close()
    assert Lg <= L * (1 + 1e-5)
    assert Lg >= L * (1 - 2e-2), (Lg, L)


def test_plan_vectors_at_odd_float_offsets(cs):
    """The n-vectors of cs_forward / cs_adjoint / cs_ista must be 8-byte
    aligned: one that starts 4 bytes past an 8-byte boundary is an argument
    error reported before anything is launched.  The m-vectors (y, r) and
    ADMM's z may start there and give the same bits as aligned ones (the
    batch calls, whose concatenations put odd-length instances at such
    offsets, are covered by test_gpu_batch_smooth)."""
    torch, dev = torch_dev()
    n, m = 1 << 12, 1 << 10
    g = synth.rng(3100)
    c = synth.gaussian_c(g, n, m)
    rows = synth.draw_rows(g, n, m)
    x = to_dev(g.standard_normal(n).astype(np.float32))
    plan = cs.cs_plan(n, m, rows, c, torch.cuda.current_stream(dev))

    def odd(k):
        return torch.zeros(k + 1, dtype=torch.float32, device=dev)[1:]
    try:
        xo = odd(n)
        assert xo.data_ptr() % 8 == 4
        ya = torch.zeros(m, device=dev)
        for call in (lambda: cs.cs_forward(plan, xo, ya), lambda: cs.cs_adjoint(plan, ya, xo),
                     lambda: cs.cs_ista(plan, ya, 1e-3, 0.05, 5, xo)):
            with pytest.raises(cs.CsError) as e:
                call()
            assert e.value.code == cs.CS_ERR_ARG
        yo = odd(m)
        cs.cs_forward(plan, x, ya)
        cs.cs_forward(plan, x, yo)
        ga, go = torch.zeros(n, device=dev), torch.zeros(n, device=dev)
        cs.cs_adjoint(plan, ya, ga)
        cs.cs_adjoint(plan, yo, go)
        za, zo = torch.zeros(n, device=dev), odd(n)
        cs.cs_admm(plan, ya, 1e-3, 1.0, 10, za)
        cs.cs_admm(plan, yo, 1e-3, 1.0, 10, zo)
        assert cs.cs_status_sync(plan) == cs.CS_OK
        assert torch.equal(ya, yo) and torch.equal(ga, go) and torch.equal(za, zo)
    finally:
        plan.close()
