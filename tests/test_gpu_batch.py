"""GPU parity of the batched solves (cs_batch_ista / cs_batch_admm) against
the FP64 oracle, instance by instance, on a batch of uneven sizes that
covers every single-CTA size class (n = 64 .. 8192), repeated sizes, and
instances above that limit (solved by per-instance plans inside the batch).

Bars as for the plain solver: relative l2 <= 1e-5 after 100 iterations.
"""
import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import f32, host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5
SIZES = [8192, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 4096, 16384, 64, 1 << 16, 2048]


@pytest.fixture(scope="module")
def cs():
    import paper_1707_02244_gb300 as cs
    return cs


@pytest.fixture(scope="module")
def batch_data():
    g = synth.rng(7100)
    n = np.array(SIZES, dtype=np.int64)
    m = np.maximum(1, np.rint(g.uniform(0.2, 0.5, size=len(n)) * n)).astype(np.int64)
    insts = synth.batch_instances(n, m, seed=7200)
    ys = [(O.forward_fft(O.spectrum(i.c), i.rows, i.x_true) + i.noise).astype(np.float32) for i in insts]
    lam = np.array([f32(2e-3 * (1 + 0.1 * (j % 3))) for j in range(len(n))])
    tau = np.array([f32(1.0 / np.max(np.abs(O.spectrum(i.c)) ** 2)) for i in insts])
    rho = np.array([f32(0.8 + 0.1 * (j % 4)) for j in range(len(n))])
    return n, m, insts, ys, lam, tau, rho


def _batch(cs, n, m, insts):
    torch, dev = torch_dev()
    rows = np.concatenate([i.rows for i in insts])
    c = np.concatenate([i.c for i in insts])
    return cs.cs_batch_plan(n, m, rows, c, torch.cuda.current_stream(dev))


def _split(v, offs, sizes):
    return [v[o:o + s] for o, s in zip(offs, sizes)]


def test_batch_ista_matches_oracle_per_instance(cs, batch_data):
    """100 iterations from x(0) = 0, run as 60 + 40 through the x(0) input."""
    torch, dev = torch_dev()
    n, m, insts, ys, lam, tau, _ = batch_data
    b = _batch(cs, n, m, insts)
    try:
        x = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
        y = to_dev(np.concatenate(ys))
        cs.cs_batch_ista(b, y, lam, tau, 60, x)
        cs.cs_batch_ista(b, y, lam, tau, 40, x)
        assert cs.cs_batch_status_sync(b) == cs.CS_OK
        xs = _split(host(x), b.noff, n)
    finally:
        b.close()
    for j, inst in enumerate(insts):
        xo = O.ista_fft(inst.c, inst.rows, ys[j].astype(np.float64), lam[j], tau[j], 100)
        assert rel_l2(xs[j], xo) <= ITER_TOL, (j, int(n[j]), rel_l2(xs[j], xo))


def test_batch_admm_matches_oracle_per_instance(cs, batch_data):
    torch, dev = torch_dev()
    n, m, insts, ys, lam, _, rho = batch_data
    b = _batch(cs, n, m, insts)
    try:
        z = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
        y = to_dev(np.concatenate(ys))
        cs.cs_batch_admm(b, y, lam, rho, 100, z)
        # a second call with other rho re-tabulates B's spectrum
        z2 = torch.zeros_like(z)
        cs.cs_batch_admm(b, y, lam, rho * 0 + f32(1.0), 100, z2)
        assert cs.cs_batch_status_sync(b) == cs.CS_OK
        zs = _split(host(z), b.noff, n)
        zs2 = _split(host(z2), b.noff, n)
    finally:
        b.close()
    for j, inst in enumerate(insts):
        y64 = ys[j].astype(np.float64)
        o = O.admm_fft(inst.c, inst.rows, y64, lam[j], sigma=rho[j], rho=rho[j], iters=100)
        assert rel_l2(zs[j], o["z"]) <= ITER_TOL, (j, int(n[j]), rel_l2(zs[j], o["z"]))
        o1 = O.admm_fft(inst.c, inst.rows, y64, lam[j], sigma=1.0, rho=1.0, iters=100)
        assert rel_l2(zs2[j], o1["z"]) <= ITER_TOL, (j, int(n[j]), rel_l2(zs2[j], o1["z"]))


def test_batch_equals_plain_solver_on_small_instance(cs):
    """One instance of the paper's small configuration solved by the batch
    (one CTA) and by a plan (multipass path): both within the oracle's bar,
    and within 2e-5 of each other."""
    torch, dev = torch_dev()
    inst = synth.small_instance()
    y32 = (O.forward_dense(inst.c, inst.rows, inst.x_true)).astype(np.float32)
    lam, tau = f32(1e-3), f32(1.0 / O.opnorm2_dense(inst.c, inst.rows))
    b = cs.cs_batch_plan([inst.n], [inst.m], inst.rows, inst.c, torch.cuda.current_stream(dev))
    p = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        xb = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        xp = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        cs.cs_batch_ista(b, to_dev(y32), lam, tau, 100, xb)
        cs.cs_ista(p, to_dev(y32), lam, tau, 100, xp)
        torch.cuda.synchronize()
        xb, xp = host(xb), host(xp)
    finally:
        b.close()
        p.close()
    xo = O.ista_dense(inst.c, inst.rows, y32.astype(np.float64), lam, tau, 100)
    assert rel_l2(xb, xo) <= ITER_TOL, rel_l2(xb, xo)
    assert rel_l2(xb, xp) <= 2 * ITER_TOL, rel_l2(xb, xp)


def test_batch_zero_iterations(cs):
    torch, dev = torch_dev()
    n = np.array([256, 1 << 14], dtype=np.int64)
    m = np.array([100, 5000], dtype=np.int64)
    insts = synth.batch_instances(n, m, seed=7300)
    b = _batch(cs, n, m, insts)
    try:
        x0 = synth.random_vector(int(n.sum()), 7301).astype(np.float32)
        x = to_dev(x0)
        y = torch.zeros(int(m.sum()), dtype=torch.float32, device=dev)
        cs.cs_batch_ista(b, y, 1e-3, 0.1, 0, x)
        z = to_dev(x0)
        cs.cs_batch_admm(b, y, 1e-3, 1.0, 0, z)
        torch.cuda.synchronize()
        assert np.array_equal(host(x), x0.astype(np.float64))
        assert not np.any(host(z))
    finally:
        b.close()


def test_batch_rejects_nonfinite_measurements(cs):
    torch, dev = torch_dev()
    n = np.array([128, 512], dtype=np.int64)
    m = np.array([40, 200], dtype=np.int64)
    insts = synth.batch_instances(n, m, seed=7400)
    b = _batch(cs, n, m, insts)
    try:
        y = np.zeros(int(m.sum()), dtype=np.float32)
        y[57] = np.nan
        x = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
        cs.cs_batch_ista(b, to_dev(y), 1e-3, 0.1, 5, x)
        assert cs.cs_batch_status_sync(b) == cs.CS_ERR_NONFINITE
        # reported once; a finite call afterwards is clean
        y[57] = 0.0
        cs.cs_batch_ista(b, to_dev(y), 1e-3, 0.1, 5, x)
        assert cs.cs_batch_status_sync(b) == cs.CS_OK
    finally:
        b.close()
