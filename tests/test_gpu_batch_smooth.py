"""GPU parity of the batched solves on 7-smooth sizes (the mixed-radix
solver: radices 8, 4, 2, 7, 5, 3; one persistent launch per solve) against
the FP64 oracle, instance by instance.

The batch mixes whole-CTA instances (n <= 4096, odd and even), four-step
instances (4096 < n <= 2^20, odd and even, several splits) and power-of-two
instances (the radix-16 solvers), so the three paths run side by side in one
call.  Bar as for the plain solver: relative l2 <= 1e-5 after 100 iterations.
"""
import os

import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import f32, host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5
SIZES = [4000, 18, 60, 105, 1000, 2187, 3969, 4116, 5000, 6615, 10080, 46656, 250047, 1000000, 64, 8192, 16384,
         105, 5000]


@pytest.fixture(scope="module")
def cs():
    import paper_1707_02244_gb300 as cs
    return cs


def _data(sizes, seed):
    g = synth.rng(seed)
    n = np.array(sizes, dtype=np.int64)
    m = np.maximum(1, np.rint(g.uniform(0.2, 0.5, size=len(n)) * n)).astype(np.int64)
    insts = synth.batch_instances(n, m, seed=seed + 100)
    ys = [(O.forward_fft(O.spectrum(i.c), i.rows, i.x_true) + i.noise).astype(np.float32) for i in insts]
    lam = np.array([f32(2e-3 * (1 + 0.1 * (j % 3))) for j in range(len(n))])
    tau = np.array([f32(1.0 / np.max(np.abs(O.spectrum(i.c)) ** 2)) for i in insts])
    rho = np.array([f32(0.8 + 0.1 * (j % 4)) for j in range(len(n))])
    return n, m, insts, ys, lam, tau, rho


@pytest.fixture(scope="module")
def batch_data():
    return _data(SIZES, 7300)


def _plan(cs, n, m, insts):
    torch, dev = torch_dev()
    return cs.cs_batch_plan(n, m, np.concatenate([i.rows for i in insts]), np.concatenate([i.c for i in insts]),
                            torch.cuda.current_stream(dev))


def _split(v, offs, sizes):
    return [v[o:o + s] for o, s in zip(offs, sizes)]


def _ista(cs, b, n, ys, lam, tau, parts):
    torch, dev = torch_dev()
    x = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
    y = to_dev(np.concatenate(ys))
    for T in parts:
        cs.cs_batch_ista(b, y, lam, tau, T, x)
    assert cs.cs_batch_status_sync(b) == cs.CS_OK
    return _split(host(x), b.noff, n)


def _admm(cs, b, n, ys, lam, rho, T):
    torch, dev = torch_dev()
    z = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
    cs.cs_batch_admm(b, to_dev(np.concatenate(ys)), lam, rho, T, z)
    assert cs.cs_batch_status_sync(b) == cs.CS_OK
    return _split(host(z), b.noff, n)


def test_smooth_batch_ista_matches_oracle(cs, batch_data):
    """100 iterations from x(0) = 0, run as 60 + 40 through the x(0) input."""
    n, m, insts, ys, lam, tau, _ = batch_data
    b = _plan(cs, n, m, insts)
    try:
        xs = _ista(cs, b, n, ys, lam, tau, (60, 40))
    finally:
        b.close()
    errs = []
    for j, inst in enumerate(insts):
        xo = O.ista_fft(inst.c, inst.rows, ys[j].astype(np.float64), lam[j], tau[j], 100)
        errs.append((int(n[j]), rel_l2(xs[j], xo)))
    print("ISTA rel l2:", errs)
    assert all(e <= ITER_TOL for _, e in errs), errs


def test_smooth_batch_admm_matches_oracle(cs, batch_data):
    """100 iterations from the zero state; a second call with other rho
    re-tabulates B's spectrum."""
    n, m, insts, ys, lam, _, rho = batch_data
    b = _plan(cs, n, m, insts)
    try:
        zs = _admm(cs, b, n, ys, lam, rho, 100)
        zs2 = _admm(cs, b, n, ys, lam, rho * 0 + f32(1.0), 100)
    finally:
        b.close()
    errs = []
    for j, inst in enumerate(insts):
        y64 = ys[j].astype(np.float64)
        o = O.admm_fft(inst.c, inst.rows, y64, lam[j], sigma=rho[j], rho=rho[j], iters=100)
        o1 = O.admm_fft(inst.c, inst.rows, y64, lam[j], sigma=1.0, rho=1.0, iters=100)
        errs.append((int(n[j]), rel_l2(zs[j], o["z"]), rel_l2(zs2[j], o1["z"])))
    print("ADMM rel l2:", errs)
    assert all(a <= ITER_TOL and c <= ITER_TOL for _, a, c in errs), errs


def test_smooth_batch_is_deterministic_and_split_independent(cs):
    """Bitwise equal across calls (the queue order varies, the arithmetic of
    a tile does not); the heuristic split (CS_BATCH_AUTOTUNE=0) agrees with
    the tuned one within the bar."""
    n, m, insts, ys, lam, tau, rho = _data([6615, 1000, 46656, 3000], 7400)
    b = _plan(cs, n, m, insts)
    old = os.environ.get("CS_BATCH_AUTOTUNE")
    os.environ["CS_BATCH_AUTOTUNE"] = "0"
    try:
        bh = _plan(cs, n, m, insts)
    finally:
        if old is None:
            del os.environ["CS_BATCH_AUTOTUNE"]
        else:
            os.environ["CS_BATCH_AUTOTUNE"] = old
    try:
        a = _ista(cs, b, n, ys, lam, tau, (50,))
        a2 = _ista(cs, b, n, ys, lam, tau, (50,))
        h = _ista(cs, bh, n, ys, lam, tau, (50,))
        za = _admm(cs, b, n, ys, lam, rho, 40)
        za2 = _admm(cs, b, n, ys, lam, rho, 40)
    finally:
        b.close()
        bh.close()
    for j in range(len(n)):
        assert np.array_equal(a[j], a2[j]) and np.array_equal(za[j], za2[j]), j
        assert rel_l2(h[j], a[j]) <= 2 * ITER_TOL, (j, rel_l2(h[j], a[j]))


def test_smooth_batch_zero_iterations_and_bad_rows(cs):
    torch, dev = torch_dev()
    n, m, insts, ys, lam, tau, rho = _data([105, 5000], 7500)
    b = _plan(cs, n, m, insts)
    try:
        x0 = synth.random_vector(int(n.sum()), 7501).astype(np.float32)
        x = to_dev(x0)
        cs.cs_batch_ista(b, to_dev(np.concatenate(ys)), lam, tau, 0, x)
        z = to_dev(x0)
        cs.cs_batch_admm(b, to_dev(np.concatenate(ys)), lam, rho, 0, z)
        assert cs.cs_batch_status_sync(b) == cs.CS_OK
        assert np.array_equal(host(x), x0)
        assert not np.any(host(z))
    finally:
        b.close()
    rows = [i.rows.copy() for i in insts]
    rows[1][1] = rows[1][0]   # duplicate row in the four-step instance
    with pytest.raises(cs.CsError) as e:
        cs.cs_batch_plan(n, m, np.concatenate(rows), np.concatenate([i.c for i in insts]),
                         torch.cuda.current_stream(dev))
    assert e.value.code == cs.CS_ERR_ARG
    rows = [i.rows.copy() for i in insts]
    rows[0][0] = 105          # out of range
    with pytest.raises(cs.CsError) as e:
        cs.cs_batch_plan(n, m, np.concatenate(rows), np.concatenate([i.c for i in insts]),
                         torch.cuda.current_stream(dev))
    assert e.value.code == cs.CS_ERR_ARG


def test_smooth_batch_nonfinite_measurement_is_reported(cs):
    n, m, insts, ys, lam, tau, _ = _data([1000, 5000], 7600)
    b = _plan(cs, n, m, insts)
    try:
        yb = [y.copy() for y in ys]
        yb[1][3] = np.nan
        _, dev = torch_dev()
        import torch
        x = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
        cs.cs_batch_ista(b, to_dev(np.concatenate(yb)), lam, tau, 5, x)
        assert cs.cs_batch_status_sync(b) == cs.CS_ERR_NONFINITE
        cs.cs_batch_ista(b, to_dev(np.concatenate(ys)), lam, tau, 5, x)
        assert cs.cs_batch_status_sync(b) == cs.CS_OK
    finally:
        b.close()


def test_smooth_batch_bounded_wait_times_out(cs):
    """Every device-side wait of the persistent launch is bounded.  The test
    arms, from the host, a count that instance 0's tiles wait for and that no
    tile ever reaches (CS_BATCH_STALL_TEST): the wait gives up after its
    limit, latches the timeout, every CTA stops taking work and the launch
    returns; the host reads CS_ERR_TIMEOUT.  The same batch then solves
    normally, matching the oracle."""
    import time
    n, m, insts, ys, lam, tau, _ = _data([5000, 1000], 7700)
    b = _plan(cs, n, m, insts)
    torch, dev = torch_dev()
    try:
        x = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
        y = to_dev(np.concatenate(ys))
        os.environ["CS_BATCH_STALL_TEST"] = str(1 << 40)
        try:
            t0 = time.perf_counter()
            cs.cs_batch_ista(b, y, lam, tau, 5, x)
            st = cs.cs_batch_status_sync(b)
            secs = time.perf_counter() - t0
        finally:
            del os.environ["CS_BATCH_STALL_TEST"]
        print(f"stalled solve returned {st} after {secs:.2f} s")
        assert st == cs.CS_ERR_TIMEOUT
        assert secs < 20.0
        got = _ista(cs, b, n, ys, lam, tau, [30])
        for i, inst in enumerate(insts):
            want = O.ista_fft(inst.c, inst.rows, ys[i].astype(np.float64), lam[i], tau[i], 30)
            assert rel_l2(got[i], want) <= ITER_TOL
    finally:
        b.close()


def test_tuner_cache_file_round_trip(tmp_path):
    """With CS_BATCH_TUNE_CACHE set, the plan-time tuner keeps its chosen
    splits in a JSON file keyed by the GPU's name.  A first process tunes two
    four-step sizes and writes them; a second process reads the file and
    tunes nothing (the file is not rewritten).  Each process starts with an
    empty in-memory cache, so the file is what the second one uses."""
    import json
    import pathlib
    import subprocess
    import sys
    root = str(pathlib.Path(__file__).resolve().parents[1])
    path = tmp_path / "tune.json"
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np, torch\n"
        "import paper_1707_02244_gb300 as cs, synth\n"
        "n = np.array([6615, 10080], dtype=np.int64); m = n // 4\n"
        "insts = synth.batch_instances(n, m)\n"
        "b = cs.cs_batch_plan(n, m, np.concatenate([i.rows for i in insts]),\n"
        "                     np.concatenate([i.c for i in insts]), torch.cuda.current_stream())\n"
        "b.close()\n"
        "print(torch.cuda.get_device_name(0))\n" % root)
    env = dict(os.environ, CS_BATCH_TUNE_CACHE=str(path))
    env.pop("CS_BATCH_AUTOTUNE", None)
    first = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, check=True,
                           capture_output=True, text=True)
    data = json.loads(path.read_text())
    assert data["device"] == first.stdout.strip().splitlines()[-1]
    assert set(data["splits"]) == {"6615", "10080"}
    for key, (n1, n2, g) in data["splits"].items():
        assert n1 * n2 == int(key) and 1 <= g <= 8
    stamp = path.stat().st_mtime_ns
    subprocess.run([sys.executable, "-c", code], env=env, cwd=root, check=True, capture_output=True)
    assert path.stat().st_mtime_ns == stamp
