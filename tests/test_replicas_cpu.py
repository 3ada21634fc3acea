"""The multi-process (replicas) path of bench.py, run as two gloo ranks on
the CPU: per-rank instances, the job time as the maximum over ranks, the
whole-job rate, and the reference arm doing no work on ranks other than 0.
"""
import importlib.util
import multiprocessing as mp
import os
import pathlib
import socket
import types

ROOT = pathlib.Path(__file__).resolve().parents[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        r, w, loc = b.dist_env()
        t = b.max_over_ranks(1.0 + r, w, torch.device("cpu"))
        rate = b.job_rate(w, 1200, t)
        rc = None
        if r != 0:
            args = types.SimpleNamespace(n=1 << 22, warmup=3, steps=3, gpus=w)
            rc = b.run_reference(args)   # rank != 0: returns at once, no work
        q.put((r, w, loc, t, rate, b.replica_seed(r), rc))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, t0, rate0, s0, rc0), (r1, w1, l1, t1, rate1, s1, rc1) = out
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert t0 == t1 == 2.0                 # the slower rank's time
    assert rate0 == rate1 == 2 * 1200 / 2.0
    assert s0 != s1                        # each rank its own instance
    assert rc1 == 0


def test_single_process_is_unchanged():
    b = _bench()
    assert b.max_over_ranks(1.5, 1, None) == 1.5
    assert b.job_rate(1, 400, 2.0) == 200.0
