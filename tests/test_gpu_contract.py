"""C-ABI behaviour that needs a device: rejected row sets, argument checks,
non-finite input reported through the status word (no GPU fault involved)."""
import numpy as np
import pytest

import synth
from gpu_util import f32, host, to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    import paper_1707_02244_gb300 as cs
    return cs


def test_duplicate_and_out_of_range_rows(cs):
    torch, dev = torch_dev()
    n = 256
    c = synth.random_vector(n, 1)
    with pytest.raises(cs.CsError) as e:
        cs.cs_plan(n, 4, np.array([3, 9, 3, 1]), c, torch.cuda.current_stream(dev))
    assert e.value.code == cs.CS_ERR_ARG
    for bad in ([0, 256], [-1, 5]):
        with pytest.raises(cs.CsError) as e:
            cs.cs_plan(n, 2, np.array(bad), c, torch.cuda.current_stream(dev))
        assert e.value.code == cs.CS_ERR_ARG


def test_bad_solver_arguments(cs):
    torch, dev = torch_dev()
    inst = synth.instance(512, 100, k=5, seed=2)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        y = torch.zeros(inst.m, dtype=torch.float32, device=dev)
        x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        for lam, tau, it in ((-1.0, 0.1, 1), (0.1, 0.0, 1), (0.1, -1.0, 1), (0.1, 0.1, -1),
                             (float("nan"), 0.1, 1), (0.1, float("inf"), 1)):
            with pytest.raises(cs.CsError) as e:
                cs.cs_ista(plan, y, lam, tau, it, x)
            assert e.value.code == cs.CS_ERR_ARG
        with pytest.raises(cs.CsError) as e:
            cs.cs_admm(plan, y, 0.1, 0.0, 1, x)
        assert e.value.code == cs.CS_ERR_ARG
        vs = [torch.zeros(inst.n, dtype=torch.float32, device=dev) for _ in range(4)]
        with pytest.raises(cs.CsError) as e:
            cs.cs_admm_ex(plan, y, 0.1, 1.0, 1.0, 0.0, 1.0, 1, False, None, *vs)
        assert e.value.code == cs.CS_ERR_ARG
        with pytest.raises(cs.CsError) as e:
            cs.cs_set_monitor(plan, None, 0.0, 0)
        assert e.value.code == cs.CS_ERR_ARG
        with pytest.raises(cs.CsError) as e:   # all-zero ground truth
            cs.cs_set_monitor(plan, torch.zeros(inst.n, dtype=torch.float32, device=dev), 0.0, 10)
        assert e.value.code == cs.CS_ERR_ARG
    finally:
        plan.close()


def test_nonfinite_measurement_is_reported(cs):
    torch, dev = torch_dev()
    inst = synth.instance(1024, 200, k=5, seed=3)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    try:
        y = np.zeros(inst.m, dtype=np.float32)
        y[17] = np.nan
        x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
        with pytest.raises(cs.CsError) as e:
            cs.cs_ista(plan, to_dev(y), f32(1e-3), f32(0.1), 3, x)
        assert e.value.code == cs.CS_ERR_NONFINITE
        # the latch is cleared by cs_status_sync; a clean solve then succeeds
        cs.cs_status_sync(plan)
        y[17] = 0.0
        st = cs.cs_ista(plan, to_dev(y), f32(1e-3), f32(0.1), 3, torch.zeros_like(x))
        assert st["iters_run"] == 3
    finally:
        plan.close()


def test_plan_on_side_stream(cs):
    """A plan bound to a non-default stream orders its work on that stream."""
    torch, dev = torch_dev()
    inst = synth.instance(4096, 1000, k=10, seed=4)
    s = torch.cuda.Stream(dev)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, s)
    try:
        with torch.cuda.stream(s):
            x = to_dev(synth.random_vector(inst.n, 5).astype(np.float32))
            y = torch.empty(inst.m, dtype=torch.float32, device=dev)
            cs.cs_forward(plan, x, y)
        s.synchronize()
        assert np.all(np.isfinite(host(y)))
    finally:
        plan.close()
