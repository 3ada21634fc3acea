"""The allocation-free circulant product, checked against the planned path and
against the FP64 oracle.

cs_circulant_apply_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or an allocation's implicit
synchronisation is too costly): it needs no plan and keeps its FFT work space
in a fixed array inside the library.  Here it is called through the C ABI
twice in a row (C x, then C^T x on another vector) and each result is checked
element by element against the oracle's FFT product (Sec. 4.2's circulant)
and against cs_forward / cs_adjoint of a plan that keeps every row (A = C),
with the element and l2 tolerances of the other product tests.  A second
test checks that further calls leave the device's free memory unchanged.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu

REL = 2e-6
ELEM = 2e-5


def _check(got, want):
    assert rel_l2(got, want) <= REL, rel_l2(got, want)
    rms = np.sqrt(np.mean(want ** 2))
    assert np.max(np.abs(got - want)) <= ELEM * rms


def _raw_fn():
    import paper_1707_02244_gb300 as cs
    lib = ctypes.CDLL(str(cs.LIB_PATH))
    fn = lib.cs_circulant_apply_static
    fn.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return cs, fn


@pytest.mark.parametrize("n", [64, 4096, 16384])
def test_static_product_matches_oracle_and_planned_product(n):
    cs, fn = _raw_fn()
    torch, dev = torch_dev()
    g = synth.rng(900 + n)
    c = synth.gaussian_c(g, n, n // 4)
    x1 = g.standard_normal(n).astype(np.float32)
    x2 = g.standard_normal(n).astype(np.float32)
    stream = torch.cuda.current_stream(dev)
    c_d = torch.from_numpy(c).to(dev)                   # float64
    x1_d, x2_d = to_dev(x1), to_dev(x2)
    y1_d = torch.empty(n, dtype=torch.float32, device=dev)
    y2_d = torch.empty(n, dtype=torch.float32, device=dev)
    # two calls in a row through the C ABI: C x1, then C^T x2
    assert fn(n, c_d.data_ptr(), x1_d.data_ptr(), y1_d.data_ptr(), 0, stream.cuda_stream) == cs.CS_OK
    assert fn(n, c_d.data_ptr(), x2_d.data_ptr(), y2_d.data_ptr(), 1, stream.cuda_stream) == cs.CS_OK
    torch.cuda.synchronize()
    y1, y2 = host(y1_d), host(y2_d)

    # the oracle on the same fp32 inputs (promoted to FP64)
    chat = O.spectrum(c)
    _check(y1, O.circulant_apply_fft(chat, x1.astype(np.float64)))
    _check(y2, O.circulant_apply_fft(chat, x2.astype(np.float64), transpose=True))

    # the planned entry points on the same inputs
    plan = cs.cs_plan(n, n, np.arange(n), c, stream)
    try:
        r1 = torch.empty(n, dtype=torch.float32, device=dev)
        r2 = torch.empty(n, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, x1_d, r1)
        cs.cs_adjoint(plan, x2_d, r2)
        torch.cuda.synchronize()
        want1, want2 = host(r1), host(r2)
    finally:
        plan.close()
    _check(y1, want1)
    _check(y2, want2)


def test_static_product_allocates_no_device_memory():
    """After a first call (which may load the library's device code and its
    fixed work array), further calls leave the device's free memory as it
    was: nothing is taken from cudaMalloc or any other allocator."""
    cs, fn = _raw_fn()
    torch, dev = torch_dev()
    n = 16384
    g = synth.rng(977)
    c_d = torch.from_numpy(synth.gaussian_c(g, n, n // 4)).to(dev)
    x_d = to_dev(g.standard_normal(n))
    y_d = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    assert fn(n, c_d.data_ptr(), x_d.data_ptr(), y_d.data_ptr(), 0, stream.cuda_stream) == cs.CS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for k in range(4):
        assert fn(n, c_d.data_ptr(), x_d.data_ptr(), y_d.data_ptr(), k & 1, stream.cuda_stream) == cs.CS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)


def test_static_product_rejects_sizes_beyond_the_limit():
    import paper_1707_02244_gb300 as cs
    torch, dev = torch_dev()
    n = 2 * 16384
    c_d = torch.zeros(n, dtype=torch.float64, device=dev)
    x_d = torch.zeros(n, dtype=torch.float32, device=dev)
    with pytest.raises(cs.CsError) as e:
        cs.cs_circulant_apply_static(n, c_d, x_d, x_d)
    assert e.value.code == cs.CS_ERR_UNSUPPORTED
    with pytest.raises(cs.CsError) as e:
        cs.cs_circulant_apply_static(100, c_d, x_d, x_d)
    assert e.value.code == cs.CS_ERR_UNSUPPORTED
