"""C-ABI contract checks that need no GPU: the library loads, exports every
entry point include/cs.h declares, and rejects bad arguments before touching
the device."""
import ctypes
import pathlib
import re

import numpy as np
import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "cs.h"


def _declared():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def cs():
    lib = ROOT / "paper_1707_02244_gb300" / "libcsgb.so"
    if not lib.exists():
        pytest.skip("libcsgb.so not built (run __graft_entry__.build())")
    import paper_1707_02244_gb300 as cs
    return cs


def test_header_declares_expected_calls():
    names = _declared()
    for n in ("cs_plan", "cs_plan_destroy", "cs_forward", "cs_adjoint", "cs_ista", "cs_admm",
              "cs_admm_ex", "cs_opnorm2", "cs_set_monitor", "cs_status_sync"):
        assert n in names, n


def test_every_declared_symbol_is_exported(cs):
    lib = ctypes.CDLL(str(cs.LIB_PATH))
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(cs.EXPORTS) <= set(_declared())


def test_version_and_strings(cs):
    assert cs.cs_version() >= 100
    assert cs.status_string(0) == "CS_OK"
    assert cs.status_string(1) == "CS_ERR_ARG"
    assert cs.status_string(6) == "CS_ERR_UNSUPPORTED"


def test_plan_rejects_bad_arguments_without_device(cs):
    h = ctypes.c_void_p()
    rows = np.arange(8, dtype=np.int64)
    c = np.zeros(64)
    # null out / rows / c
    assert cs.raw_call("cs_plan", None, 64, 8, rows.ctypes.data, c.ctypes.data, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_plan", ctypes.byref(h), 64, 8, None, c.ctypes.data, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_plan", ctypes.byref(h), 64, 8, rows.ctypes.data, None, None) == cs.CS_ERR_ARG
    # m out of range
    assert cs.raw_call("cs_plan", ctypes.byref(h), 64, 0, rows.ctypes.data, c.ctypes.data, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_plan", ctypes.byref(h), 64, 65, rows.ctypes.data, c.ctypes.data, None) == cs.CS_ERR_ARG
    # unsupported n: not a power of two, too small, too large
    for n in (100, 32, 1 << 23):
        cn = np.zeros(min(n, 128))
        assert cs.raw_call("cs_plan", ctypes.byref(h), n, 8, rows.ctypes.data, cn.ctypes.data,
                           None) == cs.CS_ERR_UNSUPPORTED, n


def test_null_plan_is_an_argument_error(cs):
    st = cs.CsStats()
    assert cs.raw_call("cs_plan_destroy", None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_forward", None, None, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_adjoint", None, None, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_ista", None, None, ctypes.c_float(0.1), ctypes.c_float(1.0), 1, None,
                       ctypes.byref(st)) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_admm", None, None, ctypes.c_float(0.1), ctypes.c_float(1.0), 1, None,
                       None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_status_sync", None) == cs.CS_ERR_ARG
    L = ctypes.c_double()
    assert cs.raw_call("cs_opnorm2", None, 10, ctypes.byref(L)) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_set_monitor", None, None, ctypes.c_double(0.0), 10) == cs.CS_ERR_ARG
    prm = cs.CsAdmmParams(1.0, 1.0, 1.0, 1.0)
    buf = ctypes.c_void_p(8)
    assert cs.raw_call("cs_grad_admm", None, buf, ctypes.c_float(0.1), ctypes.byref(prm), 10, 5, buf, None, buf,
                       buf, buf) == cs.CS_ERR_ARG


def test_batch_plan_rejects_bad_arguments_without_device(cs):
    h = ctypes.c_void_p()
    n = np.array([64, 128], dtype=np.int64)
    m = np.array([8, 16], dtype=np.int64)
    rows = np.zeros(24, dtype=np.int64)
    c = np.zeros(192)
    args = [n.ctypes.data, m.ctypes.data, rows.ctypes.data, c.ctypes.data, None]
    assert cs.raw_call("cs_batch_plan", None, 2, *args) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_batch_plan", ctypes.byref(h), 0, *args) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_batch_plan", ctypes.byref(h), 2, n.ctypes.data, m.ctypes.data, None,
                       c.ctypes.data, None) == cs.CS_ERR_ARG
    bad_m = np.array([8, 129], dtype=np.int64)
    assert cs.raw_call("cs_batch_plan", ctypes.byref(h), 2, n.ctypes.data, bad_m.ctypes.data,
                       rows.ctypes.data, c.ctypes.data, None) == cs.CS_ERR_ARG
    for bad in (88, 32, 12, 1 << 22, 1 << 23, 1200000):
        bn = np.array([64, bad], dtype=np.int64)
        assert cs.raw_call("cs_batch_plan", ctypes.byref(h), 2, bn.ctypes.data, m.ctypes.data,
                           rows.ctypes.data, c.ctypes.data, None) == cs.CS_ERR_UNSUPPORTED, bad


def test_null_batch_is_an_argument_error(cs):
    lam = np.ones(2, dtype=np.float32)
    assert cs.raw_call("cs_batch_destroy", None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_batch_ista", None, None, lam.ctypes.data, lam.ctypes.data, 1, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_batch_admm", None, None, lam.ctypes.data, lam.ctypes.data, 1, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_batch_status_sync", None) == cs.CS_ERR_ARG


def test_direct_product_rejects_bad_arguments_without_device(cs):
    buf = ctypes.c_void_p(8)
    assert cs.raw_call("cs_forward_direct", 0, 1, buf, buf, buf, buf, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_forward_direct", 16, 17, buf, buf, buf, buf, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_forward_direct", 16, 4, None, buf, buf, buf, None) == cs.CS_ERR_ARG


def test_plan_2d_rejects_bad_arguments_without_device(cs):
    h = ctypes.c_void_p()
    pix = np.arange(8, dtype=np.int64)
    c2 = np.zeros(8 * 16)
    assert cs.raw_call("cs_plan_2d", None, 8, 16, 8, pix.ctypes.data, c2.ctypes.data, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_plan_2d", ctypes.byref(h), 8, 16, 8, None, c2.ctypes.data, None) == cs.CS_ERR_ARG
    assert cs.raw_call("cs_plan_2d", ctypes.byref(h), 8, 16, 0, pix.ctypes.data, c2.ctypes.data,
                       None) == cs.CS_ERR_ARG
    for n0, n1 in ((8, 8), (4, 16), (8192, 16), (12, 16), (8, 24)):
        assert cs.raw_call("cs_plan_2d", ctypes.byref(h), n0, n1, 8, pix.ctypes.data, c2.ctypes.data,
                           None) == cs.CS_ERR_UNSUPPORTED, (n0, n1)


def _declared_arity():
    """Parameter count of every call declared in the header."""
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(cs_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        p = params.strip()
        out[name] = 0 if p in ("", "void") else len([x for x in p.split(",") if x.strip()])
    return out


def test_binding_signatures_match_header(cs):
    """Every entry point the binding sets argtypes for takes as many
    arguments as the header declares (a mismatch would corrupt the call)."""
    arity = _declared_arity()
    lib = cs._lib
    for name in cs.EXPORTS:
        fn = getattr(lib, name)
        if fn.argtypes is None:
            continue
        assert name in arity, name
        assert len(fn.argtypes) == arity[name], (name, len(fn.argtypes), arity[name])


def test_static_product_binding_rejects_bad_tensors_before_any_launch(cs):
    """cs_circulant_apply_static's binding checks dtype, residency and length
    of c, x and y before the library is called (no device is touched)."""
    import torch
    n = 64
    c64 = torch.zeros(n, dtype=torch.float64)        # host tensor
    c32 = torch.zeros(n, dtype=torch.float32)
    x = torch.zeros(n, dtype=torch.float32)
    with pytest.raises(TypeError):                   # float32 c: 4n bytes where 8n are read
        cs.cs_circulant_apply_static(n, c32, x, x)
    with pytest.raises(ValueError):                  # host c
        cs.cs_circulant_apply_static(n, c64, x, x)


def test_ptr_checks_length(cs):
    import torch
    with pytest.raises(ValueError):
        cs._ptr(torch.zeros(4, dtype=torch.float32), numel=8)
    with pytest.raises(TypeError):
        cs._ptr(torch.zeros(4, dtype=torch.float64))


class _FakeDeviceTensor:
    """Looks like a contiguous float32 CUDA tensor of `k` elements; the
    binding checks it without touching a device (its address is never used,
    because every call below fails the length check first)."""

    def __init__(self, k, dtype="torch.float32"):
        self.k, self.dtype = k, dtype

    def data_ptr(self):
        return 1 << 20

    def is_contiguous(self):
        return True

    is_cuda = True

    def numel(self):
        return self.k


def test_binding_rejects_short_vectors_before_any_call(cs):
    """Every binding call that takes device vectors checks their lengths
    against the plan (n-vectors, m-vectors, the batch's concatenations)
    before the library is called: a short tensor would otherwise make the
    kernels read or write past its end."""
    n, m = 64, 16
    plan = cs.Plan(None, n, m)          # no library handle: nothing may reach the library
    good_n, good_m = _FakeDeviceTensor(n), _FakeDeviceTensor(m)
    short_n, short_m = _FakeDeviceTensor(n - 1), _FakeDeviceTensor(m - 1)
    calls = [
        lambda: cs.cs_forward(plan, short_n, good_m),
        lambda: cs.cs_forward(plan, good_n, short_m),
        lambda: cs.cs_adjoint(plan, short_m, good_n),
        lambda: cs.cs_adjoint(plan, good_m, short_n),
        lambda: cs.cs_set_monitor(plan, short_n, 1e-4, 10),
        lambda: cs.cs_ista(plan, short_m, 1e-3, 0.1, 1, good_n),
        lambda: cs.cs_ista(plan, good_m, 1e-3, 0.1, 1, short_n),
        lambda: cs.cs_admm(plan, good_m, 1e-3, 1.0, 1, short_n),
        lambda: cs.cs_admm_ex(plan, good_m, 1e-3, 1.0, 1.0, 1.0, 1.0, 1, False, None, good_n, good_n,
                              short_n, good_n),
        lambda: cs.cs_grad(plan, good_m, 1e-3, 0.1, 4, 2, good_n, good_n, _FakeDeviceTensor(0), good_m),
        lambda: cs.cs_grad(plan, good_m, 1e-3, 0.1, 4, 2, good_n, short_n, _FakeDeviceTensor(1), good_m),
        lambda: cs.cs_forward_direct(n, m, short_n, _FakeDeviceTensor(m, "torch.int32"), good_n, good_m),
        lambda: cs.cs_forward_direct(n, m, good_n, _FakeDeviceTensor(m - 1, "torch.int32"), good_n, good_m),
    ]
    batch = cs.BatchPlan(None, [32, 32], [8, 8])
    calls += [
        lambda: cs.cs_batch_ista(batch, _FakeDeviceTensor(15), 1e-3, 0.1, 1, _FakeDeviceTensor(64)),
        lambda: cs.cs_batch_admm(batch, _FakeDeviceTensor(16), 1e-3, 1.0, 1, _FakeDeviceTensor(63)),
    ]
    for k, call in enumerate(calls):
        with pytest.raises(ValueError, match="expected at least"):
            call()
    # an int32 row list is required by the direct product
    with pytest.raises(TypeError):
        cs.cs_forward_direct(n, m, good_n, _FakeDeviceTensor(m), good_n, good_m)
