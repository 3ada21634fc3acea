"""The direct circulant product (one O(n) dot product per kept row, the
context comparator) against the FP64 oracle, at power-of-two and other n."""
import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import host, rel_l2, to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m", [(64, 64), (1000, 300), (4096, 1024), (1 << 16, 1 << 14)])
def test_direct_forward_matches_oracle(n, m):
    import paper_1707_02244_gb300 as cs
    torch, dev = torch_dev()
    inst = synth.instance(n, m, k=3, seed=9000 + n)
    c32 = inst.c.astype(np.float32)
    x = synth.random_vector(n, 9001 + n).astype(np.float32)
    y = torch.empty(m, dtype=torch.float32, device=dev)
    rows = torch.from_numpy(inst.rows.astype(np.int32)).to(dev)
    cs.cs_forward_direct(n, m, to_dev(c32), rows, to_dev(x), y, torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    c64, x64 = c32.astype(np.float64), x.astype(np.float64)
    want = O.forward_dense(c64, inst.rows, x64) if n <= 4096 else O.forward_fft(O.spectrum(c64), inst.rows, x64)
    got = host(y)
    assert rel_l2(got, want) <= 2e-6, rel_l2(got, want)
    assert np.max(np.abs(got - want)) <= 2e-5 * np.sqrt(np.mean(want ** 2)) * np.sqrt(n / 1024 + 1)


def test_direct_forward_invalid_row_is_nan_not_a_read():
    import paper_1707_02244_gb300 as cs
    torch, dev = torch_dev()
    n, m = 256, 4
    c = to_dev(synth.random_vector(n, 9050).astype(np.float32))
    x = to_dev(synth.random_vector(n, 9051).astype(np.float32))
    rows = torch.tensor([3, -1, n, 7], dtype=torch.int32, device=dev)
    y = torch.zeros(m, dtype=torch.float32, device=dev)
    cs.cs_forward_direct(n, m, c, rows, x, y, torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    got = host(y)
    assert np.isfinite(got[0]) and np.isfinite(got[3])
    assert np.isnan(got[1]) and np.isnan(got[2])
