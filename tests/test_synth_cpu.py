"""Host-side checks of the seeded input generators (no method arithmetic):
the 7-smooth size list and the batch size draw."""
import numpy as np

import synth


def _smooth(v):
    for p in (2, 3, 5, 7):
        while v % p == 0:
            v //= p
    return v == 1


def test_smooth_numbers_brute_force():
    got = synth.smooth_numbers(5000)
    want = [v for v in range(1, 5001) if _smooth(v)]
    assert got.tolist() == want


def test_batch_sizes_smooth_snap():
    n, m = synth.batch_sizes(512, 12, 20, synth.BATCH_SEED, snap="smooth")
    assert all(_smooth(int(v)) for v in n)
    assert n.min() >= 2 ** 12 - 1 and n.max() <= 2 ** 20
    assert np.all(m >= 0.2 * n - 1) and np.all(m <= 0.5 * n + 1)
    # nearest: no 7-smooth integer strictly closer to the drawn target
    g = synth.rng(synth.BATCH_SEED)
    target = np.exp2(g.uniform(12, 20, size=512))
    cand = synth.smooth_numbers(1 << 21)
    for t, v in zip(target[:64], n[:64]):
        assert np.min(np.abs(cand - t)) == abs(v - t)
    # most draws are not powers of two (they take the mixed-radix solver)
    assert np.sum((n & (n - 1)) == 0) < 32


def test_batch_sizes_pow2_snap_unchanged():
    n, _ = synth.batch_sizes(64, 12, 20, 5, snap="pow2")
    assert np.all((n & (n - 1)) == 0)
