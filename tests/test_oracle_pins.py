"""The FP64 oracle against its pins (CPU only)."""
import pytest

import oracle.cs_oracle as O
from oracle_pins import ALL_CHECKS


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check(O)


def test_threaded_fft_step_matches_numpy():
    """The oracle's FFT library step on several threads (scipy's FFT, used to
    time the oracle on all host cores) gives the same ISTA and ADMM iterates
    as the default numpy step, to FP64 rounding."""
    pytest.importorskip("scipy")
    import numpy as np
    import synth
    inst = synth.instance(1 << 14, 1 << 12, k=80, noise_std=1e-3, seed=4242)
    chat = O.spectrum(inst.c)
    y = O.forward_fft(chat, inst.rows, inst.x_true) + inst.noise
    tau = 1.0 / float(np.max(np.abs(chat) ** 2))
    x1 = O.ista_fft(inst.c, inst.rows, y, 1e-3, tau, 30)
    z1 = O.admm_fft(inst.c, inst.rows, y, 1e-3, sigma=1.0, rho=1.0, iters=30)["z"]
    old = O.set_fft_threads(4)
    try:
        x4 = O.ista_fft(inst.c, inst.rows, y, 1e-3, tau, 30)
        z4 = O.admm_fft(inst.c, inst.rows, y, 1e-3, sigma=1.0, rho=1.0, iters=30)["z"]
    finally:
        O.set_fft_threads(old)
    assert np.linalg.norm(x4 - x1) <= 1e-12 * np.linalg.norm(x1)
    assert np.linalg.norm(z4 - z1) <= 1e-12 * np.linalg.norm(z1)
