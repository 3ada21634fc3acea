"""Final-solution parity at the timed size (Algorithm 1 and Algorithm 3 at
n = 2^22, m = n/4, lambda = 5e-3, the Bernoulli(1/200)-Gaussian instance).

ISTA runs 970 iterations and ADMM (sigma = rho = 1, tau1 = tau2 = 1) 250
iterations from the zero state: the iteration counts at which the timed
workload reaches NMSE 1e-4 against x*.  Both sides get the same inputs (c in
FP64, y rounded once to fp32, the same fp32 lambda and tau); the oracle runs
its FFT step on every host core.

Bar: NMSE(gpu, oracle) <= 1e-6 for the ISTA solution x and for ADMM's x,
z, mu and nu.  The multipliers mu and nu are running sums of v - C x and
x - z, whose fp32 error grows with |v| and |x| rather than with their own
(smaller) size; their error relative to |v| and |x| is printed beside it.
"""
import os

import numpy as np
import pytest

import oracle.cs_oracle as O
import synth
from gpu_util import f32, host, to_dev, torch_dev

pytestmark = pytest.mark.gpu

FINAL_NMSE = 1e-6
ISTA_ITERS = 970
ADMM_ITERS = 250


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


@pytest.fixture(scope="module")
def setup():
    import paper_1707_02244_gb300 as cs
    torch, dev = torch_dev()
    inst = synth.large_instance()
    chat = O.spectrum(inst.c)
    y32 = (O.forward_fft(chat, inst.rows, inst.x_true) + inst.noise).astype(np.float32)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    tau = f32(1.0 / cs.cs_opnorm2(plan, 100))   # an input to both sides
    old = O.set_fft_threads(_cores())
    yield cs, inst, y32, plan, tau
    O.set_fft_threads(old)
    plan.close()


def test_ista_final_solution_full_size(setup):
    cs, inst, y32, plan, tau = setup
    torch, dev = torch_dev()
    lam = f32(5e-3)
    x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
    cs.cs_ista(plan, to_dev(y32), lam, tau, ISTA_ITERS, x)
    xg = host(x)
    xo = O.ista_fft(inst.c, inst.rows, y32.astype(np.float64), lam, tau, ISTA_ITERS)
    e = O.nmse(xg, xo)
    print(f"ISTA {ISTA_ITERS} iterations: NMSE(gpu, oracle) {e:.3e}, NMSE(oracle, x*) "
          f"{O.nmse(xo, inst.x_true):.3e}")
    assert e <= FINAL_NMSE, e


def test_admm_final_solution_full_size(setup):
    cs, inst, y32, plan, tau = setup
    torch, dev = torch_dev()
    lam = f32(5e-3)
    n = inst.n
    x, z, mu, nu, v = (torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(5))
    cs.cs_admm_ex(plan, to_dev(y32), lam, 1.0, 1.0, 1.0, 1.0, ADMM_ITERS, False, x, z, mu, nu, v)
    g = {"x": host(x), "z": host(z), "mu": host(mu), "nu": host(nu)}
    o = O.admm_fft(inst.c, inst.rows, y32.astype(np.float64), lam, sigma=1.0, rho=1.0, iters=ADMM_ITERS)
    errs = {k: O.nmse(g[k], o[k]) for k in g}
    scaled = {"mu": np.sum((g["mu"] - o["mu"]) ** 2) / np.sum(o["v"] ** 2),
              "nu": np.sum((g["nu"] - o["nu"]) ** 2) / np.sum(o["x"] ** 2)}
    print(f"ADMM {ADMM_ITERS} iterations: NMSE(gpu, oracle) " +
          ", ".join(f"{k} {v:.3e}" for k, v in errs.items()) +
          f"; mu err^2/|v|^2 {scaled['mu']:.3e}, nu err^2/|x|^2 {scaled['nu']:.3e}; "
          f"NMSE(oracle z, x*) {O.nmse(o['z'], inst.x_true):.3e}")
    for k in ("x", "z", "mu", "nu"):
        assert errs[k] <= FINAL_NMSE, (k, errs)
