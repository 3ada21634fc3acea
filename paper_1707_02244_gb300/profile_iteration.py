"""Small fixed workload for ncu captures of the iteration kernels.

Builds a plan for the n = 2^22, m = n/4 instance, forms y = A x*, and runs
3 ISTA and 3 ADMM iterations.  With CS_GRAPHS=0 every kernel is a separate
launch, so ncu's -k / -s / -c select individual passes:

    CS_GRAPHS=0 python -m paper_1707_02244_gb300.profile_iteration
"""
import sys

import numpy as np
import torch

import paper_1707_02244_gb300 as cs


def main(n: int = 1 << 22) -> int:
    sys.path.insert(0, str(cs.LIB_PATH.parents[1]))
    import synth
    dev = torch.device("cuda:0")
    inst = synth.large_instance(n=n)
    plan = cs.cs_plan(inst.n, inst.m, inst.rows, inst.c, torch.cuda.current_stream(dev))
    xt = torch.from_numpy(inst.x_true.astype(np.float32)).to(dev)
    y = torch.empty(inst.m, dtype=torch.float32, device=dev)
    cs.cs_forward(plan, xt, y)
    x = torch.zeros(inst.n, dtype=torch.float32, device=dev)
    z = torch.zeros(inst.n, dtype=torch.float32, device=dev)
    cs.cs_ista(plan, y, 5e-3, 0.05, 3, x)
    cs.cs_admm(plan, y, 5e-3, 1.0, 3, z)
    torch.cuda.synchronize()
    plan.close()
    print("ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
