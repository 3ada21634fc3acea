"""Small fixed workloads for ncu captures of the batched, 2D and gradient
kernels (direct launches with CS_GRAPHS=0):

    CS_GRAPHS=0 python -m paper_1707_02244_gb300.profile_extras batch
    CS_GRAPHS=0 python -m paper_1707_02244_gb300.profile_extras deblur2d
    CS_GRAPHS=0 python -m paper_1707_02244_gb300.profile_extras grad

batch: 128 instances (64 of n = 8192, 64 of n = 4096), 5 ISTA and 5 ADMM
iterations in the single-CTA kernels.  deblur2d: the 4096 x 4096 star field,
3 ISTA and 3 ADMM iterations.  grad: n = 2^20, m = n/4, 4 unrolled ISTA
steps, checkpoints every 2.
"""
import sys

import numpy as np
import torch

import paper_1707_02244_gb300 as cs


def main(mode: str) -> int:
    sys.path.insert(0, str(cs.LIB_PATH.parents[1]))
    import synth
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    if mode == "batch":
        n = np.array([8192] * 64 + [4096] * 64, dtype=np.int64)
        m = n // 4
        insts = synth.batch_instances(n, m)
        b = cs.cs_batch_plan(n, m, np.concatenate([i.rows for i in insts]), np.concatenate([i.c for i in insts]),
                             stream)
        y = torch.from_numpy(np.random.default_rng(0).standard_normal(int(m.sum())).astype(np.float32)).to(dev)
        x = torch.zeros(int(n.sum()), dtype=torch.float32, device=dev)
        z = torch.zeros_like(x)
        cs.cs_batch_ista(b, y, 1e-3, 0.05, 5, x)
        cs.cs_batch_admm(b, y, 1e-3, 1.0, 5, z)
        assert cs.cs_batch_status_sync(b) == cs.CS_OK
        b.close()
    elif mode == "deblur2d":
        img = synth.star_field()
        plan = cs.cs_plan_2d(img.n0, img.n1, img.m, img.pix, img.c2, stream)
        xt = torch.from_numpy(img.x_true.astype(np.float32)).to(dev)
        y = torch.empty(img.m, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, xt, y)
        x = torch.zeros(img.n, dtype=torch.float32, device=dev)
        z = torch.zeros_like(x)
        cs.cs_ista(plan, y, 2e-4, 1.0, 3, x)
        cs.cs_admm(plan, y, 2e-4, 1.0, 3, z)
        plan.close()
    elif mode == "grad":
        n = 1 << 20
        inst = synth.instance(n, n // 4, k=n // 100, noise_std=1e-3, seed=8300)
        plan = cs.cs_plan(n, inst.m, inst.rows, inst.c, stream)
        xt = torch.from_numpy(inst.x_true.astype(np.float32)).to(dev)
        y = torch.empty(inst.m, dtype=torch.float32, device=dev)
        cs.cs_forward(plan, xt, y)
        gx = torch.ones(n, dtype=torch.float32, device=dev)
        dc = torch.empty(n, dtype=torch.float32, device=dev)
        dl = torch.empty(1, dtype=torch.float32, device=dev)
        dy = torch.empty(inst.m, dtype=torch.float32, device=dev)
        cs.cs_grad(plan, y, 5e-3, 0.05, 4, 2, gx, dc, dl, dy)
        assert cs.cs_status_sync(plan) == cs.CS_OK
        plan.close()
    else:
        raise SystemExit(f"unknown mode {mode}")
    torch.cuda.synchronize()
    print("ok")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1] if len(sys.argv) > 1 else "batch"))
