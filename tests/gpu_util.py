"""Helpers shared by the GPU tests (inputs come from synth, expectations
from the FP64 oracle; nothing here computes the method)."""
from __future__ import annotations

import numpy as np


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def to_dev(a, dtype=np.float32):
    torch, dev = torch_dev()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(dev)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def f32(v):
    """Round a scalar to fp32 and return it as a Python float (both sides of
    a parity test see exactly this value)."""
    return float(np.float32(v))
