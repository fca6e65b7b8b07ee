"""Helpers shared by the GPU parity tests (host <-> device marshalling, tolerances)."""
import numpy as np


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    """max |a - b| / max |b| (the max-norm relative error used for every FP64 parity check)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# FP64 parity bar: the GPU path must match the oracle to 1e-10 relative.
TOL = 1e-10
