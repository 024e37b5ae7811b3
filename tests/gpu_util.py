"""Helpers of the GPU parity tests."""
import numpy as np
import torch


def dev():
    return torch.device("cuda", 0)


def cu(rel):
    return tuple(torch.from_numpy(np.ascontiguousarray(np.asarray(c, dtype=np.int32))).to(dev())
                 for c in rel)


def sorted_rows(a):
    a = np.asarray(a)
    if a.size == 0:
        return a.reshape(0, a.shape[1] if a.ndim == 2 else 0)
    order = np.lexsort(a.T[::-1])
    return a[order]
