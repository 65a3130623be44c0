"""Helpers shared by the GPU tests (inputs from initial_conditions only)."""
import numpy as np

import initial_conditions as ic


def cuda():
    import torch
    return torch


def sorted_plummer(n, seed=1, masses="equal"):
    import oracle
    d = ic.plummer(n, seed=seed, masses=masses)
    perm = oracle.sort_perm(d["r"], d["id"])
    return {k: v[perm].copy() for k, v in d.items()}


def dev(a):
    import torch
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32).copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    a = t.cpu().numpy()
    if t.dtype == torch.int32:
        return a.view(np.uint32)
    return a
