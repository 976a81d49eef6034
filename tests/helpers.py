"""Shared helpers of the GPU tests: build a plan from a synthetic workload, pack profiles."""
import numpy as np

import paper_1606_05474_b300 as hp

_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        _CTX = hp.Context(0)
    return _CTX


def make_plan(wl, **params):
    import torch
    kap = [torch.from_numpy(t.kappa32).cuda().contiguous() for t in wl.tables]
    p = hp.default_params(**params)
    if wl.grey:
        p.grey_mode = 1
    if wl.n_scat != 4:
        p.n_scat = wl.n_scat
    return hp.Plan(ctx(), wl.atms, wl.tables, kap, p)


def pack(profiles):
    import torch
    return torch.from_numpy(np.concatenate([np.asarray(x, np.float64) for x in profiles])).cuda()


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))
