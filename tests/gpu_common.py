"""Shared fixtures of the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

import oracle as O
from paper_2605_25149_gb300 import hq, inputs


def torch_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def dev(a, dtype=None):
    torch = torch_mod()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch_mod().cuda.synchronize()
    return t.detach().double().cpu().numpy()


def make(m, N, potential="wells", seed=2, useed=102, precision="fp64", **kw):
    V = inputs.wells(m, seed) if potential == "wells" else inputs.harmonic(m)
    U0 = inputs.initial_block(m, N, useed)
    s = hq.Solver(m, N, precision=precision, **kw)
    s.set_potential(V)
    s.set_initial(U0)
    return s, V, U0


def oracle_mg(s, V):
    c = s.cfg
    return O.MG(s.m, V, s.info()["sigma"], lo=c.lo, hi=c.hi, nu1=c.mg_nu1, nu2=c.mg_nu2,
                omega=c.mg_omega, coarsest=c.mg_coarsest)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
