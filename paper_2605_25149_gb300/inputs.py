"""Seeded synthetic inputs: potentials and initial blocks.

This module is shared by the CUDA path, the oracle and the tests.  It holds
none of the eigensolver's arithmetic: it only draws random numbers and
evaluates the potential functions on the grid, in FP64 on the host.

Workloads follow the paper's model problems: the harmonic oscillator
V = |x|^2/2 of Example 5.1 (here in 3D on a finite-difference grid), and the
same oscillator with eight attractive Gaussian wells (depth U[1,5], width
U[0.5,1.5], centres uniform in the box) drawn from ``numpy.random.default_rng``
in the fixed order depths, widths, centres.  Initial data are i.i.d. N(0,1)
(Section 5 starts from random, non-orthogonal U0).
"""
from __future__ import annotations

import numpy as np

LO, HI = -6.0, 6.0


def grid_h(m: int, lo: float = LO, hi: float = HI) -> float:
    return (hi - lo) / (m + 1)


def coords(m: int, lo: float = LO, hi: float = HI):
    """x, y, z of the m^3 interior nodes, flattened with x fastest."""
    h = grid_h(m, lo, hi)
    t = lo + h * np.arange(1, m + 1, dtype=np.float64)
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def harmonic(m: int, lo: float = LO, hi: float = HI) -> np.ndarray:
    x, y, z = coords(m, lo, hi)
    return 0.5 * (x * x + y * y + z * z)


def well_params(seed: int, n_wells: int = 8, lo: float = LO, hi: float = HI):
    rng = np.random.default_rng(seed)
    depth = rng.uniform(1.0, 5.0, n_wells)
    width = rng.uniform(0.5, 1.5, n_wells)
    centre = rng.uniform(lo, hi, (n_wells, 3))
    return depth, width, centre


def wells(m: int, seed: int, n_wells: int = 8, lo: float = LO, hi: float = HI) -> np.ndarray:
    """Harmonic oscillator plus seeded attractive Gaussian wells."""
    x, y, z = coords(m, lo, hi)
    V = 0.5 * (x * x + y * y + z * z)
    depth, width, centre = well_params(seed, n_wells, lo, hi)
    for d, w, c in zip(depth, width, centre):
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        V = V - d * np.exp(-r2 / (2.0 * w * w))
    return V


def initial_block(m: int, N: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) n x N block, point-major (row p = grid node)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m ** 3, N))


# Workloads of the benchmark suite: (name, m, N, potential, U0 seed, tau, precision;
# mg_fp32 = 1: FP64 block PCG with the multigrid preconditioner in FP32)
WORKLOADS = {
    "harmonic16_N8": dict(m=16, N=8, potential=("harmonic", None), u0_seed=1, tau=0.5,
                          precision="fp64", cg_rtol=1e-10, eps=1e-8, mg_fp32=1),
    "wells64_N64": dict(m=64, N=64, potential=("wells", 2), u0_seed=102, tau=0.4,
                        precision="fp64", cg_rtol=1e-10, eps=1e-8, mg_fp32=1, mg_nu=3),
    "wells128_N256": dict(m=128, N=256, potential=("wells", 3), u0_seed=103, tau=0.4,
                          precision="mixed", cg_rtol=1e-6, eps=1e-5),
    "wells64_N32": dict(m=64, N=32, potential=("wells", 5), u0_seed=105, tau=0.4,
                        precision="fp64", cg_rtol=1e-10, eps=1e-8),
}


def potential(spec, m: int) -> np.ndarray:
    kind, seed = spec
    if kind == "harmonic":
        return harmonic(m)
    if kind == "wells":
        return wells(m, seed)
    raise ValueError(kind)


def workload(name: str):
    """(V, U0, parameters) of a named workload."""
    w = dict(WORKLOADS[name])
    V = potential(w["potential"], w["m"])
    U0 = initial_block(w["m"], w["N"], w["u0_seed"])
    return V, U0, w


# The batched workload: 32 independent problems, grid sides and block widths
# drawn uniformly from these sets by default_rng(4) (sides first, then widths),
# wells potential k from default_rng(1000 + k), U0 k from default_rng(2000 + k),
# tau = 0.4, mixed precision.
BATCH_SIDES = (32, 48, 64, 96)
BATCH_WIDTHS = (16, 32, 64, 128)


def batch_shapes(count: int = 32, seed: int = 4):
    """[(m_k, N_k)] of the batched workload."""
    rng = np.random.default_rng(seed)
    ms = rng.choice(BATCH_SIDES, count)
    Ns = rng.choice(BATCH_WIDTHS, count)
    return [(int(m), int(N)) for m, N in zip(ms, Ns)]


def batch_problem(k: int, m: int, N: int):
    """(V, U0) of problem k of the batched workload."""
    return wells(m, 1000 + k), initial_block(m, N, 2000 + k)
