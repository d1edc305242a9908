"""Differentiation at the full size of the differentiation workload
(wells64_N32: 64^3 grid, N = 32, harmonic + wells potential from
default_rng(5), U0 from default_rng(105), FP64): d(sum of the 32 lowest
eigenvalues)/dV and the gradient of the L2 density mismatch to the density
of a second potential (default_rng(6)), against central finite differences
(h = 1e-6) at 20 grid points drawn by default_rng(505) and against the
oracle's gradients (orc_grad_eigs, orc_grad_density) evaluated on the GPU's
converged eigenpairs.

Converged eigenpairs: Algorithm 1 (FP64 block PCG with the FP32 multigrid
preconditioner, adaptive time step) to g < 1e-4, then the FP64 residual
refinement (hq_refine) to g < 1e-10.  Each finite-difference evaluation
starts from those eigenpairs and refines them for the perturbed potential:
Newton's method for the invariant subspace converges quadratically from a
start that is O(h) away, so two rounds reach the rounding level."""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import hq, inputs
from tests.gpu_common import torch_mod

pytestmark = pytest.mark.gpu

FD_H = 1e-6


def _converged(V, U0, N):
    m = round(len(V) ** (1 / 3))
    s = hq.Solver(m, N, tau=0.4, cg_rtol=1e-10, mg_fp32=1, adaptive_tau=1, tau_max=10.0)
    s.set_potential(V)
    s.set_initial(U0)
    s.solve(1e-4, 60000)
    s.refine(rounds=3, rtol=1e-10, maxit=2000)
    _, g = s.solve(1e-10, 0, raise_on_unconverged=False)
    assert g < 1e-10, g
    return s


def test_full_size_gradients_match_finite_differences_and_oracle():
    torch = torch_mod()
    V, U0, w = inputs.workload("wells64_N32")
    m, N = w["m"], w["N"]
    h3 = inputs.grid_h(m) ** 3
    s = _converged(V, U0, N)
    ev = s.eigenpairs(vectors=True)
    lam, U = ev["lam_rr"], ev["vectors"]
    Ud, st = s.state_device()
    # target density: the N lowest eigenvectors of a second potential
    s6 = _converged(inputs.wells(m, 6), inputs.initial_block(m, N, 106), N)
    rho_t = s6.density()
    del s6
    g = s.grad_eigs()
    dV, L, its = s.grad_density(rho_target=rho_t, rtol=1e-11, maxit=4000)
    assert np.sum(g) == pytest.approx(N, rel=1e-9)          # constant shift moves every level
    assert abs(np.sum(dV)) <= 1e-6 * np.abs(dV).sum()       # and leaves rho unchanged
    # finite differences of the converged, refined eigenpairs of V +- h e_p
    f = hq.Solver(m, N, tau=0.4, cg_rtol=1e-10, mg_fp32=1)
    pts = np.random.default_rng(505).choice(m ** 3, 20, replace=False)
    fd_s, fd_l = [], []
    for p in pts:
        vals = []
        for sgn in (1.0, -1.0):
            Vx = V.copy()
            Vx[p] += sgn * FD_H
            f.set_potential(Vx)
            f.set_state_device(Ud, st)
            f.refine(rounds=2, rtol=1e-12, maxit=4000)
            lx = f.eigenpairs()["lam_rr"]
            rho = f.density()
            vals.append((np.sum(lx), 0.5 * h3 * np.sum((rho - rho_t) ** 2)))
        fd_s.append((vals[0][0] - vals[1][0]) / (2 * FD_H))
        fd_l.append((vals[0][1] - vals[1][1]) / (2 * FD_H))
    fd_s, fd_l = np.array(fd_s), np.array(fd_l)
    # the sum of ~32 eigenvalues (~150) is accurate to ~1e-13 absolute, so a
    # central difference carries ~1e-7 of noise
    np.testing.assert_allclose(g[pts], fd_s, rtol=1e-5, atol=3e-7)
    np.testing.assert_allclose(dV[pts], fd_l, rtol=1e-4, atol=3e-7 * max(1.0, L))
    # the oracle's gradients on the same eigenpairs
    np.testing.assert_allclose(g, O.grad_eigs(m, U), rtol=1e-9, atol=1e-14)
    dV_or, L_or, _ = O.grad_density(m, V, U, lam, rho_t, rtol=1e-10, maxit=20000)
    assert L == pytest.approx(L_or, rel=1e-9)
    np.testing.assert_allclose(dV, dV_or, rtol=1e-5, atol=1e-7 * np.abs(dV_or).max())
