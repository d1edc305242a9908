"""Differentiation through the converged eigenpairs (FP64 contexts):
d(sum lambda_i)/dV by Hellmann-Feynman and the adjoint of a density loss,
against central finite differences (h = 1e-6, 20 random grid points) of
dense eigensolves of the same discrete operator."""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import hq, inputs
from tests.gpu_common import make, torch_mod
from tests.helpers import dense_h

pytestmark = pytest.mark.gpu

M, N = 8, 4
FD_H = 1e-6
# central differences of dense eigenvalues (accurate to ~1e-15 relative) carry
# an absolute noise of ~1e-15 * |sum lambda| / FD_H ~ 1e-8
FD_NOISE = 2e-8


def _dense(V):
    h = inputs.grid_h(M)
    lam, vec = np.linalg.eigh(dense_h(M, h, V))
    vec = vec / np.sqrt(h ** 3)          # <u,u> = h^3 u^T u = 1
    return lam, vec


def _solved(seed=2):
    torch_mod()
    s, V, U0 = make(M, N, seed=seed, cg_rtol=1e-12, cg_maxit=400, adaptive_tau=1, tau_max=5.0)
    lam, _ = _dense(V)
    assert lam[N] - lam[N - 1] > 0.05          # gap for a well-defined subspace
    s.solve(1e-11, 50000)
    return s, V


def test_grad_sum_of_eigenvalues_matches_finite_differences():
    s, V = _solved()
    g = s.grad_eigs()
    rng = np.random.default_rng(505)
    pts = rng.choice(M ** 3, 20, replace=False)
    for p in pts:
        Vp, Vm = V.copy(), V.copy()
        Vp[p] += FD_H
        Vm[p] -= FD_H
        fd = (np.sum(_dense(Vp)[0][:N]) - np.sum(_dense(Vm)[0][:N])) / (2 * FD_H)
        assert g[p] == pytest.approx(fd, rel=1e-5, abs=FD_NOISE)
    # weighted form: d lambda_2 / dV = h^3 u_2^2
    w = np.zeros(N)
    w[1] = 1.0
    g2 = s.grad_eigs(w)
    lam, vec = _dense(V)
    np.testing.assert_allclose(g2, inputs.grid_h(M) ** 3 * vec[:, 1] ** 2, rtol=1e-7, atol=1e-12)


def test_density_matches_dense_eigenvectors():
    s, V = _solved()
    lam, vec = _dense(V)
    np.testing.assert_allclose(s.density(), np.sum(vec[:, :N] ** 2, axis=1), rtol=1e-7, atol=1e-10)


def test_grad_density_loss_matches_finite_differences():
    s, V = _solved()
    V2 = inputs.wells(M, 6)
    rho_t = np.sum(_dense(V2)[1][:, :N] ** 2, axis=1)
    h3 = inputs.grid_h(M) ** 3

    def loss(Vx):
        rho = np.sum(_dense(Vx)[1][:, :N] ** 2, axis=1)
        return 0.5 * h3 * np.sum((rho - rho_t) ** 2)

    dV, L, its = s.grad_density(rho_target=rho_t, rtol=1e-12, maxit=1000)
    assert L == pytest.approx(loss(V), rel=1e-8)
    assert its > 0
    rng = np.random.default_rng(506)
    for p in rng.choice(M ** 3, 20, replace=False):
        Vp, Vm = V.copy(), V.copy()
        Vp[p] += FD_H
        Vm[p] -= FD_H
        fd = (loss(Vp) - loss(Vm)) / (2 * FD_H)
        assert dV[p] == pytest.approx(fd, rel=1e-4, abs=FD_NOISE * max(1.0, loss(V)))


def test_differentiation_needs_fp64_context():
    torch_mod()
    s, V, U0 = make(M, N, precision="mixed", cg_rtol=1e-6)
    with pytest.raises(hq.HQError) as e:
        s.grad_eigs()
    assert e.value.status == 2


def test_gradients_match_the_oracle():
    """hq_grad_eigs / hq_grad_density against the oracle's gradients
    (orc_grad_eigs, orc_grad_density) evaluated on the dense eigenpairs."""
    s, V = _solved()
    lam, vec = _dense(V)
    g_or = O.grad_eigs(M, vec[:, :N])
    np.testing.assert_allclose(s.grad_eigs(), g_or, rtol=1e-8, atol=1e-12 * np.abs(g_or).max())
    rho_t = np.sum(_dense(inputs.wells(M, 6))[1][:, :N] ** 2, axis=1)
    dV_or, L_or, _ = O.grad_density(M, V, vec[:, :N], lam[:N], rho_t)
    dV, L, _ = s.grad_density(rho_target=rho_t, rtol=1e-12, maxit=1000)
    assert L == pytest.approx(L_or, rel=1e-9)
    np.testing.assert_allclose(dV, dV_or, rtol=1e-6, atol=1e-8 * np.abs(dV_or).max())


def test_autograd_functions():
    """EigenvalueSum / Density through torch.autograd give the C-ABI gradients."""
    import torch
    from paper_2605_25149_gb300.autograd import Density, EigenvalueSum
    s, V = _solved()
    Vt = torch.tensor(V, dtype=torch.float64, device="cuda", requires_grad=True)
    lam_sum = EigenvalueSum.apply(Vt, s, 1e-11, 50000)
    lam_sum.backward()
    lam, vec = _dense(V)
    assert lam_sum.item() == pytest.approx(np.sum(lam[:N]), rel=1e-12)
    np.testing.assert_allclose(Vt.grad.cpu().numpy(), O.grad_eigs(M, vec[:, :N]), rtol=1e-8,
                               atol=1e-14)
    rho_t = torch.tensor(np.sum(_dense(inputs.wells(M, 6))[1][:, :N] ** 2, axis=1),
                         device="cuda")
    Vt.grad = None
    rho = Density.apply(Vt, s, 1e-11, 50000, 1e-12, 1000)
    h3 = inputs.grid_h(M) ** 3
    loss = 0.5 * h3 * ((rho - rho_t) ** 2).sum()
    loss.backward()
    dV_ref, L_ref, _ = s.grad_density(rho_target=rho_t.cpu().numpy(), rtol=1e-12, maxit=1000)
    assert loss.item() == pytest.approx(L_ref, rel=1e-10)
    np.testing.assert_allclose(Vt.grad.cpu().numpy(), dV_ref, rtol=1e-7,
                               atol=1e-10 * np.abs(dV_ref).max())


def test_gradient_shift_rules_at_a_larger_size():
    """16^3, N = 8 wells: a constant shift of V moves every eigenvalue by the
    same amount (sum_p d(sum lambda)/dV_p = N) and leaves rho unchanged
    (sum_p dL/dV_p = 0) -- properties that hold at any size."""
    torch_mod()
    m, n_ev = 16, 8
    s, V, U0 = make(m, n_ev, seed=5, useed=105, cg_rtol=1e-12, cg_maxit=400, adaptive_tau=1,
                    tau_max=5.0)
    s.solve(1e-10, 50000)
    g = s.grad_eigs()
    assert np.sum(g) == pytest.approx(n_ev, rel=1e-8)
    rho_t = np.full(m ** 3, n_ev / (m ** 3 * inputs.grid_h(m) ** 3))
    dV, L, its = s.grad_density(rho_target=rho_t, rtol=1e-12, maxit=2000)
    assert its > 0 and L > 0
    assert abs(np.sum(dV)) <= 1e-6 * np.abs(dV).sum()
