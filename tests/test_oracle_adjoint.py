"""Pins of the oracle's differentiation functions (orc_grad_eigs,
orc_grad_density) on small grids: central finite differences of dense
eigensolves, an independent sum-over-states formula, and the invariance of
the density under a constant shift of V."""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import inputs
from tests.helpers import dense_h

M = 5
FD_H = 1e-6


def _eig(V, m=M):
    h = inputs.grid_h(m)
    lam, vec = np.linalg.eigh(dense_h(m, h, V))
    return lam, vec / np.sqrt(h ** 3)          # <u,u> = h^3 u^T u = 1


def _case(N=4, seed=2):
    V = inputs.wells(M, seed)
    lam, vec = _eig(V)
    assert lam[N] - lam[N - 1] > 0.05
    return V, lam, vec


def _rho(vec, N):
    return np.sum(vec[:, :N] ** 2, axis=1)


def test_grad_eigs_matches_finite_differences_and_shift_rule():
    N = 4
    V, lam, vec = _case(N)
    g = O.grad_eigs(M, vec[:, :N])
    rng = np.random.default_rng(11)
    for p in rng.choice(M ** 3, 12, replace=False):
        Vp, Vm = V.copy(), V.copy()
        Vp[p] += FD_H
        Vm[p] -= FD_H
        fd = (np.sum(_eig(Vp)[0][:N]) - np.sum(_eig(Vm)[0][:N])) / (2 * FD_H)
        assert g[p] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    # a constant shift c of V moves every eigenvalue by c: sum_p dV_p = N
    assert np.sum(g) == pytest.approx(N, rel=1e-12)
    # weights select single eigenvalues
    w = np.array([0.0, 0.0, 1.0, 0.0])
    g3 = O.grad_eigs(M, vec[:, :N], w)
    assert np.sum(g3) == pytest.approx(1.0, rel=1e-12)
    np.testing.assert_allclose(g3, inputs.grid_h(M) ** 3 * vec[:, 2] ** 2, rtol=1e-13, atol=0)


def _loss_fn(rho_t, N):
    h3 = inputs.grid_h(M) ** 3

    def loss(Vx):
        return 0.5 * h3 * np.sum((_rho(_eig(Vx)[1], N) - rho_t) ** 2)
    return loss


def test_grad_density_matches_finite_differences():
    N = 4
    V, lam, vec = _case(N)
    rho_t = _rho(_eig(inputs.wells(M, 6))[1], N)
    loss = _loss_fn(rho_t, N)
    dV, L, its = O.grad_density(M, V, vec[:, :N], lam[:N], rho_t)
    assert L == pytest.approx(loss(V), rel=1e-12)
    assert its > 0
    rng = np.random.default_rng(12)
    for p in rng.choice(M ** 3, 12, replace=False):
        Vp, Vm = V.copy(), V.copy()
        Vp[p] += FD_H
        Vm[p] -= FD_H
        fd = (loss(Vp) - loss(Vm)) / (2 * FD_H)
        assert dV[p] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, L))
    # rho does not change under V -> V + c: the gradient sums to zero
    assert abs(np.sum(dV)) <= 1e-9 * np.abs(dV).sum()


def test_grad_density_matches_sum_over_states():
    """dL/dV_p = 2 h^3 sum_{i occ} sum_{j unocc} u_i(p) u_j(p) <g u_i, u_j> /
    (lambda_i - lambda_j), from first-order perturbation theory with the full
    dense spectrum (occupied-occupied terms cancel in rho)."""
    N = 4
    V, lam, vec = _case(N)
    h3 = inputs.grid_h(M) ** 3
    rho_t = _rho(_eig(inputs.wells(M, 7))[1], N)
    g = _rho(vec, N) - rho_t
    ref = np.zeros(M ** 3)
    for i in range(N):
        for j in range(N, M ** 3):
            c = h3 * np.sum(g * vec[:, i] * vec[:, j]) / (lam[i] - lam[j])
            ref += 2.0 * h3 * c * vec[:, i] * vec[:, j]
    dV, _, _ = O.grad_density(M, V, vec[:, :N], lam[:N], rho_t, rtol=1e-14)
    np.testing.assert_allclose(dV, ref, rtol=1e-8, atol=1e-12 * np.abs(ref).max())
