"""Pins of the oracle's finite-difference operator, CG and shift rule.

Each check is against something other than the oracle itself: a dense
Kronecker-sum assembly, 1D tridiagonal eigenpairs (the 3D operator of a
separable potential is a Kronecker sum, so its eigenvalues are sums of 1D
ones), a closed form, or numpy's dense solver.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import inputs as I
from tests.helpers import dense_h, harmonic_1d, separable_levels


def test_grid_spacing():
    assert O.grid_h(16) == pytest.approx(12.0 / 17.0, rel=1e-15)
    assert O.grid_h(64) == pytest.approx(12.0 / 65.0, rel=1e-15)


@pytest.mark.parametrize("m", [3, 5, 6])
def test_apply_matches_dense_kronecker_sum(m):
    rng = np.random.default_rng(10 + m)
    h = O.grid_h(m)
    V = rng.uniform(-3, 3, m ** 3)
    sigma = 0.7
    X = rng.standard_normal((m ** 3, 3))
    Y = O.apply_h(m, h, V, sigma, X)
    A = dense_h(m, h, V, sigma)
    np.testing.assert_allclose(Y, A @ X, rtol=1e-13, atol=1e-12)


def test_tensor_product_eigenvectors():
    """H (phi_a x phi_b x phi_c) = (mu_a + mu_b + mu_c)(phi_a x phi_b x phi_c)
    for the separable harmonic potential of Example 5.1 (in 3D)."""
    m = 8
    h = O.grid_h(m)
    mu, phi = np.linalg.eigh(harmonic_1d(m, -6.0, 6.0))
    V = I.harmonic(m)
    cols, lams = [], []
    for a, b, c in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 1, 4)]:
        # flattened index i + m(j + m k): C order over (k, j, i)
        u = np.einsum("k,j,i->kji", phi[:, c], phi[:, b], phi[:, a]).ravel()
        cols.append(u)
        lams.append(mu[a] + mu[b] + mu[c])
    U = np.stack(cols, axis=1)
    HU = O.apply_h(m, h, V, 0.0, U)
    np.testing.assert_allclose(HU, U * np.array(lams), atol=1e-12)


def test_laplacian_lowest_eigenvalue_closed_form():
    """lambda_min(-Delta_h/2) = 3 (2/h^2) sin^2(pi / (2(m+1))); with V = 0 the
    shift rule must see a positive bound and return sigma = 0."""
    m = 6
    h = O.grid_h(m)
    A = dense_h(m, h, np.zeros(m ** 3))
    lmin = np.linalg.eigvalsh(A)[0]
    closed = 3.0 * (2.0 / h ** 2) * np.sin(np.pi / (2 * (m + 1))) ** 2
    assert lmin == pytest.approx(closed, rel=1e-12)
    assert O.auto_shift(m, np.zeros(m ** 3)) == 0.0


def test_auto_shift_makes_operator_coercive():
    """Wells make H_h indefinite; the shifted operator has lambda_1 >= 1."""
    m = 6
    V = I.wells(m, seed=2) - 30.0
    sigma = O.auto_shift(m, V)
    h = O.grid_h(m)
    lam = np.linalg.eigvalsh(dense_h(m, h, V, sigma))
    assert sigma > 0
    assert lam[0] >= 1.0 - 1e-12
    # closed-form lower bound is tight for a constant potential
    Vc = np.full(m ** 3, -4.0)
    sc = O.auto_shift(m, Vc)
    assert np.linalg.eigvalsh(dense_h(m, h, Vc, sc))[0] == pytest.approx(1.0, rel=1e-12)


def test_harmonic_levels_are_kronecker_sums():
    """The 16^3 harmonic levels used as the converged-result pin are sums of
    three 1D tridiagonal eigenvalues: brute force against a dense eigensolve of
    the assembled 3D operator on a small grid, and the degeneracies the cubic
    symmetry forces at 16^3 (the first excited level threefold; lambda_8 =
    lambda_10, a triplet cut by the first N = 8 columns)."""
    m = 6
    lam = np.linalg.eigvalsh(dense_h(m, O.grid_h(m), I.harmonic(m)))
    np.testing.assert_allclose(separable_levels(m, -6.0, 6.0, 20), lam[:20], rtol=1e-12)
    lv = separable_levels(16, -6.0, 6.0, 11)
    assert lv[1] == pytest.approx(lv[3], rel=1e-13) and lv[0] < lv[1] * (1 - 1e-3)
    assert lv[7] == pytest.approx(lv[9], rel=1e-13)


def test_cg_matches_dense_solve():
    m = 6
    rng = np.random.default_rng(3)
    h = O.grid_h(m)
    V = I.wells(m, seed=4)
    sigma = O.auto_shift(m, V)
    B = rng.standard_normal((m ** 3, 4))
    X, its = O.cg(m, h, V, sigma, B, rtol=1e-14)
    Xd = np.linalg.solve(dense_h(m, h, V, sigma), B)
    np.testing.assert_allclose(X, Xd, rtol=1e-11, atol=1e-12)
    assert (its > 0).all()


def test_cg_warm_start_from_solution_takes_no_iterations():
    m = 5
    rng = np.random.default_rng(4)
    h = O.grid_h(m)
    V = I.harmonic(m)
    B = rng.standard_normal((m ** 3, 2))
    X, _ = O.cg(m, h, V, 0.0, B, rtol=1e-13)
    X2, its = O.cg(m, h, V, 0.0, B, X0=X, rtol=1e-10)
    assert (its == 0).all()
    np.testing.assert_array_equal(X, X2)


def test_cg_reports_breakdown_on_negative_definite_operator():
    m = 4
    h = O.grid_h(m)
    V = np.zeros(m ** 3)
    B = np.ones((m ** 3, 1))
    with pytest.raises(O.OracleError, match="breakdown"):
        O.cg(m, h, V, -1000.0, B)


def test_zero_rhs_gives_zero_solution():
    m = 4
    h = O.grid_h(m)
    X, its = O.cg(m, h, I.harmonic(m), 0.0, np.zeros((m ** 3, 2)))
    assert (X == 0).all() and (its == 0).all()
