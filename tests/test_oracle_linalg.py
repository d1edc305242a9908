"""Pins of the oracle's Gram products, LU solve and Jacobi eigensolver."""
import numpy as np
import pytest

import oracle as O


def test_gram_matches_numpy():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((1000, 5))
    B = rng.standard_normal((1000, 3))
    np.testing.assert_allclose(O.gram(A, B, 0.25), 0.25 * A.T @ B, rtol=1e-13, atol=1e-13)


def test_gram_compensated_sum_is_exact_on_cancelling_data():
    """1e16 + 1 - 1e16 style cancellation: a compensated sum recovers the
    exact value where naive summation loses it."""
    a = np.array([[1e16], [1.0], [-1e16], [1.0]])
    b = np.ones((4, 1))
    assert O.gram(a, b, 1.0)[0, 0] == 2.0


def test_lu_solve_matches_numpy_and_pivots():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((12, 12))
    A[0, 0] = 0.0  # forces a row exchange
    B = rng.standard_normal((12, 4))
    np.testing.assert_allclose(O.lu_solve(A, B), np.linalg.solve(A, B), rtol=1e-11, atol=1e-12)


def test_lu_singular():
    A = np.ones((3, 3))
    with pytest.raises(O.OracleError, match="singular"):
        O.lu_solve(A, np.ones((3, 1)))


@pytest.mark.parametrize("n", [1, 2, 7, 20])
def test_jacobi_eig_tridiagonal_closed_form(n):
    """tridiag(-1, 2, -1) has eigenvalues 2 - 2 cos(k pi / (n + 1))."""
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    ev, V = O.sym_eig(T)
    k = np.arange(1, n + 1)
    np.testing.assert_allclose(ev, np.sort(2 - 2 * np.cos(k * np.pi / (n + 1))), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(T @ V, V * ev, atol=1e-12)


def test_jacobi_eig_random_symmetric():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((16, 16))
    A = A + A.T
    ev, V = O.sym_eig(A)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(A), atol=1e-12)
    np.testing.assert_allclose(A @ V, V * ev, atol=1e-11)


def test_scale_initial_puts_block_in_quasi_stiefel_set():
    rng = np.random.default_rng(4)
    U = rng.standard_normal((500, 6))
    h3 = 0.1
    Us, f = O.scale_initial(U, h3)
    lam = np.linalg.eigvalsh(h3 * Us.T @ Us)
    assert lam[0] == pytest.approx(1.0, rel=1e-12)
    assert lam[-1] > 1.0
    np.testing.assert_allclose(Us, U * f, rtol=1e-15)
