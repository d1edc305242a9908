"""Pins of the test-side reference constructions (tests/helpers.py) that the
GPU tests use as the definition of the converged result: the N lowest
eigenpairs of the assembled H_h by sparse shift-invert Lanczos."""
import numpy as np
import pytest

pytest.importorskip("scipy")

from paper_2605_25149_gb300 import inputs as I
from tests.helpers import clusters, dense_h, lowest_eigenpairs, separable_levels, sparse_h


def test_sparse_operator_equals_dense():
    m = 5
    h = I.grid_h(m)
    V = I.wells(m, 3)
    np.testing.assert_allclose(sparse_h(m, h, V, 0.7).toarray(), dense_h(m, h, V, 0.7),
                               rtol=0, atol=0)


def test_lowest_eigenpairs_match_dense_eigh_on_wells():
    m, k = 6, 9
    V = I.wells(m, 5)
    h = I.grid_h(m)
    lam, vec = lowest_eigenpairs(m, V, k)
    ld, vd = np.linalg.eigh(dense_h(m, h, V))
    np.testing.assert_allclose(lam, ld[:k], rtol=1e-12)
    # normalised in <u,u> = h^3 u^T u, spanning the same eigenvectors
    np.testing.assert_allclose(h ** 3 * vec.T @ vec, np.eye(k), atol=1e-10)
    A = dense_h(m, h, V)
    np.testing.assert_allclose(A @ vec, vec * lam, atol=1e-9 * np.abs(vec).max())


def test_lowest_eigenpairs_match_separable_closed_form():
    m, k = 16, 10
    lam, _ = lowest_eigenpairs(m, I.harmonic(m), k)
    np.testing.assert_allclose(lam, separable_levels(m, -6.0, 6.0, k), rtol=1e-12)


def test_clusters_keep_complete_groups_only():
    lam = np.array([1.0, 2.0, 2.0005, 3.0, 3.0002, 3.0004])
    assert clusters(lam, 5, 1e-3) == [[0], [1, 2]]
    assert clusters(lam, 3, 1e-3) == [[0], [1, 2]]
    assert clusters(lam[:3], 3, 1e-3) == [[0]]
