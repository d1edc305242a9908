"""Pins of the oracle's FP64 residual refinement (orc_refine): Rayleigh-Ritz
followed by per-column Newton corrections on the complement of span(U).

Not in the paper; it is the final FP64 refinement of a lower-precision result.
Pinned by the plain definition of the converged result (the N lowest
eigenpairs of the assembled H_h, dense eigh), the fixed point at exact
eigenvectors, quadratic convergence from a perturbed subspace, and
invariance under a change of basis of span(U)."""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import inputs as I
from tests.helpers import dense_h, subspace_sin


def _dense(m, V, N):
    h = O.grid_h(m)
    lam, vec = np.linalg.eigh(dense_h(m, h, V))
    return lam[: N + 1], vec[:, :N] / np.sqrt(h ** 3)


def test_refine_converges_quadratically_to_dense_eigenpairs():
    m, N = 8, 6
    V = I.wells(m, 11)
    lam_ref, vec_ref = _dense(m, V, N)
    assert lam_ref[N] - lam_ref[N - 1] > 0.05
    rng = np.random.default_rng(3)
    errs = []
    for eps in (1e-2, 1e-3):
        U0 = vec_ref + eps * rng.standard_normal(vec_ref.shape) / np.sqrt(len(V))
        e0 = subspace_sin(U0, vec_ref)
        U1, lam1, _, its = O.refine(m, V, U0, 1, rtol=1e-13)
        e1 = subspace_sin(U1, vec_ref)
        errs.append((e0, e1))
        # Newton: the subspace error is squared up to a modest constant
        assert e1 <= 100.0 * e0 ** 2 + 1e-12, (e0, e1)
    # two more rounds: eigenvalues and vectors at FP64 accuracy
    U2, lam2, res2, its = O.refine(m, V, U1, 2, rtol=1e-13)
    np.testing.assert_allclose(lam2, lam_ref[:N], rtol=1e-13)
    assert subspace_sin(U2, vec_ref) < 1e-11
    assert res2.max() < 1e-10
    h3 = O.grid_h(m) ** 3
    np.testing.assert_allclose(h3 * U2.T @ U2, np.eye(N), atol=1e-12)
    # each eigenvector individually (the levels are simple)
    for i in range(N):
        c = h3 * U2[:, i] @ vec_ref[:, i]
        assert abs(abs(c) - 1.0) < 1e-11


def test_refine_fixes_exact_eigenvectors_and_ignores_the_basis():
    m, N = 7, 3
    V = I.wells(m, 2)
    lam_ref, vec_ref = _dense(m, V, N)
    assert lam_ref[N] - lam_ref[N - 1] > 0.3
    # exact eigenvectors leave residuals at the rounding level: a relative
    # inner tolerance of 1e-10 ends the CG before it runs on rounding noise
    U, lam, res, its = O.refine(m, V, vec_ref, 1, rtol=1e-10)
    np.testing.assert_allclose(lam, lam_ref[:N], rtol=1e-13)
    assert subspace_sin(U, vec_ref) < 1e-12
    assert res.max() < 1e-10
    # the same subspace in another, non-orthonormal basis gives the same result
    rng = np.random.default_rng(9)
    Ub = vec_ref + 1e-3 * rng.standard_normal(vec_ref.shape)
    C = rng.standard_normal((N, N)) + 3.0 * np.eye(N)
    Ua, la, _, _ = O.refine(m, V, Ub, 1, rtol=1e-12)
    Uc, lc, _, _ = O.refine(m, V, Ub @ C, 1, rtol=1e-12)
    np.testing.assert_allclose(lc, la, rtol=1e-12)
    assert subspace_sin(Uc, Ua) < 1e-10


def test_refine_reports_a_failed_inner_solve():
    m, N = 6, 3
    V = I.wells(m, 4)
    _, vec_ref = _dense(m, V, N)
    U0 = vec_ref + 1e-2 * np.random.default_rng(1).standard_normal(vec_ref.shape)
    with pytest.raises(O.OracleError):
        O.refine(m, V, U0, 1, rtol=1e-14, maxit=1)
