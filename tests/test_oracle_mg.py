"""Pins of the oracle's multigrid preconditioner.

The transfer operators are checked against scipy's independent trilinear
interpolator and against the L2-adjoint identity that defines restriction;
the V-cycle against symmetry, linearity, exactness on one level and
contraction as a stationary iteration.
"""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import inputs as I
from tests.helpers import dense_h

scipy_interp = pytest.importorskip("scipy.interpolate")


def test_level_sequence():
    assert O.mg_levels(64) == [64, 32, 16, 8, 4]
    assert O.mg_levels(48) == [48, 24, 12, 6, 3]
    assert O.mg_levels(96) == [96, 48, 24, 12, 6, 3]
    assert O.mg_levels(128) == [128, 64, 32, 16, 8, 4]
    assert O.mg_levels(16) == [16, 8, 4]
    assert O.mg_levels(3) == [3]
    assert O.mg_levels(5) == [5, 2]


def _padded_axes(m):
    h = 12.0 / (m + 1)
    return -6.0 + h * np.arange(0, m + 2)


@pytest.mark.parametrize("mc,mf", [(4, 8), (3, 7), (5, 11), (6, 13), (8, 16)])
def test_prolongation_is_trilinear_interpolation(mc, mf):
    """P e = trilinear interpolant of the coarse nodal values (zero on the
    boundary nodes), evaluated at the fine nodes, by scipy."""
    rng = np.random.default_rng(mc * 100 + mf)
    ec = rng.standard_normal(mc ** 3)
    padded = np.zeros((mc + 2,) * 3)
    padded[1:-1, 1:-1, 1:-1] = ec.reshape(mc, mc, mc)      # axes (k, j, i)
    ax = _padded_axes(mc)
    f = scipy_interp.RegularGridInterpolator((ax, ax, ax), padded, method="linear")
    x, y, z = I.coords(mf)
    expect = f(np.stack([z, y, x], axis=1))
    got = O.prolong_add(mc, mf, ec[:, None], np.zeros((mf ** 3, 1)))[:, 0]
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("mf,mc", [(8, 4), (7, 3), (11, 5), (16, 8)])
def test_restriction_is_scaled_adjoint_of_prolongation(mf, mc):
    """h_c^3 <R r, e>_c = h_f^3 <r, P e>_f (R is the L2 adjoint of P).  The
    oracle implements R and P as separate loops, so this pins both."""
    rng = np.random.default_rng(mf)
    r = rng.standard_normal((mf ** 3, 2))
    e = rng.standard_normal((mc ** 3, 2))
    Rr = O.restrict(mf, mc, r)
    Pe = O.prolong_add(mc, mf, e, np.zeros((mf ** 3, 2)))
    hf, hc = 12.0 / (mf + 1), 12.0 / (mc + 1)
    lhs = hc ** 3 * np.sum(Rr * e, axis=0)
    rhs = hf ** 3 * np.sum(r * Pe, axis=0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_nested_prolongation_injects_and_averages():
    """For odd m_f = 2 m_c + 1 the grids are nested: coarse nodes are copied
    and fine midpoints in x get the average of their two coarse neighbours."""
    mc, mf = 3, 7
    ec = np.arange(1, mc ** 3 + 1, dtype=np.float64)
    ef = O.prolong_add(mc, mf, ec[:, None], np.zeros((mf ** 3, 1)))[:, 0].reshape(mf, mf, mf)
    C = ec.reshape(mc, mc, mc)
    assert ef[1, 1, 1] == C[0, 0, 0]
    assert ef[3, 5, 3] == C[1, 2, 1]
    assert ef[1, 1, 2] == pytest.approx(0.5 * (C[0, 0, 0] + C[0, 0, 1]), rel=1e-15)
    assert ef[1, 1, 0] == pytest.approx(0.5 * C[0, 0, 0], rel=1e-15)


@pytest.mark.parametrize("mf,mc", [(8, 4), (16, 8), (9, 4)])
def test_coarse_potential_is_trilinear_sample(mf, mc):
    rng = np.random.default_rng(mf + mc)
    Vf = rng.uniform(-2, 2, mf ** 3)
    h = 12.0 / (mf + 1)
    ax = -6.0 + h * np.arange(1, mf + 1)
    f = scipy_interp.RegularGridInterpolator((ax, ax, ax), Vf.reshape(mf, mf, mf),
                                             method="linear")
    x, y, z = I.coords(mc)
    np.testing.assert_allclose(O.coarse_potential(mf, Vf, mc), f(np.stack([z, y, x], 1)),
                               rtol=1e-13, atol=1e-14)


def _mg(m, seed=2, **kw):
    V = I.wells(m, seed)
    sigma = O.auto_shift(m, V)
    return O.MG(m, V, sigma, **kw), V, sigma


def test_vcycle_is_symmetric_and_linear():
    mg, V, sigma = _mg(16)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((16 ** 3, 3))
    y = rng.standard_normal((16 ** 3, 3))
    Mx, My = mg.vcycle(x), mg.vcycle(y)
    np.testing.assert_allclose(np.sum(Mx * y, 0), np.sum(x * My, 0), rtol=1e-12)
    np.testing.assert_allclose(mg.vcycle(2.0 * x - 3.0 * y), 2.0 * Mx - 3.0 * My,
                               rtol=1e-11, atol=1e-13)
    # positive definite on these vectors
    assert (np.sum(Mx * x, 0) > 0).all()


def test_single_level_vcycle_is_exact_solve():
    m = 3
    mg, V, sigma = _mg(m)
    assert mg.levels == [3]
    rng = np.random.default_rng(6)
    b = rng.standard_normal((m ** 3, 2))
    z = mg.vcycle(b)
    np.testing.assert_allclose(dense_h(m, O.grid_h(m), V, sigma) @ z, b, rtol=1e-12, atol=1e-12)
    # PCG with an exact preconditioner converges in one iteration
    x, its = mg.pcg(b, rtol=1e-12)
    assert (its == 1).all()


def test_coarse_solve_matches_dense():
    mg, V, sigma = _mg(8)
    mc = mg.levels[-1]
    Vc = mg.level_potential(len(mg.levels) - 1)
    rng = np.random.default_rng(7)
    b = rng.standard_normal((mc ** 3, 2))
    z = mg.coarse_solve(b)
    A = dense_h(mc, O.grid_h(mc), Vc, sigma)
    np.testing.assert_allclose(z, np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)


def test_smoother_is_damped_jacobi():
    m = 8
    mg, V, sigma = _mg(m, omega=0.8)
    rng = np.random.default_rng(8)
    r = rng.standard_normal((m ** 3, 2))
    z = rng.standard_normal((m ** 3, 2))
    h = O.grid_h(m)
    A = dense_h(m, h, V, sigma)
    D = np.diag(A)[:, None]
    expect = z + 0.8 * (r - A @ z) / D
    np.testing.assert_allclose(mg.smooth(0, r, z), expect, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m", [16, 24])
def test_vcycle_contracts_error(m):
    """x <- x + M (b - A x) reduces the A-norm of the error by at least 4x
    per cycle: the hierarchy is a working multigrid, not just symmetric."""
    mg, V, sigma = _mg(m)
    h = O.grid_h(m)
    rng = np.random.default_rng(9)
    b = rng.standard_normal((m ** 3, 1))
    xs, _ = O.cg(m, h, V, sigma, b, rtol=1e-14)
    x = np.zeros_like(b)

    def anorm(e):
        return float(np.sqrt(np.sum(e * O.apply_h(m, h, V, sigma, e))))

    e0 = anorm(x - xs)
    for _ in range(3):
        x = x + mg.vcycle(b - O.apply_h(m, h, V, sigma, x))
    e3 = anorm(x - xs)
    assert e3 < e0 / 4 ** 3


def test_pcg_converges_and_beats_plain_cg():
    m = 16
    mg, V, sigma = _mg(m)
    h = O.grid_h(m)
    rng = np.random.default_rng(11)
    b = rng.standard_normal((m ** 3, 3))
    x, its = mg.pcg(b, rtol=1e-10)
    res = np.linalg.norm(b - O.apply_h(m, h, V, sigma, x), axis=0) / np.linalg.norm(b, axis=0)
    assert (res <= 1e-10).all()
    _, its_cg = O.cg(m, h, V, sigma, b, rtol=1e-10)
    assert its.max() * 2 < its_cg.min()


def test_pcg_fixed_iteration_mode():
    mg, V, sigma = _mg(8)
    rng = np.random.default_rng(12)
    b = rng.standard_normal((8 ** 3, 2))
    x3, its = mg.pcg(b, rtol=0.0, maxit=3)
    assert (its == 3).all()
    x2, _ = mg.pcg(b, rtol=0.0, maxit=2)
    assert not np.array_equal(x2, x3)


def test_block_pcg_single_column_is_pcg_and_solves_the_system():
    """O'Leary's block PCG (N x N alpha, beta) with one column is the
    per-column PCG iterate by iterate; with several columns it converges to
    the dense solve of (H + sigma) X = B in no more iterations than the
    slowest column of the per-column PCG (its block Krylov space contains
    every column's Krylov space)."""
    m = 9
    V = I.wells(m, 6)
    sigma = O.auto_shift(m, V)
    mg = O.MG(m, V, sigma)
    rng = np.random.default_rng(21)
    b = rng.standard_normal((m ** 3, 1))
    for k in (1, 2, 5):
        xb, _ = mg.block_pcg(b, rtol=0.0, maxit=k)
        xc, _ = mg.pcg(b, rtol=0.0, maxit=k)
        np.testing.assert_allclose(xb, xc, rtol=1e-12, atol=1e-14 * np.abs(xc).max())
    N = 6
    B = rng.standard_normal((m ** 3, N))
    Xb, itb = mg.block_pcg(B, rtol=1e-12, maxit=500)
    Xc, itc = mg.pcg(B, rtol=1e-12, maxit=500)
    A = dense_h(m, O.grid_h(m), V, sigma)
    Xd = np.linalg.solve(A, B)
    np.testing.assert_allclose(Xb, Xd, rtol=1e-10, atol=1e-12 * np.abs(Xd).max())
    assert itb <= itc.max()
    # the block residual is below the tolerance in every column
    R = B - A @ Xb
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-12 * np.linalg.norm(B, axis=0) * 1.0001)
