"""The whole-phase CUDA graphs of hq_step / hq_solve against the host-driven
path of the same context type.

With graphs, the two phases of a step of Eq. (4.1) (A: W = G U, the Gram of
[U W] and g; B: predictor system, Uh, Z = G Uh, corrector) are replayed as
captured graphs whose inner PCG loop is a conditional WHILE node.  The
operation sequence is the host path's, so the trajectories must agree
bit for bit; HQ_NO_GRAPHS=1 at context creation selects the host path.
"""
import os

import numpy as np
import pytest

from paper_2605_25149_gb300 import hq
from tests.gpu_common import make

pytestmark = pytest.mark.gpu


def _make(graphs, *a, **kw):
    old = os.environ.pop("HQ_NO_GRAPHS", None)
    try:
        if not graphs:
            os.environ["HQ_NO_GRAPHS"] = "1"
        return make(*a, **kw)
    finally:
        os.environ.pop("HQ_NO_GRAPHS", None)
        if old is not None:
            os.environ["HQ_NO_GRAPHS"] = old


@pytest.mark.parametrize("precision,adaptive,warm", [("fp64", 0, 1), ("fp64", 1, 1),
                                                     ("fp64", 0, 0), ("mixed", 1, 1)])
def test_graph_steps_are_bit_identical_to_host_steps(precision, adaptive, warm):
    m, N = 20, 12
    kw = dict(precision=precision, tau=0.4, cg_rtol=1e-10, adaptive_tau=adaptive,
              z_warm_start=warm)
    a, _, _ = _make(True, m, N, **kw)
    b, _, _ = _make(False, m, N, **kw)
    a.profile()
    b.profile()
    for k in (1, 3, 4):
        ga = a.step(k)
        gb = b.step(k)
        assert ga == gb
        Ua, Za, sa = a.get_state(with_warm_start=True)
        Ub, Zb, sb = b.get_state(with_warm_start=True)
        assert sa == sb
        assert np.array_equal(Ua, Ub)
        assert np.array_equal(Za, Zb)
    assert a.pcg_stats() == b.pcg_stats()
    # the stencil, smoother and transfer launches are the same kernels in both
    pa, pb = a.profile_read(), b.profile_read()
    for cls in ("stencil", "residual", "smooth", "transfer", "coarse", "gram", "blockgemm"):
        assert pa[cls][0] == pb[cls][0], cls


def test_graph_solve_matches_host_solve():
    m, N = 16, 8
    kw = dict(tau=0.4, cg_rtol=1e-10, adaptive_tau=1)
    a, _, _ = _make(True, m, N, **kw)
    b, _, _ = _make(False, m, N, **kw)
    ra = a.solve(1e-7, 300, raise_on_unconverged=False)
    rb = b.solve(1e-7, 300, raise_on_unconverged=False)
    assert ra == rb
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    assert a.time_step() == b.time_step()


def test_graph_step_reports_inner_pcg_limit():
    """cg_maxit reached inside a replayed graph: hq_step returns
    HQ_ERR_NOT_CONVERGED, as the host path does."""
    m, N = 16, 8
    a, _, _ = _make(True, m, N, tau=0.4, cg_rtol=1e-10)
    a.step(2)
    U, Z, step = a.get_state(with_warm_start=True)
    b, _, _ = _make(True, m, N, tau=0.4, cg_rtol=1e-14, cg_maxit=2)
    b.set_state(U, step, Z)
    with pytest.raises(hq.HQError) as ei:
        b.step(2)
    assert ei.value.status == 7   # HQ_ERR_NOT_CONVERGED


def test_graphs_follow_a_new_potential():
    """A new potential changes the shift sigma, which the captured graphs hold
    by value: hq_set_potential must discard them."""
    from paper_2605_25149_gb300 import inputs
    m, N = 16, 8
    kw = dict(tau=0.4, cg_rtol=1e-10, adaptive_tau=1)
    a, _, U0 = _make(True, m, N, **kw)
    b, _, _ = _make(False, m, N, **kw)
    for s in (a, b):
        s.step(3)
        s.set_potential(inputs.harmonic(m) - 3.0)
        s.set_initial(U0)
        s.step(4)
    assert a.info()["sigma"] == b.info()["sigma"] > 0.0
    assert np.array_equal(a.get_state()[0], b.get_state()[0])


def _zm_pair(precision, m=20, N=12):
    out = []
    for flag in ("1", "0"):
        old = os.environ.get("HQ_ZMARCH")
        os.environ["HQ_ZMARCH"] = flag
        try:
            s, _, _ = make(m, N, precision=precision, tau=0.4,
                           cg_rtol=1e-10 if precision == "fp64" else 1e-6)
        finally:
            if old is None:
                os.environ.pop("HQ_ZMARCH", None)
            else:
                os.environ["HQ_ZMARCH"] = old
        out.append(s)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zmarch_kernels_match_the_linear_order(precision):
    """The z-marching CTAs (used for finest-level blocks beyond about three
    quarters of L2; HQ_ZMARCH=1 forces them) form every element with the
    same sums in the same order as the linear-order kernels: the operator,
    a smoothing sweep and a V-cycle are bit-identical.  Their per-column
    PCG partial sums (p.q, r.z, r.r, b.b) are reduced per CTA, a different
    order, so PCG solves and trajectories agree to rounding."""
    from tests.gpu_common import dev, host, rel
    torch = pytest.importorskip("torch")
    a, b = _zm_pair(precision)
    n, N = a.n, a.N
    dt = torch.float64 if precision == "fp64" else torch.float32
    rng = np.random.default_rng(5)
    x = dev(rng.standard_normal((n, N)), dt)
    r = dev(rng.standard_normal((n, N)), dt)
    assert np.array_equal(host(a.apply_operator(x)), host(b.apply_operator(x)))
    assert np.array_equal(host(a.mg_smooth(0, r, x)), host(b.mg_smooth(0, r, x)))
    assert np.array_equal(host(a.mg_vcycle(r)), host(b.mg_vcycle(r)))
    tol_x = 1e-8 if precision == "fp64" else 1e-4
    Xa, ia = a.block_pcg(r, rtol=1e-10 if precision == "fp64" else 1e-6)
    Xb, ib = b.block_pcg(r, rtol=1e-10 if precision == "fp64" else 1e-6)
    assert np.abs(ia - ib).max() <= 1
    assert rel(host(Xa), host(Xb)) < tol_x
    a.step(3)
    b.step(3)
    assert rel(a.get_state()[0], b.get_state()[0]) < (1e-8 if precision == "fp64" else 1e-4)
