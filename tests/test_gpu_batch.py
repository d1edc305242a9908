"""The batched form (hq_batch_*): heterogeneous problems advanced together in
one graph launch must follow, bit for bit, the trajectories their contexts
follow alone (hq_step / hq_solve), stop individually, and report per-problem
status; the converged result is checked against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import hq, inputs
from tests.gpu_common import make, torch_mod

pytestmark = pytest.mark.gpu

# (m, N, potential, precision, extra config)
PROBLEMS = [
    (12, 4, "wells", "fp64", dict(tau=0.4)),
    (16, 8, "harmonic", "mixed", dict(tau=0.5, cg_rtol=1e-6)),
    (10, 6, "wells", "fp64", dict(tau=0.4, adaptive_tau=1)),
    (20, 12, "wells", "mixed", dict(tau=0.4, cg_rtol=1e-6, adaptive_tau=1)),
]


def _pair(spec):
    m, N, pot, prec, kw = spec
    kw = dict(kw)
    kw.setdefault("cg_rtol", 1e-10)
    a, V, U0 = make(m, N, potential=pot, precision=prec, **kw)
    b, _, _ = make(m, N, potential=pot, precision=prec, **kw)
    return a, b, V, U0


def test_batch_steps_match_single_contexts():
    torch_mod()
    pairs = [_pair(p) for p in PROBLEMS]
    batch = hq.Batch([a for a, _, _, _ in pairs])
    for n in (1, 4, 3):
        g, stat = batch.step(n)
        assert (stat == 0).all()
        for k, (a, b, _, _) in enumerate(pairs):
            gb = b.step(n)
            assert g[k] == gb, k
            Ua, _, sa = a.get_state()
            Ub, _, sb = b.get_state()
            assert sa == sb
            assert np.array_equal(Ua, Ub), k
    kernels, iters = batch.launches()
    assert iters == (1 + 1) + (4 + 1) + (3 + 1)   # one arm-only iteration per call
    assert kernels == 3 * 1 + 2 * iters
    for a, b, _, _ in pairs:
        assert a.pcg_stats() == b.pcg_stats()


def test_batch_follows_a_new_potential():
    torch_mod()
    pairs = [_pair(p) for p in PROBLEMS[:2]]
    batch = hq.Batch([a for a, _, _, _ in pairs])
    batch.step(2)
    for a, b, _, U0 in pairs:
        b.step(2)
        for s in (a, b):
            s.set_potential(inputs.harmonic(s.m) - 2.0)
            s.set_initial(U0)
    batch.step(3)
    for a, b, _, _ in pairs:
        b.step(3)
        assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_batch_solve_stops_each_problem_like_hq_solve():
    torch_mod()
    specs = [(8, 4, "harmonic", "fp64", dict(tau=0.5)),
             (10, 5, "wells", "fp64", dict(tau=0.4, adaptive_tau=1)),
             (12, 6, "wells", "mixed", dict(tau=0.4, cg_rtol=1e-6, adaptive_tau=1))]
    eps = np.array([1e-8, 1e-8, 1e-4])
    pairs = [_pair(p) for p in specs]
    batch = hq.Batch([a for a, _, _, _ in pairs])
    steps, g, stat = batch.solve(eps, 20000)
    assert (stat == 0).all()
    for k, (a, b, _, _) in enumerate(pairs):
        nb, gb = b.solve(eps[k], 20000)
        assert steps[k] == nb and g[k] == gb, k
        assert np.array_equal(a.get_state()[0], b.get_state()[0])
        ea, eb = a.eigenpairs(), b.eigenpairs()
        assert np.array_equal(ea["lam_rr"], eb["lam_rr"])
    # the first problem against the oracle's Algorithm 1 (Section 5) and the
    # eigenvalues of H_h
    a, _, V, U0 = pairs[0]
    m, N = 8, 4
    h = O.grid_h(m)
    Uo, _ = O.scale_initial(U0, h ** 3)
    Ue, We, so, go, _ = O.solve(m, V, a.info()["sigma"], Uo, 0.5, 1e-8, 20000, cg_rtol=1e-10)
    assert abs(so - steps[0]) <= 2
    ex = O.extract(m, V, a.info()["sigma"], Ue, We, want_vectors=False)
    np.testing.assert_allclose(a.eigenpairs()["lam_rr"], ex["lam_rr"], rtol=1e-10)


def test_batch_reports_per_problem_status():
    torch_mod()
    specs = [(10, 4, "wells", "fp64", dict(tau=0.4)),
             (10, 4, "wells", "fp64", dict(tau=0.4, cg_rtol=1e-14, cg_maxit=1)),
             (12, 4, "harmonic", "fp64", dict(tau=0.5))]
    pairs = [_pair(p) for p in specs]
    batch = hq.Batch([a for a, _, _, _ in pairs])
    steps, g, stat = batch.solve([1e-8] * 3, 5, raise_on_error=False)
    assert list(stat) == [7, 7, 7]            # HQ_ERR_NOT_CONVERGED each
    assert steps[0] == 5 and steps[2] == 5    # cap reached
    assert steps[1] == 0                      # stopped by its inner PCG limit
    # the members that did not fail match hq_solve, which also stops at the cap
    for k in (0, 2):
        a, b = pairs[k][0], pairs[k][1]
        with pytest.raises(hq.HQError) as ei:
            b.solve(1e-8, 5)
        assert ei.value.status == 7
        assert np.array_equal(a.get_state()[0], b.get_state()[0])
    with pytest.raises(hq.HQError) as ei:
        pairs[1][1].solve(1e-8, 5)
    assert ei.value.status == 7
    with pytest.raises(hq.HQError):
        batch.solve([1e-8] * 3, 5)


def test_batch_wall_clock_limit():
    torch_mod()
    pairs = [_pair(p) for p in PROBLEMS[:2]]
    batch = hq.Batch([a for a, _, _, _ in pairs])
    steps, g, stat = batch.solve([1e-12, 1e-12], 1000, timeout_s=1e-9, raise_on_error=False)
    assert list(stat) == [8, 8]               # HQ_ERR_TIMEOUT
    assert list(steps) == [1, 1]              # the limit is tested after each loop iteration


@pytest.mark.parametrize("prec,N,gb", [("mixed", 128, 64), ("mixed", 128, 128), ("fp64", 64, 64)])
def test_small_blocks_form_every_partial_sum(prec, N, gb):
    """Grid kernels of 64- and 128-thread CTAs with 32 column groups (N = 128
    in FP32, vector width 4: more per-column outputs of a CTA's reduction
    than threads) follow the default shape's trajectory to rounding."""
    torch_mod()
    m = 10
    kw = dict(precision="mixed", cg_rtol=1e-6) if prec == "mixed" else dict(cg_rtol=1e-12)
    sd, _, _ = make(m, N, tau=0.4, **kw)
    st, _, _ = make(m, N, tau=0.4, grid_block=gb, grid_ctas=8, **kw)
    sd.step(3)
    st.step(3)
    Ud, Ut = sd.get_state()[0], st.get_state()[0]
    tol = 1e-4 if prec == "mixed" else 1e-10
    assert np.abs(Ud - Ut).max() <= tol * np.abs(Ud).max()


def test_tuned_launch_shape_keeps_the_trajectory(tmp_path):
    """hq_tune picks a candidate launch shape; a context using it follows the
    default-shape trajectory to rounding (only reduction orders change) and a
    batch of tuned contexts matches the same tuned contexts stepped alone."""
    torch_mod()
    m, N = 16, 8
    b, c = hq.tuned_shape(m, N, "fp64", cache=str(tmp_path / "tune.json"))
    assert b in (64, 128, 256) and c in (4, 8, 16, 32)
    assert hq.tuned_shape(m, N, "fp64", cache=str(tmp_path / "tune.json")) == (b, c)
    sd, _, _ = make(m, N, tau=0.4, cg_rtol=1e-12)
    st, _, _ = make(m, N, tau=0.4, cg_rtol=1e-12, grid_block=64, grid_ctas=4)
    sd.step(5)
    st.step(5)
    Ud, Ut = sd.get_state()[0], st.get_state()[0]
    assert np.abs(Ud - Ut).max() <= 1e-10 * np.abs(Ud).max()
    specs = [(12, 4, 64, 8), (16, 8, 128, 32)]
    pairs = []
    for m2, N2, gb, gc in specs:
        a, _, _ = make(m2, N2, tau=0.4, grid_block=gb, grid_ctas=gc)
        a2, _, _ = make(m2, N2, tau=0.4, grid_block=gb, grid_ctas=gc)
        pairs.append((a, a2))
    batch = hq.Batch([a for a, _ in pairs])
    batch.step(3)
    for a, a2 in pairs:
        a2.step(3)
        assert np.array_equal(a.get_state()[0], a2.get_state()[0])
