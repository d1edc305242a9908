"""GPU parity of the hot-path operations against the CPU oracle, element by
element, through the C ABI (FP64 contexts unless stated).  Sizes span several
CTAs with ragged tails (odd m, odd N) and the degenerate cases (N = 1,
single-level multigrid)."""
import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import inputs
from tests.gpu_common import dev, host, make, oracle_mg, rel, torch_mod

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.mark.parametrize("m,N", [(5, 1), (8, 3), (13, 17), (16, 8), (24, 64)])
def test_operator_matches_oracle(m, N):
    torch = torch_mod()
    s, V, _ = make(m, N)
    rng = np.random.default_rng(m * 7 + N)
    X = rng.standard_normal((m ** 3, N))
    Y = host(s.apply_operator(dev(X)))
    Yo = O.apply_h(m, inputs.grid_h(m), V, s.info()["sigma"], X)
    assert rel(Y, Yo) < TOL64


@pytest.mark.parametrize("m,N", [(9, 2), (16, 5), (20, 8)])
def test_multigrid_pieces_match_oracle(m, N):
    s, V, _ = make(m, N)
    mg = oracle_mg(s, V)
    assert s.levels() == mg.levels
    rng = np.random.default_rng(m + N)
    for l, ml in enumerate(mg.levels):
        np.testing.assert_allclose(host(s.mg_level_potential(l)), mg.level_potential(l),
                                   rtol=1e-14, atol=1e-14)
        r = rng.standard_normal((ml ** 3, N))
        z = rng.standard_normal((ml ** 3, N))
        assert rel(host(s.mg_smooth(l, dev(r), dev(z))), mg.smooth(l, r, z)) < TOL64
        if l + 1 < len(mg.levels):
            mc = mg.levels[l + 1]
            assert rel(host(s.mg_restrict(l, dev(r))), O.restrict(ml, mc, r)) < TOL64
            ec = rng.standard_normal((mc ** 3, N))
            assert rel(host(s.mg_prolong(l, dev(ec), dev(z))), O.prolong_add(mc, ml, ec, z)) < TOL64
    mc = mg.levels[-1]
    r = rng.standard_normal((mc ** 3, N))
    assert rel(host(s.mg_coarse_solve(dev(r))), mg.coarse_solve(r)) < 1e-11


@pytest.mark.parametrize("m,N", [(9, 2), (17, 5), (24, 8)])
def test_prescaled_sweep_matches_oracle_sweep(m, N):
    """The FP64 V-cycle's sweep from rt = omega D^-1 r (D = 6c + V_l + sigma,
    c = 1/(2 h_l^2)) equals the damped-Jacobi sweep of r on every level above
    the coarsest; the coarsest level and FP32 contexts refuse it."""
    from paper_2605_25149_gb300 import hq
    s, V, _ = make(m, N)
    mg = oracle_mg(s, V)
    om, sigma = s.cfg.mg_omega, s.info()["sigma"]
    rng = np.random.default_rng(3 * m + N)
    for l, ml in enumerate(mg.levels[:-1]):
        D = 6.0 / (2.0 * inputs.grid_h(ml) ** 2) + mg.level_potential(l) + sigma
        r = rng.standard_normal((ml ** 3, N))
        z = rng.standard_normal((ml ** 3, N))
        rt = (om / D)[:, None] * r
        got = host(s.mg_smooth_prescaled(l, dev(rt), dev(z)))
        assert rel(got, mg.smooth(l, r, z)) < TOL64, l
    mc = mg.levels[-1]
    with pytest.raises(hq.HQError) as ei:
        s.mg_smooth_prescaled(len(mg.levels) - 1, dev(np.zeros((mc ** 3, N))),
                              dev(np.zeros((mc ** 3, N))))
    assert ei.value.status == 1   # HQ_ERR_ARG
    t, _, _ = make(m, N, precision="mixed", cg_rtol=1e-6)
    z32 = dev(np.zeros((m ** 3, N), np.float32))
    with pytest.raises(hq.HQError) as ei:
        t.mg_smooth_prescaled(0, z32, z32.clone())
    assert ei.value.status == 2   # HQ_ERR_STATE


@pytest.mark.parametrize("m,N", [(9, 3), (16, 6), (20, 8), (33, 12)])
def test_mixed_transfers_match_oracle(m, N):
    """FP32 restriction and prolongation-with-correction on every level
    against the oracle's FP64 transfers of the same FP32 data; all three
    vector widths, nested and non-nested level pairs."""
    s, V, _ = make(m, N, precision="mixed", cg_rtol=1e-6)
    levels = s.levels()
    rng = np.random.default_rng(m * N)
    for l in range(len(levels) - 1):
        ml, mc = levels[l], levels[l + 1]
        r = rng.standard_normal((ml ** 3, N)).astype(np.float32)
        got = host(s.mg_restrict(l, dev(r)))
        assert rel(got, O.restrict(ml, mc, r.astype(np.float64))) < 2e-6, l
        ec = rng.standard_normal((mc ** 3, N)).astype(np.float32)
        z = rng.standard_normal((ml ** 3, N)).astype(np.float32)
        got = host(s.mg_prolong(l, dev(ec), dev(z)))
        ref = O.prolong_add(mc, ml, ec.astype(np.float64), z.astype(np.float64))
        assert rel(got, ref) < 2e-6, l


@pytest.mark.parametrize("m,N", [(3, 2), (16, 4), (21, 9)])
def test_vcycle_matches_oracle(m, N):
    s, V, _ = make(m, N)
    mg = oracle_mg(s, V)
    r = np.random.default_rng(5).standard_normal((m ** 3, N))
    assert rel(host(s.mg_vcycle(dev(r))), mg.vcycle(r)) < 1e-11


@pytest.mark.parametrize("m,N,k", [(12, 3, 1), (16, 8, 4), (19, 5, 6)])
def test_pcg_recurrence_matches_oracle_iteration_by_iteration(m, N, k):
    """rtol = 0: both sides run exactly k PCG iterations of the same recurrence."""
    s, V, _ = make(m, N)
    mg = oracle_mg(s, V)
    B = np.random.default_rng(7).standard_normal((m ** 3, N))
    X, its = s.block_pcg(dev(B), rtol=0.0, maxit=k)
    Xo, itso = mg.pcg(B, rtol=0.0, maxit=k)
    assert (its == k).all() and (itso == k).all()
    assert rel(host(X), Xo) < 1e-10


def test_pcg_converges_to_inverse_operator():
    m, N = 24, 6
    s, V, _ = make(m, N)
    sigma = s.info()["sigma"]
    B = np.random.default_rng(8).standard_normal((m ** 3, N))
    X, its = s.block_pcg(dev(B), rtol=1e-11, maxit=100)
    X = host(X)
    res = np.linalg.norm(B - O.apply_h(m, inputs.grid_h(m), V, sigma, X), axis=0)
    assert (res <= 1e-11 * np.linalg.norm(B, axis=0) * 1.0001).all()
    Xo, _ = O.cg(m, inputs.grid_h(m), V, sigma, B, rtol=1e-13)
    assert rel(X, Xo) < 1e-8
    mg = oracle_mg(s, V)
    _, itso = mg.pcg(B, rtol=1e-11, maxit=100)
    np.testing.assert_array_equal(its, itso)


@pytest.mark.parametrize("m,N,k", [(12, 1, 4), (12, 3, 1), (16, 8, 3), (19, 5, 6), (17, 40, 2)])
def test_coupled_block_pcg_matches_oracle_iteration_by_iteration(m, N, k):
    """O'Leary's block PCG, rtol = 0: both sides run exactly k iterations with
    the N x N step matrices (N = 40: the blocked elimination of the small
    solves instead of the one-CTA Cholesky)."""
    s, V, _ = make(m, N)
    mg = oracle_mg(s, V)
    B = np.random.default_rng(11 + N).standard_normal((m ** 3, N))
    X0 = np.random.default_rng(12).standard_normal((m ** 3, N)) * 1e-2
    X, its = s.block_pcg_coupled(dev(B), dev(X0), rtol=0.0, maxit=k)
    Xo, itso = mg.block_pcg(B, X0, rtol=0.0, maxit=k)
    assert its == k and itso == k
    assert rel(host(X), Xo) < 1e-10


def test_coupled_block_pcg_converges_with_the_oracle_count():
    m, N = 24, 12
    s, V, _ = make(m, N)
    sigma = s.info()["sigma"]
    B = np.random.default_rng(9).standard_normal((m ** 3, N))
    X, its = s.block_pcg_coupled(dev(B), rtol=1e-11, maxit=200)
    X = host(X)
    res = np.linalg.norm(B - O.apply_h(m, inputs.grid_h(m), V, sigma, X), axis=0)
    assert (res <= 2e-11 * np.linalg.norm(B, axis=0)).all()
    _, itso = oracle_mg(s, V).block_pcg(B, rtol=1e-11, maxit=200)
    assert abs(its - itso) <= 1
    # the block Krylov space holds every column's: no more iterations than
    # the slowest column of the per-column PCG
    _, itc = s.block_pcg(dev(B), rtol=1e-11, maxit=200)
    assert its <= itc.max()


def test_coupled_block_pcg_mixed_and_errors():
    from paper_2605_25149_gb300 import hq
    torch = torch_mod()
    m, N = 20, 8
    s, V, _ = make(m, N, precision="mixed", cg_rtol=1e-6)
    sigma = s.info()["sigma"]
    B = np.random.default_rng(4).standard_normal((m ** 3, N)).astype(np.float32)
    X, its = s.block_pcg_coupled(dev(B), rtol=1e-5, maxit=100)
    assert 0 < its < 100
    res = np.linalg.norm(B - O.apply_h(m, inputs.grid_h(m), V, sigma, host(X)), axis=0)
    assert (res <= 2e-5 * np.linalg.norm(B.astype(np.float64), axis=0)).all()
    with pytest.raises(hq.HQError) as ei:
        s.block_pcg_coupled(dev(B), rtol=1e-12, maxit=2)
    assert ei.value.status == 7   # HQ_ERR_NOT_CONVERGED
    with pytest.raises(hq.HQError) as ei:
        s.block_pcg_coupled(dev(B), rtol=-1.0, maxit=2)
    assert ei.value.status == 1   # HQ_ERR_ARG
    # a zero right-hand side is solved before the first iteration
    Z = torch.zeros((m ** 3, N), dtype=torch.float32, device="cuda")
    X, its = s.block_pcg_coupled(Z, rtol=1e-6, maxit=5)
    assert its == 0 and float(X.abs().max()) == 0.0


@pytest.mark.parametrize("m,Na,Nb", [(10, 3, 3), (16, 16, 9), (17, 70, 128), (12, 1, 5)])
def test_gram_matches_oracle(m, Na, Nb):
    N = max(Na, Nb)
    s, V, _ = make(m, (N + 1) // 2 if N > 1 else 1)
    rng = np.random.default_rng(Na * 31 + Nb)
    A = rng.standard_normal((m ** 3, Na))
    B = rng.standard_normal((m ** 3, Nb))
    w = inputs.grid_h(m) ** 3
    out = host(s.gram(dev(A), dev(B), w))
    assert rel(out, O.gram(A, B, w)) < TOL64
    outs = host(s.gram(dev(A), dev(A), w))     # symmetric path
    assert rel(outs, O.gram(A, A, w)) < TOL64


def test_determinism_bitwise():
    m, N = 16, 8
    outs = []
    for _ in range(2):
        s, V, U0 = make(m, N)
        s.step(2)
        outs.append(s.get_state()[0])
    np.testing.assert_array_equal(outs[0], outs[1])


# ---------------------------------------------------------------------------
# mixed precision (FP32 blocks, tcgen05 3xTF32 Gram)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m,N,Na", [(16, 4, 8), (16, 32, 64), (17, 65, 130), (24, 128, 256)])
def test_tensor_core_gram_matches_oracle(m, N, Na):
    """Symmetric Gram of an FP32 block on tcgen05 (kind::tf32, 3xTF32 split):
    relative error at FP32 level against the FP64 oracle of the same data."""
    torch = torch_mod()
    s, V, _ = make(m, N, precision="mixed", cg_rtol=1e-6)
    rng = np.random.default_rng(Na)
    A = rng.standard_normal((m ** 3, Na)).astype(np.float32)
    w = inputs.grid_h(m) ** 3
    Ad = dev(A)
    out = host(s.gram(Ad, Ad, w))          # same tensor twice: the tensor-core path
    ref = O.gram(A.astype(np.float64), A.astype(np.float64), w)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
    np.testing.assert_array_equal(out, out.T)
    # a second call is bit-identical (fixed-order reduction)
    np.testing.assert_array_equal(host(s.gram(Ad, Ad, w)), out)


def test_tensor_core_gram_has_no_accumulation_bias():
    """The tcgen05 FP32 accumulator truncates each addition relative to its
    own magnitude, so a Gram summed over thousands of points in one TMEM
    accumulator comes out biased low.  With every 32-point slice in a fresh
    accumulator and the slices summed in FP32 registers, a positive block
    (no cancellation: every entry accumulates the bias) of 110,592 points x
    512 columns (3,686 points per chunk) stays at FP32 level, unbiased."""
    torch_mod()
    m, N, Na = 48, 256, 512
    s, V, _ = make(m, N, precision="mixed", cg_rtol=1e-6)
    rng = np.random.default_rng(17)
    A = np.abs(rng.standard_normal((m ** 3, Na))).astype(np.float32)
    Ad = dev(A)
    out = host(s.gram(Ad, Ad, 1.0))        # same tensor twice: the tensor-core path
    A64 = A.astype(np.float64)
    ref = A64.T @ A64          # FP64 BLAS: its rounding is far below the bound tested
    relerr = (out - ref) / ref
    # measured on GB300: max 2.7e-7, mean -1.3e-7 (the bias of one slice);
    # one TMEM accumulator per chunk gave -5e-5 here
    assert np.abs(relerr).max() < 1e-6, np.abs(relerr).max()
    assert abs(relerr.mean()) < 3e-7, relerr.mean()


@pytest.mark.parametrize("m,N", [(8, 3), (16, 8), (33, 5)])
def test_mixed_operator_and_vcycle_match_oracle(m, N):
    s, V, _ = make(m, N, precision="mixed", cg_rtol=1e-6)
    torch = torch_mod()
    rng = np.random.default_rng(3)
    X = rng.standard_normal((m ** 3, N)).astype(np.float32)
    Y = host(s.apply_operator(dev(X)))
    Yo = O.apply_h(m, inputs.grid_h(m), V, s.info()["sigma"], X.astype(np.float64))
    assert rel(Y, Yo) < 1e-6
    mg = oracle_mg(s, V)
    Z = host(s.mg_vcycle(dev(X)))
    assert rel(Z, mg.vcycle(X.astype(np.float64))) < 1e-5


@pytest.mark.parametrize("prec,m,N,k1,k2,tol", [("fp64", 12, 8, 8, 8, 1e-13), ("fp64", 13, 17, 5, 0, 1e-13),
                                               ("mixed", 16, 64, 64, 64, 2e-6),
                                               ("mixed", 13, 24, 24, 7, 2e-6),
                                               ("mixed", 12, 80, 80, 0, 2e-6),
                                               ("mixed", 10, 9, 9, 9, 2e-6),
                                               ("mixed", 11, 40, 40, 33, 2e-6),
                                               ("mixed", 12, 256, 256, 256, 2e-6),
                                               ("mixed", 13, 128, 128, 128, 2e-6),
                                               ("mixed", 11, 128, 128, 0, 2e-6),
                                               ("mixed", 9, 256, 256, 40, 2e-6),
                                               ("mixed", 10, 128, 128, 7, 2e-6)])
def test_block_gemm_matches_numpy(prec, m, N, k1, k2, tol):
    """Out = A1 M1 + A2 M2 + Cin, the products of the predictor / corrector
    updates: SIMT FP64, or tcgen05 3xTF32 in mixed precision (ragged tile
    widths and K not a multiple of 32 included; 128 and 256 output columns
    with ragged point blocks)."""
    torch = torch_mod()
    s, V, _ = make(m, N, precision=prec, cg_rtol=1e-10 if prec == "fp64" else 1e-6)
    rng = np.random.default_rng(N + k1 + k2)
    dt = np.float64 if prec == "fp64" else np.float32
    n = m ** 3
    A1 = rng.standard_normal((n, k1)).astype(dt)
    M1 = rng.standard_normal((k1, N))
    A2 = rng.standard_normal((n, k2)).astype(dt) if k2 else None
    M2 = rng.standard_normal((k2, N)) if k2 else None
    Cin = rng.standard_normal((n, N)).astype(dt)
    out = host(s.block_gemm(dev(A1), dev(M1), None if A2 is None else dev(A2),
                            None if M2 is None else dev(M2), dev(Cin)))
    ref = A1.astype(np.float64) @ M1 + Cin.astype(np.float64)
    if k2:
        ref += A2.astype(np.float64) @ M2
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err < tol, err


@pytest.mark.parametrize("m,N,k1,k2", [(13, 64, 64, 64), (12, 40, 40, 0), (13, 17, 17, 9)])
def test_fp64_tensor_core_products_match_fp64(m, N, k1, k2):
    """FP64 block products on tensor cores (exact integer digit slicing) against
    numpy FP64 and the FP64 SIMT kernel: rows spanning 1e-9..1e3 in scale, a
    zero row, ragged point count and column tiles.  The error bound of the
    slicing is 2^-53 |row max| |column max| per term."""
    torch = torch_mod()
    rng = np.random.default_rng(m * N + k1 + k2)
    n = m ** 3
    A1 = rng.standard_normal((n, k1)) * np.exp(rng.uniform(-20, 7, (n, 1)))
    A1[5] = 0.0
    M1 = rng.standard_normal((k1, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    A2 = rng.standard_normal((n, k2)) * np.exp(rng.uniform(-20, 7, (n, 1))) if k2 else None
    M2 = rng.standard_normal((k2, N)) if k2 else None
    Cin = rng.standard_normal((n, N))
    ref = A1 @ M1 + Cin + (A2 @ M2 if k2 else 0.0)
    outs = []
    for tc in (2, 0):
        s, _, _ = make(m, N, fp64_tc=tc)
        outs.append(host(s.block_gemm(dev(A1), dev(M1), None if A2 is None else dev(A2),
                                      None if M2 is None else dev(M2), dev(Cin))))
    rowmax = np.abs(A1).max(axis=1, keepdims=True)
    colmax = np.abs(M1).max(axis=0, keepdims=True)
    if k2:
        rowmax = np.maximum(rowmax, np.abs(A2).max(axis=1, keepdims=True))
        colmax = np.maximum(colmax, np.abs(M2).max(axis=0, keepdims=True))
    bound = 4 * 2.0 ** -53 * (k1 + k2) * rowmax * colmax + 4 * 2.0 ** -53 * np.abs(ref)
    for out in outs:
        assert np.all(np.abs(out - ref) <= bound)
    assert np.array_equal(outs[0][5], (Cin + (A2 @ M2 if k2 else 0.0))[5]) or k2


@pytest.mark.parametrize("m,N", [(16, 64), (13, 9)])
def test_fp64_tensor_core_gram_matches_simt(m, N):
    """The Gram of [U W] of one step by digit slicing on tensor cores
    (fp64_tc = 2) against the FP64 SIMT Gram (fp64_tc = 0) on the same state:
    exactly symmetric, and equal to within 2^-50 |col max_i| |col max_j| n h^3."""
    torch_mod()
    grams, Ws = [], []
    for tc in (2, 0):
        s, V, U0 = make(m, N, fp64_tc=tc, cg_rtol=1e-12)
        tr = s.step_trace()
        grams.append(host(tr["gram"]))
        Ws.append(host(tr["W"]))
    g_tc, g_ref = grams
    assert np.array_equal(g_tc, g_tc.T)
    scale = np.sqrt(np.abs(np.diag(g_ref)))
    bound = 2.0 ** -44 * np.outer(scale, scale) * (m ** 3)
    assert np.all(np.abs(g_tc - g_ref) <= bound + 1e-14 * np.abs(g_ref).max())


@pytest.mark.parametrize("m,N,prec", [(16, 8, "mg32"), (8, 3, "mixed"), (20, 6, "mixed"),
                                      (33, 5, "mixed"), (48, 4, "mixed"), (24, 3, "mg32")])
def test_fused_coarse_vcycle_matches_separate_kernels(m, N, prec, monkeypatch):
    """The coarse levels of an FP32 V-cycle as one launch (one CTA per column,
    every level from about 16^3 points down in shared memory) against the
    same V-cycle as separate kernels (HQ_FUSED_COARSE=0): each operation
    repeats its separate kernel's expression, so the V-cycle and three steps
    of the scheme agree bit for bit.  Cases: the whole V-cycle fused (m <= 16),
    fused from level 1 (20, 33, 48), FP64 contexts with the FP32 preconditioner."""
    torch_mod()
    kw = dict(precision="mixed", cg_rtol=1e-6) if prec == "mixed" else dict(mg_fp32=1)
    outs = []
    for fused in (True, False):
        if fused:
            monkeypatch.delenv("HQ_FUSED_COARSE", raising=False)
        else:
            monkeypatch.setenv("HQ_FUSED_COARSE", "0")
        s, V, _ = make(m, N, **kw)
        rng = np.random.default_rng(m + N)
        X = rng.standard_normal((m ** 3, N))
        if prec == "mixed":
            X = X.astype(np.float32)
        z = host(s.mg_vcycle(dev(X)))
        s.profile()
        s.step(3)
        launches = s.profile_read()
        outs.append((z, s.get_state()[0], launches))
    (zf, uf, lf), (zs, us, ls) = outs
    np.testing.assert_array_equal(zf, zs)
    np.testing.assert_array_equal(uf, us)
    # the steps' V-cycles fuse below the finest level (mixed: the finest sweep
    # forms the PCG's dot products) once there are three levels or more
    nl, nf = sum(v[0] for v in ls.values()), sum(v[0] for v in lf.values())
    if len(s.levels()) >= 3:
        assert nf < nl, (nf, nl)
    else:
        assert nf == nl
