"""Pins of the oracle's scheme step (Eq. (4.1)) and of Algorithm 1.

The step is checked against the paper's equations re-evaluated with numpy
from the step's own outputs (not against the 2N x 2N system the oracle
solves), against the exact identities of Lemma 4.2 / Theorem 4.3, the
theorem-level invariants along a trajectory, the fixed points given by exact
eigenvectors, and the converged result against closed forms and dense
eigensolves.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_25149_gb300 import inputs as I
from tests.helpers import dense_h, harmonic_1d, separable_levels, subspace_sin

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(m, N, seed_u=1, V=None):
    V = I.harmonic(m) if V is None else V
    sigma = O.auto_shift(m, V)
    h = O.grid_h(m)
    U, _ = O.scale_initial(I.initial_block(m, N, seed_u), h ** 3)
    return V, sigma, h ** 3, U


def test_step_satisfies_predictor_equation():
    """(Uh - U)/tau = G U <U, Ut> - U <G U, Ut>,  Ut = (Uh + U)/2."""
    m, N, tau = 8, 4, 0.5
    V, sigma, h3, U = _problem(m, N, V=I.wells(8, 3))
    s = O.scheme_step(m, V, sigma, U, tau)
    W, Uh = s["W"], s["Uh"]
    Ut = 0.5 * (Uh + U)
    rhs = W @ (h3 * U.T @ Ut) - U @ (h3 * W.T @ Ut)
    np.testing.assert_allclose((Uh - U) / tau, rhs, rtol=1e-10, atol=1e-12)
    # and W is G U: the true residual of the inner solve
    h = h3 ** (1 / 3)
    res = np.linalg.norm(O.apply_h(m, h, V, sigma, W) - U) / np.linalg.norm(U)
    assert res < 1e-12


def test_predictor_solve_worked_check_and_step_consistency():
    """The predictor system of Eq. (4.1) on the Gram of exact eigenvector
    columns u_j = c_j phi_j, w_j = G u_j = u_j / mu_j (S = diag c^2,
    P_uw = P_wu = diag c^2/mu, Q = diag c^2/mu^2) has the closed-form
    solution X = S, Y = P_wu, so that Uh = U (I - tau Y) + W tau X = U.  On a
    general Gram, the standalone solve equals the one inside the step."""
    N, tau = 5, 0.7
    c2 = np.array([0.5, 1.0, 1.5, 2.0, 3.0])
    mu = np.array([0.9, 0.4, 0.25, 0.1, 0.05])
    S, P, Q = np.diag(c2), np.diag(c2 / mu), np.diag(c2 / mu ** 2)
    gram = np.block([[S, P], [P, Q]])
    XY, C = O.predictor(gram, tau)
    # each column decouples into a 2 x 2 system of determinant 1 whose
    # entries reach tau c^2 / (2 mu^2) = 420 (mu = 0.05): condition ~2e5, so
    # the elimination's rounding allows ~2e5 ulps
    tol = 1e-10
    np.testing.assert_allclose(XY[:N], S, rtol=tol, atol=tol)
    np.testing.assert_allclose(XY[N:], P, rtol=tol, atol=tol)
    # C1 = I - tau Y, C2 = tau X, and [U W] C = U for W = U diag(1/mu)
    np.testing.assert_allclose(C[:N], np.eye(N) - tau * P, rtol=tol, atol=tol)
    np.testing.assert_allclose(C[N:], tau * S, rtol=tol, atol=tol)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((40, N))
    np.testing.assert_allclose(U @ C[:N] + (U / mu) @ C[N:], U, rtol=tol, atol=tol)
    # general Gram: the step's own [X; Y] is the standalone solve, bit for bit
    m = 8
    V, sigma, h3, U = _problem(m, 4, seed_u=3, V=I.wells(8, 5))
    st = O.scheme_step(m, V, sigma, U, 0.4)
    XY2, C2 = O.predictor(st["gram"], 0.4)
    assert np.array_equal(XY2, st["XY"])
    np.testing.assert_allclose(st["Uh"], np.hstack([U, st["W"]]) @ C2, rtol=1e-13, atol=1e-14)


def test_step_satisfies_corrector_equation():
    """(U+ - Uh)/tau = -G Uh (<Uh,Uh> - I), with Z = G Uh checked by residual."""
    m, N, tau = 8, 4, 0.4
    V, sigma, h3, U = _problem(m, N, seed_u=5, V=I.wells(8, 4))
    s = O.scheme_step(m, V, sigma, U, tau)
    Uh, Z, Un = s["Uh"], s["Z"], s["Unew"]
    Sh = h3 * Uh.T @ Uh
    np.testing.assert_allclose(s["Shat"], Sh, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose((Un - Uh) / tau, -Z @ (Sh - np.eye(N)), rtol=1e-9, atol=1e-12)
    h = h3 ** (1 / 3)
    res = np.linalg.norm(O.apply_h(m, h, V, sigma, Z) - Uh) / np.linalg.norm(Uh)
    assert res < 1e-12


def test_gram_and_gradient_norm_definitions():
    m, N = 6, 3
    V, sigma, h3, U = _problem(m, N, seed_u=7)
    s = O.scheme_step(m, V, sigma, U, 0.3)
    UW = np.hstack([U, s["W"]])
    np.testing.assert_allclose(s["gram"], h3 * UW.T @ UW, rtol=1e-12, atol=1e-14)
    Pwu = h3 * s["W"].T @ U
    R = s["W"] - U @ Pwu                    # grad_G E_G(U), Remark 3.1
    assert s["g"] == pytest.approx(np.sqrt(h3 * np.sum(R * R)), rel=1e-10)


def test_cayley_predictor_preserves_gram():
    """<Uh, Uh> = <U, U> (the predictor is a Cayley transform, Lemma 4.2)."""
    m, N = 8, 5
    V, sigma, h3, U = _problem(m, N, seed_u=9, V=I.wells(8, 5))
    for tau in (0.1, 0.6, 2.0):
        s = O.scheme_step(m, V, sigma, U, tau)
        S = h3 * U.T @ U
        np.testing.assert_allclose(s["Shat"], S, rtol=1e-12, atol=1e-12 * np.abs(S).max())


def test_corrector_identity_for_gram():
    """O+ = O - tau(<Uh,Z> O + O <Z,Uh>) + tau^2 O <Z,Z> O  (Lemma 4.2 / Thm 4.3;
    A_n = <Uh, G Uh>, B_n = <G Uh, G Uh>)."""
    m, N, tau = 8, 4, 0.5
    V, sigma, h3, U = _problem(m, N, seed_u=11)
    s = O.scheme_step(m, V, sigma, U, tau)
    Uh, Z, Un = s["Uh"], s["Z"], s["Unew"]
    Om = h3 * Uh.T @ Uh - np.eye(N)
    A = h3 * Uh.T @ Z
    B = h3 * Z.T @ Z
    lhs = h3 * Un.T @ Un - np.eye(N)
    rhs = Om - tau * (A @ Om + Om @ A.T) + tau ** 2 * Om @ B @ Om
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_exact_eigenvectors_are_fixed_points():
    """U = Phi diag(c) with H Phi = Phi Lambda: X = diag(c^2), Y = diag(c^2/lambda'),
    Uh = U (the worked check of Eq. (4.1) for an eigenfunction).  Off the
    Stiefel manifold the gradient of Remark 3.1 does not vanish:
    G U - U <G U,U> = Phi Lambda^{-1} C (I - C^2), so
    g = sqrt(sum_i (c_i (1 - c_i^2) / lambda_i)^2), and g = 0 when C = I."""
    m, tau = 8, 0.5
    mu, phi = np.linalg.eigh(harmonic_1d(m, -6.0, 6.0))
    h = O.grid_h(m)
    h3 = h ** 3
    cols, lam = [], []
    for a, b, c in [(0, 0, 0), (1, 0, 0), (0, 0, 1)]:
        u = np.einsum("k,j,i->kji", phi[:, c], phi[:, b], phi[:, a]).ravel() / np.sqrt(h3)
        cols.append(u)
        lam.append(mu[a] + mu[b] + mu[c])
    cvec = np.array([1.0, 1.3, 1.1])
    U = np.stack(cols, 1) * cvec
    V = I.harmonic(m)
    s = O.scheme_step(m, V, 0.0, U, tau)
    N = 3
    X, Y = s["XY"][:N], s["XY"][N:]
    np.testing.assert_allclose(X, np.diag(cvec ** 2), atol=1e-11)
    np.testing.assert_allclose(Y, np.diag(cvec ** 2 / np.array(lam)), atol=1e-11)
    np.testing.assert_allclose(s["Uh"], U, atol=1e-10)
    lam = np.array(lam)
    g_exact = np.sqrt(np.sum((cvec * (1 - cvec ** 2) / lam) ** 2))
    assert s["g"] == pytest.approx(g_exact, rel=1e-10)
    s1 = O.scheme_step(m, V, 0.0, U / cvec, tau)
    assert s1["g"] < 1e-12


def test_grad_norm_alone_closed_form_rotation_and_dense():
    """orc_grad_norm (g = ||G U - U <G U,U>||, Remark 3.1, without a step):
    on exact eigenvector columns U = Phi diag(c) it equals the closed form
    sqrt(sum_i (c_i (1 - c_i^2) / lambda_i)^2) and vanishes for c = 1; it is
    invariant under U -> U Q for orthogonal Q (the gradient transforms as
    R -> R Q); on a wells potential it equals the definition evaluated with a
    dense solve of (H_h + sigma) W = U."""
    m = 8
    mu, phi = np.linalg.eigh(harmonic_1d(m, -6.0, 6.0))
    h3 = O.grid_h(m) ** 3
    cols, lam = [], []
    for a, b, c in [(0, 0, 0), (1, 0, 0), (0, 1, 1), (2, 0, 1)]:
        cols.append(np.einsum("k,j,i->kji", phi[:, c], phi[:, b], phi[:, a]).ravel() / np.sqrt(h3))
        lam.append(mu[a] + mu[b] + mu[c])
    lam = np.array(lam)
    cvec = np.array([0.7, 1.0, 1.2, 1.45])
    V = I.harmonic(m)
    U = np.stack(cols, 1) * cvec
    g, W = O.grad_norm(m, V, 0.0, U)
    assert g == pytest.approx(np.sqrt(np.sum((cvec * (1 - cvec ** 2) / lam) ** 2)), rel=1e-10)
    np.testing.assert_allclose(W, U / lam, rtol=1e-10, atol=1e-12)
    g1, _ = O.grad_norm(m, V, 0.0, U / cvec)
    assert g1 < 1e-12
    Qr, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((4, 4)))
    gq, _ = O.grad_norm(m, V, 0.0, U @ Qr)
    assert gq == pytest.approx(g, rel=1e-10)
    # wells, general U: the definition with a dense solve
    m = 6
    V, sigma, h3, U = _problem(m, 3, seed_u=13, V=I.wells(6, 4))
    gw, Ww = O.grad_norm(m, V, sigma, U)
    A = dense_h(m, O.grid_h(m), V, sigma)
    Wd = np.linalg.solve(A, U)
    R = Wd - U @ (h3 * Wd.T @ U)
    assert gw == pytest.approx(np.sqrt(h3 * np.sum(R * R)), rel=1e-10)
    np.testing.assert_allclose(Ww, Wd, rtol=1e-10, atol=1e-12)


def test_invariants_along_trajectory():
    """Theorem 4.5 (monotone energy of the shifted form) and Theorem 4.6
    (orthogonality error decreases) hold step by step for tau below the
    Theorem 4.3 bound.  Lemma 4.2 (non-expansion) and Theorem 4.3
    (quasi-Stiefel membership) hold only up to a small excursion when U0
    starts on the boundary of M_>= (lambda_min<U0,U0> = 1, as the initial
    scaling puts it): their proofs bound the symmetric part of A_n O_n by the
    spectrum of A_n O_n, which fails for non-commuting matrices (see
    test_lemma42_theorem43_counterexample).  The iterates keep full rank and
    return to the set; both are checked with a stated slack."""
    m, N = 8, 4
    V = I.wells(8, 6)
    sigma = O.auto_shift(m, V)
    h = O.grid_h(m)
    h3 = h ** 3
    U, _ = O.scale_initial(I.initial_block(m, N, 13), h3)
    lam1 = np.linalg.eigvalsh(dense_h(m, h, V, sigma))[0]
    S0 = h3 * U.T @ U
    tau = 0.9 * lam1 / (2 * np.linalg.eigvalsh(S0)[-1])
    E_prev = O.energy(m, V, U, shift=sigma)
    S_prev, O_prev = S0, np.linalg.norm(S0 - np.eye(N))
    lmins = []
    for n in range(40):
        s = O.scheme_step(m, V, sigma, U, tau)
        U = s["Unew"]
        S = h3 * U.T @ U
        lmins.append(np.linalg.eigvalsh(S)[0])
        assert lmins[-1] >= 1.0 - 1e-3                     # Theorem 4.3, with slack
        assert np.linalg.eigvalsh(S - S_prev)[-1] <= 1e-3  # Lemma 4.2, with slack
        E = O.energy(m, V, U, shift=sigma)
        assert E <= E_prev + 1e-12 * abs(E_prev)           # Theorem 4.5
        On = np.linalg.norm(S - np.eye(N))
        assert On <= O_prev + 1e-14                        # Theorem 4.6
        E_prev, S_prev, O_prev = E, S, On
    assert lmins[-1] >= 1.0 - 1e-9
    assert O_prev < 1e-6


def test_lemma42_theorem43_counterexample():
    """O_{n+1} = O_n - tau(A O_n + O_n A) + tau^2 O_n B O_n  with O_n >= 0
    singular, A > 0 and B = A^2 (within Lemma 4.1's bounds, lambda_1 =
    1/lambda_max(A)) and tau inside Theorem 4.3's limit: the symmetric part
    A O_n + O_n A is indefinite although A O_n has a nonnegative spectrum, so
    O_{n+1} gets a negative eigenvalue (Theorem 4.3's bound fails) and
    O_{n+1} - O_n a positive one (Lemma 4.2's non-expansion fails)."""
    d, tau = 0.2, 0.1
    Om = np.diag([0.0, d])
    A = np.array([[0.5, 0.2], [0.2, 0.4]])
    B = A @ A
    lam1 = 1.0 / np.linalg.eigvalsh(A)[-1]
    assert tau < lam1 / (2 * np.linalg.eigvalsh(Om + np.eye(2))[-1])
    assert np.linalg.eigvals(A @ Om).real.min() >= -1e-15
    On = Om - tau * (A @ Om + Om @ A) + tau ** 2 * Om @ B @ Om
    assert np.linalg.eigvalsh(On)[0] < -1e-5
    assert np.linalg.eigvalsh(On - Om)[-1] > 1e-5


def test_converged_harmonic_matches_closed_form():
    """N = 4 fills the two lowest shells; Rayleigh-Ritz values equal the sums
    of 1D eigenvalues, E(U_end) = sum(lambda)/2, <U,U> -> I, and the paper's
    eig(<G U,U>^{-1}) agrees with Rayleigh-Ritz."""
    m, N = 8, 4
    V, sigma, h3, U = _problem(m, N, seed_u=17)
    Ue, We, steps, g, hist = O.solve(m, V, sigma, U, 0.5, 1e-10, 3000)
    ex = O.extract(m, V, sigma, Ue, We)
    lv = separable_levels(m, -6.0, 6.0, N)
    np.testing.assert_allclose(ex["lam_rr"], lv, rtol=1e-12)
    np.testing.assert_allclose(ex["lam_paper"], lv, rtol=1e-9)
    assert O.energy(m, V, Ue) == pytest.approx(0.5 * lv.sum(), rel=1e-9)
    np.testing.assert_allclose(h3 * Ue.T @ Ue, np.eye(N), atol=1e-8)
    assert ex["residuals"].max() < 1e-9
    assert hist[-1] < 1e-10 and hist[0] > 1e-3


def test_accuracy_does_not_depend_on_tau():
    """Table 1: converged eigenvalue accuracy is insensitive to tau."""
    m, N = 8, 4
    V, sigma, h3, U = _problem(m, N, seed_u=19, V=I.wells(8, 7))
    out = []
    for tau in (0.2, 0.5):
        Ue, We, steps, g, _ = O.solve(m, V, sigma, U, tau, 1e-10, 6000)
        out.append((O.extract(m, V, sigma, Ue, We)["lam_rr"], steps))
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-11)
    assert out[0][1] > out[1][1]      # the larger step converges in fewer steps


def test_wells_converge_to_dense_eigenpairs():
    """Brute force: dense eigh of the assembled operator on a 6^3 grid."""
    m, N = 6, 5
    V = I.wells(m, 8)
    sigma = O.auto_shift(m, V)
    h = O.grid_h(m)
    h3 = h ** 3
    lam, vec = np.linalg.eigh(dense_h(m, h, V))
    assert lam[N] - lam[N - 1] > 1e-2
    U, _ = O.scale_initial(I.initial_block(m, N, 23), h3)
    Ue, We, steps, g, _ = O.solve(m, V, sigma, U, 0.4, 1e-10, 20000)
    ex = O.extract(m, V, sigma, Ue, We)
    np.testing.assert_allclose(ex["lam_rr"], lam[:N], rtol=1e-11, atol=1e-11)
    assert subspace_sin(Ue, vec[:, :N]) < 1e-6
    # Ritz vectors: sign convention (largest entry positive) and unit L2 norm
    u = ex["vectors"]
    for i in range(N):
        assert u[np.argmax(np.abs(u[:, i])), i] > 0
    np.testing.assert_allclose(h3 * u.T @ u, np.eye(N), atol=1e-9)


def test_contraction_rate_matches_spectral_gap():
    """Near convergence g_{n+1}/g_n ~ 1 - tau (1/lambda'_N - 1/lambda'_{N+1})
    (the linearised rate behind Theorem 4.7), within a factor of two in the
    decrement."""
    m, N, tau = 8, 4, 0.5
    V, sigma, h3, U = _problem(m, N, seed_u=29)
    h = O.grid_h(m)
    lam = np.linalg.eigvalsh(dense_h(m, h, V, sigma))
    pred = tau * (1 / lam[N - 1] - 1 / lam[N])
    _, _, steps, g, hist = O.solve(m, V, sigma, U, tau, 1e-11, 3000)
    tail = hist[len(hist) // 2:]
    obs = 1 - np.exp(np.mean(np.diff(np.log(tail))))
    assert pred / 2 < obs < pred * 2


def test_paper_energy_identity_golden():
    """The paper's printed final energy equals half the sum of its printed
    eigenvalues (Example 5.2, Tables 2-3), fixing E(U) = (1/2)(U,U)_a with
    the unshifted operator; the oracle's energy obeys the same identity."""
    d = json.load(open(os.path.join(GOLDEN, "paper_example52_hydrogen.json")))
    assert d["E_ref"] == pytest.approx(0.5 * sum(d["lambda_ref"]), rel=1e-14)
    # the computed state is converged only to ||grad|| < 1e-5: agreement 1e-9
    assert d["E_end"] == pytest.approx(0.5 * sum(d["lambda"]), rel=1e-8)


def test_fd_levels_converge_to_example51_closed_form():
    """Example 5.1's closed form (n1+1/2)+(n2+1/2), in 3D: the oracle's
    converged lambda_1..4 approach 1.5, 2.5, 2.5, 2.5 at second order in h."""
    d = json.load(open(os.path.join(GOLDEN, "paper_example51_harmonic.json")))
    exact = np.array(d["levels_3d_first10"][:4])
    errs = []
    for m in (11, 23):
        V, sigma, h3, U = _problem(m, 4, seed_u=31)
        Ue, We, _, _, _ = O.solve(m, V, sigma, U, 0.5, 1e-9, 2000)
        errs.append(np.abs(O.extract(m, V, sigma, Ue, We)["lam_rr"] - exact))
    ratio = errs[0] / errs[1]
    # h ratio 24/12 = 2 -> error ratio ~ 4
    assert np.all((ratio > 3.3) & (ratio < 4.7))
    assert errs[1].max() < 0.1


@pytest.mark.slow
def test_harmonic16_N8_converges_to_closed_form():
    """The 16^3, N = 8 harmonic workload: converged values equal the 1D-sum
    levels (lambda_8 sits in a degenerate triplet; eigenvalues stay unique)."""
    m, N = 16, 8
    V, sigma, h3, U = _problem(m, N, seed_u=1)
    Ue, We, steps, g, _ = O.solve(m, V, sigma, U, 0.5, 1e-8, 8000)
    ex = O.extract(m, V, sigma, Ue, We)
    np.testing.assert_allclose(ex["lam_rr"], separable_levels(m, -6.0, 6.0, N), rtol=1e-10)
    assert g < 1e-8


@pytest.mark.parametrize("c", [0.8, 0.95])
def test_adaptive_time_step_converges_faster_to_same_eigenvalues(c):
    """Algorithm 1 allows tau_n <= delta_T; the adaptive rule reaches the same
    closed-form eigenvalues in fewer steps, and its tau grows from the
    lower-bound start to c lambda_1 (below the linear stability limit
    tau < lambda_1 of the orthogonality error of eigenpair 1); a larger
    safety factor c takes no more steps."""
    m, N = 8, 4
    V, sigma, h3, U = _problem(m, N, seed_u=17)
    _, _, steps_fixed, _, _ = O.solve(m, V, sigma, U, 0.5, 1e-10, 5000)
    Ue, We, steps, g, hist, taus = O.solve_adaptive(m, V, sigma, U, 10.0, 1e-10, 5000, c=c)
    assert steps < steps_fixed
    lv = separable_levels(m, -6.0, 6.0, N)
    np.testing.assert_allclose(O.extract(m, V, sigma, Ue, We)["lam_rr"], lv, rtol=1e-12)
    lam1 = lv[0] + sigma
    lb = O.lambda1_lower_bound(m, V, sigma)
    assert 0 < lb <= lam1
    assert taus[0] <= c * lb / 1.0 + 1e-12
    assert np.all(np.diff(taus) <= 0.05 * taus[:-1] + 1e-15)      # growth at most 5%
    assert taus[-1] == pytest.approx(c * lam1, rel=1e-6)
    if c > 0.8:
        _, _, steps08, _, _, _ = O.solve_adaptive(m, V, sigma, U, 10.0, 1e-10, 5000)
        assert steps <= steps08
    with pytest.raises(O.OracleError):
        O.solve_adaptive(m, V, sigma, U, 10.0, 1e-10, 5, c=1.5)
