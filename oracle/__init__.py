"""Plain FP64 CPU oracle of the quasi-orthogonal inverse-operator scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_2605_25149_gb300``)
and does not import it; the seeded input generators are the only module both
sides use.

The arithmetic lives in ``hq_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so x86_64 and aarch64 agree bit for bit).  This module
only compiles it, loads it with ctypes and marshals numpy arrays.

Every function cites the passage of Wang & Zhou (arXiv 2605.25149) that it
follows; the readings of passages the paper leaves open are stated in
``hq_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhq_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_SINGULAR, ERR_ARG, ERR_NOMEM = range(6)


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile hq_oracle.c into oracle/_build/libhq_oracle.so (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-shared",
           "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_long
_P = ctypes.c_void_p


def _sig(lib):
    spec = {
        "orc_grid_h": (_D, [_I, _D, _D]),
        "orc_apply_h": (None, [_I, _D, _P, _D, _I, _P, _P]),
        "orc_cg": (_I, [_I, _D, _P, _D, _I, _P, _P, _D, _I, _P]),
        "orc_mg_levels": (_I, [_I, _I, _P]),
        "orc_coarse_potential": (None, [_I, _P, _I, _P]),
        "orc_prolong_add": (None, [_I, _I, _I, _P, _P]),
        "orc_restrict": (None, [_I, _I, _I, _P, _P]),
        "orc_mg_create": (_P, [_I, _D, _D, _P, _D, _I, _I, _D, _I]),
        "orc_mg_destroy": (None, [_P]),
        "orc_mg_nlevels": (_I, [_P]),
        "orc_mg_level_m": (_I, [_P, _I]),
        "orc_mg_level_potential": (None, [_P, _I, _P]),
        "orc_mg_vcycle": (None, [_P, _I, _P, _P]),
        "orc_mg_smooth": (None, [_P, _I, _I, _P, _P]),
        "orc_mg_coarse_solve": (None, [_P, _I, _P, _P]),
        "orc_pcg_mg": (_I, [_P, _I, _P, _P, _D, _I, _P]),
        "orc_gram": (None, [_L, _I, _P, _I, _P, _D, _P]),
        "orc_lu_solve": (_I, [_I, _P, _I, _P]),
        "orc_predictor": (_I, [_I, _D, _P, _P, _P]),
        "orc_sym_eig": (_I, [_I, _P, _P, _P]),
        "orc_auto_shift": (_D, [_I, _D, _D, _P]),
        "orc_scale_initial": (_D, [_L, _I, _D, _P]),
        "orc_scheme_step": (_I, [_I, _D, _D, _P, _D, _I, _D, _D, _I, _P, _P, _P,
                                 _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "orc_grad_norm": (_I, [_I, _D, _D, _P, _D, _I, _D, _I, _P, _P, _P]),
        "orc_solve": (_I, [_I, _D, _D, _P, _D, _I, _D, _D, _I, _D, _L, _P, _P,
                           _P, _P, _P]),
        "orc_extract": (_I, [_I, _D, _D, _P, _D, _I, _P, _P, _P, _P, _P, _P]),
        "orc_lambda1_lower_bound": (_D, [_I, _D, _D, _P, _D]),
        "orc_solve_adaptive": (_I, [_I, _D, _D, _P, _D, _I, _D, _D, _D, _I, _D, _L, _P, _P,
                                    _P, _P, _P, _P]),
        "orc_energy": (_D, [_I, _D, _D, _P, _D, _I, _P]),
        "orc_grad_eigs": (_I, [_I, _D, _D, _I, _P, _P, _P]),
        "orc_grad_density": (_I, [_I, _D, _D, _P, _I, _P, _P, _P, _D, _I, _P, _P, _P]),
        "orc_refine": (_I, [_I, _D, _D, _P, _I, _P, _I, _D, _I, _P, _P, _P]),
        "orc_block_pcg_mg": (_I, [_P, _I, _P, _P, _D, _I, _P]),
    }
    for name, (res, args) in spec.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _sig(_lib)
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(st, what):
    if st != OK:
        names = {1: "breakdown", 2: "not converged", 3: "singular", 4: "bad argument",
                 5: "out of memory"}
        raise OracleError("%s: %s (status %d)" % (what, names.get(st, "?"), st))


# --------------------------------------------------------------------------
# grid and operator (Section 2; -Delta/2 + V scaling of Example 5.1)
# --------------------------------------------------------------------------
def grid_h(m, lo=-6.0, hi=6.0):
    return lib().orc_grid_h(m, lo, hi)


def apply_h(m, h, V, sigma, X):
    """Y = (H_h + sigma) X for a point-major (n, N) block."""
    V = _f64(V).ravel()
    X = _f64(X)
    X2 = X.reshape(m ** 3, -1)
    Y = np.empty_like(X2)
    lib().orc_apply_h(m, h, _ptr(V), sigma, X2.shape[1], _ptr(X2), _ptr(Y))
    return Y.reshape(X.shape)


def cg(m, h, V, sigma, B, X0=None, rtol=1e-13, maxit=10000):
    """Per-column CG for (H_h + sigma) X = B; returns (X, iterations)."""
    V = _f64(V).ravel()
    B = _f64(B).reshape(m ** 3, -1)
    X = np.zeros_like(B) if X0 is None else _f64(X0).reshape(B.shape).copy()
    its = np.zeros(B.shape[1], dtype=np.int32)
    st = lib().orc_cg(m, h, _ptr(V), sigma, B.shape[1], _ptr(B), _ptr(X), rtol, maxit,
                      _ptr(its))
    _check(st, "orc_cg")
    return X, its


def auto_shift(m, V, lo=-6.0, hi=6.0):
    """Garding shift sigma (reading of Section 2.2): 0 if H_h is already
    positive by the closed-form bound, else 1 - bound."""
    return lib().orc_auto_shift(m, lo, hi, _ptr(_f64(V).ravel()))


# --------------------------------------------------------------------------
# multigrid preconditioner (not in the paper; stated readings in hq_oracle.c)
# --------------------------------------------------------------------------
def mg_levels(m, coarsest=4):
    ms = np.zeros(32, dtype=np.int32)
    L = lib().orc_mg_levels(m, coarsest, _ptr(ms))
    return [int(x) for x in ms[:L]]


def coarse_potential(mf, Vf, mc):
    Vf = _f64(Vf).ravel()
    Vc = np.empty(mc ** 3)
    lib().orc_coarse_potential(mf, _ptr(Vf), mc, _ptr(Vc))
    return Vc


def prolong_add(mc, mf, Ec, Ef):
    """Ef + P Ec (trilinear interpolation, zero boundary)."""
    Ec = _f64(Ec).reshape(mc ** 3, -1)
    Ef = _f64(Ef).reshape(mf ** 3, -1).copy()
    lib().orc_prolong_add(mc, mf, Ec.shape[1], _ptr(Ec), _ptr(Ef))
    return Ef


def restrict(mf, mc, Rf):
    """((mc+1)/(mf+1))^3 P^T Rf."""
    Rf = _f64(Rf).reshape(mf ** 3, -1)
    Rc = np.empty((mc ** 3, Rf.shape[1]))
    lib().orc_restrict(mf, mc, Rf.shape[1], _ptr(Rf), _ptr(Rc))
    return Rc


class MG:
    """V-cycle hierarchy for H_h + sigma on one potential."""

    def __init__(self, m, V, sigma, lo=-6.0, hi=6.0, nu1=2, nu2=2, omega=0.8, coarsest=4):
        self.m, self.lo, self.hi, self.sigma = m, lo, hi, sigma
        V = _f64(V).ravel()
        self._h = lib().orc_mg_create(m, lo, hi, _ptr(V), sigma, nu1, nu2, omega, coarsest)
        if not self._h:
            raise OracleError("orc_mg_create failed (coarsest matrix not SPD?)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_mg_destroy(h)
            self._h = None

    @property
    def levels(self):
        return [lib().orc_mg_level_m(self._h, l) for l in range(lib().orc_mg_nlevels(self._h))]

    def level_potential(self, l):
        m = self.levels[l]
        out = np.empty(m ** 3)
        lib().orc_mg_level_potential(self._h, l, _ptr(out))
        return out

    def vcycle(self, R):
        R = _f64(R).reshape(self.m ** 3, -1)
        Z = np.empty_like(R)
        lib().orc_mg_vcycle(self._h, R.shape[1], _ptr(R), _ptr(Z))
        return Z

    def smooth(self, level, R, Z):
        m = self.levels[level]
        R = _f64(R).reshape(m ** 3, -1)
        Z = _f64(Z).reshape(m ** 3, -1).copy()
        lib().orc_mg_smooth(self._h, level, R.shape[1], _ptr(R), _ptr(Z))
        return Z

    def coarse_solve(self, R):
        m = self.levels[-1]
        R = _f64(R).reshape(m ** 3, -1)
        Z = np.empty_like(R)
        lib().orc_mg_coarse_solve(self._h, R.shape[1], _ptr(R), _ptr(Z))
        return Z

    def block_pcg(self, B, X0=None, rtol=1e-13, maxit=1000):
        """O'Leary's block PCG with this V-cycle (an alternative inner solver,
        not in the paper): N x N step matrices alpha = (P^T A P)^-1 Z^T R,
        beta = (Z^T R)^-1 Z'^T R'.  rtol = 0 runs exactly maxit iterations.
        Returns (X, iterations)."""
        B = _f64(B)
        X = np.zeros_like(B) if X0 is None else np.array(_f64(X0), copy=True)
        its = ctypes.c_int()
        st = lib().orc_block_pcg_mg(self._h, B.shape[1], _ptr(B), _ptr(X), rtol, maxit,
                                    ctypes.byref(its))
        _check(st, "orc_block_pcg_mg")
        return X, its.value

    def pcg(self, B, X0=None, rtol=1e-13, maxit=1000):
        """MG-preconditioned CG per column; rtol = 0 runs exactly maxit steps."""
        B = _f64(B).reshape(self.m ** 3, -1)
        X = np.zeros_like(B) if X0 is None else _f64(X0).reshape(B.shape).copy()
        its = np.zeros(B.shape[1], dtype=np.int32)
        st = lib().orc_pcg_mg(self._h, B.shape[1], _ptr(B), _ptr(X), rtol, maxit, _ptr(its))
        _check(st, "orc_pcg_mg")
        return X, its


# --------------------------------------------------------------------------
# inner products and small dense algebra (Section 2.1, Eq. (4.1))
# --------------------------------------------------------------------------
def gram(A, B, w):
    """w A^T B for point-major blocks A (n, Na), B (n, Nb), compensated sums."""
    A = _f64(A)
    B = _f64(B)
    A = A.reshape(A.shape[0], -1)
    B = B.reshape(B.shape[0], -1)
    out = np.empty((A.shape[1], B.shape[1]))
    lib().orc_gram(A.shape[0], A.shape[1], _ptr(A), B.shape[1], _ptr(B), w, _ptr(out))
    return out


def lu_solve(A, B):
    A = _f64(A).copy()
    B = _f64(B).copy()
    B2 = B.reshape(A.shape[0], -1)
    st = lib().orc_lu_solve(A.shape[0], _ptr(A), B2.shape[1], _ptr(B2))
    _check(st, "orc_lu_solve")
    return B2.reshape(B.shape)


def predictor(gram, tau):
    """Step 4 of Eq. (4.1) and the small matrices of its predictor update from
    the 2N x 2N Gram of [U W] (S, <U,W>, <W,U>, Q): the 2N x 2N predictor
    system solved by LU with partial pivoting, XY = [X; Y] (2N x N), and
    C = [I - tau Y; tau X] with Uh = [U W] C.  The routine the oracle's own
    step uses (orc_scheme_step)."""
    G = _f64(gram)
    N = G.shape[0] // 2
    XY = np.empty((2 * N, N))
    C = np.empty((2 * N, N))
    _check(lib().orc_predictor(N, tau, _ptr(G), _ptr(XY), _ptr(C)), "orc_predictor")
    return XY, C


def sym_eig(A):
    """Cyclic Jacobi: ascending eigenvalues and unit eigenvectors (columns)."""
    A = _f64(A)
    n = A.shape[0]
    ev = np.empty(n)
    V = np.empty((n, n))
    lib().orc_sym_eig(n, _ptr(A), _ptr(ev), _ptr(V))
    return ev, V


def scale_initial(U, h3):
    """U / sqrt(lambda_min(<U,U>)): puts U in the quasi-Stiefel set."""
    U = _f64(U).copy()
    f = lib().orc_scale_initial(U.shape[0], U.shape[1], h3, _ptr(U))
    return U, f


# --------------------------------------------------------------------------
# the scheme (Eq. (4.1)) and Algorithm 1
# --------------------------------------------------------------------------
def scheme_step(m, V, sigma, U, tau, lo=-6.0, hi=6.0, cg_rtol=1e-13, cg_maxit=20000,
                W0=None, Z0=None):
    """One step of Eq. (4.1).  Returns a dict with W = G U, the 2N x 2N Gram of
    [U W], g = ||G U - U <G U,U>||, [X; Y], Uh, Shat = <Uh,Uh>, Z = G Uh and
    Unew = U_{n+1}."""
    V = _f64(V).ravel()
    U = _f64(U)
    n, N = U.shape
    out = dict(W=np.empty((n, N)), gram=np.empty((2 * N, 2 * N)), g=ctypes.c_double(),
               XY=np.empty((2 * N, N)), Uh=np.empty((n, N)), Shat=np.empty((N, N)),
               Z=np.empty((n, N)), Unew=np.empty((n, N)),
               iters=np.zeros(2 * N, dtype=np.int32))
    W0 = None if W0 is None else _f64(W0)
    Z0 = None if Z0 is None else _f64(Z0)
    st = lib().orc_scheme_step(m, lo, hi, _ptr(V), sigma, N, tau, cg_rtol, cg_maxit,
                               _ptr(U), _ptr(W0), _ptr(Z0), _ptr(out["W"]), _ptr(out["gram"]),
                               ctypes.byref(out["g"]), _ptr(out["XY"]), _ptr(out["Uh"]),
                               _ptr(out["Shat"]), _ptr(out["Z"]), _ptr(out["Unew"]),
                               _ptr(out["iters"]))
    _check(st, "orc_scheme_step")
    out["g"] = out["g"].value
    return out


def grad_norm(m, V, sigma, U, lo=-6.0, hi=6.0, cg_rtol=1e-13, cg_maxit=20000):
    """g = ||G U - U <G U, U>|| (Remark 3.1), the quantity Algorithm 1 tests."""
    V = _f64(V).ravel()
    U = _f64(U)
    W = np.zeros_like(U)
    g = ctypes.c_double()
    st = lib().orc_grad_norm(m, lo, hi, _ptr(V), sigma, U.shape[1], cg_rtol, cg_maxit,
                             _ptr(U), _ptr(W), ctypes.byref(g))
    _check(st, "orc_grad_norm")
    return g.value, W


def solve(m, V, sigma, U0, tau, eps, max_steps, lo=-6.0, hi=6.0, cg_rtol=1e-13,
          cg_maxit=20000, allow_unconverged=False):
    """Algorithm 1 with fixed tau.  U0 must already be scaled (scale_initial).
    Returns (U_end, W_end = G U_end, steps, g_end, g_history)."""
    V = _f64(V).ravel()
    U = _f64(U0).copy()
    W = np.empty_like(U)
    steps = ctypes.c_long()
    g = ctypes.c_double()
    hist = np.full(max_steps + 1, np.nan)
    st = lib().orc_solve(m, lo, hi, _ptr(V), sigma, U.shape[1], tau, cg_rtol, cg_maxit, eps,
                         max_steps, _ptr(U), _ptr(W), ctypes.byref(steps), ctypes.byref(g),
                         _ptr(hist))
    if not (allow_unconverged and st == ERR_NOT_CONVERGED):
        _check(st, "orc_solve")
    return U, W, steps.value, g.value, hist[: steps.value + 1]


def lambda1_lower_bound(m, V, sigma, lo=-6.0, hi=6.0):
    """Closed-form lower bound of the smallest eigenvalue of H_h + sigma."""
    return lib().orc_lambda1_lower_bound(m, lo, hi, _ptr(_f64(V).ravel()), sigma)


def solve_adaptive(m, V, sigma, U0, tau_max, eps, max_steps, lo=-6.0, hi=6.0, cg_rtol=1e-13,
                   cg_maxit=20000, allow_unconverged=False, c=0.8):
    """Algorithm 1 with the adaptive time step (tau_n <= tau_max = delta_T):
    tau_n = min(delta_T, c lam_hat / lambda_max<U,U>, 1.05 tau_{n-1}), 0 < c <= 1.
    Returns (U_end, W_end, steps, g_end, g_history, tau_history)."""
    V = _f64(V).ravel()
    U = _f64(U0).copy()
    W = np.empty_like(U)
    steps = ctypes.c_long()
    g = ctypes.c_double()
    hist = np.full(max_steps + 1, np.nan)
    th = np.full(max_steps + 1, np.nan)
    st = lib().orc_solve_adaptive(m, lo, hi, _ptr(V), sigma, U.shape[1], tau_max, c, cg_rtol,
                                  cg_maxit, eps, max_steps, _ptr(U), _ptr(W), ctypes.byref(steps),
                                  ctypes.byref(g), _ptr(hist), _ptr(th))
    if not (allow_unconverged and st == ERR_NOT_CONVERGED):
        _check(st, "orc_solve_adaptive")
    return U, W, steps.value, g.value, hist[: steps.value + 1], th[: steps.value]


def extract(m, V, sigma, U, W, lo=-6.0, hi=6.0, want_vectors=True):
    """Eigenvalues as the paper defines them (eig <G U,U>^{-1}, Section 5,
    shifted back by sigma) plus FP64 Rayleigh-Ritz values, Ritz vectors and
    residuals ||H u_i - lambda_i u_i||."""
    V = _f64(V).ravel()
    U = _f64(U)
    W = _f64(W)
    n, N = U.shape
    lp = np.empty(N)
    lr = np.empty(N)
    vec = np.empty((n, N)) if want_vectors else None
    res = np.empty(N)
    st = lib().orc_extract(m, lo, hi, _ptr(V), sigma, N, _ptr(U), _ptr(W), _ptr(lp), _ptr(lr),
                           _ptr(vec), _ptr(res))
    _check(st, "orc_extract")
    return dict(lam_paper=lp, lam_rr=lr, vectors=vec, residuals=res)


def energy(m, V, U, shift=0.0, lo=-6.0, hi=6.0):
    """E(U) = (1/2)(U,U)_a (Section 2.2), with a = H_h + shift."""
    V = _f64(V).ravel()
    U = _f64(U)
    return lib().orc_energy(m, lo, hi, _ptr(V), shift, U.shape[1], _ptr(U))


# --------------------------------------------------------------------------
# differentiation through converged eigenpairs (not in the paper; the
# derivations are in the comments of orc_grad_eigs / orc_grad_density)
# --------------------------------------------------------------------------
def grad_eigs(m, U, w=None, lo=-6.0, hi=6.0):
    """d(sum_i w_i lambda_i)/dV = h^3 sum_i w_i u_i^2 for eigenvectors U
    (point-major n x N, <u_i,u_j> = delta_ij)."""
    U = _f64(U)
    n, N = U.shape
    wv = None if w is None else _f64(w).ravel()
    dV = np.empty(n)
    _check(lib().orc_grad_eigs(m, lo, hi, N, _ptr(U), _ptr(wv), _ptr(dV)), "orc_grad_eigs")
    return dV


def grad_density(m, V, U, lam, rho_target, rtol=1e-12, maxit=20000, lo=-6.0, hi=6.0):
    """Loss L = (1/2) h^3 |rho - rho_target|^2 with rho = sum_i u_i^2 and its
    gradient dL/dV by the adjoint solves (H - lambda_i) xi_i = Q (g u_i).
    Returns (dV, L, largest CG iteration count)."""
    V = _f64(V).ravel()
    U = _f64(U)
    n, N = U.shape
    lam = _f64(lam).ravel()
    rt = _f64(rho_target).ravel()
    dV = np.empty(n)
    L = ctypes.c_double()
    its = ctypes.c_int()
    st = lib().orc_grad_density(m, lo, hi, _ptr(V), N, _ptr(U), _ptr(lam), _ptr(rt), rtol, maxit,
                                _ptr(dV), ctypes.byref(L), ctypes.byref(its))
    _check(st, "orc_grad_density")
    return dV, L.value, its.value


def refine(m, V, U, rounds, rtol=1e-12, maxit=20000, lo=-6.0, hi=6.0):
    """FP64 residual refinement of span(U) (not in the paper; the final FP64
    refinement of a lower-precision result): per round, Rayleigh-Ritz pairs
    (theta_i, u_i), then Newton corrections t_i in the complement of span(U)
    from Q (H - theta_i) Q t_i = -(H u_i - theta_i u_i) by CG, U <- u + t; a
    last Rayleigh-Ritz returns (Ritz vectors, Ritz values, residual norms,
    largest CG count per round)."""
    V = _f64(V).ravel()
    U = np.array(_f64(U), copy=True)
    n, N = U.shape
    lam = np.zeros(N)
    res = np.zeros(N)
    its = np.zeros(max(rounds, 1), dtype=np.int32)
    st = lib().orc_refine(m, lo, hi, _ptr(V), N, _ptr(U), rounds, rtol, maxit, _ptr(lam),
                          _ptr(res), _ptr(its))
    _check(st, "orc_refine")
    return U, lam, res, its[:rounds]
