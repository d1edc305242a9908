"""ctypes binding of libhq (include/hq.h): argument marshalling only.

Every step of the eigensolver runs in libhq's CUDA kernels; PyTorch provides
the device workspace (one uint8 tensor) and the CUDA stream.  Importing this
module loads the in-tree ``_build/libhq.so`` and raises if it is missing:
there is no CPU fallback.

Host arrays are numpy FP64 arrays; device arrays are CUDA torch tensors of
the context's element type (float64 for ``precision="fp64"``, float32 for
``precision="mixed"`` where a call takes the working precision, float64 where
the header says FP64).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhq.so")

OK = 0
STATUS_NAMES = {
    0: "HQ_OK", 1: "HQ_ERR_ARG", 2: "HQ_ERR_STATE", 3: "HQ_ERR_CUDA", 4: "HQ_ERR_NOMEM",
    5: "HQ_ERR_BREAKDOWN", 6: "HQ_ERR_SINGULAR", 7: "HQ_ERR_NOT_CONVERGED",
    8: "HQ_ERR_TIMEOUT", 9: "HQ_ERR_NONFINITE",
}
FP64, MIXED = 0, 1

EXPORTED = [
    "hq_default_config", "hq_workspace_bytes", "hq_init", "hq_set_potential", "hq_set_initial",
    "hq_step", "hq_solve", "hq_eigenpairs", "hq_monitor", "hq_time_step", "hq_density",
    "hq_grad_eigs", "hq_grad_density", "hq_refine", "hq_get_state", "hq_set_state", "hq_problem_info",
    "hq_apply_operator", "hq_mg_vcycle", "hq_block_pcg", "hq_block_pcg_coupled", "hq_gram",
    "hq_block_gemm",
    "hq_step_trace",
    "hq_mg_smooth", "hq_mg_smooth_prescaled", "hq_mg_restrict", "hq_mg_prolong",
    "hq_mg_coarse_solve",
    "hq_mg_level_potential", "hq_gram_static", "hq_profile", "hq_profile_read", "hq_pcg_stats",
    "hq_last_error",
    "hq_status_string", "hq_destroy",
    "hq_tune_workspace_bytes", "hq_tune",
    "hq_batch_create", "hq_batch_solve", "hq_batch_step", "hq_batch_launches",
    "hq_batch_last_error", "hq_batch_destroy",
]
KERNEL_CLASSES = ["stencil", "residual", "smooth", "transfer", "coarse", "vector", "reduce", "gram",
                  "blockgemm", "small", "setup", "coarse_grids"]


class HQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int), ("lo", ctypes.c_double), ("hi", ctypes.c_double),
        ("nev", ctypes.c_int), ("tau", ctypes.c_double), ("shift", ctypes.c_double),
        ("precision", ctypes.c_int), ("cg_rtol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
        ("mg_nu1", ctypes.c_int), ("mg_nu2", ctypes.c_int), ("mg_coarsest", ctypes.c_int),
        ("mg_omega", ctypes.c_double), ("timeout_s", ctypes.c_double),
        ("z_warm_start", ctypes.c_int), ("adaptive_tau", ctypes.c_int),
        ("tau_max", ctypes.c_double), ("grid_block", ctypes.c_int), ("grid_ctas", ctypes.c_int),
        ("fp64_tc", ctypes.c_int), ("mg_fp32", ctypes.c_int), ("tau_safety", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_L = ctypes.c_long
_lib = None


def load():
    """Load libhq.so (built by paper_2605_25149_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhq.so is not built (%s); run "
                           "paper_2605_25149_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "hq_default_config": (None, [_P]),
        "hq_workspace_bytes": (ctypes.c_size_t, [_P]),
        "hq_init": (_I, [_P, _P, ctypes.c_size_t, _P, _P]),
        "hq_set_potential": (_I, [_P, _P, _I]),
        "hq_set_initial": (_I, [_P, _P, _I]),
        "hq_step": (_I, [_P, _I, _P]),
        "hq_solve": (_I, [_P, _D, _L, _P, _P]),
        "hq_eigenpairs": (_I, [_P, _P, _P, _P, _I, _P]),
        "hq_monitor": (_I, [_P, _P, _P, _P, _P]),
        "hq_time_step": (_I, [_P, _P]),
        "hq_density": (_I, [_P, _P, _I]),
        "hq_grad_eigs": (_I, [_P, _P, _P, _I]),
        "hq_grad_density": (_I, [_P, _P, _P, _I, _D, _I, _P, _P, _P]),
        "hq_refine": (_I, [_P, _I, _D, _I, _P, _P]),
        "hq_get_state": (_I, [_P, _P, _P, _I, _P]),
        "hq_set_state": (_I, [_P, _P, _P, _I, _L]),
        "hq_problem_info": (_I, [_P, _P, _P, _P, _P]),
        "hq_apply_operator": (_I, [_P, _P, _P, _I]),
        "hq_mg_vcycle": (_I, [_P, _P, _P]),
        "hq_block_pcg": (_I, [_P, _P, _P, _D, _I, _P]),
        "hq_block_pcg_coupled": (_I, [_P, _P, _P, _D, _I, _P]),
        "hq_gram": (_I, [_P, _P, _I, _P, _I, _D, _P]),
        "hq_block_gemm": (_I, [_P, _P, _I, _P, _P, _I, _P, _P, _P]),
        "hq_step_trace": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "hq_mg_smooth": (_I, [_P, _I, _P, _P, _P]),
        "hq_mg_smooth_prescaled": (_I, [_P, _I, _P, _P, _P]),
        "hq_mg_restrict": (_I, [_P, _I, _P, _P]),
        "hq_mg_prolong": (_I, [_P, _I, _P, _P, _P]),
        "hq_mg_coarse_solve": (_I, [_P, _P, _P]),
        "hq_mg_level_potential": (_I, [_P, _I, _P]),
        "hq_gram_static": (_I, [_P, _I, _P, _I, _L, _D, _P, _P]),
        "hq_profile": (_I, [_P, _I]),
        "hq_profile_read": (_I, [_P, _P, _P, _P]),
        "hq_pcg_stats": (_I, [_P, _P, _P]),
        "hq_last_error": (ctypes.c_char_p, [_P]),
        "hq_status_string": (ctypes.c_char_p, [_I]),
        "hq_destroy": (None, [_P]),
        "hq_tune_workspace_bytes": (ctypes.c_size_t, [_P]),
        "hq_tune": (_I, [_P, _P, ctypes.c_size_t, _P, _P, _P]),
        "hq_batch_create": (_I, [_P, _I, _P, _P]),
        "hq_batch_solve": (_I, [_P, _P, _L, _D, _P, _P, _P]),
        "hq_batch_step": (_I, [_P, _L, _P, _P]),
        "hq_batch_launches": (_I, [_P, _P, _P]),
        "hq_batch_last_error": (ctypes.c_char_p, [_P]),
        "hq_batch_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_config(m, nev, **kw) -> Config:
    c = Config()
    load().hq_default_config(ctypes.byref(c))
    c.m, c.nev = m, nev
    if "precision" in kw and isinstance(kw["precision"], str):
        kw["precision"] = {"fp64": FP64, "mixed": MIXED}[kw["precision"]]
    for k, v in kw.items():
        if v is None:
            continue
        setattr(c, k, v)
    return c


def workspace_bytes(cfg: Config) -> int:
    return int(load().hq_workspace_bytes(ctypes.byref(cfg)))


def tune(cfg: Config, stream=None):
    """hq_tune: (grid_block, grid_ctas, ms per PCG iteration) for cfg."""
    import torch
    lib = load()
    nbytes = int(lib.hq_tune_workspace_bytes(ctypes.byref(cfg)))
    if nbytes == 0:
        raise HQError(1, "invalid configuration")
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = ws.data_ptr()
    off = (-base) % 256
    stream = stream if stream is not None else torch.cuda.current_stream()
    out = Config()
    ms = ctypes.c_double()
    st = lib.hq_tune(ctypes.byref(cfg), ctypes.c_void_p(base + off), nbytes,
                     ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out), ctypes.byref(ms))
    del ws
    if st != OK:
        raise HQError(st, "hq_tune failed")
    return out.grid_block, out.grid_ctas, ms.value


def tuned_shape(m, nev, precision="fp64", cache=None, **cfg_kw):
    """(grid_block, grid_ctas) for this problem shape on this GPU: from the JSON
    cache (path `cache`, else $HQ_TUNE_CACHE, else ~/.cache/hq_tune.json), or
    measured by hq_tune and stored there."""
    import json
    import torch
    path = cache or os.environ.get("HQ_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "hq_tune.json")
    key = "%s|m=%d|N=%d|%s" % (torch.cuda.get_device_name(), m, nev, precision)
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        table = {}
    if key in table:
        e = table[key]
        return int(e["grid_block"]), int(e["grid_ctas"])
    b, c, ms = tune(default_config(m, nev, precision=precision, **cfg_kw))
    table[key] = {"grid_block": b, "grid_ctas": c, "ms_per_pcg_iteration": ms}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return b, c


def _dptr(t):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Solver:
    """One eigenproblem context (C handle hq_ctx) on the current CUDA device."""

    def __init__(self, m, nev, stream=None, **cfg_kw):
        import torch
        self._torch = torch
        self.lib = load()
        self.cfg = default_config(m, nev, **cfg_kw)
        nbytes = workspace_bytes(self.cfg)
        if nbytes == 0:
            raise HQError(1, "invalid configuration")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = ctypes.c_void_p()
        st = self.lib.hq_init(ctypes.byref(self.cfg), ctypes.c_void_p(base + off), nbytes,
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._ctx))
        if st != OK:
            raise HQError(st, "hq_init failed")
        self.m, self.N = m, nev
        self.n = m ** 3
        self.dtype = torch.float64 if self.cfg.precision == FP64 else torch.float32

    # -- plumbing ---------------------------------------------------------
    def _check(self, st, what):
        if st != OK:
            msg = self.lib.hq_last_error(self._ctx)
            raise HQError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self.lib.hq_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _host_f64(a, shape):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.size != int(np.prod(shape)):
            raise ValueError("expected %s values" % (shape,))
        return a

    def _buf(self, a, shape):
        """(pointer, on_device, keepalive) for an FP64 host array or CUDA tensor."""
        if hasattr(a, "is_cuda") and a.is_cuda:
            if a.dtype != self._torch.float64 or a.numel() != int(np.prod(shape)):
                raise ValueError("expected a float64 CUDA tensor of %s values" % (shape,))
            return _dptr(a), 1, a
        h = self._host_f64(a, shape)
        return _hptr(h), 0, h

    # -- the five calls of the problem statement ---------------------------
    def set_potential(self, V):
        p, dev, keep = self._buf(V, (self.n,))
        self._check(self.lib.hq_set_potential(self._ctx, p, dev), "hq_set_potential")

    def set_initial(self, U0):
        p, dev, keep = self._buf(U0, (self.n, self.N))
        self._check(self.lib.hq_set_initial(self._ctx, p, dev), "hq_set_initial")

    def step(self, nsteps=1):
        g = ctypes.c_double()
        self._check(self.lib.hq_step(self._ctx, nsteps, ctypes.byref(g)), "hq_step")
        return g.value

    def solve(self, eps, max_steps, raise_on_unconverged=True):
        steps, g = ctypes.c_long(), ctypes.c_double()
        st = self.lib.hq_solve(self._ctx, eps, max_steps, ctypes.byref(steps), ctypes.byref(g))
        if st == 7 and not raise_on_unconverged:
            return steps.value, g.value
        self._check(st, "hq_solve")
        return steps.value, g.value

    def eigenpairs(self, vectors=False, vectors_on_device=False):
        N = self.N
        lp, lr, res = np.empty(N), np.empty(N), np.empty(N)
        vec = None
        vptr = None
        if vectors:
            if vectors_on_device:
                vec = self._torch.empty((self.n, N), dtype=self._torch.float64, device="cuda")
                vptr = _dptr(vec)
            else:
                vec = np.empty((self.n, N))
                vptr = _hptr(vec)
        self._check(self.lib.hq_eigenpairs(self._ctx, _hptr(lp), _hptr(lr), vptr,
                                           1 if vectors_on_device else 0, _hptr(res)),
                    "hq_eigenpairs")
        return dict(lam_paper=lp, lam_rr=lr, vectors=vec, residuals=res)

    def density(self):
        """rho = sum_i u_i^2 of the Ritz vectors (host FP64 array)."""
        rho = np.empty(self.n)
        self._check(self.lib.hq_density(self._ctx, _hptr(rho), 0), "hq_density")
        return rho

    def grad_eigs(self, w=None):
        """sum_i w_i d lambda_i / dV (w = None: d(sum lambda)/dV)."""
        dV = np.empty(self.n)
        wh = None if w is None else self._host_f64(w, (self.N,))
        self._check(self.lib.hq_grad_eigs(self._ctx, _hptr(wh), _hptr(dV), 0), "hq_grad_eigs")
        return dV

    def grad_density(self, G=None, rho_target=None, rtol=1e-10, maxit=500):
        """dL/dV for a density loss: G = dL/drho, or the L2 mismatch to
        rho_target; returns (dV, loss, iterations)."""
        dV = np.empty(self.n)
        loss = ctypes.c_double()
        its = ctypes.c_int()
        Gh = None if G is None else self._host_f64(G, (self.n,))
        Th = None if rho_target is None else self._host_f64(rho_target, (self.n,))
        self._check(self.lib.hq_grad_density(self._ctx, _hptr(Gh), _hptr(Th), 0, rtol, maxit,
                                             _hptr(dV), ctypes.byref(loss), ctypes.byref(its)),
                    "hq_grad_density")
        return dV, loss.value, its.value

    def refine(self, rounds=2, rtol=1e-8, maxit=500):
        """FP64 residual refinement of span(U) (hq_refine): `rounds` Newton
        corrections of the Ritz pairs; returns (final residual norms
        ||H u_i - theta_i u_i|| as a host array, PCG iterations)."""
        res = np.empty(self.N)
        its = ctypes.c_int()
        self._check(self.lib.hq_refine(self._ctx, rounds, rtol, maxit, _hptr(res),
                                       ctypes.byref(its)), "hq_refine")
        return res, its.value

    def time_step(self):
        """tau_n of the last step taken."""
        t = ctypes.c_double()
        self._check(self.lib.hq_time_step(self._ctx, ctypes.byref(t)), "hq_time_step")
        return t.value

    def monitor(self):
        """Energy E(U), ||<U,U> - I||_F, extreme eigenvalues of <U,U>."""
        e, o, lo, hi = (ctypes.c_double() for _ in range(4))
        self._check(self.lib.hq_monitor(self._ctx, ctypes.byref(e), ctypes.byref(o),
                                        ctypes.byref(lo), ctypes.byref(hi)), "hq_monitor")
        return dict(energy=e.value, onorm=o.value, smin=lo.value, smax=hi.value)

    def get_state(self, with_warm_start=False, U_out=None, Z_out=None):
        """(U, Z or None, step).  U_out / Z_out: optional preallocated host
        FP64 arrays (e.g. pinned) to copy into."""
        U = np.empty((self.n, self.N)) if U_out is None else U_out
        Z = None
        if with_warm_start:
            Z = np.empty((self.n, self.N)) if Z_out is None else Z_out
        for a in (U, Z):
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous or
                                  a.size != self.n * self.N):
                raise ValueError("expected a C-contiguous float64 array of n x N values")
        step = ctypes.c_long()
        self._check(self.lib.hq_get_state(self._ctx, _hptr(U), _hptr(Z), 0, ctypes.byref(step)),
                    "hq_get_state")
        return U, Z, step.value

    def state_device(self):
        """The current block as a device FP64 tensor (n x N) and the step count."""
        U = self._torch.empty((self.n, self.N), dtype=self._torch.float64, device="cuda")
        step = ctypes.c_long()
        self._check(self.lib.hq_get_state(self._ctx, _dptr(U), None, 1, ctypes.byref(step)),
                    "hq_get_state")
        return U, step.value

    def set_state(self, U, step, Z=None):
        U = self._host_f64(U, (self.n, self.N))
        Zh = None if Z is None else self._host_f64(Z, (self.n, self.N))
        self._check(self.lib.hq_set_state(self._ctx, _hptr(U), _hptr(Zh), 0, step),
                    "hq_set_state")

    def set_state_device(self, U, step, Z=None):
        """hq_set_state from device FP64 tensors (n x N), e.g. the state of
        another context read with state_device()."""
        for t in (U, Z):
            if t is not None and (t.dtype != self._torch.float64 or not t.is_cuda or
                                  not t.is_contiguous() or t.numel() != self.n * self.N):
                raise ValueError("expected a contiguous CUDA float64 tensor of n x N values")
        self._check(self.lib.hq_set_state(self._ctx, _dptr(U), None if Z is None else _dptr(Z), 1,
                                          step), "hq_set_state")

    def info(self):
        h, s, L = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        ms = (ctypes.c_int * 24)()
        self._check(self.lib.hq_problem_info(self._ctx, ctypes.byref(h), ctypes.byref(s),
                                             ctypes.byref(L), ms), "hq_problem_info")
        return dict(h=h.value, sigma=s.value, levels=[ms[i] for i in range(L.value)])

    # -- kernel-level operations on device tensors -------------------------
    def _dev(self, t, rows, cols=None):
        cols = self.N if cols is None else cols
        if t.dtype != self.dtype or t.numel() != rows * cols:
            raise ValueError("expected %s tensor with %d x %d values" % (self.dtype, rows, cols))
        return _dptr(t)

    def apply_operator(self, x, ncol=None):
        ncol = self.N if ncol is None else ncol
        y = self._torch.empty_like(x)
        self._check(self.lib.hq_apply_operator(self._ctx, self._dev(x, self.n, ncol),
                                               _dptr(y), ncol), "hq_apply_operator")
        return y

    def mg_vcycle(self, r):
        z = self._torch.empty_like(r)
        self._check(self.lib.hq_mg_vcycle(self._ctx, self._dev(r, self.n), _dptr(z)),
                    "hq_mg_vcycle")
        return z

    def block_pcg(self, B, X0=None, rtol=1e-10, maxit=200):
        X = self._torch.zeros_like(B) if X0 is None else X0.clone()
        its = np.zeros(self.N, dtype=np.int32)
        self._check(self.lib.hq_block_pcg(self._ctx, self._dev(B, self.n), _dptr(X), rtol, maxit,
                                          _hptr(its)), "hq_block_pcg")
        return X, its

    def block_pcg_coupled(self, B, X0=None, rtol=1e-10, maxit=200):
        """O'Leary's block PCG (N x N step matrices): (X, iterations)."""
        X = self._torch.zeros_like(B) if X0 is None else X0.clone()
        its = ctypes.c_int()
        self._check(self.lib.hq_block_pcg_coupled(self._ctx, self._dev(B, self.n), self._dev(X, self.n),
                                                  rtol, maxit, ctypes.byref(its)),
                    "hq_block_pcg_coupled")
        return X, its.value

    def gram(self, A, B, w):
        Na, Nb = A.shape[1], B.shape[1]
        out = self._torch.empty((Na, Nb), dtype=self._torch.float64, device="cuda")
        self._check(self.lib.hq_gram(self._ctx, self._dev(A, self.n, Na), Na,
                                     self._dev(B, self.n, Nb), Nb, w, _dptr(out)), "hq_gram")
        return out

    def block_gemm(self, A1, M1, A2=None, M2=None, Cin=None):
        """Out = A1 M1 + A2 M2 (+ Cin) (device tensors; M's FP64)."""
        k1 = A1.shape[1]
        k2 = 0 if A2 is None else A2.shape[1]
        Out = self._torch.empty((self.n, self.N), dtype=self.dtype, device="cuda")
        self._check(self.lib.hq_block_gemm(
            self._ctx, self._dev(A1, self.n, k1), k1, _dptr(M1),
            None if A2 is None else self._dev(A2, self.n, k2), k2, _dptr(M2),
            None if Cin is None else self._dev(Cin, self.n), _dptr(Out)), "hq_block_gemm")
        return Out

    def step_trace(self):
        t = self._torch
        n, N = self.n, self.N
        o = dict(W=t.empty((n, N), dtype=self.dtype, device="cuda"),
                 gram=t.empty((2 * N, 2 * N), dtype=t.float64, device="cuda"),
                 g=t.empty(1, dtype=t.float64, device="cuda"),
                 XY=t.empty((2 * N, N), dtype=t.float64, device="cuda"),
                 Uh=t.empty((n, N), dtype=self.dtype, device="cuda"),
                 Shat=t.empty((N, N), dtype=t.float64, device="cuda"),
                 Z=t.empty((n, N), dtype=self.dtype, device="cuda"),
                 Unew=t.empty((n, N), dtype=self.dtype, device="cuda"))
        self._check(self.lib.hq_step_trace(self._ctx, *[_dptr(o[k]) for k in
                                                        ("W", "gram", "g", "XY", "Uh", "Shat",
                                                         "Z", "Unew")]), "hq_step_trace")
        return o

    def profile(self, timing=False):
        """Reset the launch counters; timing=True brackets launches with events."""
        self._check(self.lib.hq_profile(self._ctx, 1 if timing else 0), "hq_profile")

    def profile_read(self):
        """{class: (launches, ms, point-columns)} since the last profile() call."""
        n = len(KERNEL_CLASSES)
        la = (ctypes.c_long * n)()
        ms = (ctypes.c_double * n)()
        el = (ctypes.c_double * n)()
        self._check(self.lib.hq_profile_read(self._ctx, la, ms, el), "hq_profile_read")
        return {k: (la[i], ms[i], el[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def pcg_stats(self):
        """(solves, iterations) of the inner block PCG since profile()."""
        a, b = ctypes.c_long(), ctypes.c_long()
        self._check(self.lib.hq_pcg_stats(self._ctx, ctypes.byref(a), ctypes.byref(b)),
                    "hq_pcg_stats")
        return a.value, b.value

    def levels(self):
        return self.info()["levels"]

    def mg_smooth(self, level, r, zin):
        m = self.levels()[level]
        zout = self._torch.empty_like(zin)
        self._check(self.lib.hq_mg_smooth(self._ctx, level, self._dev(r, m ** 3),
                                          self._dev(zin, m ** 3), _dptr(zout)), "hq_mg_smooth")
        return zout

    def mg_smooth_prescaled(self, level, rt, zin):
        """The FP64 V-cycle's sweep from rt = omega D^-1 r (FP64 contexts)."""
        m = self.levels()[level]
        zout = self._torch.empty_like(zin)
        self._check(self.lib.hq_mg_smooth_prescaled(self._ctx, level, self._dev(rt, m ** 3),
                                                    self._dev(zin, m ** 3), _dptr(zout)),
                    "hq_mg_smooth_prescaled")
        return zout

    def mg_restrict(self, level, rf):
        ms = self.levels()
        rc = self._torch.empty((ms[level + 1] ** 3, self.N), dtype=self.dtype, device="cuda")
        self._check(self.lib.hq_mg_restrict(self._ctx, level, self._dev(rf, ms[level] ** 3),
                                            _dptr(rc)), "hq_mg_restrict")
        return rc

    def mg_prolong(self, level, ec, efin):
        ms = self.levels()
        efout = self._torch.empty_like(efin)
        self._check(self.lib.hq_mg_prolong(self._ctx, level, self._dev(ec, ms[level + 1] ** 3),
                                           self._dev(efin, ms[level] ** 3), _dptr(efout)),
                    "hq_mg_prolong")
        return efout

    def mg_coarse_solve(self, r):
        mc = self.levels()[-1]
        z = self._torch.empty_like(r)
        self._check(self.lib.hq_mg_coarse_solve(self._ctx, self._dev(r, mc ** 3), _dptr(z)),
                    "hq_mg_coarse_solve")
        return z

    def mg_level_potential(self, level):
        m = self.levels()[level]
        out = self._torch.empty(m ** 3, dtype=self._torch.float64, device="cuda")
        self._check(self.lib.hq_mg_level_potential(self._ctx, level, _dptr(out)),
                    "hq_mg_level_potential")
        return out


class Batch:
    """Several Solver contexts advanced together in one CUDA-graph launch per
    call (hq_batch_*).  The solvers must outlive the batch."""

    def __init__(self, solvers, stream=None):
        import torch
        self.lib = load()
        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._ctx.value for s in self.solvers])
        self._b = ctypes.c_void_p()
        st = self.lib.hq_batch_create(arr, len(self.solvers),
                                      ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(self._b))
        if st != OK:
            raise HQError(st, "hq_batch_create failed")

    def _check(self, st, what):
        if st != OK:
            msg = self.lib.hq_batch_last_error(self._b)
            raise HQError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def solve(self, eps, max_steps, timeout_s=0.0, raise_on_error=True):
        """Algorithm 1 for every member; returns (steps, g, status) arrays."""
        K = len(self.solvers)
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (K,)))
        steps = np.zeros(K, dtype=np.int64)
        g = np.zeros(K)
        stat = np.zeros(K, dtype=np.int32)
        st = self.lib.hq_batch_solve(self._b, _hptr(e), max_steps, timeout_s,
                                     steps.ctypes.data_as(ctypes.c_void_p), _hptr(g),
                                     stat.ctypes.data_as(ctypes.c_void_p))
        if raise_on_error:
            self._check(st, "hq_batch_solve")
        return steps, g, stat

    def step(self, nsteps=1, raise_on_error=True):
        """nsteps steps for every member; returns (g, status) arrays."""
        K = len(self.solvers)
        g = np.zeros(K)
        stat = np.zeros(K, dtype=np.int32)
        st = self.lib.hq_batch_step(self._b, nsteps, _hptr(g),
                                    stat.ctypes.data_as(ctypes.c_void_p))
        if raise_on_error:
            self._check(st, "hq_batch_step")
        return g, stat

    def launches(self):
        """(batch-level kernels, time-loop iterations) since creation."""
        a, b = ctypes.c_long(), ctypes.c_long()
        self._check(self.lib.hq_batch_launches(self._b, ctypes.byref(a), ctypes.byref(b)),
                    "hq_batch_launches")
        return a.value, b.value

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self.lib.hq_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def status_string(st: int) -> str:
    return load().hq_status_string(st).decode()
