#!/usr/bin/env python3
"""Benchmark of the quasi-orthogonal inverse-operator eigensolver on GB300.

Workload (one replica per GPU): 64^3 finite-difference grid on [-6,6]^3,
V = |x|^2/2 minus 8 seeded Gaussian wells, N = 64 eigenpairs, tau = 0.4,
inner block PCG to relative residual 1e-10, plain FP64.  A "step" is one
step of Eq. (4.1): two multigrid-preconditioned block-PCG solves, the Gram of
[U W], the gradient norm, the predictor system, the predictor and corrector
updates.

Printed (rank 0, one JSON line): steps/s over K timed steps after W warm-up
steps (CUDA events on the solver's stream, barrier + synchronize on both
sides, max over ranks), the mixed-precision path on the same workload, the
time to residual 1e-8, a roofline entry for the dominant kernel class timed
live with CUDA events, an end-to-end figure through host buffers, SM clocks
sampled during the timed region and the CPU oracle timed on the host cores.

--impl reference times the CPU oracle (the reference arm of this build) on
the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-residual 1e-8 for N eigenpairs; stencil HBM GB/s; mixed vs FP64"
WORKLOAD = "wells64_N64"
# FP64 issue rate of GB300: 2 FMA / clk / SM x 152 SMs x 2.07 GHz x 2 flop
FP64_PEAK_GFLOPS = 2 * 152 * 2.07 * 2
# algorithmic cost per point-column written, per kernel class: (flops, words)
#   smooth   z' = z + omega D^-1 (r - A z): 6-neighbour sum (5 add), r + c s
#            (fma), (1-omega) z (mul), + wD (...) (fma): 10 flops; reads r, z,
#            writes z': 3 words
#   stencil  y = D x - c s: 5 add + mul + fma = 8 flops, + the per-column
#            partial x.y of the PCG operator (fma): 10 flops; reads x, writes
#            y: 2 words
#   residual (b - D x) + c s: 5 add + 2 fma = 9 flops; 3 words
ALGO = {"smooth": (10.0, 3.0), "stencil": (10.0, 2.0), "residual": (9.0, 3.0)}
# FP64 V-cycles sweep from the pre-scaled right-hand side rt = omega D^-1 r:
#   z' = (omega c D^-1) s + ((1 - omega) z + rt): 5 add + 2 fma = 9 flops in 7
#   FP64-pipe instructions; reads rt, z, writes z': 3 words
ALGO_F64 = dict(ALGO, smooth=(9.0, 3.0))
# FP64-pipe instructions per point-column (an add takes an issue slot as an FMA does)
FP64_OPS = {"smooth": 7.0, "stencil": 8.0, "residual": 7.0}
# DRAM bytes per point-column of the roofline kernels from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch / point-columns
# of that launch): keys (class, dtype); an entry is removed whenever its
# kernel changes, until it is captured again.
TRAFFIC_PER_ELEMENT = {("smooth", "f32"): (136.215040e6 + 44.029440e6) / 16777216,
                       ("stencil", "f64"): (136.446208e6 + 96.011008e6) / 16777216,
                       # the z-marching FP32 sweep (blocks of 100 MB or more),
                       # captured on 64^3 x 256 and scaled by point-columns
                       ("smooth_zm", "f32"): (553.649408e6 + 240.579328e6) / 67108864}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    """Maximum of a per-rank scalar over all ranks (the slowest replica)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, ms_per_step_max):
    """Whole-job steps/s: every rank advances its own replica by one step in
    ms_per_step_max (the slowest rank's time)."""
    return ws * 1000.0 / ms_per_step_max


def time_steps(torch, s, K, ws, label=None):
    """ms per step over K steps: events on the solver stream, barrier + sync.
    `label` names an NVTX range around the timed steps (for ncu --nvtx)."""
    st = s.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    if label:
        torch.cuda.nvtx.range_push(label)
    e0.record(st)
    g = s.step(K) if K > 0 else float("nan")
    e1.record(st)
    torch.cuda.synchronize()
    if label:
        torch.cuda.nvtx.range_pop()
    barrier(ws)
    return e0.elapsed_time(e1) / max(K, 1), g


GRID_CLASSES = ("stencil", "smooth", "residual")
KERNEL_NAME = {"stencil": "finest-level operator y = (H + sigma) x with per-column x.y partials "
                          "(k_stencil_zm for blocks of 100 MB or more, else k_stencil)",
               "smooth": "finest-level damped-Jacobi sweep (k_jacobi_zm for blocks of 100 MB or "
                         "more, else k_jacobi)",
               "residual": "finest-level residual sweep (k_stencil_zm / k_stencil, mode 1)"}


def dominant(prof):
    """The finest-level grid kernel class with the most in-step time."""
    cand = {k: v for k, v in prof.items() if k in GRID_CLASSES and v[1] > 0}
    return max(cand, key=lambda c: cand[c][1]) if cand else None


def roofline(prof, kind, dtype_tag):
    """In-step figures of kernel class `kind` from an instrumented region."""
    if kind not in prof or prof[kind][0] == 0:
        return None
    launches, ms, elems = prof[kind]
    flops_e, words_e = (ALGO_F64 if dtype_tag == "f64" else ALGO)[kind]
    w = 8 if dtype_tag == "f64" else 4
    t = ms / 1e3 / launches
    el = elems / launches
    return {"kernel": kind, "launches": launches, "ms_per_launch": ms / launches,
            "elements_per_launch": el, "share": ms / sum(v[1] for v in prof.values()),
            "gbs": words_e * w * el / t / 1e9, "tflops": flops_e * el / t / 1e12}


def kernel_alone(torch, s, kind, mg_prescaled, reps=40):
    """One finest-level kernel of the step timed alone: `reps` back-to-back
    launches through the C ABI on n x N blocks of the context's working
    precision (ping-pong between two blocks; the blocks exceed L2, so every
    launch streams from HBM), CUDA events on the context's stream around the
    whole sequence.  kind "stencil": hq_apply_operator with ncol = N (the PCG's
    operator launch); "smooth": hq_mg_smooth_prescaled for FP64 V-cycles, else
    hq_mg_smooth.  Returns ms per launch."""
    import ctypes
    n, N = s.n, s.N
    g = torch.Generator(device="cuda").manual_seed(7)
    r = torch.rand((n, N), generator=g, device="cuda", dtype=s.dtype)
    za = torch.rand((n, N), generator=g, device="cuda", dtype=s.dtype)
    zb = torch.empty_like(za)
    st = s.stream
    lib = s.lib
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    if kind == "stencil":
        calls = [lambda: lib.hq_apply_operator(s._ctx, P(za), P(zb), N),
                 lambda: lib.hq_apply_operator(s._ctx, P(zb), P(za), N)]
        name = "hq_apply_operator"
    else:
        fn, name = lib.hq_mg_smooth, "hq_mg_smooth"
        if mg_prescaled:
            fn, name = lib.hq_mg_smooth_prescaled, "hq_mg_smooth_prescaled"
        calls = [lambda: fn(s._ctx, 0, P(r), P(za), P(zb)),
                 lambda: fn(s._ctx, 0, P(r), P(zb), P(za))]
    for i in range(4):
        s._check(calls[i & 1](), name)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(reps):
        s._check(calls[i & 1](), name)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def roofline_alone(kind, ms_launch, n_el, dtype_tag, hbm_peak, hbm_kind, in_step):
    """Roofline entry of kernel class `kind` from its stand-alone launch time:
    FP64 kernels against the derived FP64 issue peak ("alu"), FP32 kernels
    against the measured HBM copy bandwidth."""
    flops_e, words_e = (ALGO_F64 if dtype_tag == "f64" else ALGO)[kind]
    w = 8 if dtype_tag == "f64" else 4
    t = ms_launch / 1e3
    tr = TRAFFIC_PER_ELEMENT.get((kind, dtype_tag))
    traffic = None if tr is None else tr * n_el
    out = {"kernel": "%s: %s" % (kind, KERNEL_NAME[kind]),
           "timing": "alone: back-to-back launches on the step's block shape, CUDA events; "
                     "inputs exceed L2",
           "ms_per_launch": ms_launch, "elements_per_launch": n_el, "traffic": traffic,
           "algorithmic_bytes": words_e * w * n_el, "algorithmic_flops": flops_e * n_el}
    if dtype_tag == "f64":
        achieved = flops_e * n_el / t / 1e12
        peak = FP64_PEAK_GFLOPS / 1e3
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz",
                    "hbm_gbs": words_e * w * n_el / t / 1e9,
                    "fp64_issue_frac": FP64_OPS[kind] * n_el / t / (FP64_PEAK_GFLOPS / 2 * 1e9)})
    else:
        achieved = words_e * w * n_el / t / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "peak_source": hbm_kind})
    out["in_step"] = in_step
    return out


def breakdown(prof, K):
    """Per kernel class: launches and event-timed ms per step, share."""
    tot = sum(v[1] for v in prof.values()) or 1.0
    return {k: {"launches_per_step": v[0] / K, "ms_per_step": v[1] / K,
                "share": v[1] / tot} for k, v in prof.items() if v[0] > 0}


def fd_harmonic_levels(m, N, lo=-6.0, hi=6.0):
    """The N lowest eigenvalues of the 7-point H_h for V = |x|^2/2: sums of
    three eigenvalues of the 1-D tridiagonal operator (separation of
    variables)."""
    import numpy as np
    h = (hi - lo) / (m + 1)
    x = lo + h * np.arange(1, m + 1)
    T = np.diag(1.0 / h ** 2 + 0.5 * x ** 2) - np.diag(np.full(m - 1, 0.5 / h ** 2), 1) \
        - np.diag(np.full(m - 1, 0.5 / h ** 2), -1)
    e = np.linalg.eigvalsh(T)[: min(m, N)]
    return np.sort((e[:, None, None] + e[None, :, None] + e[None, None, :]).ravel())[:N]


def ttr_small(torch, hq, inputs):
    """Algorithm 1 run to residual 1e-8 on the 16^3, N = 8 harmonic workload
    (fixed tau = 0.5): wall time from hq_solve entry (potential and U0
    already uploaded) to the converged flag, and the Rayleigh-Ritz error
    against the separable closed form."""
    import numpy as np
    V, U0, w = inputs.workload("harmonic16_N8")
    s = hq.Solver(w["m"], w["N"], **solver_kw(w))
    s.set_potential(V)
    s.set_initial(U0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, g = s.solve(w["eps"], 100000)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    lam = s.eigenpairs()["lam_rr"]
    ref = fd_harmonic_levels(w["m"], w["N"])
    out = {"value": el, "unit": "s", "steps": steps, "g": g, "eps": w["eps"], "how": "measured",
           "workload": "harmonic16_N8: 16^3, V=|x|^2/2, N=8, tau=0.5, FP64 block PCG with the "
                       "FP32 multigrid preconditioner",
           "eig_rel_err_vs_closed_form": float(np.max(np.abs(lam - ref) / np.abs(ref)))}
    # the same problem by the scheme and the final FP64 refinement: the mixed
    # scheme (fixed tau 0.5, inner rtol 1e-4) to g < 1e-3, the state handed to
    # the FP64 context above, refinement rounds to g < 1e-8 (a hand-over whose
    # refinement breaks down continues the scheme to a 3x lower g first)
    sm = hq.Solver(w["m"], w["N"], tau=w["tau"], cg_rtol=1e-4, precision="mixed")
    sm.set_potential(V)
    sm.set_initial(U0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n1, failed = 0, []
    for tgt in (1e-3, 3e-4, 1e-4, 3e-5):
        n, g1 = sm.solve(tgt, 100000)
        n1 += n
        U, st = sm.state_device()
        s.set_state_device(U, st)
        try:
            rounds, its, g = refine_to(torch, s, w["eps"])
            break
        except hq.HQError as err:
            if err.status not in (5, 7):
                raise
            failed.append(g1)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    lam = s.eigenpairs()["lam_rr"]
    out["mixed_refined"] = {
        "value": el, "unit": "s", "how": "measured", "scheme_steps": n1,
        "g_at_handoff": g1, "refine_rounds": rounds, "refine_pcg_iterations": its, "g": g,
        "converged": bool(g < w["eps"]), "failed_handoffs": failed,
        "eig_rel_err_vs_closed_form": float(np.max(np.abs(lam - ref) / np.abs(ref)))}
    return out


def solve_history(torch, s, eps, chunk, max_steps, lam_ref=None, stop_err=None, stall=None):
    """Algorithm 1 in chunks of at most `chunk` steps (consecutive hq_solve
    calls continue one trajectory).  Each chunk is timed with CUDA events on
    the solver stream; g and the Rayleigh-Ritz values are read after it
    (outside the timed region).  Stops at g < eps, at max_steps, at
    eigenvalue error <= stop_err against lam_ref, or when that error (g
    without lam_ref) has not dropped by 10% over `stall` chunks."""
    import numpy as np
    hist, steps, t = [], 0, 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    while steps < max_steps:
        torch.cuda.synchronize()
        e0.record(s.stream)
        n, g = s.solve(eps, min(chunk, max_steps - steps), raise_on_unconverged=False)
        e1.record(s.stream)
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        steps += n
        lam = s.eigenpairs()["lam_rr"]
        err = None if lam_ref is None else float(np.max(np.abs(lam - lam_ref) / np.abs(lam_ref)))
        hist.append({"steps": steps, "s": t, "g": g, "err": err, "tau": s.time_step(), "lam": lam})
        if g < eps or (stop_err is not None and err is not None and err <= stop_err):
            break
        key = "g" if lam_ref is None else "err"
        if stall and len(hist) > stall and hist[-1][key] > 0.9 * hist[-1 - stall][key]:
            break
    return hist


def first_below(hist, key, thr):
    for h in hist:
        if h[key] is not None and h[key] <= thr:
            return h
    return None


def run_ttr(args):
    """The long time-to-residual legs on the 64^3, N = 64 wells workload,
    scheme only (no refinement), adaptive time step, SM clocks sampled:
    the FP64 scheme (FP64 PCG, FP32 V-cycle) from U0 to g < 1e-8 (its
    Rayleigh-Ritz values are the reference), the mixed scheme to g < 2e-6
    handed device to device to the FP64 scheme and continued to g < 1e-8, and
    the steps and seconds each needs to eigenvalue error 1e-6."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2605_25149_gb300 import hq, inputs
    V, U0, w = inputs.workload(WORKLOAD)
    m, N = w["m"], w["N"]
    chunk = args.ttr_chunk
    common = dict(tau=w["tau"], adaptive_tau=1, tau_max=args.tau_max,
                  tau_safety=args.tau_safety)
    clk = ClockSampler(0)
    clk.start()
    s = hq.Solver(m, N, cg_rtol=w["cg_rtol"], precision="fp64", mg_fp32=1, **common, **nu_kw(w))
    s.set_potential(V)
    s.set_initial(U0)
    h64 = solve_history(torch, s, w["eps"], chunk, args.ttr_steps)
    lam_ref = h64[-1]["lam"]
    for h in h64:
        h["err"] = float(np.max(np.abs(h["lam"] - lam_ref) / np.abs(lam_ref)))
    del s
    torch.cuda.empty_cache()
    sm = hq.Solver(m, N, cg_rtol=args.mixed_rtol, precision="mixed", **common)
    sm.set_potential(V)
    sm.set_initial(U0)
    hmx = solve_history(torch, sm, 2e-6, chunk, args.ttr_steps, lam_ref=lam_ref)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U, st = sm.state_device()
    s4 = hq.Solver(m, N, cg_rtol=w["cg_rtol"], precision="fp64", mg_fp32=1, **common, **nu_kw(w))
    s4.set_potential(V)
    s4.set_state_device(U, st)
    torch.cuda.synchronize()
    t_hand = time.perf_counter() - t0
    h4 = solve_history(torch, s4, w["eps"], chunk, args.ttr_steps, lam_ref=lam_ref)
    clocks = clk.stop()

    def pick(hh):
        return [{k: v for k, v in h.items() if k != "lam"} for h in hh]

    a64, amx = first_below(h64, "err", 1e-6), first_below(hmx, "err", 1e-6)
    out = {"workload": WORKLOAD,
           "tau_rule": "adaptive, tau_max %g, safety factor %g" % (args.tau_max, args.tau_safety),
           "chunk": chunk, "eps": w["eps"], "clocks": clocks,
           "fp64": {"time_to_residual_s": h64[-1]["s"], "steps": h64[-1]["steps"],
                    "g": h64[-1]["g"], "to_err_1e-6": a64 and {"s": a64["s"], "steps": a64["steps"]}},
           "mixed": {"to_err_1e-6": amx and {"s": amx["s"], "steps": amx["steps"]},
                     "last": pick(hmx[-1:])[0], "cg_rtol": args.mixed_rtol},
           "speedup_mixed_vs_fp64_at_err_1e-6": (a64["s"] / amx["s"]) if (a64 and amx) else None,
           "mixed_then_fp64": {
               "time_to_residual_s": hmx[-1]["s"] + t_hand + h4[-1]["s"],
               "mixed_s": hmx[-1]["s"], "mixed_steps": hmx[-1]["steps"], "handover_s": t_hand,
               "fp64_s": h4[-1]["s"], "fp64_steps": h4[-1]["steps"], "g": h4[-1]["g"],
               "err": h4[-1]["err"]},
           "history": {"fp64": pick(h64), "mixed": pick(hmx), "fp64_after_mixed": pick(h4)}}
    print(json.dumps(out), flush=True)


def run_large_accuracy(args):
    """The 128^3, N = 256 mixed workload run for accuracy (not part of the
    default run): Algorithm 1 in mixed precision with the adaptive time step
    (tau_max 10) in chunks of 500 steps timed with CUDA events, until g <
    --large-g or --large-steps steps; after every 1000 steps (untimed) the
    FP64 Rayleigh-Ritz eigenpairs with their FP64 residual norms
    r_i = ||H u_i - lambda_i u_i||.  H is symmetric, so an eigenvalue lies
    within r_i of each Ritz value lambda_i (and lambda_i is an upper bound of
    the i-th eigenvalue): max_i r_i / |lambda_i| bounds the relative
    eigenvalue error without an FP64 reference run.  SM clocks sampled."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2605_25149_gb300 import hq, inputs
    V, U0, w = inputs.workload("wells128_N256")
    m, N = w["m"], w["N"]
    clk = ClockSampler(0)
    clk.start()
    s = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="mixed", adaptive_tau=1,
                  tau_max=args.tau_max)
    s.set_potential(V)
    s.set_initial(U0)
    del U0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    hist, steps, t, g = [], 0, 0.0, float("inf")
    while steps < args.large_steps and g >= args.large_g:
        torch.cuda.synchronize()
        e0.record(s.stream)
        n, g = s.solve(args.large_g, min(500, args.large_steps - steps),
                       raise_on_unconverged=False)
        e1.record(s.stream)
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        steps += n
        row = {"steps": steps, "s": t, "g": g, "tau": s.time_step()}
        if steps % 1000 == 0 or g < args.large_g or steps >= args.large_steps:
            ev = s.eigenpairs()
            lam, res = ev["lam_rr"], ev["residuals"]
            row.update({"max_rel_resid": float(np.max(res / np.abs(lam))),
                        "lam_first": lam[:3].tolist(), "lam_last": lam[-3:].tolist()})
        hist.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    clocks = clk.stop()
    print(json.dumps({"workload": "wells128_N256: 128^3 grid, V=|x|^2/2 + 8 wells "
                                  "(default_rng(3)), N=256, mixed, PCG rtol 1e-6, adaptive tau",
                      "steps": steps, "scheme_s": t, "g": g, "clocks": clocks,
                      "history": hist}), flush=True)


def bench_batched(torch, hq, inputs, K, W, tune=True):
    """The batched workload: 32 wells problems, grid sides in {32,48,64,96}^3
    and N in {16,32,64,128} (seeded), tau = 0.4, mixed precision, advanced
    together by hq_batch_step (one graph launch per call), with the default
    launch shape and with the shapes hq_tune picks per (m, N).  Compared with
    the same problems stepped one after another, mixed and plain FP64."""
    shapes = inputs.batch_shapes()
    probs = [inputs.batch_problem(k, m, N) for k, (m, N) in enumerate(shapes)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def make(shape_of):
        out = []
        for (m, N), (V, U0) in zip(shapes, probs):
            gb, gc = shape_of(m, N)
            s = hq.Solver(m, N, tau=0.4, cg_rtol=1e-6, precision="mixed", grid_block=gb,
                          grid_ctas=gc)
            s.set_potential(V)
            s.set_initial(U0)
            out.append(s)
        return out

    def time_batch(solvers, label):
        b = hq.Batch(solvers)
        b.step(W)
        for s in solvers:
            s.profile()
        k0, _ = b.launches()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(label)
        e0.record(b.stream)
        b.step(K)
        e1.record(b.stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        k1, _ = b.launches()
        launches = (k1 - k0) + sum(sum(v[0] for v in s.profile_read().values()) for s in solvers)
        return e0.elapsed_time(e1) / K, launches / K

    per_problem = []

    def seq(solvers, record=False):
        tot = 0.0
        for s in solvers:
            s.step(W)
            torch.cuda.synchronize()
            e0.record(s.stream)
            s.step(K)
            e1.record(s.stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / K
            if record:
                per_problem.append(t)
            tot += t
        return tot

    solvers = make(lambda m, N: (0, 0))
    ms_default, launches = time_batch(solvers, "batch_timed")
    ms_seq_mixed = seq(solvers, record=True)
    del solvers
    torch.cuda.empty_cache()
    out = {}
    if tune:
        cache = os.path.join(tempfile.gettempdir(), "hq_tune_bench_%d.json" % os.getpid())
        t0 = time.perf_counter()
        tuned = {(m, N): hq.tuned_shape(m, N, "mixed", cache=cache, tau=0.4, cg_rtol=1e-6)
                 for m, N in sorted(set(shapes))}
        t_tune = time.perf_counter() - t0
        try:
            os.unlink(cache)
        except OSError:
            pass
        solvers = make(lambda m, N: tuned[(m, N)])
        ms_tuned, launches_t = time_batch(solvers, "batch_tuned_timed")
        del solvers
        torch.cuda.empty_cache()
        out = {"tuned_ms_per_batch_step": ms_tuned, "tuning_s": t_tune,
               "tuned_shapes": {"%dx%d" % k: list(v) for k, v in tuned.items()}}
    else:
        ms_tuned = ms_default
    ms_seq_fp64 = 0.0
    for i, (m, N) in enumerate(shapes):
        s = hq.Solver(m, N, tau=0.4, cg_rtol=1e-10, precision="fp64")
        s.set_potential(probs[i][0])
        s.set_initial(probs[i][1])
        ms_seq_fp64 += seq([s])
        del s
    torch.cuda.empty_cache()
    # many small problems: 32 problems of the 16^3, N = 8 harmonic workload
    # (U0 from default_rng(3000 + k)) in one batch, against one of them alone
    Vh, _, wh = inputs.workload("harmonic16_N8")
    small = []
    for k in range(32):
        sh = hq.Solver(wh["m"], wh["N"], **solver_kw(wh))
        sh.set_potential(Vh)
        sh.set_initial(inputs.initial_block(wh["m"], wh["N"], 3000 + k))
        small.append(sh)
    ms_small_one = seq(small[:1])
    ms_small_batch, _ = time_batch(small, "batch_small_timed")
    del small
    torch.cuda.empty_cache()
    out["small_problems"] = {
        "problems": 32, "workload": "harmonic16_N8 (16^3, N = 8, FP64 PCG, FP32 multigrid "
                                    "preconditioner), U0 from default_rng(3000 + k)",
        "ms_per_batch_step": ms_small_batch, "ms_per_step_one_problem": ms_small_one,
        "problem_steps_per_s": 32 * 1000.0 / ms_small_batch,
        "speedup_vs_one_at_a_time": 32 * ms_small_one / ms_small_batch}
    ms_batch = min(ms_default, ms_tuned)
    pc = sum(m ** 3 * N for m, N in shapes)
    res = {"value": len(shapes) * 1000.0 / ms_batch, "unit": "problem-steps/s",
           "ms_per_batch_step": ms_batch, "default_ms_per_batch_step": ms_default,
           "problems": len(shapes), "point_columns": pc,
           "gpu_launches_per_batch_step": launches, "graph_launches_per_call": 1,
           "sequential_mixed_ms": ms_seq_mixed, "sequential_fp64_ms": ms_seq_fp64,
           "speedup_vs_sequential_mixed": ms_seq_mixed / ms_batch,
           "sequential_mixed_ms_by_shape": {
               "%dx%d" % k: round(sum(t for (mm, nn), t in zip(shapes, per_problem)
                                      if (mm, nn) == k), 3)
               for k in sorted(set(shapes))},
           "largest_problem_ms": max(per_problem),
           "speedup_vs_fp64": ms_seq_fp64 / ms_batch,
           "workload": "32 wells problems, sides/N drawn by default_rng(4) from "
                       "{32,48,64,96} x {16,32,64,128}; tau 0.4; mixed, PCG rtol 1e-6; "
                       "FP64 baseline: the same problems stepped one at a time, rtol 1e-10",
           "note": "per-step throughput; the mixed path reaches eigenvalue error 1e-6 in "
                   "the same number of steps as FP64 (mixed.to_eig_err_1e-6)"}
    res.update(out)
    return res


def bench_large(torch, hq, inputs, K, W, hbm_peak, hbm_kind, shape=(128, 256)):
    """The 128^3, N = 256 wells workload in mixed precision (FP32 blocks of
    2.15 GB: every grid kernel streams from HBM): ms per step, the smooth
    sweep timed alone against the HBM roofline, and the per-class split of
    an instrumented pass.  `shape` = (m, N) overrides the size (same
    potential family and seeds), e.g. for a profiler capture of a smaller
    case."""
    V, U0, w = inputs.workload("wells128_N256")
    if tuple(shape) != (w["m"], w["N"]):
        w = dict(w, m=shape[0], N=shape[1])
        V = inputs.wells(w["m"], w["potential"][1])
        U0 = inputs.initial_block(w["m"], w["N"], w["u0_seed"])
    m, N = w["m"], w["N"]
    s = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="mixed")
    s.set_potential(V)
    s.set_initial(U0)
    del U0
    for _ in range(W):
        s.step(1)
    ms, _ = time_steps(torch, s, K, 1, "large_timed")
    s.profile(timing=True)
    time_steps(torch, s, 1, 1)
    prof = s.profile_read()
    s.profile(timing=False)
    kind = dominant(prof) or "smooth"
    roof = roofline_alone(kind, kernel_alone(torch, s, kind, False, reps=10), m ** 3 * N, "f32",
                          hbm_peak, hbm_kind, roofline(prof, kind, "f32"))
    # the block (>= 100 MB) runs the z-marching sweep: its own capture
    zm = TRAFFIC_PER_ELEMENT.get((kind + "_zm", "f32"))
    roof["traffic"] = zm * m ** 3 * N if (zm is not None and 4 * m ** 3 * N >= 100e6) else None
    out = {"workload": "wells: %d^3 grid, V=|x|^2/2 + 8 wells (default_rng(3)), "
                       "N=%d, tau=0.4, mixed, PCG rtol 1e-6" % (m, N),
           "ms_per_step": ms, "value": 1000.0 / ms, "unit": "steps/s", "roofline": roof,
           "breakdown": breakdown(prof, 1),
           "workspace_gb": s.workspace.numel() / 1e9}
    del s
    torch.cuda.empty_cache()
    return out


def nu_kw(w):
    """Damped-Jacobi sweeps per level of a workload's V-cycle (default 2)."""
    return {"mg_nu1": w["mg_nu"], "mg_nu2": w["mg_nu"]} if w.get("mg_nu") else {}


def solver_kw(w):
    """Solver options of a workload."""
    kw = dict(tau=w["tau"], cg_rtol=w["cg_rtol"], precision=w["precision"], **nu_kw(w))
    if w.get("mg_fp32"):
        kw["mg_fp32"] = 1
    return kw


def refine_to(torch, s, eps, max_rounds=8, rtol=1e-2, maxit=1000):
    """FP64 residual refinement rounds (hq_refine) until the state passes
    Algorithm 1's stopping test g < eps (evaluated with an FP64 inner solve:
    hq_solve with max_steps = 0).  Each round is an inexact Newton step: its
    correction equations are solved to rtol (1e-2: on wells64_N64 from the
    g = 3e-4 hand-off, four rounds reach g = 1.3e-9 in 192 PCG iterations,
    against 367 at rtol 1e-6 for the same four rounds).  Returns (rounds,
    PCG iterations, g)."""
    rounds, its, g = 0, 0, float("inf")
    while rounds < max_rounds:
        _, k = s.refine(rounds=1, rtol=rtol, maxit=maxit)
        rounds += 1
        its += k
        _, g = s.solve(eps, 0, raise_on_unconverged=False)
        if g < eps:
            break
    return rounds, its, g


def ttr_live(torch, hq, inputs, args):
    """Time to residual 1e-8 on the 64^3, N = 64 wells workload, measured in
    this run (host wall clock between synchronisations, from hq_solve entry
    with the potential and U0 uploaded, to the state that passes Algorithm 1's
    stopping test g < 1e-8 in FP64).  Adaptive time step (tau_max 10) in every
    leg.

    mixed_refined: the mixed-precision scheme (inner PCG rtol 1e-4: the
      warm-started solves then take ~0.5 iterations on average and the
      scheme reaches the hand-over in the same number of steps as at 1e-6)
      until g < g_hand, the state handed device to device to an FP64 context
      (FP32 multigrid preconditioner), then FP64 residual refinement rounds
      (hq_refine) until g < 1e-8 (a hand-over whose refinement breaks down
      continues the scheme to a 3x lower g first; that time counts).  The
      refined eigenvalues are the FP64 reference of this run.
    mixed_to_err: the mixed scheme alone (inner rtol 1e-6) from U0 until its
      own Rayleigh-Ritz eigenvalues are within 1e-6 of the reference (the
      mixed form's stated accuracy), in chunks of 500 steps.
    fp64_refined: the same with the FP64 scheme (FP64 PCG, FP32 V-cycle)
      until g < g_hand, then refinement.  Its ms per step gives the FP64
      scheme's time to eigenvalue error 1e-6 at the mixed leg's step count
      (the two trajectories agree to rounding, so the step counts are equal;
      labelled projected)."""
    import numpy as np
    V, U0, w = inputs.workload(WORKLOAD)
    m, N, eps = w["m"], w["N"], w["eps"]
    g_hand = args.ttr_handoff
    common = dict(tau=w["tau"], adaptive_tau=1, tau_max=args.tau_max,
                  tau_safety=args.tau_safety)
    out = {"workload": "%s: %d^3 wells, N=%d" % (WORKLOAD, m, N), "eps": eps,
           "tau_rule": "adaptive, tau_max %g, safety factor %g" % (args.tau_max, args.tau_safety),
           "handoff_g": g_hand}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def leg(prec_kw, label):
        s = hq.Solver(m, N, **common, **prec_kw)
        s.set_potential(V)
        s.set_initial(U0)
        s64 = hq.Solver(m, N, cg_rtol=w["cg_rtol"], precision="fp64", mg_fp32=1, **common, **nu_kw(w))
        s64.set_potential(V)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(label)
        t0 = time.perf_counter()
        n1, scheme_s, failed = 0, 0.0, []
        # hand over at g_hand; if the refinement's inner solve breaks down (the
        # Ritz values not yet below the rest of the spectrum), continue the
        # scheme to a 3x lower g and hand over again (all time counted)
        for tgt in (g_hand, g_hand / 3, g_hand / 10, g_hand / 30):
            e0.record(s.stream)
            n, g1 = s.solve(tgt, 60000)
            e1.record(s.stream)
            e1.synchronize()
            n1 += n
            scheme_s += e0.elapsed_time(e1) / 1e3
            U, st = s.state_device()
            s64.set_state_device(U, st)
            t_hand = time.perf_counter()
            try:
                rounds, its, g = refine_to(torch, s64, eps)
                break
            except hq.HQError as err:
                if err.status not in (5, 7):   # breakdown / not converged
                    raise
                failed.append({"g_at_handoff": g1, "status": err.status})
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        torch.cuda.nvtx.range_pop()
        return s, s64, {"value": t1 - t0, "unit": "s", "how": "measured", "scheme_steps": n1,
                        "scheme_s": scheme_s, "scheme_ms_per_step": 1e3 * scheme_s / max(n1, 1),
                        "g_at_handoff": g1, "handoff_and_refine_s": t1 - t_hand,
                        "refine_rounds": rounds, "refine_pcg_iterations": its, "g": g,
                        "converged": bool(g < eps), "failed_handoffs": failed}

    sm, sr, res_m = leg(dict(precision="mixed", cg_rtol=args.ttr_mixed_rtol), "ttr_mixed")
    lam_ref = sr.eigenpairs()["lam_rr"]
    lam_hand = sm.eigenpairs()["lam_rr"]
    res_m["eig_err_at_handoff"] = float(np.max(np.abs(lam_hand - lam_ref) / np.abs(lam_ref)))
    res_m["mixed_cg_rtol"] = args.ttr_mixed_rtol
    out["mixed_refined"] = res_m
    del sr, sm
    torch.cuda.empty_cache()
    # the mixed scheme alone (inner rtol --mixed-rtol) from U0 until its
    # Rayleigh-Ritz eigenvalues are within 1e-6 of the refined values, in
    # chunks of 500 steps
    sm = hq.Solver(m, N, precision="mixed", cg_rtol=args.mixed_rtol, **common)
    sm.set_potential(V)
    sm.set_initial(U0)
    t, steps, err = 0.0, 0, float("inf")
    while err > 1e-6 and steps < 30000:
        torch.cuda.synchronize()
        e0.record(sm.stream)
        n, _ = sm.solve(1e-300, 500, raise_on_unconverged=False)
        e1.record(sm.stream)
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        steps += n
        lam = sm.eigenpairs()["lam_rr"]
        err = float(np.max(np.abs(lam - lam_ref) / np.abs(lam_ref)))
    out["mixed_to_eig_err_1e-6"] = {"s": t, "steps": steps, "err": err, "how": "measured",
                                    "reached": bool(err <= 1e-6), "mixed_cg_rtol": args.mixed_rtol}
    del sm
    torch.cuda.empty_cache()
    s64, sr64, res_f = leg(dict(precision="fp64", cg_rtol=w["cg_rtol"], mg_fp32=1, **nu_kw(w)), "ttr_fp64")
    lam64 = sr64.eigenpairs()["lam_rr"]
    res_f["eig_agreement_with_mixed_refined"] = float(np.max(np.abs(lam64 - lam_ref) /
                                                             np.abs(lam_ref)))
    res_f["fp64_cg_rtol"] = w["cg_rtol"]
    out["fp64_refined"] = res_f
    del s64, sr64
    torch.cuda.empty_cache()
    st = out["mixed_to_eig_err_1e-6"]["steps"]
    out["fp64_to_eig_err_1e-6"] = {"s": st * res_f["scheme_ms_per_step"] / 1e3, "steps": st,
                                   "how": "projected: the mixed leg's step count x the FP64 "
                                          "scheme's ms/step measured above"}
    out["speedup_mixed_vs_fp64_at_eig_err_1e-6"] = (out["fp64_to_eig_err_1e-6"]["s"] /
                                                    out["mixed_to_eig_err_1e-6"]["s"])
    out["speedup_mixed_refined_vs_fp64_refined"] = res_f["value"] / res_m["value"]
    return out


def bench_inner(torch, hq, V, U0, w, reps=3):
    """The inner solve (H + sigma) X = U of the step, from a zero start to the
    workload's rtol, with the per-column block PCG the step uses and with
    O'Leary's block PCG (N x N step matrices, one block Krylov space): time,
    iterations and launches of each.  Both host-driven (one synchronisation
    per iteration), so wall time brackets each solve."""
    import numpy as np
    m, N = w["m"], w["N"]
    s = hq.Solver(m, N, **solver_kw(w))
    s.set_potential(V)
    s.set_initial(U0)
    B = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
    rt = w["cg_rtol"]
    out = {"rtol": rt, "start": "zero", "rhs": "the initial block U_0"}
    for name, solve in (("per_column", lambda: s.block_pcg(B, rtol=rt, maxit=1000)),
                        ("oleary_block", lambda: s.block_pcg_coupled(B, rtol=rt, maxit=1000))):
        solve()
        s.profile(timing=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            X, its = solve()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        launches = sum(v[0] for v in s.profile_read().values()) / reps
        its = np.asarray(its)
        out[name] = {"ms": ms, "iterations_max": int(its.max()),
                     "iterations_mean": float(its.mean()), "launches": launches}
        del X
    out["oleary_speedup"] = out["per_column"]["ms"] / out["oleary_block"]["ms"]
    del s
    torch.cuda.empty_cache()
    return out


def bench_grad(torch, hq, inputs, n_fd=6):
    """The differentiation workload (64^3, N = 32, wells default_rng(5), FP64):
    converged eigenpairs (mixed scheme to g < 1e-4, then FP64 residual
    refinement to g < 1e-10 in an FP64 context), the target density of a second
    potential (default_rng(6)) the same way, then timed: d(sum lambda)/dV
    (hq_grad_eigs) and the adjoint of the density loss (hq_grad_density, rtol
    1e-11).  Central finite differences (h = 1e-6) of the refined eigenpairs of
    V +- h e_p at the first n_fd / 2 of the 20 points drawn by default_rng(505)
    check both gradients (the other half: the points of largest gradient)."""
    import numpy as np
    V, U0, w = inputs.workload("wells64_N32")
    m, N = w["m"], w["N"]
    h3 = inputs.grid_h(m) ** 3

    def converged(Vx, U0x):
        sm = hq.Solver(m, N, tau=0.4, cg_rtol=1e-6, precision="mixed", adaptive_tau=1, tau_max=10.0)
        sm.set_potential(Vx)
        sm.set_initial(U0x)
        sm.solve(1e-4, 60000)
        U, st = sm.state_device()
        s = hq.Solver(m, N, tau=0.4, cg_rtol=1e-10, mg_fp32=1)
        s.set_potential(Vx)
        s.set_state_device(U, st)
        refine_to(torch, s, 1e-10, rtol=1e-8, maxit=2000)
        return s

    t0 = time.perf_counter()
    s = converged(V, U0)
    s6 = converged(inputs.wells(m, 6), inputs.initial_block(m, N, 106))
    rho_t = s6.density()
    del s6
    torch.cuda.synchronize()
    t_conv = time.perf_counter() - t0
    Ud, st = s.state_device()
    _, g = s.solve(1e-10, 0, raise_on_unconverged=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ge = s.grad_eigs()
    torch.cuda.synchronize()
    t_eigs = time.perf_counter() - t0
    t0 = time.perf_counter()
    dV, L, its = s.grad_density(rho_target=rho_t, rtol=1e-11, maxit=4000)
    torch.cuda.synchronize()
    t_dens = time.perf_counter() - t0
    f = hq.Solver(m, N, tau=0.4, cg_rtol=1e-10, mg_fp32=1)
    # the first of the 20 seeded points (mostly far from the wells, where the
    # density is small) and the points of largest |d(sum lambda)/dV|
    seeded = np.random.default_rng(505).choice(m ** 3, 20, replace=False)[:n_fd // 2]
    pts = np.concatenate([seeded, np.argsort(-np.abs(ge))[:n_fd - len(seeded)]])
    fds, fdl = [], []
    for p in pts:
        vals = []
        for sgn in (1.0, -1.0):
            Vx = V.copy()
            Vx[p] += sgn * 1e-6
            f.set_potential(Vx)
            f.set_state_device(Ud, st)
            f.refine(rounds=2, rtol=1e-12, maxit=4000)
            rho = f.density()
            vals.append((np.sum(f.eigenpairs()["lam_rr"]), 0.5 * h3 * np.sum((rho - rho_t) ** 2)))
        fds.append((vals[0][0] - vals[1][0]) / 2e-6)
        fdl.append((vals[0][1] - vals[1][1]) / 2e-6)
    fds, fdl = np.array(fds), np.array(fdl)

    def errs(g_all, fd):
        # max |g - fd| over the points, relative to the gradient's largest
        # entry, and the largest relative error where |g| > 1e-3 max |g|
        scale = float(np.abs(g_all).max())
        gp = g_all[pts]
        big = np.abs(gp) > 1e-3 * scale
        rel = float(np.max(np.abs(gp - fd)[big] / np.abs(gp)[big])) if big.any() else None
        return float(np.abs(gp - fd).max() / scale), rel
    return {"workload": "wells64_N32: 64^3 grid, V=|x|^2/2 + 8 wells (default_rng(5)), N=32, FP64",
            "g_converged": g, "converge_s": t_conv,
            "grad_eigs_s": t_eigs, "grad_density_s": t_dens, "grad_density_pcg_iterations": its,
            "loss": L, "fd_points": int(len(pts)),
            "fd_err_grad_eigs": dict(zip(("max_abs_over_max_grad", "max_rel_where_large"),
                                         errs(ge, fds))),
            "fd_err_grad_density": dict(zip(("max_abs_over_max_grad", "max_rel_where_large"),
                                            errs(dV, fdl))),
            "how": "converged eigenpairs: mixed scheme to g < 1e-4, FP64 refinement to g < "
                   "1e-10; gradients timed with synchronisation on both sides; finite "
                   "differences h = 1e-6 of refined eigenpairs (all 20 points: "
                   "tests/test_gpu_adjoint_fullsize.py)"}


def run_hq(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as ge
    if rank == 0 or ws == 1:
        ge.build()
    barrier(ws)
    ge.build()
    from paper_2605_25149_gb300 import hq, inputs

    V, U0, w = inputs.workload(WORKLOAD)
    m, N = w["m"], w["N"]
    K, W = args.steps, args.warmup
    hbm_peak, hbm_kind = peaks()

    # ---- FP64 path: headline ------------------------------------------------
    s = hq.Solver(m, N, **solver_kw(w))
    s.set_potential(V)
    s.set_initial(U0)
    for _ in range(W):
        s.step(1)
    clk = ClockSampler(local)
    clk.start()
    s.profile(timing=False)
    ms, g = time_steps(torch, s, K, ws, "fp64_timed")
    launches = sum(v[0] for v in s.profile_read().values())
    clocks = clk.stop()
    ms = max_over_ranks(ws, ms)
    # instrumented region (per-class CUDA events) for the roofline
    s.profile(timing=True)
    ms_instr, _ = time_steps(torch, s, K, ws)
    prof = s.profile_read()
    pcg_solves, pcg_iters = s.pcg_stats()
    s.profile(timing=False)
    # the dominant kernel: with the FP32 preconditioner the FP64 operator
    # (k_stencil_zm, the largest single kernel of the step's launch list); the
    # smooth class there is the FP32 sweeps of every level, split over ~115
    # launches a step, with their own roofline in the mixed leg
    kind = "stencil" if w.get("mg_fp32") else dominant(prof)
    roof = roofline_alone(kind, kernel_alone(torch, s, kind, not w.get("mg_fp32")), m ** 3 * N,
                          "f64", hbm_peak, hbm_kind, roofline(prof, kind, "f64"))
    brk = breakdown(prof, K)
    # end to end through host buffers: state in from pinned host memory,
    # step, state and gradient norm back to pinned host memory
    Uh_host = torch.empty((m ** 3, N), dtype=torch.float64, pin_memory=True).numpy()
    Zh_host = torch.empty((m ** 3, N), dtype=torch.float64, pin_memory=True).numpy()
    _, _, stp = s.get_state(with_warm_start=True, U_out=Uh_host, Z_out=Zh_host)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        s.set_state(Uh_host, stp, Z=Zh_host)
        s.step(1)
        _, _, stp = s.get_state(with_warm_start=True, U_out=Uh_host, Z_out=Zh_host)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / max(K, 1)
    barrier(ws)
    e2e_s = max_over_ranks(ws, e2e_s)
    blk_bytes = m ** 3 * N * 8
    del s
    torch.cuda.empty_cache()

    # ---- time to residual (rank 0 of a single-GPU run) ---------------------------
    ttr = {}
    if not args.no_ttr:
        ttr["harmonic16_N8"] = ttr_small(torch, hq, inputs)
        if ws == 1:
            clk2 = ClockSampler(local)
            clk2.start()
            ttr[WORKLOAD] = ttr_live(torch, hq, inputs, args)
            ttr[WORKLOAD]["clocks"] = clk2.stop()

    # ---- FP64 with the FP64 V-cycle (mg_fp32 = 0) ---------------------------------
    v64 = None
    if not args.no_mixed:
        s3 = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64", **nu_kw(w))
        s3.set_potential(V)
        s3.set_initial(U0)
        for _ in range(W):
            s3.step(1)
        s3.profile(timing=False)
        ms3, _ = time_steps(torch, s3, K, ws)
        ms3 = max_over_ranks(ws, ms3)
        sol3, it3 = s3.pcg_stats()
        v64 = {"value": job_value(ws, ms3), "unit": "steps/s", "ms_per_step": ms3,
               "headline_speedup_over_this": ms3 / ms,
               "pcg_iterations_per_solve": it3 / max(sol3, 1),
               "dtype": "f64 throughout (FP64 multigrid V-cycle)",
               "note": "the same solve with an FP64 preconditioner; not the headline"}
        del s3
        torch.cuda.empty_cache()

    # ---- mixed-precision path on the same workload -----------------------------
    mixed = None
    if not args.no_mixed:
        sm = hq.Solver(m, N, tau=w["tau"], cg_rtol=args.mixed_rtol, precision="mixed")
        sm.set_potential(V)
        sm.set_initial(U0)
        for _ in range(W):
            sm.step(1)
        sm.profile(timing=False)
        ms_m, _ = time_steps(torch, sm, K, ws, "mixed_timed")
        ms_m = max_over_ranks(ws, ms_m)
        sm.profile(timing=True)
        time_steps(torch, sm, K, ws)
        prof_m = sm.profile_read()
        sm.profile(timing=False)
        kind_m = dominant(prof_m) or "smooth"
        mixed = {"value": job_value(ws, ms_m), "unit": "steps/s", "ms_per_step": ms_m,
                 "speedup_vs_fp64": ms / ms_m, "dtype": "f32 (FP64 small solve / extraction)",
                 "cg_rtol": args.mixed_rtol,
                 "roofline": roofline_alone(kind_m, kernel_alone(torch, sm, kind_m, False),
                                            m ** 3 * N, "f32", hbm_peak, hbm_kind,
                                            roofline(prof_m, kind_m, "f32")),
                 "breakdown": breakdown(prof_m, K)}
        del sm
        torch.cuda.empty_cache()

    # ---- 128^3, N = 256 in mixed precision ---------------------------------------
    large = None
    if not args.no_large:
        large = bench_large(torch, hq, inputs, max(1, min(K, 3)), max(1, min(W, 2)), hbm_peak,
                            hbm_kind, tuple(args.large_shape))

    # ---- batched form ---------------------------------------------------------
    batched = None
    if not args.no_batch:
        batched = bench_batched(torch, hq, inputs, max(1, min(K, 3)), max(1, min(W, 1)),
                                tune=not args.no_tune)

    # ---- inner solver: per-column against O'Leary's block PCG --------------------
    inner = None
    if not args.no_inner:
        inner = bench_inner(torch, hq, V, U0, w)

    # ---- differentiation workload (64^3, N = 32) ------------------------------
    grad = None
    if not args.no_grad:
        grad = bench_grad(torch, hq, inputs)
        torch.cuda.empty_cache()

    # ---- CPU oracle on the host cores (rank 0, N = 1) ------------------------
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(V, U0, w, steps=1)
        if not args.no_ttr:
            cpu["time_to_residual"] = cpu_ttr_small()

    value = job_value(ws, ms)
    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s: %d^3 grid on [-6,6]^3, V=|x|^2/2 + 8 seeded Gaussian wells, "
                               "N=%d, tau=%g, FP64 block PCG to rtol %g with an FP32 multigrid "
                               "preconditioner, FP64 step algebra"
                               % (WORKLOAD, m, N, w["tau"], w["cg_rtol"]),
                   "n_points": m ** 3, "nev": N, "parallelism": "replicas (one problem per GPU)",
                   "l2": "working set %.2f GB per GPU > 126 MB L2; no flush needed" %
                         (9 * blk_bytes / 1e9)},
        "time_to_residual": ttr,
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "ms_per_step_instrumented": ms_instr,
        "pcg_iterations_per_solve": pcg_iters / max(pcg_solves, 1),
        "breakdown": brk,
        "e2e": {"value": ws / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": 2 * blk_bytes,
                "d2h_bytes_per_step": 2 * blk_bytes + 8,
                "how": "hq_set_state from pinned host (U and warm start), hq_step, "
                       "hq_get_state to pinned host, every step"},
        "mixed": mixed,
        "fp64_fp64_vcycle": v64,
        "large": large,
        "batched": batched,
        "differentiation": grad,
        "inner_solvers": inner,
        "cpu_baseline": cpu,
        "gradient_norm_last": g,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(V, U0, w, steps):
    """Time the CPU oracle's scheme step on this workload (bounded sample)."""
    import numpy as np

    import oracle as O
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    m, N = w["m"], w["N"]
    h = O.grid_h(m)
    sigma = O.auto_shift(m, V)
    U, _ = O.scale_initial(U0, h ** 3)
    Zprev = None
    t0 = time.perf_counter()
    for _ in range(steps):
        o = O.scheme_step(m, V, sigma, U, w["tau"], cg_rtol=w["cg_rtol"], W0=Zprev)
        U, Zprev = o["Unew"], o["Z"]
    el = time.perf_counter() - t0
    return {"value": steps / el, "unit": "steps/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample": "%d step(s) of Eq. (4.1) on the full %s workload "
                                        "(plain CG inner solves, rtol %g)" % (steps, WORKLOAD, w["cg_rtol"]),
            "seconds": el}


def cpu_ttr_small():
    """The oracle's Algorithm 1 to residual 1e-8 on the 16^3, N = 8 harmonic
    workload (same tau, tolerances and U0 as the GPU run)."""
    import oracle as O
    from paper_2605_25149_gb300 import inputs
    V, U0, w = inputs.workload("harmonic16_N8")
    m = w["m"]
    U, _ = O.scale_initial(U0, O.grid_h(m) ** 3)
    sigma = O.auto_shift(m, V)
    t0 = time.perf_counter()
    _, _, steps, g, _ = O.solve(m, V, sigma, U, w["tau"], w["eps"], 100000, cg_rtol=w["cg_rtol"])
    out = {"value": time.perf_counter() - t0, "unit": "s", "steps": steps, "g": g,
           "workload": "harmonic16_N8", "how": "measured"}
    # the scheme (FP64, as the oracle computes) to g < 1e-3, then the
    # oracle's refinement rounds (inner rtol 1e-2) to g < 1e-8: the GPU's
    # scheme-plus-refinement path on the host cores
    t0 = time.perf_counter()
    Uc, n1, failed = U, 0, []
    for tgt in (1e-3, 3e-4, 1e-4, 3e-5):
        Uc, _, n, g1, _ = O.solve(m, V, sigma, Uc, w["tau"], tgt, 100000, cg_rtol=w["cg_rtol"])
        n1 += n
        Ur, rounds, g = Uc, 0, g1
        try:
            while g >= w["eps"] and rounds < 8:
                Ur, _, _, _ = O.refine(m, V, Ur, 1, rtol=1e-2)
                rounds += 1
                _, _, _, g, _ = O.solve(m, V, sigma, Ur, w["tau"], w["eps"], 0,
                                        cg_rtol=w["cg_rtol"], allow_unconverged=True)
            break
        except O.OracleError:
            failed.append(g1)
    out["refined"] = {"value": time.perf_counter() - t0, "unit": "s", "how": "measured",
                      "scheme_steps": n1, "refine_rounds": rounds, "g": g,
                      "failed_handoffs": failed}
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    from paper_2605_25149_gb300 import inputs
    V, U0, w = inputs.workload(WORKLOAD)
    K = max(1, min(args.steps, 2))
    Wm = min(args.warmup, 1)
    if Wm:
        cpu_baseline(V, U0, w, steps=Wm)
    cb = cpu_baseline(V, U0, w, steps=K)
    cb["sample"] += "; timed steps capped at 2, warm-up at 1"
    out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "steps/s",
           "n_gpus": ws, "steps": K, "warmup": Wm, "ms_per_step": 1000.0 / cb["value"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "host cores"},
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def spawn_command(argv, n, port):
    """torchrun command that runs this script on n local ranks (one per GPU)
    with the same arguments; rendezvous on 127.0.0.1."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            "--nproc-per-node", str(n), "--master-addr", "127.0.0.1", "--master-port", str(port),
            os.path.join(ROOT, "bench.py")] + list(argv)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hq", "reference"], default="hq")
    ap.add_argument("--ttr", action="store_true",
                    help="only the long scheme-only time-to-residual legs on %s "
                         "(adaptive tau; several minutes)" % WORKLOAD)
    ap.add_argument("--no-ttr", action="store_true",
                    help="skip the time-to-residual legs")
    ap.add_argument("--ttr-steps", type=int, default=40000, help="step cap of each --ttr leg")
    ap.add_argument("--ttr-chunk", type=int, default=250)
    ap.add_argument("--tau-max", type=float, default=10.0)
    ap.add_argument("--tau-safety", type=float, default=0.9,
                    help="safety factor c of the adaptive time step in the time-to-residual "
                         "legs (tau_n <= c lam / s_max)")
    ap.add_argument("--ttr-mixed-rtol", type=float, default=1e-4,
                    help="inner PCG rtol of the mixed scheme in the time-to-residual leg that "
                         "hands over to the FP64 refinement")
    ap.add_argument("--ttr-handoff", type=float, default=3e-4,
                    help="g at which the time-to-residual legs hand the scheme's state to "
                         "the FP64 residual refinement")
    ap.add_argument("--large-accuracy", action="store_true",
                    help="only the accuracy run of the 128^3, N = 256 mixed workload (minutes)")
    ap.add_argument("--large-g", type=float, default=1e-4)
    ap.add_argument("--large-steps", type=int, default=4000)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-grad", action="store_true", help="skip the differentiation workload")
    ap.add_argument("--no-large", action="store_true", help="skip the 128^3, N = 256 workload")
    ap.add_argument("--no-inner", action="store_true",
                    help="skip the per-column / O'Leary block PCG comparison")
    ap.add_argument("--large-shape", type=int, nargs=2, default=[128, 256], metavar=("M", "N"),
                    help="grid side and block width of the large mixed workload")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload with the default launch shape only")
    ap.add_argument("--mixed-rtol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1 or args.gpus < 1:
        ap.error("need --steps >= 1, --warmup >= 0 and --gpus >= 1")
    ws = int(os.environ.get("WORLD_SIZE", "0"))
    if ws == 0 and args.gpus > 1:
        # launched without torchrun: start one rank per GPU ourselves
        cmd = spawn_command(sys.argv[1:], args.gpus, _free_port())
        sys.exit(subprocess.call(cmd, cwd=ROOT))
    if ws and ws != args.gpus:
        ap.error("--gpus %d but WORLD_SIZE=%d" % (args.gpus, ws))
    if ws > 1:
        # replicas: the timed headline step only (the other legs hold every GPU for minutes)
        args.no_ttr = args.no_mixed = args.no_large = args.no_batch = args.no_grad = True
        args.no_inner = True
    if args.impl == "reference":
        run_reference(args)
    elif args.ttr:
        run_ttr(args)
    elif args.large_accuracy:
        run_large_accuracy(args)
    else:
        run_hq(args)


if __name__ == "__main__":
    main()
