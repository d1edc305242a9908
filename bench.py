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
#   stencil  y = D x - c s: 5 add + mul + fma = 8 flops; 2 words
#   residual (b - D x) + c s: 5 add + 2 fma = 9 flops; 3 words
ALGO = {"smooth": (10.0, 3.0), "stencil": (8.0, 2.0), "residual": (9.0, 3.0)}
# FP64 V-cycles sweep from the pre-scaled right-hand side rt = omega D^-1 r:
#   z' = (omega c D^-1) s + ((1 - omega) z + rt): 5 add + 2 fma = 9 flops in 7
#   FP64-pipe instructions; reads rt, z, writes z': 3 words
ALGO_F64 = dict(ALGO, smooth=(9.0, 3.0))
FP64_OPS = {"smooth": 7.0, "stencil": 7.0, "residual": 7.0}
# DRAM bytes per point-column of the finest-level smooth kernel measured by
# ncu (dram__bytes_read.sum + dram__bytes_write.sum of one launch / 16.78 M
# point-columns, profiles/k_jacobi_k_jacobi_zm_wells64_N64.md: the pre-scaled
# k_jacobi_zm of a post-smoothing sweep for the 134 MB FP64 block, k_jacobi
# for the 67 MB FP32 block); set to None whenever the kernel changes until it
# is captured again.
TRAFFIC_PER_ELEMENT = {("smooth", "f64"): (272.048896e6 + 107.949824e6) / 16777216,
                       ("smooth", "f32"): (136.215040e6 + 44.029440e6) / 16777216}


# Recorded by `python bench.py --ttr` on a GB300 (profiles/ttr_wells64_N64.md):
# Algorithm 1 with the adaptive time step, steps and seconds to g < 1e-8 in
# FP64, and steps / seconds to a Rayleigh-Ritz eigenvalue error <= 1e-6
# (against the FP64 result) in FP64 and in mixed precision.  The default run
# reports them as "recorded" beside a projection from its own ms/step.
TTR_STEPS = {"wells64_N64": {"command": "python bench.py --ttr", "steps": 15113, "s": 288.3,
                             "fp64_err1e-6_steps": 6250, "fp64_err1e-6_s": 140.0,
                             "mixed_err1e-6_steps": 6250, "mixed_err1e-6_s": 25.7,
                             "fp64_mg32_s": 171.8, "mixed_then_fp64_mg32_s": 105.5,
                             "mixed_then_fp64_mg32_steps": 7750 + 7379}}


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


def roofline(prof, dtype_tag, hbm_peak, hbm_kind):
    """Dominant grid kernel class of an instrumented region."""
    cand = {k: v for k, v in prof.items() if k in ALGO and v[1] > 0}
    if not cand:
        return None
    k = max(cand, key=lambda c: cand[c][1])
    launches, ms, elems = cand[k]
    flops_e, words_e = (ALGO_F64 if dtype_tag == "f64" else ALGO)[k]
    w = 8 if dtype_tag == "f64" else 4
    per_launch_s = ms / 1e3 / launches
    per_launch_elems = elems / launches
    tr = TRAFFIC_PER_ELEMENT.get((k, dtype_tag))
    traffic = None if tr is None else tr * per_launch_elems
    if dtype_tag == "f64":
        achieved = flops_e * per_launch_elems / per_launch_s / 1e12
        peak = FP64_PEAK_GFLOPS / 1e3
        out = {"bound": "alu", "kernel": k, "achieved": achieved, "peak": peak,
               "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
               "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz",
               "hbm_gbs": words_e * w * per_launch_elems / per_launch_s / 1e9,
               "fp64_issue_frac": FP64_OPS[k] * per_launch_elems / per_launch_s
               / (FP64_PEAK_GFLOPS / 2 * 1e9)}
    else:
        achieved = words_e * w * per_launch_elems / per_launch_s / 1e9
        out = {"bound": "hbm", "kernel": k, "achieved": achieved, "peak": hbm_peak,
               "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
               "peak_source": hbm_kind}
    out.update({"launches": launches, "ms_per_launch": ms / launches,
                "elements_per_launch": per_launch_elems, "share": ms / sum(v[1] for v in prof.values())})
    return out


def smooth_alone(torch, hq, s, reps=40):
    """The finest-level damped-Jacobi sweep (the dominant kernel class) timed
    alone, in the form the context's V-cycle launches it (hq_mg_smooth_prescaled
    for FP64 contexts, hq_mg_smooth otherwise): `reps` back-to-back launches on
    n x N blocks of the working precision (ping-pong z_in / z_out; the three
    blocks exceed L2, so every sweep streams from HBM), CUDA events on the
    context's stream around the whole sequence.  Returns ms per launch."""
    import ctypes
    n, N = s.n, s.N
    g = torch.Generator(device="cuda").manual_seed(7)
    r = torch.rand((n, N), generator=g, device="cuda", dtype=s.dtype)
    za = torch.rand((n, N), generator=g, device="cuda", dtype=s.dtype)
    zb = torch.empty_like(za)
    st = s.stream
    lib = s.lib
    args = [(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(za.data_ptr()),
             ctypes.c_void_p(zb.data_ptr())),
            (ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(zb.data_ptr()),
             ctypes.c_void_p(za.data_ptr()))]
    fn, name = lib.hq_mg_smooth, "hq_mg_smooth"
    if s.dtype == torch.float64 and not s.cfg.mg_fp32:
        fn, name = lib.hq_mg_smooth_prescaled, "hq_mg_smooth_prescaled"
    for i in range(4):
        s._check(fn(s._ctx, 0, *args[i & 1]), name)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(reps):
        s._check(fn(s._ctx, 0, *args[i & 1]), name)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def roofline_alone(ms_launch, n_el, dtype_tag, hbm_peak, hbm_kind, in_step):
    """Roofline entry of the smooth kernel from its stand-alone launch time."""
    flops_e, words_e = (ALGO_F64 if dtype_tag == "f64" else ALGO)["smooth"]
    w = 8 if dtype_tag == "f64" else 4
    t = ms_launch / 1e3
    tr = TRAFFIC_PER_ELEMENT.get(("smooth", dtype_tag))
    traffic = None if tr is None else tr * n_el
    out = {"kernel": "smooth (finest-level damped-Jacobi sweep: k_jacobi_zm for blocks of "
           "100 MB or more, else k_jacobi)", "timing": "alone: back-to-back "
           "launches on the step's block shape, CUDA events; inputs exceed L2",
           "ms_per_launch": ms_launch, "elements_per_launch": n_el, "traffic": traffic,
           "algorithmic_bytes": words_e * w * n_el, "algorithmic_flops": flops_e * n_el}
    if dtype_tag == "f64":
        achieved = flops_e * n_el / t / 1e12
        peak = FP64_PEAK_GFLOPS / 1e3
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz",
                    "hbm_gbs": words_e * w * n_el / t / 1e9,
                    "fp64_issue_frac": FP64_OPS["smooth"] * n_el / t
                    / (FP64_PEAK_GFLOPS / 2 * 1e9)})
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
    s = hq.Solver(w["m"], w["N"], tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64")
    s.set_potential(V)
    s.set_initial(U0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, g = s.solve(w["eps"], 100000)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    lam = s.eigenpairs()["lam_rr"]
    ref = fd_harmonic_levels(w["m"], w["N"])
    return {"value": el, "unit": "s", "steps": steps, "g": g, "eps": w["eps"], "how": "measured",
            "workload": "harmonic16_N8: 16^3, V=|x|^2/2, N=8, tau=0.5, FP64",
            "eig_rel_err_vs_closed_form": float(np.max(np.abs(lam - ref) / np.abs(ref)))}


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
    """Time to residual and to eigenvalue error on the 64^3, N = 64 wells
    workload with the adaptive time step: FP64 to g < 1e-8 (its Rayleigh-Ritz
    values are the reference), the mixed path to eigenvalue error <= 1e-6,
    and the mixed path followed by FP64 to g < 1e-8."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2605_25149_gb300 import hq, inputs
    V, U0, w = inputs.workload(WORKLOAD)
    m, N = w["m"], w["N"]
    chunk = args.ttr_chunk
    s = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64", adaptive_tau=1,
                  tau_max=args.tau_max)
    s.set_potential(V)
    s.set_initial(U0)
    h64 = solve_history(torch, s, w["eps"], chunk, args.ttr_steps)
    lam_ref = h64[-1]["lam"]
    for h in h64:
        h["err"] = float(np.max(np.abs(h["lam"] - lam_ref) / np.abs(lam_ref)))
    del s
    torch.cuda.empty_cache()
    sm = hq.Solver(m, N, tau=w["tau"], cg_rtol=args.mixed_rtol, precision="mixed", adaptive_tau=1,
                   tau_max=args.tau_max)
    sm.set_potential(V)
    sm.set_initial(U0)
    hmx = solve_history(torch, sm, 1e-300, chunk, args.ttr_steps, lam_ref=lam_ref, stop_err=1e-7,
                        stall=8)
    # FP64 PCG with the FP32 preconditioner, to g < 1e-8, and the same after
    # the mixed leg (state handed over through host memory)
    s3 = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64", adaptive_tau=1,
                   tau_max=args.tau_max, mg_fp32=1)
    s3.set_potential(V)
    s3.set_initial(U0)
    h32 = solve_history(torch, s3, w["eps"], chunk, args.ttr_steps, lam_ref=lam_ref)
    del s3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Um, Zm, stpm = sm.get_state(with_warm_start=True)
    s4 = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64", adaptive_tau=1,
                   tau_max=args.tau_max, mg_fp32=1)
    s4.set_potential(V)
    s4.set_state(Um, stpm, Zm)
    torch.cuda.synchronize()
    t_hand4 = time.perf_counter() - t0
    h4 = solve_history(torch, s4, w["eps"], chunk, args.ttr_steps, lam_ref=lam_ref)
    del s4
    torch.cuda.empty_cache()
    hpol, t_hand = None, None
    if args.ttr_pipeline:
        # hand over to FP64 (state through host memory), then to g < 1e-8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U, Z, stp = sm.get_state(with_warm_start=True)
        s2 = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64",
                       adaptive_tau=1, tau_max=args.tau_max)
        s2.set_potential(V)
        s2.set_state(U, stp, Z)
        torch.cuda.synchronize()
        t_hand = time.perf_counter() - t0
        hpol = solve_history(torch, s2, w["eps"], chunk, args.ttr_steps, lam_ref=lam_ref)
    del sm

    def pick(hh):
        return [{k: v for k, v in h.items() if k != "lam"} for h in hh]

    a64, amx = first_below(h64, "err", 1e-6), first_below(hmx, "err", 1e-6)
    out = {"workload": WORKLOAD, "tau_rule": "adaptive, tau_max %g" % args.tau_max,
           "chunk": chunk, "eps": w["eps"],
           "fp64": {"time_to_residual_s": h64[-1]["s"], "steps": h64[-1]["steps"],
                    "g": h64[-1]["g"], "to_err_1e-6": a64 and {"s": a64["s"], "steps": a64["steps"]}},
           "mixed": {"to_err_1e-6": amx and {"s": amx["s"], "steps": amx["steps"]},
                     "last": pick(hmx[-1:])[0], "cg_rtol": args.mixed_rtol},
           "speedup_mixed_vs_fp64_at_err_1e-6": (a64["s"] / amx["s"]) if (a64 and amx) else None,
           "mixed_then_fp64": hpol and {
               "time_to_residual_s": hmx[-1]["s"] + t_hand + hpol[-1]["s"],
               "mixed_s": hmx[-1]["s"], "handover_s": t_hand, "fp64_s": hpol[-1]["s"],
               "fp64_steps": hpol[-1]["steps"], "g": hpol[-1]["g"]},
           "fp64_mg32": {"time_to_residual_s": h32[-1]["s"], "steps": h32[-1]["steps"],
                         "g": h32[-1]["g"], "err": h32[-1]["err"]},
           "mixed_then_fp64_mg32": {
               "time_to_residual_s": hmx[-1]["s"] + t_hand4 + h4[-1]["s"],
               "mixed_s": hmx[-1]["s"], "mixed_steps": hmx[-1]["steps"], "handover_s": t_hand4,
               "fp64_mg32_s": h4[-1]["s"], "fp64_mg32_steps": h4[-1]["steps"], "g": h4[-1]["g"],
               "err": h4[-1]["err"]},
           "history": {"fp64": pick(h64), "mixed": pick(hmx),
                       "fp64_after_mixed": hpol and pick(hpol), "fp64_mg32": pick(h32),
                       "fp64_mg32_after_mixed": pick(h4)}}
    print(json.dumps(out), flush=True)


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

    def seq(solvers):
        tot = 0.0
        for s in solvers:
            s.step(W)
            torch.cuda.synchronize()
            e0.record(s.stream)
            s.step(K)
            e1.record(s.stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1) / K
        return tot

    solvers = make(lambda m, N: (0, 0))
    ms_default, launches = time_batch(solvers, "batch_timed")
    ms_seq_mixed = seq(solvers)
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
    ms_batch = min(ms_default, ms_tuned)
    pc = sum(m ** 3 * N for m, N in shapes)
    res = {"value": len(shapes) * 1000.0 / ms_batch, "unit": "problem-steps/s",
           "ms_per_batch_step": ms_batch, "default_ms_per_batch_step": ms_default,
           "problems": len(shapes), "point_columns": pc,
           "gpu_launches_per_batch_step": launches, "graph_launches_per_call": 1,
           "sequential_mixed_ms": ms_seq_mixed, "sequential_fp64_ms": ms_seq_fp64,
           "speedup_vs_sequential_mixed": ms_seq_mixed / ms_batch,
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
    ms_sm = smooth_alone(torch, hq, s, reps=10)
    roof = roofline_alone(ms_sm, m ** 3 * N, "f32", hbm_peak, hbm_kind, None)
    roof["traffic"] = None
    out = {"workload": "wells: %d^3 grid, V=|x|^2/2 + 8 wells (default_rng(3)), "
                       "N=%d, tau=0.4, mixed, PCG rtol 1e-6" % (m, N),
           "ms_per_step": ms, "value": 1000.0 / ms, "unit": "steps/s", "roofline": roof,
           "breakdown": breakdown(prof, 1),
           "workspace_gb": s.workspace.numel() / 1e9}
    del s
    torch.cuda.empty_cache()
    return out


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
    result = {}

    # ---- FP64 path: headline ------------------------------------------------
    s = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64")
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
    roof = roofline_alone(smooth_alone(torch, hq, s), m ** 3 * N, "f64", hbm_peak, hbm_kind,
                          roofline(prof, "f64", hbm_peak, hbm_kind))
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
    ttr = {} if args.no_ttr else {"harmonic16_N8": ttr_small(torch, hq, inputs)}
    if WORKLOAD in TTR_STEPS:
        rec = TTR_STEPS[WORKLOAD]
        ttr[WORKLOAD] = {"value": rec["s"], "unit": "s", "how": "recorded (%s)" % rec["command"],
                         "steps": rec["steps"], "eps": w["eps"], "tau": "adaptive",
                         "projected_s": rec["steps"] * ms / 1e3,
                         "projected_basis": "recorded steps x this run's fixed-tau ms/step "
                                            "(early steps cost more PCG iterations than late ones)",
                         "fp64_fp32_preconditioner_s": rec["fp64_mg32_s"],
                         "mixed_then_fp64_fp32_preconditioner_s": rec["mixed_then_fp64_mg32_s"],
                         "mixed_then_fp64_steps": rec["mixed_then_fp64_mg32_steps"],
                         "note": "all three end at g < 1e-8 with FP64 blocks; eigenvalues agree "
                                 "with the plain FP64 run to 1e-14"}
    del s
    torch.cuda.empty_cache()

    # ---- FP64 PCG with an FP32 multigrid preconditioner (mg_fp32) --------------
    mg32 = None
    if not args.no_mixed:
        s3 = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64", mg_fp32=1)
        s3.set_potential(V)
        s3.set_initial(U0)
        for _ in range(W):
            s3.step(1)
        s3.profile(timing=False)
        ms3, _ = time_steps(torch, s3, K, ws)
        ms3 = max_over_ranks(ws, ms3)
        sol3, it3 = s3.pcg_stats()
        mg32 = {"value": job_value(ws, ms3), "unit": "steps/s", "ms_per_step": ms3,
                "speedup_vs_fp64": ms / ms3, "pcg_iterations_per_solve": it3 / max(sol3, 1),
                "dtype": "f64 PCG (residuals, updates, stopping test, step algebra); "
                         "f32 multigrid V-cycle inside the preconditioner",
                "note": "W = G U solved to the same FP64 rtol 1e-10; not the headline"}
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
        mixed = {"value": job_value(ws, ms_m), "unit": "steps/s", "ms_per_step": ms_m,
                 "speedup_vs_fp64": ms / ms_m, "dtype": "f32 (FP64 small solve / extraction)",
                 "to_eig_err_1e-6": None if WORKLOAD not in TTR_STEPS else {
                     "recorded_fp64_s": TTR_STEPS[WORKLOAD]["fp64_err1e-6_s"],
                     "recorded_mixed_s": TTR_STEPS[WORKLOAD]["mixed_err1e-6_s"],
                     "recorded_speedup": TTR_STEPS[WORKLOAD]["fp64_err1e-6_s"] /
                                         TTR_STEPS[WORKLOAD]["mixed_err1e-6_s"],
                     "steps_fp64": TTR_STEPS[WORKLOAD]["fp64_err1e-6_steps"],
                     "steps_mixed": TTR_STEPS[WORKLOAD]["mixed_err1e-6_steps"],
                     "how": "recorded (%s); same step count, so the speedup at error 1e-6 "
                            "equals the per-step ratio" % TTR_STEPS[WORKLOAD]["command"]},
                 "cg_rtol": args.mixed_rtol,
                 "roofline": roofline_alone(smooth_alone(torch, hq, sm), m ** 3 * N, "f32",
                                            hbm_peak, hbm_kind,
                                            roofline(prof_m, "f32", hbm_peak, hbm_kind)),
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
                               "N=%d, tau=%g, PCG rtol %g, FP64" % (WORKLOAD, m, N, w["tau"], w["cg_rtol"]),
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
        "fp64_fp32_preconditioner": mg32,
        "large": large,
        "batched": batched,
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
    return {"value": time.perf_counter() - t0, "unit": "s", "steps": steps, "g": g,
            "workload": "harmonic16_N8", "how": "measured"}


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


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hq", "reference"], default="hq")
    ap.add_argument("--ttr", action="store_true",
                    help="only measure time to residual / eigenvalue error on %s "
                         "(adaptive tau; several minutes)" % WORKLOAD)
    ap.add_argument("--no-ttr", action="store_true",
                    help="skip the time-to-residual run of the 16^3 workload")
    ap.add_argument("--ttr-steps", type=int, default=40000, help="step cap of each --ttr leg")
    ap.add_argument("--ttr-chunk", type=int, default=250)
    ap.add_argument("--ttr-pipeline", action="store_true",
                    help="with --ttr: also hand the mixed state to FP64 and run to 1e-8")
    ap.add_argument("--tau-max", type=float, default=10.0)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-large", action="store_true", help="skip the 128^3, N = 256 workload")
    ap.add_argument("--large-shape", type=int, nargs=2, default=[128, 256], metavar=("M", "N"),
                    help="grid side and block width of the large mixed workload")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload with the default launch shape only")
    ap.add_argument("--mixed-rtol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.ttr:
        run_ttr(args)
    else:
        run_hq(args)


if __name__ == "__main__":
    main()
