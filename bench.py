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
#   residual b - (D x - c s): 9 flops; 3 words
ALGO = {"smooth": (10.0, 3.0), "stencil": (8.0, 2.0), "residual": (9.0, 3.0)}
# DRAM bytes per point-column of the finest-level smooth kernel measured by
# ncu (dram__bytes_read.sum + dram__bytes_write.sum of one launch / 16.78 M
# point-columns, profiles/k_jacobi_wells64_N64.md); set to None whenever the
# kernel changes until it is captured again.
TRAFFIC_PER_ELEMENT = {("smooth", "f64"): (278.660352e6 + 112.328704e6) / 16777216,
                       ("smooth", "f32"): (135.338240e6 + 44.317696e6) / 16777216}


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


def time_steps(torch, s, K, ws):
    """ms per step over K steps: events on the solver stream, barrier + sync."""
    st = s.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(st)
    g = s.step(K) if K > 0 else float("nan")
    e1.record(st)
    torch.cuda.synchronize()
    barrier(ws)
    return e0.elapsed_time(e1) / max(K, 1), g


def roofline(prof, dtype_tag, hbm_peak, hbm_kind):
    """Dominant grid kernel class of an instrumented region."""
    cand = {k: v for k, v in prof.items() if k in ALGO and v[1] > 0}
    if not cand:
        return None
    k = max(cand, key=lambda c: cand[c][1])
    launches, ms, elems = cand[k]
    flops_e, words_e = ALGO[k]
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
               "hbm_gbs": words_e * w * per_launch_elems / per_launch_s / 1e9}
    else:
        achieved = words_e * w * per_launch_elems / per_launch_s / 1e9
        out = {"bound": "hbm", "kernel": k, "achieved": achieved, "peak": hbm_peak,
               "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
               "peak_source": hbm_kind}
    out.update({"launches": launches, "ms_per_launch": ms / launches,
                "elements_per_launch": per_launch_elems, "share": ms / sum(v[1] for v in prof.values())})
    return out


def breakdown(prof, K):
    """Per kernel class: launches and event-timed ms per step, share."""
    tot = sum(v[1] for v in prof.values()) or 1.0
    return {k: {"launches_per_step": v[0] / K, "ms_per_step": v[1] / K,
                "share": v[1] / tot} for k, v in prof.items() if v[0] > 0}


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
    ms, g = time_steps(torch, s, K, ws)
    launches = sum(v[0] for v in s.profile_read().values())
    clocks = clk.stop()
    ms = max_over_ranks(ws, ms)
    # instrumented region (per-class CUDA events) for the roofline
    s.profile(timing=True)
    ms_instr, _ = time_steps(torch, s, K, ws)
    prof = s.profile_read()
    pcg_solves, pcg_iters = s.pcg_stats()
    s.profile(timing=False)
    roof = roofline(prof, "f64", hbm_peak, hbm_kind)
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
    fp64_lam = None
    ttr = None
    if args.ttr_steps > 0:
        s2 = hq.Solver(m, N, tau=w["tau"], cg_rtol=w["cg_rtol"], precision="fp64",
                       timeout_s=args.ttr_timeout)
        s2.set_potential(V)
        s2.set_initial(U0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            steps, gend = s2.solve(w["eps"], args.ttr_steps)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            ttr = {"value": el, "unit": "s", "steps": steps, "g": gend, "how": "measured",
                   "eps": w["eps"]}
            fp64_lam = s2.eigenpairs()["lam_rr"]
        except hq.HQError as e:
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            _, _, steps_done = s2.get_state()
            ttr = {"value": None, "unit": "s", "steps": steps_done, "how": "not reached",
                   "wall_s": el, "reason": str(e)[:120]}
        del s2
    del s
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
        ms_m, _ = time_steps(torch, sm, K, ws)
        ms_m = max_over_ranks(ws, ms_m)
        sm.profile(timing=True)
        time_steps(torch, sm, K, ws)
        prof_m = sm.profile_read()
        sm.profile(timing=False)
        mixed = {"value": job_value(ws, ms_m), "unit": "steps/s", "ms_per_step": ms_m,
                 "speedup_vs_fp64": ms / ms_m, "dtype": "f32 (FP64 small solve / extraction)",
                 "cg_rtol": args.mixed_rtol,
                 "roofline": roofline(prof_m, "f32", hbm_peak, hbm_kind),
                 "breakdown": breakdown(prof_m, K)}
        if fp64_lam is not None and args.ttr_steps > 0:
            sm2 = hq.Solver(m, N, tau=w["tau"], cg_rtol=args.mixed_rtol, precision="mixed",
                            timeout_s=args.ttr_timeout)
            sm2.set_potential(V)
            sm2.set_initial(U0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                steps_m, g_m = sm2.solve(args.mixed_eps, args.ttr_steps)
                torch.cuda.synchronize()
                el = time.perf_counter() - t0
                lam_m = sm2.eigenpairs()["lam_rr"]
                err = float(np.max(np.abs(lam_m - fp64_lam) / np.abs(fp64_lam)))
                mixed["time_to_residual"] = {"value": el, "unit": "s", "steps": steps_m,
                                             "eps": args.mixed_eps, "how": "measured"}
                mixed["eig_rel_err_vs_fp64"] = err
            except hq.HQError as e:
                mixed["time_to_residual"] = {"value": None, "how": "not reached",
                                             "reason": str(e)[:120]}
            del sm2
        del sm
        torch.cuda.empty_cache()

    # ---- CPU oracle on the host cores (rank 0, N = 1) ------------------------
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(V, U0, w, steps=1)

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
    ap.add_argument("--ttr-steps", type=int, default=0,
                    help="also run Algorithm 1 to residual 1e-8 (at most this many steps)")
    ap.add_argument("--ttr-timeout", type=float, default=120.0)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--mixed-rtol", type=float, default=1e-6)
    ap.add_argument("--mixed-eps", type=float, default=1e-5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_hq(args)


if __name__ == "__main__":
    main()
