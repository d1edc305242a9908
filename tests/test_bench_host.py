"""Host-side arithmetic of bench.py (no GPU): the roofline entries, the
dominant-class pick, the whole-job value, the clock-record parser and the
separable closed form the time-to-residual check compares against."""
import os

import numpy as np
import pytest

import bench
from tests.helpers import dense_h


@pytest.mark.parametrize("kind,ops", [("smooth", 7), ("stencil", 8)])
def test_roofline_alone_fp64_is_alu_bound_with_issue_fraction(kind, ops):
    n, ms = 16777216, 0.24
    r = bench.roofline_alone(kind, ms, n, "f64", 6778.7, "measured", None)
    t = ms / 1e3
    flops, words = bench.ALGO_F64[kind]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["kernel"].startswith(kind)
    assert r["achieved"] == pytest.approx(flops * n / t / 1e12)
    assert r["peak"] == pytest.approx(2 * 152 * 2.07 * 2 / 1e3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # FP64-pipe instructions per point-column against 2 per clock per SM
    assert r["fp64_issue_frac"] == pytest.approx(ops * n / t / (2 * 152 * 2.07e9))
    assert r["hbm_gbs"] == pytest.approx(words * 8 * n / t / 1e9)
    assert r["algorithmic_bytes"] == words * 8 * n
    tr = bench.TRAFFIC_PER_ELEMENT.get((kind, "f64"))
    assert r["traffic"] == (None if tr is None else pytest.approx(tr * n))


def test_roofline_alone_fp32_is_hbm_bound():
    n, ms = 16777216, 0.04
    r = bench.roofline_alone("smooth", ms, n, "f32", 6778.7, "measured", None)
    flops, words = bench.ALGO["smooth"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(words * 4 * n / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6778.7)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_ELEMENT[("smooth", "f32")] * n)


def test_roofline_picks_the_dominant_grid_class():
    # (launches, ms, point-columns) per class; "vector" is not a grid class
    prof = {"smooth": (45, 12.0, 45 * 1e6), "stencil": (15, 4.0, 15 * 1e6),
            "residual": (17, 4.4, 17 * 1e6), "vector": (30, 30.0, 30 * 1e6)}
    assert bench.dominant(prof) == "smooth"
    r = bench.roofline(prof, "smooth", "f64")
    assert r["kernel"] == "smooth"
    assert r["launches"] == 45
    assert r["ms_per_launch"] == pytest.approx(12.0 / 45)
    assert r["elements_per_launch"] == pytest.approx(1e6)
    assert r["share"] == pytest.approx(12.0 / 50.4)
    assert r["tflops"] == pytest.approx(9.0 * 1e6 / (12.0 / 45 / 1e3) / 1e12)
    prof["stencil"] = (16, 20.0, 16 * 1e6)
    assert bench.dominant(prof) == "stencil"
    assert bench.dominant({"vector": (1, 1.0, 1.0)}) is None
    assert bench.roofline({"vector": (1, 1.0, 1.0)}, "smooth", "f64") is None


def test_job_value_counts_every_replica_at_the_slowest_time():
    assert bench.job_value(1, 36.0) == pytest.approx(1000.0 / 36.0)
    assert bench.job_value(4, 40.0) == pytest.approx(100.0)


def test_breakdown_shares_sum_to_one():
    prof = {"a": (10, 3.0, 0), "b": (5, 1.0, 0), "c": (0, 0.0, 0)}
    b = bench.breakdown(prof, 2)
    assert set(b) == {"a", "b"}
    assert b["a"]["launches_per_step"] == 5 and b["a"]["ms_per_step"] == 1.5
    assert b["a"]["share"] + b["b"]["share"] == pytest.approx(1.0)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clock_record(lines):
    c = bench.ClockSampler(0)
    c.f.write("\n".join(lines) + "\n")
    c.p = _Done()
    return c.stop()


def test_clock_record_median_and_throttle_reasons():
    base = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    lines = [base.format(sm=s, hw="Not Active", pc="Not Active") for s in (2070, 2055, 2070)]
    lines.append(base.format(sm=1980, hw="Not Active", pc="Active"))
    lines.append("garbage line")
    r = _clock_record(lines)
    assert r["samples"] == 4
    assert r["sm_mhz"] == pytest.approx(2062.5)
    assert r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]
    r = _clock_record([base.format(sm=1500, hw="Active", pc="Not Active")])
    assert r["reasons"] == ["hw_slowdown"]
    assert _clock_record(["[N/A], [N/A]"]) is None


def test_peaks_reads_the_measured_copy_bandwidth():
    hbm, kind = bench.peaks()
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        assert kind == "measured" and hbm > 1000.0
    else:
        assert (hbm, kind) == (6800.0, "fallback")


@pytest.mark.parametrize("m,N", [(4, 10), (6, 12)])
def test_fd_harmonic_levels_match_a_dense_eigensolve(m, N):
    """The separable closed form of the 7-point operator for V = |x|^2/2
    against numpy's eigensolve of the assembled dense matrix."""
    from paper_2605_25149_gb300 import inputs
    H = dense_h(m, inputs.grid_h(m), inputs.harmonic(m))
    ref = np.sort(np.linalg.eigvalsh(H))[:N]
    np.testing.assert_allclose(bench.fd_harmonic_levels(m, N), ref, rtol=1e-12, atol=1e-12)
