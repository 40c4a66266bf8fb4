"""Records the bench adds to its line, checked on the CPU.  The clock record keeps the
nvidia-smi samples taken during the timed region (or the two around it when the region
is shorter than the sampling interval) and reports every throttle reason any of them saw
(synthetic sample lines).  The phase check compares stored phasors with the oracle's
FP64 path phase."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

T = datetime.datetime(2026, 1, 2, 3, 4, 5)


def _line(ms, sm, hw="Not Active", power="Not Active"):
    t = (T + datetime.timedelta(milliseconds=ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return "%s, 0, %d, 2070, 900.5, 0x0, %s, Not Active, Not Active, %s" % (t, sm, hw, power)


def _sampler(lines, t0_ms, t1_ms):
    c = bench.ClockSampler(0)
    c.lines = lines
    c.t0 = T + datetime.timedelta(milliseconds=t0_ms)
    c.t1 = T + datetime.timedelta(milliseconds=t1_ms)
    return c


def test_samples_inside_the_region_only():
    lines = [_line(0, 1200), _line(50, 2070), _line(100, 2060), _line(150, 2070), _line(200, 900, hw="Active")]
    s = _sampler(lines, 40, 160).summary()
    assert s["window"] == "inside" and s["samples"] == 3
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == []          # the throttled sample lies after the region


def test_short_region_takes_the_samples_on_either_side():
    lines = [_line(0, 2000), _line(50, 2070, power="Active"), _line(100, 2070)]
    s = _sampler(lines, 60, 90).summary()
    assert s["window"] == "bracketing" and s["samples"] == 2
    assert s["sm_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]


def test_every_reason_seen_in_the_region_is_reported():
    lines = [_line(10, 2070, hw="Active"), _line(20, 2070, power="Active")]
    s = _sampler(lines, 0, 30).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_malformed_lines_and_no_samples():
    c = _sampler(["", "garbage", "[N/A], 0, x, y, 1, 0, a, b, c, d"], 0, 10)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_phase_error_against_the_oracle():
    """The bench's phase check reads the view records' (cone term, cos, -sin): phasors
    built from the oracle's own phase give a rounding-sized error, one phasor rotated by
    0.01 rad shows up as the largest error, and records marked by a NaN cone term (in no
    tile's list, no phase stored) are left out, whatever their phasor floats hold."""
    import numpy as np
    import oracle
    from paper_2502_01826_gb300 import synthetic
    cfg = synthetic.config_ble(K=64, n_rx=3)
    oracle.build()
    ph = np.stack([oracle.path_phase(cfg["scene"], cfg["rx"][r], cfg["tx"], cfg["f0"]) for r in range(3)])
    phasor = np.stack([np.zeros_like(ph), np.cos(ph), -np.sin(ph)], axis=-1).astype(np.float32)
    e = bench.oracle_phase_error(cfg, phasor)
    assert e["pairs"] == 3 * 64 and e["max"] < 1e-6
    ph[1, 5] += 0.01
    phasor[1, 5, 1:] = np.array([np.cos(ph[1, 5]), -np.sin(ph[1, 5])], np.float32)
    e = bench.oracle_phase_error(cfg, phasor)
    assert abs(e["max"] - 0.01) < 1e-5
    phasor[1, 5] = np.array([np.nan, 123.0, -7.0], np.float32)  # a record in no list
    e = bench.oracle_phase_error(cfg, phasor)
    assert e["pairs"] == 3 * 64 - 1 and e["max"] < 1e-6


def test_launch_count_follows_the_cluster_sort_limit():
    """The bench's per-step launch claim (18 library kernels when a receiver's depth sort
    runs in one cluster, 29 with the 12 global passes) uses the library's limit: CTAs of
    kCsThreads x kCsIpt keys, at most kCsMaxCluster of them."""
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2502_01826_gb300", "csrc", "k_dsort.cu")).read()
    const = {k: int(re.search(r"constexpr int %s = (\d+);" % k, src).group(1))
             for k in ("kCsThreads", "kCsIpt", "kCsMaxCluster")}
    limit = const["kCsThreads"] * const["kCsIpt"] * const["kCsMaxCluster"]
    assert bench.CLUSTER_SORT_MAX_GAUSSIANS == limit
    assert bench.launches_per_step(50_000) == 18
    assert bench.launches_per_step(limit) == 18
    assert bench.launches_per_step(limit + 1) == 29
