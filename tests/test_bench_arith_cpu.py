"""The bench's roofline arithmetic on the host: the derived FP32 peak, the
executed-flop count of the headline kernel against its stated per-link parts,
and the match between the committed ncu summary and the kernel sources."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_peaks_scale_with_sm_count_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.070 GHz
    assert abs(bench.fp32_peak_tflops() - 152 * 128 * 2 * 2.070e9 / 1e12) < 1e-9
    assert abs(bench.fp32_peak_tflops() - 80.548) < 1e-3
    # FP64: 2 FMAs per SM per clock, 1.26 TFLOP/s at 152 SMs and 2.07 GHz
    assert abs(bench.fp64_peak_tflops() - 1.2586) < 1e-4
    assert abs(bench.fp32_peak_tflops(148, 1800.0) - 148 * 128 * 2 * 1.8e9 / 1e12) < 1e-9
    assert abs(bench.fp64_peak_tflops(76, 1000.0) / bench.fp64_peak_tflops(152, 2000.0) - 0.25) < 1e-12
    assert bench.fp32_inst_rate(152, 2070.0) == 152 * 128 * 2070.0e6


def test_fractions_are_work_over_time_at_the_sampled_clock():
    pk = bench.Peaks(152, 1035.0)  # half the maximum clock: half the peak
    assert abs(pk.f32 - bench.fp32_peak_tflops() * 1e12 / 2) < 1.0
    t = 1e-5
    adj = bench.adjoint_report({"B8192_recompute": {"B": 8192, "mode": 2, "t": t}}, pk)
    r = adj["B8192_recompute"]
    assert adj["flop_per_link"] == 621
    assert abs(r["frac"] - 8192 * 32 * 621 / t / pk.f32) < 1e-12
    fd = bench.fd_report({"n64_B16384": {"n": 64, "B": 16384, "t64": 6e-4, "tdf": 3e-4}}, pk)
    f = fd["n64_B16384"]
    nb = 64 * 16384
    assert abs(f["frac"] - nb * (257 / pk.f32 + 400 / pk.f64) / 6e-4) < 1e-12
    assert abs(f["frac_alg"] - nb * (720 / pk.f32 + 800 / pk.f64) / 6e-4) < 1e-12
    assert abs(f["df_frac"] - nb * 3043 / pk.i32 / 3e-4) < 1e-12


def test_rounding_keeps_four_significant_digits():
    x = bench.rnd({"a": 2806440547.738912, "b": [0.5240223181402908, 3], "c": "s", "d": None})
    assert x == {"a": 2806000000.0, "b": [0.524, 3], "c": "s", "d": None}


def test_executed_flops_follow_the_per_link_parts():
    stored = 26 + 4 + 86 + 93 + 44 + 4       # sin/cos, products, step, wrench, carry, products
    rederived = stored + 86                   # plus the inverse motion step
    assert (stored, rederived) == (257, 343)
    for n, K in ((32, 24), (16, 16), (64, 12), (100, 0), (4, 4)):
        want = K * stored + (n - K) * rederived - 38 - (86 if K < n else 0)
        assert bench.dh_param_flops(n, K) == want
    assert abs(bench.dh_param_flops(32, 24) / 32 - 274.625) < 1e-12


def test_adjoint_counts_follow_the_per_sweep_parts():
    sweep1 = 26 + 4 + 86 + 39
    sweep2 = 4 + 93 + 44 + 126 + 30 + 42 + 88 + 8 + 31
    recompute_extra = 26 + 86 + 39
    assert (sweep1, sweep2, recompute_extra) == (155, 466, 151)
    assert bench.VJP_FLOP_PER_LINK[1] == sweep1 + sweep2
    assert bench.VJP_FLOP_PER_LINK[2] == sweep1 + sweep2 + recompute_extra


def test_profile_traffic_is_reported_only_for_the_profiled_sources():
    """The bench takes the headline kernel's DRAM traffic from its committed ncu
    summary only while the kernel sources hash to the value recorded there."""
    import re

    text = open(os.path.join(ROOT, "profiles", "rnea_fp32_n32_B65536.md")).read()
    recorded_hash = re.search(r"kernel_sources_sha256:\s*([0-9a-f]+)", text).group(1)
    traffic = float(re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text).group(1))
    got = bench.recorded_traffic("rnea_fp32_n32_B65536")
    if recorded_hash == bench.kernel_sources_hash():
        assert got == traffic
    else:
        assert got is None
    assert bench.recorded_traffic("no_such_profile") is None
