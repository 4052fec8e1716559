"""Host-side pieces of bench.py that decide what it reports: the source hash
that ties the committed ncu traffic figure to the kernel sources it was
measured on, and the whole-job throughput arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_and_layout():
    a = "int x = 1; // note\n/* block\n comment */ int y;"
    b = "int x = 1;\n\n   int y;   // other note"
    assert bench._code_only(a) == bench._code_only(b) == "int x = 1; int y;"
    assert bench._code_only("int x = 2;") != bench._code_only("int x = 1;")


def test_committed_traffic_is_plausible_for_the_step():
    traffic = bench.profiled_traffic()
    if traffic is None:
        pytest.skip("the committed ncu summary was taken on other kernel sources")
    # algorithmic bytes of the step: 128 B per padded block + 3 B per pixel
    side = bench.SIDE
    px = side * side
    blocks = {"444": 3 * px // 64, "422": 2 * px // 64, "420": 3 * px // 128}
    alg = sum(128 * b + 3 * px for b in blocks.values())
    # reads = coefficients + chroma halo, writes <= RGB (part stays in L2)
    assert 0.7 * alg < traffic < 1.1 * alg


def test_whole_job_throughput():
    # 2 ranks, 3 steps of 1e6 pixels each, slowest rank 1.5 ms: 4000 MPix/s
    assert bench.whole_job_mpix_s(1e6, 3, 2, 1.5) == pytest.approx(4000.0)


def test_committed_instruction_counts_are_read():
    inst = bench.profiled_inst_per_px()
    if inst is None:
        pytest.skip("the committed ncu summary was taken on other kernel sources")
    assert set(inst) == {"444", "422", "420"}
    assert all(1.0 < v < 3.0 for v in inst.values())


def test_sps_estimate_from_measured_rates():
    class Img:
        width = height = 8192
    out = {"value": 425000.0, "e2e": {"value": 37000.0}, "cpu_baseline": {"value": 830.0}}
    est = bench.sps_estimate(out, [Img(), Img(), Img()])
    assert est["executed"] is False
    dev, e2e = est["device_resident"], est["end_to_end"]
    # the host cores are ~500x slower than the device-resident GPU: a sliver
    assert 0 <= dev["cpu_share"] < 0.005 and dev["predicted_speedup"] >= 1.0
    # against the link-bound end-to-end rate they could take ~2 %
    assert 0.01 < e2e["cpu_share"] < 0.04 and e2e["predicted_speedup"] > 1.0
    assert dev["cpu_rows"] % 16 == 0 and e2e["cpu_rows"] % 16 == 0


def test_variant_stats_line():
    from paper_1311_5304_gb300 import synth
    imgs = [synth.make_image(64, 48, s, 80, seed=1) for s in ("444", "422", "420")]
    bytes_v = [im.coef_bytes() + im.rgb_bytes() for im in imgs]
    launch_ms = [[0.2, 0.1, 0.3], [0.1] * 5, [0.05, 0.06]]
    per_var_ms = [sum(x) / len(x) for x in launch_ms]
    st = bench.variant_stats(["444", "422", "420"], imgs, bytes_v, per_var_ms, launch_ms, 6674.5,
                             {"444": 1.9, "422": 1.7, "420": 1.8})
    assert st["444"]["ms_p50"] == 0.2 and st["444"]["ms_p99"] == 0.3
    assert st["422"]["warp_inst_per_px"] == 1.7
    assert 0.0 <= st["420"]["nonzero_ac"] <= 1.0
    assert st["420"]["gbs"] == round(bytes_v[2] / (per_var_ms[2] / 1e3) / 1e9, 1)
    assert bench.variant_stats(["444"], imgs[:1], bytes_v[:1], per_var_ms[:1], launch_ms[:1], 1.0)["444"][
        "warp_inst_per_px"] is None
