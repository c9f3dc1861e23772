"""The benchmark's host-side arithmetic (no GPU): the algorithmic operation
count behind the roofline, from the oracle's ladder, and the nominal FP32
peak it is divided by."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_ladder_radii_match_the_oracle(bench):
    import oracle
    t, R = bench.ladder_radii()
    t_ref = oracle.ladder(bench.N_LAYERS, bench.T_MIN, bench.T_MAX)
    assert len(t) == len(t_ref) == bench.N_LAYERS + 1
    assert max(abs(a - b) for a, b in zip(t, t_ref)) < 1e-12
    assert R == [oracle.kernel_radius(x) for x in t_ref]


def test_algorithmic_operation_count(bench):
    import oracle
    t = oracle.ladder(16, 1.0, 12.0)
    taps = [2 * oracle.kernel_radius(x) + 1 for x in t]
    # two separable passes per level, one DoG and one max/argmax operation
    # per layer, the 8 comparisons of the 3x3 max-pool
    assert bench.algorithmic_ops_per_px() == 2 * sum(taps) + 2 * 16 + 8 == 1866
    # the tensor-core kernel moves the vertical pass (one pass of taps) off
    # the FP32 pipe
    assert bench.ffma_side_ops_per_px() == 1866 - sum(taps) == 953


def test_nominal_fp32_peak(bench):
    # 152 SMs x 128 FP32 lanes x 2.07 GHz maximum SM clock
    assert abs(bench.nominal_alu_peak() - 40.27392e12) < 1e6


def test_variant_operation_counts(bench):
    import oracle
    t = oracle.ladder(16, 1.0, 12.0)
    R = [oracle.kernel_radius(x) for x in t]
    assert bench.variant_ops_per_px("dog") == 1866
    # the derived-tap Laplacian on levels t_1..t_n: vertical g (2R+1) and
    # g'' (2R+3), horizontal g'' and g on them (2R+3, 2R+1)
    assert bench.variant_ops_per_px("log") == sum(8 * r + 8 for r in R[:16]) + 2 * 16 + 8
    # the DoG stack and one threshold test per (pixel, layer)
    assert bench.variant_ops_per_px("local26") == 2 * sum(2 * r + 1 for r in R) + 2 * 16


def test_r4_keeps_four_significant_digits(bench):
    assert bench.r4(14643.263544) == 14640.0
    assert bench.r4(0.0009999840015) == 0.001
    assert bench.r4(None) is None


def test_headline_line_fits_the_kept_tail(bench):
    """The last line bench.py prints must stay under 1500 characters, the
    tail a reader of the output keeps.  Section values shaped like a real run
    (long floats everywhere; rounding keeps four digits)."""
    import json
    import math
    x = math.pi * 1234.56789

    def rate(k):
        return {"tiles_per_s": x / k, "p99_ms": x * k, "p50_ms": x}

    serving = {"rates": {str(r): rate(r) for r in (100, 500, 2000)},
               "sequential_plain": {str(r): rate(r + 1) for r in (100, 500, 2000)}}
    variants = {"fused_" + k: {"ms": x, "roofline": {"frac": x / 1e4}}
                for k in ("reflect", "reflect_vtc", "reflect_ffma", "periodic", "local26",
                          "local26_vtc", "log")}
    variants.update({"plain_" + k: {"ms": x} for k in ("dog", "local26", "log")})
    summary = bench.summary_of({"tiles_per_s": x, "speedup_vs_plain": x / 100}, serving,
                               {"fit": {"held_out_mse": x / 1e5, "held_out_target_var": x / 1e3,
                                        "held_out_spearman": x / 4e3}}, variants)
    cpu = {"value": x / 1e3, "unit": "Mpixel/s", "cores": 16, "kind": "oracle",
           "sample": "2048^2 crop, sd=0 tile, whole method, 1.4 s",
           "single_core": {"value": x}}
    e2e = {"value": x * 10, "unit": "Mpixel/s", "h2d_bytes_per_step": 167772160,
           "d2h_bytes_per_step": 4227376}
    line = bench.headline_line(
        value=x * 10, world=1, steps=20, warmup=5, total_ms=x / 100, p50=x / 1e3, p99=x / 900,
        plain={"value": x / 3, "p50_ms_per_tile": x / 70}, achieved=x / 100, peak=40.27392,
        traffic=33911552, k_avg=x / 3800, side=x / 200, cpu=cpu, e2e=e2e, launches=3600,
        clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]},
        scores=[77964.0, 54646.0, 26709.0, 11418.0, 5337.0], summary=summary,
        tensor=(x / 3, x / 1.5))
    text = json.dumps(line)
    assert len(text) < 1500, len(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "p50_ms_per_tile", "p99_ms_per_tile", "plain", "fused_vs_plain", "roofline",
                "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert "single_core" not in line["cpu_baseline"]


def test_kernel_digest_ignores_comments_only(bench, tmp_path):
    """The digest that ties the committed ncu counters to the kernel source
    changes with the code, not with its comments or layout."""
    src = "int f(int a) {\n    return a + 1;  // one more\n}\n/* block\n comment */\n"
    paths = []
    for k, text in enumerate([src, src.replace("one more", "the next"),
                              src.replace("    return", "  return"),
                              src.replace("a + 1", "a + 2")]):
        p = tmp_path / ("k%d.cuh" % k)
        p.write_text(text)
        paths.append(str(p))
    d = [bench.kernel_digest([p]) for p in paths]
    assert d[0] == d[1] == d[2] != d[3]
