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
