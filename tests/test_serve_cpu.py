"""Host-side pieces of the server: arrival process and footprint model."""
import numpy as np

from paper_2108_12050_gb300 import serve


def test_poisson_arrivals_rate_and_determinism():
    a = serve.poisson_arrivals(500, 4.0, seed=5)
    b = serve.poisson_arrivals(500, 4.0, seed=5)
    assert a == b and all(x < y for x, y in zip(a, a[1:]))
    assert 1800 < len(a) < 2200          # 500/s over 4 s, within ~4.5 sigma
    gaps = np.diff([0.0] + a)
    assert abs(gaps.mean() - 1 / 500) < 2e-4


def test_footprint_grows_with_pixels_and_dtype():
    f8 = serve.footprint((1024, 1024), np.uint8)
    f16 = serve.footprint((1024, 1024), np.uint16)
    assert f16 - f8 == 1024 * 1024
    assert serve.footprint((2048, 2048), np.uint8) == 4 * f8
