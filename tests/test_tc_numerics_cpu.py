"""The arithmetic assumptions of the tensor-core vertical pass, checked on
the CPU with IEEE half precision (numpy float16 rounds to nearest even, as
the kernel's cvt.rn.f16.f32 does):

* the window holds x = clamp(v, lo, hi) - c0, c0 = (lo + hi) >> 1, as fp16:
  exact for every integer with |x| <= 2048, so for every uint8 image and for
  uint16 images whose stretch range hi - lo is at most 4095;
* a tap g scaled by 2^10 and split into fp16 hi = rn(g 2^10) and
  lo = rn(g 2^10 - hi) keeps hi + lo within 2^-22 of g 2^10 (relative), or
  2^-25 absolute where the remainder is below fp16's normal range; over a
  whole level the split moves the taps' sum by less than 2^-21 relative.
"""
import math

import numpy as np
import pytest

import oracle


def test_window_integers_are_exact_in_half_precision():
    x = np.arange(-2048, 2049, dtype=np.float64)
    assert np.array_equal(x.astype(np.float16).astype(np.float64), x)
    # one step beyond the bound is not representable
    assert float(np.float16(2049.0)) != 2049.0


@pytest.mark.parametrize("rng_width", [0, 1, 255, 4094, 4095])
def test_centred_stretch_range_fits_the_exact_window(rng_width):
    for lo in (0, 7, 60000 - rng_width):
        hi = lo + rng_width
        c0 = (lo + hi) >> 1
        assert -2048 <= lo - c0 and hi - c0 <= 2048


def _split(v32):
    hi = v32.astype(np.float16)
    lo = (v32 - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float64) + lo.astype(np.float64)


@pytest.mark.parametrize("n,tmin,tmax", [(16, 1.0, 12.0), (10, 1.0, 10.0), (4, 1.0, 4.0),
                                         (8, 0.5, 30.0)])
def test_two_part_tap_split_error(n, tmin, tmax):
    for t in oracle.ladder(n, tmin, tmax):
        g = oracle.kernel(float(t))                       # g[-R..R], FP64
        half = g[len(g) // 2:]                            # g[0..R]
        v32 = (half.astype(np.float32) * np.float32(1024.0)).astype(np.float32)
        got = _split(v32)
        ref = v32.astype(np.float64)
        err = np.abs(got - ref)
        assert np.all(err <= np.maximum(2.0 ** -22 * np.abs(ref), 2.0 ** -25)), t
        # whole level (both sides of the symmetric kernel)
        s_err = abs((2 * got.sum() - got[0]) - (2 * ref.sum() - ref[0]))
        assert s_err <= 2.0 ** -21 * 1024.0, t


def test_second_difference_taps_split_and_sum_to_zero():
    """The LoG level's second-difference taps g''[k] = g[k-1] - 2 g[k] + g[k+1]
    (radius R + 1) sum to zero over the symmetric support, and their split
    keeps that sum within the same bound, so the stretch offset drops out."""
    for t in oracle.ladder(16, 1.0, 12.0)[:16]:
        g = oracle.kernel(float(t))
        R = len(g) // 2
        ge = np.concatenate(([0.0], g, [0.0]))             # g[-R-1..R+1]
        d2 = ge[:-2] - 2 * ge[1:-1] + ge[2:]              # g''[-R..R]
        d2 = np.concatenate(([g[0]], d2, [g[0]]))          # ends: g[-R] at -R-1, g[R] at R+1
        assert abs(d2.sum()) < 1e-15
        half = d2[R + 1:]                                  # g''[0..R+1]
        v32 = (half.astype(np.float32) * np.float32(1024.0)).astype(np.float32)
        got = _split(v32)
        full = 2 * got.sum() - got[0]
        assert abs(full) <= 2.0 ** -20 * 1024.0 * math.fsum(np.abs(half)), t
