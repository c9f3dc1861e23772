"""The seeded scene generator that feeds both the oracle and the GPU path
(no GPU): determinism, dtypes and ranges, and its closed-form defocus checked
against what a Gaussian PSF must do (mass is conserved, variances add,
numerical convolution of the in-focus scene agrees)."""
import dataclasses
import math

import numpy as np
import pytest

import synth


def _spec(**kw):
    base = synth.SceneSpec(H=96, W=96, bg=100.0, noise_std=0.0, n_blobs=0, r_range=(3.0, 3.0),
                           amp=-50.0, n_lines=0, line_w=(3, 3), dtype="f32", vmax=0.0)
    return dataclasses.replace(base, **kw)


def test_same_seed_same_tile_other_seed_other_tile():
    spec = synth.scene12bit_spec(0.0, 256, 256)
    a = synth.make_scene(5, spec)
    assert np.array_equal(a, synth.make_scene(5, spec))
    assert not np.array_equal(a, synth.make_scene(6, spec))


@pytest.mark.parametrize("dtype,top", [("u16", 4095), ("u8", 255)])
def test_integer_tiles_stay_in_their_range(dtype, top):
    img = synth.make_scene(3, synth.scene12bit_spec(2.0, 256, 256, dtype))
    assert img.dtype == (np.uint16 if dtype == "u16" else np.uint8)
    assert img.min() >= 0 and img.max() <= top
    # the 12-bit scene: mean near the background, dark features below it
    bg = 2000.0 if dtype == "u16" else 2000.0 * 255 / 4095
    assert abs(float(np.median(img)) - bg) < 0.05 * bg


def test_noise_stream_is_shared_across_defocus_levels():
    spec0 = _spec(noise_std=5.0, n_blobs=6, r_range=(2.0, 5.0))
    clean0 = synth.make_scene(9, dataclasses.replace(spec0, noise_std=0.0))
    clean4 = synth.make_scene(9, dataclasses.replace(spec0, noise_std=0.0, sigma_d=4.0))
    n0 = synth.make_scene(9, spec0).astype(np.float64) - clean0
    n4 = synth.make_scene(9, dataclasses.replace(spec0, sigma_d=4.0)).astype(np.float64) - clean4
    np.testing.assert_allclose(n0, n4, atol=1e-4)     # float32 rounding only


@pytest.mark.parametrize("sigma_d", [0.0, 1.5, 4.0])
def test_defocused_blob_conserves_mass_and_adds_variances(sigma_d):
    spec = _spec(n_blobs=1, r_range=(4.0, 4.0), sigma_d=sigma_d)
    img, truth = synth.make_scene(1, dataclasses.replace(spec, H=128, W=128), return_truth=True)
    s = float(truth["s"][0])
    d = img.astype(np.float64) - 100.0
    # mass of A exp(-rho^2/(2 s^2)) is 2 pi s^2 A, whatever the blur
    cx, cy = float(truth["cx"][0]), float(truth["cy"][0])
    margin = min(cx, cy, 128 - cx, 128 - cy)
    if margin > 5 * math.sqrt(s * s + sigma_d ** 2) + 2:
        assert abs(d.sum() - 2 * math.pi * s * s * -50.0) < 1e-3 * 2 * math.pi * s * s * 50
        # the second moment about the centre is the sum of the variances
        yy, xx = np.mgrid[0:128, 0:128]
        var = (d * ((xx - cx) ** 2)).sum() / d.sum()
        assert abs(var - (s * s + sigma_d ** 2)) < 1e-3 * (s * s + sigma_d ** 2)


def test_defocus_equals_numerical_convolution_of_the_in_focus_scene():
    """Blobs rendered sharp on a 7x supersampled grid (pixel centres on grid
    points), convolved with the PSF numerically and sampled at the pixel
    centres, against the closed-form defocused render."""
    from scipy.ndimage import gaussian_filter
    sd, f = 2.0, 7
    spec = _spec(H=64, W=64, n_blobs=3, r_range=(2.0, 4.0), sigma_d=sd)
    blurred, truth = synth.make_scene(4, spec, return_truth=True)
    blurred = blurred.astype(np.float64) - 100.0
    # fine grid index i sits at pixel coordinate (i - (f - 1) / 2) / f
    yy, xx = np.mgrid[0:64 * f, 0:64 * f]
    px = (xx - (f - 1) // 2) / f
    py = (yy - (f - 1) // 2) / f
    fine = np.zeros(px.shape)
    for x0, y0, s in zip(truth["cx"], truth["cy"], truth["s"]):
        fine += -50.0 * np.exp(-((px - x0) ** 2 + (py - y0) ** 2) / (2 * s * s))
    conv = gaussian_filter(fine, sd * f, mode="constant", truncate=6.0)
    sampled = conv[(f - 1) // 2::f, (f - 1) // 2::f]
    # away from the borders, where the numerical filter's zero extension and
    # the closed form's clipped support agree
    core = (slice(12, 52), slice(12, 52))
    err = np.abs(sampled[core] - blurred[core]).max()
    assert err < 1e-3, err          # float32 output rounding is ~1e-5


def test_defocused_line_equals_numerical_convolution_of_the_sharp_segment():
    """A hard-edged segment rendered with its closed-form erf edges against
    the sharp segment on a 15x supersampled grid convolved numerically; the
    residual is the supersampled grid's edge quantisation (it halves when the
    grid is refined), about 0.5 % of the amplitude here."""
    from scipy.ndimage import gaussian_filter
    sd, f = 1.5, 15
    spec = _spec(H=64, W=64, n_lines=1, line_w=(3, 3), sigma_d=sd)
    img, truth = synth.make_scene(11, spec, return_truth=True)
    blurred = img.astype(np.float64) - 100.0
    p0, p1 = truth["lines_p0"][0], truth["lines_p1"][0]
    w = float(truth["lines_w"][0])
    yy, xx = np.mgrid[0:64 * f, 0:64 * f]
    px = (xx - (f - 1) // 2) / f
    py = (yy - (f - 1) // 2) / f
    length = float(np.hypot(*(p1 - p0)))
    ux, uy = (p1 - p0) / length
    u = (px - p0[0]) * ux + (py - p0[1]) * uy
    v = -(px - p0[0]) * uy + (py - p0[1]) * ux
    sharp = -50.0 * ((np.abs(v) <= w / 2) & (u >= 0) & (u <= length))
    conv = gaussian_filter(sharp, sd * f, mode="constant", truncate=6.0)
    sampled = conv[(f - 1) // 2::f, (f - 1) // 2::f]
    core = (slice(10, 54), slice(10, 54))
    assert blurred[core].min() < -25.0              # the line crosses the core
    err = np.abs(sampled[core] - blurred[core]).max()
    assert err < 0.5, err
