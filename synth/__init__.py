"""Seeded synthetic SEM-like tiles for the multi-scale feature detector.

This module only draws scenes.  It holds none of the detector's arithmetic
(no sampled Gaussian taps, no discrete convolution, no responses): defocus is
rendered *analytically* from the continuous scene, so neither the CUDA path
nor the CPU oracle shares code with it beyond receiving its pixels.

Scene model (the paper's SEM focal series of §5 is not available, so these
tiles stand in for it; shapes and dtypes follow the paper's workloads):

* background level ``bg`` plus Gaussian noise of std ``noise_std``;
* ``n_blobs`` dark Gaussian blobs ``A * exp(-rho^2 / (2 s^2))`` with
  ``s = r / sqrt(2)`` and ``r`` uniform in ``r_range`` (so the scale-normalised
  Laplacian peaks at ``t = s`` and the blob radius ``sqrt(2) t`` equals ``r``);
* ``n_lines`` straight hard-edged dark segments (membrane-like) of width ``w``
  with random endpoints inside the image and the blob amplitude;
* defocus: an isotropic Gaussian PSF of std ``sigma_d`` applied to the
  noise-free scene.  A Gaussian blob stays Gaussian (variances add, amplitude
  scales by ``s^2 / (s^2 + sigma_d^2)``) and a rectangle becomes a product of
  two error-function edges, so the blurred scene is evaluated in closed form;
* noise is drawn from its own stream (same for every ``sigma_d`` of one seed),
  then values are rounded half-to-even and clipped to the dtype range
  (12-bit data lives in ``uint16`` with range [0, 4095]).
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import Optional

import numpy as np
from scipy.special import erf

__all__ = [
    "SceneSpec", "make_scene", "pair512_u8", "sweep_tile_4096_u16", "uneven_batch_tile",
    "uneven_batch_specs", "soft_tile_f32", "random_candidates",
]

_SQRT2 = math.sqrt(2.0)


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    H: int
    W: int
    bg: float
    noise_std: float
    n_blobs: int
    r_range: tuple
    amp: float
    n_lines: int
    line_w: tuple            # (lo, hi) inclusive integer widths
    dtype: str               # "u8" | "u16" | "f32"
    vmax: float              # clip ceiling for integer dtypes
    sigma_d: float = 0.0


def _phi_band(v, half, sigma):
    """Mass of N(v, sigma^2) inside [-half, half] (indicator when sigma == 0)."""
    if sigma <= 0.0:
        return (np.abs(v) <= half).astype(np.float64)
    k = 1.0 / (_SQRT2 * sigma)
    return 0.5 * (erf((half - v) * k) - erf((-half - v) * k))


def _phi_seg(u, length, sigma):
    """Mass of N(u, sigma^2) inside [0, length]."""
    if sigma <= 0.0:
        return ((u >= 0.0) & (u <= length)).astype(np.float64)
    k = 1.0 / (_SQRT2 * sigma)
    return 0.5 * (erf((length - u) * k) - erf((-u) * k))


def _add_blobs(scene, cx, cy, s, amp, sigma_d):
    H, W = scene.shape
    for x0, y0, si in zip(cx, cy, s):
        var = si * si + sigma_d * sigma_d
        a = amp * (si * si) / var
        rad = int(math.ceil(5.0 * math.sqrt(var))) + 1
        xa, xb = max(0, int(x0) - rad), min(W, int(x0) + rad + 2)
        ya, yb = max(0, int(y0) - rad), min(H, int(y0) + rad + 2)
        if xa >= xb or ya >= yb:
            continue
        xs = np.arange(xa, xb, dtype=np.float64) - x0
        ys = np.arange(ya, yb, dtype=np.float64) - y0
        ex = np.exp(-(xs * xs) / (2.0 * var))
        ey = np.exp(-(ys * ys) / (2.0 * var))
        scene[ya:yb, xa:xb] += a * np.outer(ey, ex)


def _add_line(scene, p0, p1, width, amp, sigma_d):
    """Hard-edged segment p0->p1 of the given width, blurred analytically."""
    H, W = scene.shape
    dx, dy = p1[0] - p0[0], p1[1] - p0[1]
    length = math.hypot(dx, dy)
    if length < 1e-9:
        return
    ux, uy = dx / length, dy / length
    half = 0.5 * width
    reach = half + 5.0 * sigma_d + 1.5
    # iterate along the axis the segment is most aligned with, and take the
    # bounded interval across it on each row/column
    horizontal = abs(ux) >= abs(uy)
    if horizontal:
        lo = int(math.floor(min(p0[0], p1[0]) - reach))
        hi = int(math.ceil(max(p0[0], p1[0]) + reach))
        major = np.arange(max(0, lo), min(W, hi + 1))
        # centre-line y at each x, then +- reach / |ux|
        t = (major - p0[0]) / ux if abs(ux) > 0 else np.zeros_like(major, dtype=float)
        centre = p0[1] + t * uy
        span = reach / max(abs(ux), 1e-12)
    else:
        lo = int(math.floor(min(p0[1], p1[1]) - reach))
        hi = int(math.ceil(max(p0[1], p1[1]) + reach))
        major = np.arange(max(0, lo), min(H, hi + 1))
        t = (major - p0[1]) / uy
        centre = p0[0] + t * ux
        span = reach / max(abs(uy), 1e-12)
    if major.size == 0:
        return
    limit = H if horizontal else W
    a = np.clip(np.floor(centre - span).astype(np.int64), 0, limit - 1)
    b = np.clip(np.ceil(centre + span).astype(np.int64), 0, limit - 1)
    counts = np.maximum(b - a + 1, 0)
    total = int(counts.sum())
    if total == 0:
        return
    maj = np.repeat(major, counts)
    starts = np.repeat(a - np.concatenate(([0], np.cumsum(counts)[:-1])), counts)
    minor = starts + np.arange(total)
    if horizontal:
        px, py = maj.astype(np.float64), minor.astype(np.float64)
    else:
        px, py = minor.astype(np.float64), maj.astype(np.float64)
    rx, ry = px - p0[0], py - p0[1]
    u = rx * ux + ry * uy            # along the segment
    v = -rx * uy + ry * ux           # across the segment
    val = amp * _phi_band(v, half, sigma_d) * _phi_seg(u, length, sigma_d)
    if horizontal:
        np.add.at(scene, (minor, maj), val)
    else:
        np.add.at(scene, (maj, minor), val)


def make_scene(seed: int, spec: SceneSpec, *, return_truth: bool = False,
               noise_seed: Optional[int] = None):
    """Render one tile.  Returns ``img`` (and a truth dict if asked)."""
    rng = np.random.default_rng([int(seed), 0])
    H, W = spec.H, spec.W
    cx = rng.uniform(0.0, W, spec.n_blobs)
    cy = rng.uniform(0.0, H, spec.n_blobs)
    r = rng.uniform(spec.r_range[0], spec.r_range[1], spec.n_blobs)
    s = r / _SQRT2
    lp0 = np.stack([rng.uniform(0, W, spec.n_lines), rng.uniform(0, H, spec.n_lines)], 1)
    lp1 = np.stack([rng.uniform(0, W, spec.n_lines), rng.uniform(0, H, spec.n_lines)], 1)
    lw = rng.integers(spec.line_w[0], spec.line_w[1] + 1, spec.n_lines)

    scene = np.full((H, W), float(spec.bg), dtype=np.float64)
    _add_blobs(scene, cx, cy, s, spec.amp, spec.sigma_d)
    for k in range(spec.n_lines):
        _add_line(scene, lp0[k], lp1[k], float(lw[k]), spec.amp, spec.sigma_d)

    nrng = np.random.default_rng([int(seed if noise_seed is None else noise_seed), 1])
    if spec.noise_std > 0:
        scene += nrng.normal(0.0, spec.noise_std, (H, W))
    if spec.dtype == "f32":
        img = scene.astype(np.float32)
    else:
        q = np.clip(np.rint(scene), 0.0, spec.vmax)
        img = q.astype(np.uint8 if spec.dtype == "u8" else np.uint16)
    if not return_truth:
        return img
    truth = dict(cx=cx, cy=cy, r=r, s=s, lines_p0=lp0, lines_p1=lp1, lines_w=lw)
    return img, truth


# ----------------------------------------------------------------------------
# the five workloads (seeds, sizes and value distributions)
# ----------------------------------------------------------------------------

def scene512_u8_spec(sigma_d=0.0, H=512, W=512):
    return SceneSpec(H=H, W=W, bg=128.0, noise_std=8.0, n_blobs=200, r_range=(2.0, 8.0),
                     amp=-60.0, n_lines=20, line_w=(3, 3), dtype="u8", vmax=255.0,
                     sigma_d=sigma_d)


def pair512_u8(seed=1, H=512, W=512, return_truth=False):
    """512x512 uint8 in-focus image A and the same scene defocused (sigma_d=3) B."""
    a = make_scene(seed, scene512_u8_spec(0.0, H, W), return_truth=return_truth)
    b = make_scene(seed, scene512_u8_spec(3.0, H, W), return_truth=False)
    return a, b


def scene12bit_spec(sigma_d=0.0, H=4096, W=4096, dtype="u16"):
    scale = (H * W) / float(4096 * 4096)
    n_blobs = int(round(20000 * scale))
    n_lines = int(round(300 * scale))
    if dtype == "u8":     # the 12-bit scene mapped onto 8 bits
        f = 255.0 / 4095.0
        return SceneSpec(H=H, W=W, bg=2000.0 * f, noise_std=80.0 * f, n_blobs=n_blobs,
                         r_range=(2.0, 12.0), amp=-600.0 * f, n_lines=n_lines,
                         line_w=(2, 5), dtype="u8", vmax=255.0, sigma_d=sigma_d)
    return SceneSpec(H=H, W=W, bg=2000.0, noise_std=80.0, n_blobs=n_blobs,
                     r_range=(2.0, 12.0), amp=-600.0, n_lines=n_lines, line_w=(2, 5),
                     dtype=dtype, vmax=4095.0, sigma_d=sigma_d)


def _cache_path(tag):
    """Rendered large tiles are kept (MHFD_SYNTH_CACHE, else `.synth_cache`
    at the repository root, which version control and copies skip)."""
    root = os.environ.get("MHFD_SYNTH_CACHE") or os.path.join(
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".synth_cache")
    return os.path.join(root, tag + ".npy")


def _cached(tag, fn):
    path = _cache_path(tag)
    if os.path.exists(path):
        try:
            return np.load(path)
        except Exception:
            pass
    img = fn()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path[:-4] + ".%d.tmp.npy" % os.getpid()
        np.save(tmp, img)
        os.replace(tmp, path)
    except Exception:
        pass
    return img


def sweep_tile_4096_u16(sigma_d=0.0, seed=2, H=4096, W=4096, dtype="u16", cache=True):
    """4096x4096 12-bit tile (uint16), mean 2000, noise 80, 20k blobs, 300 lines."""
    spec = scene12bit_spec(sigma_d, H, W, dtype)
    if not cache:
        return make_scene(seed, spec)
    tag = "c2_s%d_%dx%d_%s_sd%g" % (seed, H, W, dtype, sigma_d)
    return _cached(tag, lambda: make_scene(seed, spec))


_UNEVEN_SIZES = ((1024, 1024), (1536, 2048), (3072, 3072), (4096, 4096))


def uneven_batch_specs(count=256, base_seed=3000):
    """Per-tile (seed, H, W, dtype, sigma_d) of the uneven batch."""
    out = []
    for j in range(count):
        rng = np.random.default_rng([base_seed + j, 7])
        H, W = _UNEVEN_SIZES[int(rng.integers(0, len(_UNEVEN_SIZES)))]
        dtype = "u8" if rng.integers(0, 2) == 0 else "u16"
        sd = float(rng.uniform(0.0, 6.0))
        out.append((base_seed + j, H, W, dtype, sd))
    return out


def uneven_batch_tile(seed, H, W, dtype, sigma_d):
    base = scene12bit_spec(sigma_d, H, W, dtype)
    n_blobs = int(round(1.2e-3 * H * W))
    spec = dataclasses.replace(base, n_blobs=n_blobs)
    return make_scene(seed, spec)


def soft_tile_f32(j, H=2048, W=2048, base_seed=4000):
    """2048x2048 float32 tile of the 12-bit scene (not quantised), known sigma_d."""
    rng = np.random.default_rng([base_seed + j, 9])
    sd = float(rng.uniform(0.0, 8.0))
    spec = scene12bit_spec(sd, H, W, "f32")
    return make_scene(base_seed + j, spec), sd


def random_candidates(seed, n, H, W, n_levels, *, cluster=0.0):
    """Seeded synthetic candidate lists (x, y, scale index, f32 response) with
    unique (x, y, i) for exercising the overlap prune on identical inputs.
    ``cluster`` in [0,1) concentrates points so that many overlap."""
    rng = np.random.default_rng([int(seed), 3])
    if cluster > 0:
        nc = max(1, int(n * (1.0 - cluster) / 4) + 1)
        cxy = np.stack([rng.uniform(0, W, nc), rng.uniform(0, H, nc)], 1)
        pick = rng.integers(0, nc, n)
        xy = cxy[pick] + rng.normal(0, 6.0, (n, 2))
    else:
        xy = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1)
    x = np.clip(np.floor(xy[:, 0]), 0, W - 1).astype(np.int32)
    y = np.clip(np.floor(xy[:, 1]), 0, H - 1).astype(np.int32)
    i = rng.integers(0, n_levels, n).astype(np.int32)
    key = (y.astype(np.int64) * W + x) * 64 + i
    _, first = np.unique(key, return_index=True)
    first.sort()
    x, y, i = x[first], y[first], i[first]
    # responses quantised coarsely so that exact ties occur and exercise the
    # tie-break order
    resp = (np.round(rng.uniform(0.05, 1.0, x.size) * 64.0) / 64.0).astype(np.float32)
    return x, y, i, resp


def uneven_batch_tile_cached(seed, H, W, dtype, sigma_d):
    """``uneven_batch_tile`` kept in the tile cache."""
    tag = "c3_s%d_%dx%d_%s_sd%.9g" % (seed, H, W, dtype, sigma_d)
    return _cached(tag, lambda: uneven_batch_tile(seed, H, W, dtype, sigma_d))


def soft_tile_f32_cached(j, H=2048, W=2048, base_seed=4000):
    """``soft_tile_f32`` with the image kept in the tile cache."""
    rng = np.random.default_rng([base_seed + j, 9])
    sd = float(rng.uniform(0.0, 8.0))
    tag = "c4_s%d_%dx%d_f32" % (base_seed + j, H, W)
    return _cached(tag, lambda: soft_tile_f32(j, H, W, base_seed)[0]), sd


def _render_one(job):
    name, args = job
    globals()[name](*args)
    return 0


def render_parallel(name, arglist, workers=None):
    """Fills the tile cache for ``name(*args)`` over ``arglist`` (one of the
    ``*_cached`` renderers) in worker processes started with ``spawn``, then
    returns the results in order, loaded from the cache."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    todo = [(name, tuple(a)) for a in arglist]
    todo = [j for j in todo if not _is_cached(j)]
    workers = min(workers or min(16, os.cpu_count() or 1), len(todo))
    if workers > 1:
        # a worker that dies raises BrokenProcessPool here instead of hanging
        with ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            list(ex.map(_render_one, todo))
    return [globals()[name](*a) for a in arglist]


def _is_cached(job):
    name, args = job
    if name == "uneven_batch_tile_cached":
        seed, H, W, dtype, sd = args
        tag = "c3_s%d_%dx%d_%s_sd%.9g" % (seed, H, W, dtype, sd)
    elif name == "soft_tile_f32_cached":
        j = args[0]
        H, W, base = (list(args[1:]) + [2048, 2048, 4000][len(args) - 1:])[:3]
        tag = "c4_s%d_%dx%d_f32" % (base + j, H, W)
    else:
        return False
    return os.path.exists(_cache_path(tag))
