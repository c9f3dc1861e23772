"""Comparison rules between the CUDA path and the FP64 oracle.

Floating point: the response stack must satisfy, per DoG layer i,
    max |D_gpu - D_ref| <= 1e-4 * ||D_ref,i||_inf.
Integer outputs (feature lists, counts, survivors) must match exactly,
except for features the rules call *ambiguous*, where f32 rounding may
legitimately decide differently than f64 (eps = 1e-4 * ||D_ref,i||_inf):
  * the response is within eps of the threshold;
  * a neighbour in the comparison window is within eps of it;
  * (scale index only) two scales are within eps for the argmax.
Pruning decisions are compared per connected component of the conflict
graph: components that contain an ambiguous feature, or two conflicting
features of one scale whose responses are within eps (their visiting order
may flip), are excluded; every other kept/dropped decision must match.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

REL_TOL = 1e-4


def layer_eps(D_ref):
    return REL_TOL * np.abs(D_ref).reshape(D_ref.shape[0], -1).max(axis=1)


def assert_stack_close(D_gpu, D_ref, where=""):
    eps = layer_eps(D_ref)
    for i in range(D_ref.shape[0]):
        err = np.abs(D_gpu[i].astype(np.float64) - D_ref[i]).max()
        assert err <= max(eps[i], 1e-12), "%s layer %d: max err %.3g > tol %.3g" % (
            where, i, err, eps[i])


def _shift(a, dy, dx, fill):
    out = np.full_like(a, fill)
    H, W = a.shape
    ys = slice(max(0, dy), H + min(0, dy)); yd = slice(max(0, -dy), H + min(0, -dy))
    xs = slice(max(0, dx), W + min(0, dx)); xd = slice(max(0, -dx), W + min(0, -dx))
    out[yd, xd] = a[ys, xs]
    return out


def log_eps(D_ref, t, R, Lmax):
    """Per-layer tolerance of the scale-normalised Laplacian response.

    The 5-point stencil subtracts level values of size |L| to leave a
    curvature about t^2 times smaller, so the f32 rounding of L (about
    sqrt(2R+1) roundings of size 2^-24 |L| per pass) reaches the response
    multiplied by t^2 and by the stencil's weight sum 8:
        eps_i = max(1e-4 ||D_ref,i||, 16 sqrt(2R_i+1) t_i^2 2^-24 max|L|)
    (twice the 8 of the stencil: two blur passes)."""
    base = layer_eps(D_ref)
    t = np.asarray(t, dtype=np.float64)[: D_ref.shape[0]]
    R = np.asarray(R, dtype=np.float64)[: D_ref.shape[0]]
    cancel = 16.0 * np.sqrt(2 * R + 1) * t ** 2 * 2.0 ** -24 * Lmax
    return np.maximum(base, cancel)


def ambiguous_paper(D_ref, thr, eps=None):
    """Boolean (H, W) map of pixels whose paper-rule decision is ambiguous."""
    eps = float(layer_eps(D_ref).max() if eps is None else np.max(eps))
    M = D_ref.max(axis=0)
    amb = np.abs(M - thr) <= eps
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            nb = _shift(M, dy, dx, -np.inf)   # nb[y, x] = M[y+dy, x+dx]
            amb |= np.isfinite(nb) & (np.abs(nb - M) <= eps)
    srt = np.sort(D_ref, axis=0)
    amb_scale = (srt[-1] - srt[-2] <= eps) if D_ref.shape[0] > 1 else np.zeros_like(amb)
    return amb, amb_scale, eps


def ambiguous_26(D_ref, thr, eps=None):
    """Boolean (n, H, W) map of ambiguous 26-neighbour decisions."""
    eps = layer_eps(D_ref).max() if eps is None else np.max(eps)
    n = D_ref.shape[0]
    amb = np.abs(D_ref - thr) <= eps
    for di in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if di == 0 and dy == 0 and dx == 0:
                    continue
                nb = np.full_like(D_ref, -np.inf)
                for i in range(n):
                    j = i + di
                    if 0 <= j < n:
                        nb[i] = _shift(D_ref[j], dy, dx, -np.inf)
                amb |= np.isfinite(nb) & (np.abs(nb - D_ref) <= eps)
    return amb, float(eps)


def compare_feature_sets(got, want, is_ambiguous):
    """got/want: sets of (x, y, i).  Differences must all be ambiguous."""
    diff = got ^ want
    bad = [f for f in diff if not is_ambiguous(f)]
    assert not bad, "unambiguous feature mismatches (first 10): %s" % sorted(bad)[:10]
    return len(diff)


def conflict_components(feats, radius, overlap):
    """feats: list of (x, y, i).  Union-find over conflicting pairs."""
    n = len(feats)
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    if n == 0:
        return parent, []
    rmax = max(radius)
    cell = 2 * rmax + 1
    grid = {}
    for k, (x, y, i) in enumerate(feats):
        grid.setdefault((int(x // cell), int(y // cell)), []).append(k)
    pairs = []
    for k, (x, y, i) in enumerate(feats):
        cx, cy = int(x // cell), int(y // cell)
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                for m in grid.get((gx, gy), ()):
                    if m <= k:
                        continue
                    x2, y2, i2 = feats[m]
                    d = math.hypot(x - x2, y - y2)
                    if oracle.lens_overlap(radius[i], radius[i2], d) > overlap:
                        pairs.append((k, m))
                        ra, rb = find(k), find(m)
                        if ra != rb:
                            parent[ra] = rb
    return [find(k) for k in range(n)], pairs
