"""Comparison rules between the CUDA path and the FP64 oracle.

Floating point: the response stack must satisfy, per response layer i,
    max |D_gpu,i - D_ref,i| <= eps_i,    eps_i = 1e-4 * ||D_ref,i||_inf
(a wider, derived eps_i for the 5-point LoG stencil of the plain path).
Integer outputs (feature lists, counts, survivors) must match exactly,
except for decisions the rules call *ambiguous*, where f32 rounding may
legitimately decide differently than f64.  Each decision is judged with the
tolerances of the layers it involves:
  * paper rule at pixel p: the layers that compete for the argmax are the
    reference argmax a(p) and every layer j within max(eps_a, eps_j) of the
    top; e(p) is the largest eps of those layers.  The scale is ambiguous
    when another layer competes; the pixel is ambiguous when |M - tau| <=
    e(p) or an in-image 8-neighbour q has |M(q) - M(p)| <= max(e(p), e(q));
  * 26-neighbour rule at (p, i): |D_i - tau| <= eps_i, or a neighbour
    (q, j) of the 3x3x3 window has |D_j(q) - D_i(p)| <= max(eps_i, eps_j).
Pruning decisions are compared per connected component of the conflict
graph: components that contain an ambiguous feature, a feature found by
only one side, or two conflicting same-scale features whose responses are
within their layer's eps (their visiting order may flip) are excluded;
every other kept/dropped decision must match.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

REL_TOL = 1e-4


def layer_eps(D_ref):
    return REL_TOL * np.abs(D_ref).reshape(D_ref.shape[0], -1).max(axis=1)


def assert_stack_close(D_gpu, D_ref, where="", tol=None):
    eps = layer_eps(D_ref) if tol is None else np.asarray(tol, np.float64)
    for i in range(D_ref.shape[0]):
        err = np.abs(D_gpu[i].astype(np.float64) - D_ref[i]).max()
        assert err <= max(eps[i], 1e-12), "%s layer %d: max err %.3g > tol %.3g" % (
            where, i, err, eps[i])


def stack_rel_err(D_gpu, D_ref):
    """Per-layer max |D_gpu - D_ref| / ||D_ref,i||_inf (for reporting)."""
    out = []
    for i in range(D_ref.shape[0]):
        nrm = max(float(np.abs(D_ref[i]).max()), 1e-300)
        out.append(float(np.abs(D_gpu[i].astype(np.float64) - D_ref[i]).max()) / nrm)
    return np.array(out)


def _shift(a, dy, dx, fill):
    out = np.full_like(a, fill)
    H, W = a.shape
    ys = slice(max(0, dy), H + min(0, dy)); yd = slice(max(0, -dy), H + min(0, -dy))
    xs = slice(max(0, dx), W + min(0, dx)); xd = slice(max(0, -dx), W + min(0, -dx))
    out[yd, xd] = a[ys, xs]
    return out


def log_eps(D_ref, t, R, Lmax):
    """Per-layer tolerance of the 5-point scale-normalised Laplacian.

    The 5-point stencil subtracts level values of size |L| to leave a
    curvature about t^2 times smaller, so the f32 rounding of L (about
    sqrt(2R+1) roundings of size 2^-24 |L| per pass) reaches the response
    multiplied by t^2 and by the stencil's weight sum 8:
        eps_i = max(1e-4 ||D_ref,i||, 16 sqrt(2R_i+1) t_i^2 2^-24 max|L|)
    (twice the 8 of the stencil: two blur passes).  Only the plain path's
    stencil needs this; the fused kernel's derived taps are held to
    1e-4 ||D_ref,i||."""
    base = layer_eps(D_ref)
    t = np.asarray(t, dtype=np.float64)[: D_ref.shape[0]]
    R = np.asarray(R, dtype=np.float64)[: D_ref.shape[0]]
    cancel = 16.0 * np.sqrt(2 * R + 1) * t ** 2 * 2.0 ** -24 * Lmax
    return np.maximum(base, cancel)


def ambiguous_paper(D_ref, thr, tol=None):
    """Paper rule: (amb, amb_scale, e) as (H, W) maps; ``tol`` per layer."""
    n = D_ref.shape[0]
    tol = layer_eps(D_ref) if tol is None else np.asarray(tol, np.float64)
    M = D_ref.max(axis=0)
    A = D_ref.argmax(axis=0)
    eA = tol[A]
    e = eA.copy()
    amb_scale = np.zeros(M.shape, bool)
    for j in range(n):
        comp = (A != j) & (M - D_ref[j] <= np.maximum(eA, tol[j]))
        amb_scale |= comp
        np.maximum(e, np.where(comp, tol[j], 0.0), out=e)
    amb = np.abs(M - thr) <= e
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            nb = _shift(M, dy, dx, -np.inf)   # nb[y, x] = M[y+dy, x+dx]
            ne = _shift(e, dy, dx, 0.0)
            amb |= np.isfinite(nb) & (np.abs(nb - M) <= np.maximum(e, ne))
    return amb, amb_scale, e


def ambiguous_26(D_ref, thr, tol=None):
    """26-neighbour rule: boolean (n, H, W) map of ambiguous decisions."""
    tol = layer_eps(D_ref) if tol is None else np.asarray(tol, np.float64)
    n = D_ref.shape[0]
    tl = tol[:, None, None]
    amb = np.abs(D_ref - thr) <= tl
    for di in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if di == 0 and dy == 0 and dx == 0:
                    continue
                for i in range(n):
                    j = i + di
                    if not 0 <= j < n:
                        continue
                    nb = _shift(D_ref[j], dy, dx, -np.inf)
                    amb[i] |= np.isfinite(nb) & (np.abs(nb - D_ref[i]) <=
                                                 max(tol[i], tol[j]))
    return amb


def ambiguous_26_at(D_ref, thr, tol, feats):
    """``ambiguous_26`` evaluated at the items ``feats`` (x, y, i) only: the
    same predicate, without the whole-stack maps (which a 4096^2 stack of 16
    layers makes slow).  Returns the set of ambiguous items."""
    tol = layer_eps(D_ref) if tol is None else np.asarray(tol, np.float64)
    f = np.array(sorted(feats), dtype=np.int64).reshape(-1, 3)
    if not len(f):
        return set()
    n, H, W = D_ref.shape
    x, y, i = f[:, 0], f[:, 1], f[:, 2]
    v = D_ref[i, y, x]
    amb = np.abs(v - thr) <= tol[i]
    for di in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if di == 0 and dy == 0 and dx == 0:
                    continue
                j, yy, xx = i + di, y + dy, x + dx
                inside = (j >= 0) & (j < n) & (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
                jc, yc, xc = np.clip(j, 0, n - 1), np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)
                nb = D_ref[jc, yc, xc]
                amb |= inside & (np.abs(nb - v) <= np.maximum(tol[i], tol[jc]))
    return {tuple(int(c) for c in row) for row in f[amb]}


def compare_feature_sets(got, want, is_ambiguous):
    """got/want: sets of (x, y, i).  Differences must all be ambiguous."""
    diff = got ^ want
    bad = [f for f in diff if not is_ambiguous(f)]
    assert not bad, "unambiguous feature mismatches (first 10): %s" % sorted(bad)[:10]
    return len(diff)


def conflict_components(feats, radius, overlap):
    """feats: list of (x, y, i).  Union-find over conflicting pairs (the
    oracle's lens overlap above ``overlap``)."""
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
    cand_a, cand_b = [], []
    for k, (x, y, i) in enumerate(feats):
        cx, cy = int(x // cell), int(y // cell)
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                for m in grid.get((gx, gy), ()):
                    if m > k:
                        cand_a.append(k)
                        cand_b.append(m)
    pairs = []
    if cand_a:
        fa = np.asarray(feats, np.int64)
        a = np.asarray(cand_a, np.int64)
        b = np.asarray(cand_b, np.int64)
        rad = np.asarray(radius, np.float64)
        d = np.hypot((fa[a, 0] - fa[b, 0]).astype(np.float64),
                     (fa[a, 1] - fa[b, 1]).astype(np.float64))
        near = d < rad[fa[a, 2]] + rad[fa[b, 2]]
        a, b, d = a[near], b[near], d[near]
        ov = oracle.lens_overlap_many(rad[fa[a, 2]], rad[fa[b, 2]], d)
        for k, m in zip(a[ov > overlap].tolist(), b[ov > overlap].tolist()):
            pairs.append((k, m))
            ra, rb = find(k), find(m)
            if ra != rb:
                parent[ra] = rb
    return [find(k) for k in range(n)], pairs


def features(arr):
    return {(int(b["x"]), int(b["y"]), int(b["scale_idx"])) for b in arr}


def check_detection(res, ref, D_ref, tol, thr, overlap, nms, t, amb_maps=None):
    """Holds one GPU detection ``res`` (candidates kept) to the oracle's
    ``ref`` (x, y, i, resp, keep, score, mean_response) and its response
    stack ``D_ref`` with per-layer tolerances ``tol``.  ``amb_maps`` may pass
    the paper rule's ``ambiguous_paper(D_ref, thr, tol)`` computed once for
    several checks.  Returns counts of the differences the ambiguity rules
    excuse."""
    n = D_ref.shape[0]
    tol = np.asarray(tol, np.float64)
    got_c = features(res.candidates)
    want_c = set(zip(ref.x.tolist(), ref.y.tolist(), ref.i.tolist()))
    if nms == "paper":
        amb, amb_scale, _ = amb_maps if amb_maps is not None else ambiguous_paper(D_ref, thr, tol)
        is_amb = lambda f: bool(amb[f[1], f[0]] or amb_scale[f[1], f[0]])  # noqa: E731
        got_px = {(x, y) for x, y, _ in got_c}
        want_px = {(x, y) for x, y, _ in want_c}
        bad = [p for p in got_px ^ want_px if not amb[p[1], p[0]]]
        assert not bad, ("unambiguous position mismatches", bad[:10])
        bad = [(x, y, i) for x, y, i in got_c
               if (x, y) in want_px and not amb_scale[y, x] and (x, y, i) not in want_c]
        assert not bad, ("unambiguous scale mismatches", bad[:10])
        n_amb = int(sum(1 for f in got_c | want_c if is_amb(f)))
    else:
        amb = ambiguous_26_at(D_ref, thr, tol, got_c | want_c)
        is_amb = lambda f: f in amb  # noqa: E731
        compare_feature_sets(got_c, want_c, is_amb)
        n_amb = int(sum(1 for f in got_c | want_c if is_amb(f)))
    assert res.n_candidates == res.n_candidates_true == len(got_c)
    # responses of common features within their layer's tolerance
    resp_ref = {(int(x), int(y), int(i)): r for x, y, i, r in zip(ref.x, ref.y, ref.i, ref.resp)}
    bad = []
    for b in res.candidates:
        key = (int(b["x"]), int(b["y"]), int(b["scale_idx"]))
        if key in resp_ref and abs(float(b["response"]) - resp_ref[key]) > tol[key[2]]:
            bad.append((key, float(b["response"]), resp_ref[key]))
    assert not bad, ("responses outside the layer tolerance", bad[:10])
    # pruning: compare kept/dropped outside components touched by ambiguity
    kept_got = features(res.blobs)
    kept_want = {f for f, k in zip(zip(ref.x.tolist(), ref.y.tolist(), ref.i.tolist()), ref.keep)
                 if k}
    feats = sorted(got_c | want_c)
    radius = list(math.sqrt(2.0) * np.asarray(t)[:n])
    comp, pairs = conflict_components(feats, radius, overlap)
    tainted = {comp[k] for k, f in enumerate(feats) if is_amb(f) or (f in got_c) != (f in want_c)}
    resp_any = dict(resp_ref)
    for b in res.candidates:
        resp_any.setdefault((int(b["x"]), int(b["y"]), int(b["scale_idx"])), float(b["response"]))
    for a, b in pairs:
        fa, fb = feats[a], feats[b]
        if fa[2] == fb[2] and abs(resp_any[fa] - resp_any[fb]) <= tol[fa[2]]:
            tainted.add(comp[a])
    mism = [f for k, f in enumerate(feats)
            if comp[k] not in tainted and ((f in kept_got) != (f in kept_want))]
    assert not mism, ("unambiguous prune mismatches", mism[:10])
    if not tainted:
        assert res.n_blobs == ref.score
    assert res.focus_score == res.n_blobs == len(kept_got)
    per_scale = (np.bincount([f[2] for f in kept_got], minlength=n)[:n] if kept_got
                 else np.zeros(n, np.int64))
    assert np.array_equal(res.per_scale[:n], per_scale)
    # mean response of the kept features: each within its layer's tolerance
    if kept_got == kept_want:
        err = abs(res.mean_response - ref.mean_response)
        assert err <= float(tol.max()) + 1e-6 * abs(ref.mean_response), (
            res.mean_response, ref.mean_response)
    return {"candidates_gpu": len(got_c), "candidates_ref": len(want_c),
            "candidate_diffs": len(got_c ^ want_c), "ambiguous": n_amb,
            "kept_gpu": len(kept_got), "kept_ref": len(kept_want),
            "kept_diffs": len(kept_got ^ kept_want), "tainted_components": len(tainted)}


def oracle_reference(img, n, tmin, tmax, thr, overlap, nms="paper", response="dog",
                     boundary="reflect", truncate=4.0):
    """The oracle's detection of ``img`` together with its response stack
    and per-layer tolerances: (ref, D_ref, tol, t).  The stack is computed
    once and the detection composed from the oracle's own steps (stretch,
    stack, maxima, prune: the same chain as ``oracle.detect``)."""
    lo, hi = oracle.stretch_bounds(img)
    t = oracle.ladder(n, tmin, tmax)
    Ip = oracle.stretch(img, lo, hi)
    bnd = oracle.PERIODIC if boundary == "periodic" else oracle.REFLECT
    if response == "log":
        D = oracle.log_stack(Ip, t, truncate=truncate, boundary=bnd)
    else:
        D = oracle.dog_stack(Ip, t, truncate=truncate, boundary=bnd)
    ref = oracle.detect_from_stack(D, t, thr, overlap, mode=0 if nms == "paper" else 1)
    ref["lo"], ref["hi"] = lo, hi
    return ref, D, layer_eps(D), t, Ip
