"""FP64 CPU oracle of the multi-scale feature detector (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The arithmetic lives in plain C
(``mhfd_oracle.c``, compiled here with gcc); this module only marshals numpy
arrays.  It shares nothing with the CUDA path.

Every function cites the passage of the paper it follows:

* ``stretch_bounds`` / ``stretch``: §3, histogram stretching (0.175 % each end);
* ``ladder``: §2.2, ``t_i = min_t + (i-1)(max_t - min_t)/n``, ``i = 1..n+1``;
* ``kernel``: §2.2, sampled Gaussian of variance ``t^2``, truncated, normalised;
* ``blur``: §2.2, ``L = G * I`` (separable, reflect or periodic boundary);
* ``dog_stack``: Eq. 2, ``DoG_i = t_i (L_{i+1} - L_i)``;
* ``nms_paper``: Eq. 3 (argmax over scales, then 3x3 max-pool comparison);
* ``nms_local26``: 3x3x3 scale-space maxima;
* ``lens_overlap`` / ``prune``: greedy overlap pruning (not in the paper);
* ``detect``: Algorithm 1 end to end plus threshold and prune, with the
  per-image statistics: the count |C| (the DOF of Algorithm 1), the count
  per scale and the mean response of the kept features;
* ``detect_from_stack``: the same steps after the stack, on a given stack.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhfd_oracle.c")
_LIB = os.path.join(_HERE, "libmhfd_oracle.so")
_lock = threading.Lock()
_lib = None

U8, U16, F32 = 0, 1, 2
REFLECT, PERIODIC = 0, 1
MODE_PAPER, MODE_LOCAL26 = 0, 1

_DTYPE_CODE = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float32): F32}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", "-Wall"]
    tmp = _LIB + ".%d.tmp" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_stretch_bounds.argtypes = [P, i32, i64, i64, i64, dbl, P, P]
        lib.oracle_stretch_bounds.restype = i32
        lib.oracle_stretch.argtypes = [P, i32, i64, i64, i64, dbl, dbl, P]
        lib.oracle_ladder.argtypes = [i32, dbl, dbl, P]
        lib.oracle_kernel_radius.argtypes = [dbl, dbl]
        lib.oracle_kernel_radius.restype = i32
        lib.oracle_kernel.argtypes = [dbl, i32, P]
        lib.oracle_blur.argtypes = [P, i64, i64, P, i32, i32, P]
        lib.oracle_dog_stack.argtypes = [P, i64, i64, P, i32, dbl, i32, P]
        lib.oracle_nms_paper.argtypes = [P, i32, i64, i64, dbl, P, P, P, P, i64]
        lib.oracle_nms_paper.restype = i64
        lib.oracle_nms_local26.argtypes = [P, i32, i64, i64, dbl, P, P, P, P, i64]
        lib.oracle_nms_local26.restype = i64
        lib.oracle_lens_overlap.argtypes = [dbl, dbl, dbl]
        lib.oracle_lens_overlap.restype = dbl
        lib.oracle_lens_overlap_many.argtypes = [P, P, P, i64, P]
        lib.oracle_prune.argtypes = [P, P, P, P, i64, P, i32, dbl, i64, P]
        lib.oracle_prune.restype = i64
        lib.oracle_dog_at.argtypes = [P, i32, i64, i64, i64, dbl, dbl, P, i32, dbl, i64, i64, P]
        lib.oracle_dog_at_many.argtypes = [P, i32, i64, i64, i64, dbl, dbl, P, i32, dbl, P, P,
                                           i64, P]
        lib.oracle_detect.argtypes = [P, i32, i64, i64, i64, i32, dbl, dbl, dbl, dbl, dbl, dbl,
                                      i32, P, P, P, P, P, i64, P, P, P]
        lib.oracle_detect.restype = i64
        lib.oracle_log_stack.argtypes = [P, i64, i64, P, i32, dbl, i32, P]
        lib.oracle_detect_ex.argtypes = [P, i32, i64, i64, i64, i32, dbl, dbl, dbl, dbl, dbl, dbl,
                                         i32, i32, i32, P, P, P, P, P, i64, P, P, P]
        lib.oracle_detect_ex.restype = i64
        lib.oracle_blur_adjoint.argtypes = [P, i64, i64, P, i32, i32, P]
        lib.oracle_soft_score.argtypes = [P, i32, i64, i64, i64, dbl, dbl, P, i32, dbl, dbl, dbl, P,
                                          P, P]
        lib.oracle_soft_score.restype = dbl
        lib.oracle_set_threads.argtypes = [i32]
        lib.oracle_get_threads.restype = i32
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def _img_args(img):
    img = np.ascontiguousarray(img)
    if img.dtype not in _DTYPE_CODE:
        raise TypeError("image dtype must be uint8, uint16 or float32")
    H, W = img.shape
    return img, _DTYPE_CODE[img.dtype], H, W, img.strides[0]


def stretch_bounds(img, clip=0.00175):
    """§3: (lo, hi) = the k-th smallest and (N-1-k)-th smallest values, k=floor(clip*N)."""
    img, code, H, W, rs = _img_args(img)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = _load().oracle_stretch_bounds(_ptr(img), code, H, W, rs, clip, ctypes.byref(lo),
                                       ctypes.byref(hi))
    if rc != 0:
        raise ValueError("empty image")
    return lo.value, hi.value


def stretch(img, lo, hi):
    """§3: I' = clip((I - lo) / (hi - lo), 0, 1) in FP64."""
    img, code, H, W, rs = _img_args(img)
    out = np.empty((H, W), np.float64)
    _load().oracle_stretch(_ptr(img), code, H, W, rs, float(lo), float(hi), _ptr(out))
    return out


def ladder(n, tmin, tmax):
    """§2.2: the n+1 Gaussian scales t_1..t_{n+1}."""
    t = np.empty(n + 1, np.float64)
    _load().oracle_ladder(int(n), float(tmin), float(tmax), _ptr(t))
    return t


def kernel_radius(t, truncate=4.0):
    return int(_load().oracle_kernel_radius(float(t), float(truncate)))


def kernel(t, truncate=4.0, R=None):
    """§2.2: normalised sampled Gaussian taps g[-R..R]."""
    if R is None:
        R = kernel_radius(t, truncate)
    g = np.empty(2 * R + 1, np.float64)
    _load().oracle_kernel(float(t), int(R), _ptr(g))
    return g


def blur(img2d, g, boundary=REFLECT):
    """§2.2: separable convolution (columns then rows) with taps g."""
    a = np.ascontiguousarray(img2d, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    H, W = a.shape
    out = np.empty_like(a)
    _load().oracle_blur(_ptr(a), H, W, _ptr(g), (g.size - 1) // 2, int(boundary), _ptr(out))
    return out


def dog_stack(Ip, t, truncate=4.0, boundary=REFLECT):
    """Eq. 2 over the ladder t (n+1 scales) -> D of shape (n, H, W)."""
    a = np.ascontiguousarray(Ip, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    H, W = a.shape
    n = t.size - 1
    D = np.empty((n, H, W), np.float64)
    _load().oracle_dog_stack(_ptr(a), H, W, _ptr(t), n, float(truncate), int(boundary), _ptr(D))
    return D


def log_stack(Ip, t, truncate=4.0, boundary=REFLECT):
    """§2.2: t_i^2 grad^2 L(t_i) for the first n scales (5-point Laplacian) -> (n, H, W)."""
    a = np.ascontiguousarray(Ip, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    H, W = a.shape
    n = t.size - 1
    D = np.empty((n, H, W), np.float64)
    _load().oracle_log_stack(_ptr(a), H, W, _ptr(t), n, float(truncate), int(boundary), _ptr(D))
    return D


def _nms(fn, D, thr, cap):
    D = np.ascontiguousarray(D, dtype=np.float64)
    n, H, W = D.shape
    cap = int(cap if cap is not None else H * W * (1 if fn == "paper" else n))
    cap = max(cap, 1)
    x = np.empty(cap, np.int32); y = np.empty(cap, np.int32); i = np.empty(cap, np.int32)
    r = np.empty(cap, np.float64)
    f = _load().oracle_nms_paper if fn == "paper" else _load().oracle_nms_local26
    cnt = f(_ptr(D), n, H, W, float(thr), _ptr(x), _ptr(y), _ptr(i), _ptr(r), cap)
    m = min(cnt, cap)
    return x[:m].copy(), y[:m].copy(), i[:m].copy(), r[:m].copy(), int(cnt)


def nms_paper(D, thr, cap=None):
    """Eq. 3: features (x, y, i_hat, M) of the argmax / 3x3 max-pool rule."""
    return _nms("paper", D, thr, cap)


def nms_local26(D, thr, cap=None):
    """3x3x3 scale-space local maxima above thr."""
    return _nms("local26", D, thr, cap)


def lens_overlap(r1, r2, d):
    return float(_load().oracle_lens_overlap(float(r1), float(r2), float(d)))


def lens_overlap_many(r1, r2, d):
    """``lens_overlap`` elementwise over equal-length arrays."""
    r1 = np.ascontiguousarray(r1, np.float64); r2 = np.ascontiguousarray(r2, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    out = np.empty(d.size, np.float64)
    if d.size:
        _load().oracle_lens_overlap_many(_ptr(r1), _ptr(r2), _ptr(d), d.size, _ptr(out))
    return out


def prune(x, y, i, resp, radius, overlap, W):
    """Greedy overlap prune; returns a uint8 keep mask."""
    x = np.ascontiguousarray(x, np.int32); y = np.ascontiguousarray(y, np.int32)
    i = np.ascontiguousarray(i, np.int32); resp = np.ascontiguousarray(resp, np.float64)
    radius = np.ascontiguousarray(radius, np.float64)
    keep = np.zeros(x.size, np.uint8)
    if x.size:
        _load().oracle_prune(_ptr(x), _ptr(y), _ptr(i), _ptr(resp), x.size, _ptr(radius),
                             radius.size, float(overlap), int(W), _ptr(keep))
    return keep


def dog_at(img, lo, hi, t, xs, ys, truncate=4.0):
    """Eq. 2 at chosen pixels straight from the raw image -> (m, n)."""
    img, code, H, W, rs = _img_args(img)
    t = np.ascontiguousarray(t, np.float64)
    xs = np.ascontiguousarray(xs, np.int64); ys = np.ascontiguousarray(ys, np.int64)
    n = t.size - 1
    D = np.empty((xs.size, n), np.float64)
    if xs.size:
        _load().oracle_dog_at_many(_ptr(img), code, H, W, rs, float(lo), float(hi), _ptr(t), n,
                                   float(truncate), _ptr(xs), _ptr(ys), xs.size, _ptr(D))
    return D


def blur_adjoint(img2d, g, boundary=REFLECT):
    """Transpose of ``blur`` (same taps and boundary)."""
    a = np.ascontiguousarray(img2d, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    H, W = a.shape
    out = np.empty_like(a)
    _load().oracle_blur_adjoint(_ptr(a), H, W, _ptr(g), (g.size - 1) // 2, int(boundary), _ptr(out))
    return out


def soft_score(img, n, tmin, tmax, w, *, tau, T=0.01, lo=None, hi=None, truncate=4.0,
               grad=True):
    """Soft focus score S = sum_i w_i mean sigmoid((D_i - tau)/T) with the
    stretch bounds held fixed (computed from the image if not given).
    Returns (S, mean_sig (= dS/dw), dS/dI or None)."""
    img, code, H, W, rs = _img_args(img)
    if lo is None or hi is None:
        lo, hi = stretch_bounds(img)
    t = ladder(n, tmin, tmax)
    w = np.ascontiguousarray(w, np.float64)
    ms = np.empty(n, np.float64)
    dimg = np.empty((H, W), np.float64) if grad else None
    S = _load().oracle_soft_score(_ptr(img), code, H, W, rs, float(lo), float(hi), _ptr(t), n,
                                  float(truncate), float(tau), float(T), _ptr(w), _ptr(ms),
                                  _ptr(dimg) if grad else None)
    return S, ms, dimg


class OracleResult(dict):
    __getattr__ = dict.__getitem__


RESP_DOG, RESP_LOG = 0, 1


def detect(img, n, tmin, tmax, *, threshold, overlap=0.5, mode=MODE_PAPER, truncate=4.0,
           clip=0.00175, cap=None, response=RESP_DOG, boundary=REFLECT):
    """Algorithm 1 (stretch, stack, DoG, argmax + max-pool) plus threshold and prune;
    optionally the scale-normalised Laplacian response and the periodic boundary."""
    img, code, H, W, rs = _img_args(img)
    cap = int(cap if cap is not None else H * W * (1 if mode == MODE_PAPER else n))
    cap = max(cap, 1)
    x = np.empty(cap, np.int32); y = np.empty(cap, np.int32); i = np.empty(cap, np.int32)
    r = np.empty(cap, np.float64); keep = np.zeros(cap, np.uint8)
    nk = ctypes.c_int64(); lo = ctypes.c_double(); hi = ctypes.c_double()
    cnt = _load().oracle_detect_ex(_ptr(img), code, H, W, rs, int(n), float(tmin), float(tmax),
                                   float(truncate), float(clip), float(threshold), float(overlap),
                                   int(mode), int(response), int(boundary), _ptr(x), _ptr(y),
                                   _ptr(i), _ptr(r), _ptr(keep), cap, ctypes.byref(nk),
                                   ctypes.byref(lo), ctypes.byref(hi))
    if cnt < 0:
        raise ValueError("oracle_detect failed")
    m = min(cnt, cap)
    keep = keep[:m].astype(bool)
    t = ladder(n, tmin, tmax)
    return _result(x[:m].copy(), y[:m].copy(), i[:m].copy(), r[:m].copy(), keep, int(cnt),
                   int(nk.value), n, t, lo=lo.value, hi=hi.value)


def _result(x, y, i, resp, keep, n_candidates, score, n, t, **extra):
    """Per-image statistics of a detection: the kept count |C|, the count per
    scale and the mean response of the kept features (0 when none is kept)."""
    per_scale = np.bincount(i[keep], minlength=n)[:n]
    mean_response = float(resp[keep].mean()) if keep.any() else 0.0
    return OracleResult(x=x, y=y, i=i, resp=resp, keep=keep, n_candidates=n_candidates,
                        score=score, per_scale=per_scale, mean_response=mean_response, t=t,
                        **extra)


def detect_from_stack(D, t, threshold, overlap=0.5, mode=MODE_PAPER):
    """The steps of ``detect`` after the response stack (Eq. 3 maxima above the
    threshold, then the greedy prune over radii sqrt(2) t_i) on a given stack
    ``D`` of shape (n, H, W) over the ladder ``t``."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    n, H, W = D.shape
    t = np.asarray(t, np.float64)
    f = nms_paper if mode == MODE_PAPER else nms_local26
    x, y, i, r, cnt = f(D, threshold)
    radius = np.sqrt(2.0) * t[:n]
    keep = prune(x, y, i, r, radius, overlap, W).astype(bool)
    return _result(x, y, i, r, keep, cnt, int(keep.sum()), n, t)
