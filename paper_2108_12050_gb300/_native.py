"""ctypes declarations of the C ABI in include/mhfd.h (argument marshalling only).

Loading fails loudly when the in-tree library has not been built: there is
no fallback implementation anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmhfd.so")

MHFD_OK = 0
MHFD_WARN_OVERFLOW = 1
MHFD_ERR_INVALID_ARG = -1
MHFD_ERR_UNSUPPORTED = -2
MHFD_ERR_OOM = -3
MHFD_ERR_CUDA = -4
MHFD_ERR_TIMEOUT = -5
MHFD_ERR_JIT = -6
MHFD_ERR_CHECK = -7

U8, U16, F32 = 0, 1, 2
NMS_PAPER, NMS_LOCAL26 = 0, 1

# every symbol include/mhfd.h declares
EXPORTS = [
    "mhfd_default_params", "mhfd_create_detector", "mhfd_destroy_detector", "mhfd_detect",
    "mhfd_result_wait", "mhfd_detect_batch", "mhfd_result_wait_batch", "mhfd_batch_uses_graph",
    "mhfd_uses_tensor_cores", "mhfd_device_bytes", "mhfd_trim",
    "mhfd_result_ready", "mhfd_soft_score",
    "mhfd_detect_host", "mhfd_detect_host_async", "mhfd_detect_plain", "mhfd_debug_stack",
    "mhfd_prune", "mhfd_prune_noalloc", "mhfd_tile_configs", "mhfd_chosen_tile", "mhfd_precompile",
    "mhfd_last_timing", "mhfd_probe_ffma_peak", "mhfd_last_error", "mhfd_version",
]


class MhfdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mhfd error %d: %s" % (code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("t_min", ctypes.c_double),
        ("t_max", ctypes.c_double),
        ("sigmas", ctypes.POINTER(ctypes.c_double)),
        ("threshold", ctypes.c_float),
        ("overlap", ctypes.c_float),
        ("nms", ctypes.c_int32),
        ("truncate", ctypes.c_float),
        ("clip_frac", ctypes.c_double),
        ("max_candidates", ctypes.c_int64),
        ("device", ctypes.c_int32),
        ("keep_candidates", ctypes.c_int32),
        ("tile_override", ctypes.c_int32),
        ("tile_shape", ctypes.c_int32 * 6),
        ("timing", ctypes.c_int32),
        ("response", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("tensor_cores", ctypes.c_int32),
    ]


class Blob(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32), ("scale_idx", ctypes.c_int32),
                ("sigma", ctypes.c_float), ("radius", ctypes.c_float),
                ("response", ctypes.c_float)]


class Result(ctypes.Structure):
    _fields_ = [
        ("blobs", ctypes.POINTER(Blob)),
        ("n_blobs", ctypes.c_int64),
        ("candidates", ctypes.POINTER(Blob)),
        ("n_candidates", ctypes.c_int64),
        ("n_candidates_true", ctypes.c_int64),
        ("focus_score", ctypes.c_float),
        ("mean_response", ctypes.c_float),
        ("per_scale", ctypes.c_int32 * 64),
        ("lo", ctypes.c_float),
        ("hi", ctypes.c_float),
        ("status", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded C library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmhfd.so is not built: run __graft_entry__.build() "
                               "(or python -m paper_2108_12050_gb300._build)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        pP = ctypes.POINTER(Params)
        L.mhfd_default_params.argtypes = [pP]
        L.mhfd_default_params.restype = None
        L.mhfd_create_detector.argtypes = [pP, ctypes.POINTER(ctypes.c_void_p)]
        L.mhfd_destroy_detector.argtypes = [P]
        L.mhfd_detect.argtypes = [P, P, I32, I32, I32, SZ, P]
        L.mhfd_result_wait.argtypes = [P, ctypes.POINTER(Result)]
        L.mhfd_detect_host.argtypes = [P, P, I32, I32, I32, SZ, P, ctypes.POINTER(Result)]
        L.mhfd_detect_host_async.argtypes = [P, P, I32, I32, I32, SZ, P]
        L.mhfd_detect_batch.argtypes = [P, I32, P, P, P, P, P, P]
        L.mhfd_result_wait_batch.argtypes = [P, ctypes.POINTER(Result), I32]
        L.mhfd_batch_uses_graph.argtypes = [P]
        L.mhfd_uses_tensor_cores.argtypes = [P]
        L.mhfd_device_bytes.argtypes = [P, I32, I32, ctypes.POINTER(I64), ctypes.POINTER(I64)]
        L.mhfd_trim.argtypes = [P]
        L.mhfd_result_ready.argtypes = [P]
        L.mhfd_soft_score.argtypes = [P, P, I32, I32, I32, SZ, P, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, P, P, P, P, P]
        L.mhfd_detect_plain.argtypes = [P, P, I32, I32, I32, SZ, P]
        L.mhfd_debug_stack.argtypes = [P, P, I32, I32, I32, SZ, P, P, P, P]
        L.mhfd_prune.argtypes = [P, P, P, P, P, I64, I32, I32, P, P]
        L.mhfd_prune_noalloc.argtypes = [P, I32, ctypes.c_float, P, P, P, P, I64, I32, I32, P,
                                         P]
        L.mhfd_tile_configs.argtypes = [pP, P, I32]
        L.mhfd_chosen_tile.argtypes = [pP, P]
        L.mhfd_precompile.argtypes = [pP, I32]
        L.mhfd_last_timing.argtypes = [P, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float)]
        L.mhfd_probe_ffma_peak.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
        L.mhfd_last_error.restype = ctypes.c_char_p
        L.mhfd_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            fn = getattr(L, name)
            if fn.restype is ctypes.c_int:  # default
                fn.restype = ctypes.c_int
        _lib = L
        return L


def check(rc, allow_overflow=True):
    if rc == MHFD_OK or (allow_overflow and rc == MHFD_WARN_OVERFLOW):
        return rc
    raise MhfdError(rc, lib().mhfd_last_error().decode(errors="replace"))


def make_params(n=10, t_min=1.0, t_max=10.0, sigmas=None, threshold=0.1, overlap=0.5,
                nms=NMS_PAPER, truncate=4.0, clip_frac=0.00175, max_candidates=1 << 20,
                device=-1, keep_candidates=False, tile_override=0, tile_shape=None, timing=False,
                response=0, boundary=0, tensor_cores=True):
    p = Params()
    lib().mhfd_default_params(ctypes.byref(p))
    p.n = int(n)
    p.t_min = float(t_min)
    p.t_max = float(t_max)
    keep = None
    if sigmas is not None:
        arr = (ctypes.c_double * len(sigmas))(*[float(s) for s in sigmas])
        p.sigmas = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        keep = arr
    if isinstance(nms, str):
        nms = {"paper": NMS_PAPER, "local26": NMS_LOCAL26}[nms]
    p.threshold = float(threshold)
    p.overlap = float(overlap)
    p.nms = int(nms)
    p.truncate = float(truncate)
    p.clip_frac = float(clip_frac)
    p.max_candidates = int(max_candidates)
    p.device = int(device)
    p.keep_candidates = 1 if keep_candidates else 0
    p.tile_override = int(tile_override)
    if tile_shape:
        for k, v in enumerate(tile_shape):
            p.tile_shape[k] = int(v)
    p.timing = 1 if timing else 0
    if isinstance(response, str):
        response = {"dog": 0, "log": 1}[response]
    if isinstance(boundary, str):
        boundary = {"reflect": 0, "periodic": 1}[boundary]
    p.response = int(response)
    p.boundary = int(boundary)
    p.tensor_cores = 2 if tensor_cores == 2 else (1 if tensor_cores else 0)
    p._keepalive = keep
    return p


def precompile(store=0, **kw):
    p = make_params(**kw)
    return check(lib().mhfd_precompile(ctypes.byref(p), int(store)))


def tile_configs(**kw):
    p = make_params(**kw)
    n = lib().mhfd_tile_configs(ctypes.byref(p), None, 0)
    if n < 0:
        check(n)
    buf = (ctypes.c_int32 * (6 * max(n, 1)))()
    lib().mhfd_tile_configs(ctypes.byref(p), buf, n)
    return [tuple(buf[6 * k:6 * k + 6]) for k in range(n)]


def chosen_tile(**kw):
    p = make_params(**kw)
    buf = (ctypes.c_int32 * 6)()
    check(lib().mhfd_chosen_tile(ctypes.byref(p), buf))
    return tuple(buf)
