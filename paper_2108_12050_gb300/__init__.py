"""GB300 (sm_103a) multi-scale histologic feature detector (arXiv 2108.12050).

Thin Python binding of the C ABI in ``include/mhfd.h``: it marshals
arguments only.  Every step of the detection (histogram stretch of §3,
Gaussian scale space of §2.2, DoG of Eq. 2, local maxima of Eq. 3, overlap
pruning, focus score) runs in this package's CUDA kernels; PyTorch is used
only for device memory and streams.  There is no CPU fallback: if the
library is not built, or no GPU is present, calls raise.

    det = Detector(n=16, t_min=1, t_max=12, threshold=0.05, overlap=0.5)
    res = det(img_cuda_u16)            # -> DetectionResult (score, blobs, ...)
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np

from . import _native as _n
from ._native import MhfdError  # noqa: F401

__all__ = ["Detector", "DetectionResult", "MhfdError", "probe_ffma_peak", "tile_configs",
           "chosen_tile", "precompile", "version", "lib_path"]

lib_path = _n.LIB_PATH

_BLOB_DTYPE = np.dtype([("x", np.int32), ("y", np.int32), ("scale_idx", np.int32),
                        ("sigma", np.float32), ("radius", np.float32),
                        ("response", np.float32)])


def version() -> str:
    return _n.lib().mhfd_version().decode()


def tile_configs(**params):
    """Tile configurations the fused kernel offers for this ladder."""
    return _n.tile_configs(**params)


def chosen_tile(**params):
    """The (tile w, tile h, rows/step, threads, groups) the built-in heuristic picks."""
    return _n.chosen_tile(**params)


def precompile(store=0, **params):
    """Compile the ladder's fused kernel into the on-disk cache (no GPU needed)."""
    return _n.precompile(store=store, **params)


@dataclasses.dataclass
class DetectionResult:
    status: int
    focus_score: float
    n_blobs: int
    n_candidates: int
    n_candidates_true: int
    mean_response: float
    per_scale: np.ndarray
    lo: float
    hi: float
    blobs: np.ndarray            # structured array (_BLOB_DTYPE), tile order
    candidates: Optional[np.ndarray]

    @property
    def overflow(self) -> bool:
        return self.status == _n.MHFD_WARN_OVERFLOW


def _dtype_code(t):
    import torch
    if t.dtype == torch.uint8:
        return _n.U8
    if t.dtype in (torch.int16,) or str(t.dtype) == "torch.uint16":
        return _n.U16
    if t.dtype == torch.float32:
        return _n.F32
    raise TypeError("image must be uint8, uint16 (or int16 holding uint16 bits) or float32")


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _to_result(r: _n.Result, n_levels: int) -> DetectionResult:
    nb = int(r.n_blobs)
    if nb:
        buf = (_n.Blob * nb).from_address(ctypes.addressof(r.blobs.contents))
        blobs = np.frombuffer(buf, dtype=_BLOB_DTYPE, count=nb).copy()
    else:
        blobs = np.zeros(0, dtype=_BLOB_DTYPE)
    cands = None
    if r.candidates:
        nc = int(r.n_candidates)
        if nc:
            cb = (_n.Blob * nc).from_address(ctypes.addressof(r.candidates.contents))
            cands = np.frombuffer(cb, dtype=_BLOB_DTYPE, count=nc).copy()
        else:
            cands = np.zeros(0, dtype=_BLOB_DTYPE)
    return DetectionResult(status=int(r.status), focus_score=float(r.focus_score), n_blobs=nb,
                           n_candidates=int(r.n_candidates),
                           n_candidates_true=int(r.n_candidates_true),
                           mean_response=float(r.mean_response),
                           per_scale=np.array(r.per_scale[:n_levels], dtype=np.int64),
                           lo=float(r.lo), hi=float(r.hi), blobs=blobs, candidates=cands)


class Detector:
    """One detector (ladder, threshold, pruning) bound to one CUDA device.

    Parameters follow Algorithm 1 (``n``, ``t_min``, ``t_max``) plus the
    threshold, the overlap fraction of the prune (>= 1 disables it), the
    maximum rule (``"paper"``: argmax over scales then 3x3 max-pool;
    ``"local26"``: 3x3x3 scale-space maxima), the kernel truncation and the
    stretch saturation fraction.  ``sigmas`` gives an explicit ladder of
    ``n+1`` scales instead.  ``tensor_cores`` (default ``True``) runs
    detections of uint8 images and of uint16 images whose stretch range is
    at most 4095 on the tensor cores: both blur passes for the paper rule
    with the DoG response, the vertical pass otherwise (``2``: the
    vertical-pass kernel for every mode; ``False``: FFMA only).
    """

    def __init__(self, n=10, t_min=1.0, t_max=10.0, *, sigmas=None, threshold=0.1, overlap=0.5,
                 nms="paper", truncate=4.0, clip_frac=0.00175, max_candidates=1 << 20,
                 device=None, keep_candidates=False, tile_override=None, tile_shape=None,
                 timing=False, response="dog", boundary="reflect", tensor_cores=True):
        import torch
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else -1
        if tile_override is None and tile_shape is None:
            # a measured tile shape for this ladder and GPU, if the autotuner
            # recorded one; otherwise the library's built-in choice
            if sigmas is None and device >= 0:
                from . import tune
                sms = torch.cuda.get_device_properties(device).multi_processor_count
                is_log = response in ("log", 1)
                tc = bool(tensor_cores) and (nms in ("paper", 0) or not is_log)
                # the tuned shapes are the vertical-pass kernel's: the default
                # for detection with the DoG response (the 26-neighbour rule
                # up to 16 layers) is the two-pass kernel
                two_pass = (tensor_cores is True or tensor_cores == 1) and not is_log
                two_pass = two_pass and (nms in ("paper", 0) or (nms in ("local26", 1) and n <= 16))
                tile_shape = None if two_pass else tune.lookup(n, t_min, t_max, nms, sms, truncate,
                                         "log" if is_log else "dog", tensor_cores=tc)
        tile_override = tile_override or 0
        self.n = int(n)
        self.device = device
        self._p = _n.make_params(n=n, t_min=t_min, t_max=t_max, sigmas=sigmas,
                                 threshold=threshold, overlap=overlap, nms=nms,
                                 truncate=truncate, clip_frac=clip_frac,
                                 max_candidates=max_candidates, device=device,
                                 keep_candidates=keep_candidates, tile_override=tile_override,
                                 tile_shape=tile_shape, timing=timing, response=response,
                                 boundary=boundary, tensor_cores=tensor_cores)
        h = ctypes.c_void_p()
        _n.check(_n.lib().mhfd_create_detector(ctypes.byref(self._p), ctypes.byref(h)))
        self._h = h
        self._img_ref = None

    def device_bytes(self, H=0, W=0):
        """(bytes the detector holds on the device, bytes a fused detection of
        an H x W image adds) as the library allocates them."""
        f, i = ctypes.c_int64(), ctypes.c_int64()
        _n.check(_n.lib().mhfd_device_bytes(self._h, int(H), int(W), ctypes.byref(f),
                                            ctypes.byref(i)))
        return f.value, i.value

    def trim(self):
        """Give back the per-image device scratch grown so far (waits for the
        detector's work; the fixed state stays)."""
        _n.check(_n.lib().mhfd_trim(self._h))

    @property
    def uses_tensor_cores(self):
        """Whether the fused kernel runs on the tensor cores (either kernel)."""
        return bool(_n.lib().mhfd_uses_tensor_cores(self._h))

    @property
    def tensor_core_kernel(self):
        """2: both blur passes on the tensor cores; 1: the vertical pass; 0: FFMA."""
        return int(_n.lib().mhfd_uses_tensor_cores(self._h))

    # --------------------------------------------------------------- core
    def close(self):
        if getattr(self, "_h", None):
            _n.lib().mhfd_destroy_detector(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _img_args(img):
        if img.dim() != 2:
            raise ValueError("image must be 2-D (H, W)")
        if not img.is_cuda:
            raise ValueError("image must be a CUDA tensor (use detect_host for host arrays)")
        if img.stride(1) != 1:
            raise ValueError("image rows must be contiguous")
        H, W = img.shape
        return ctypes.c_void_p(img.data_ptr()), _dtype_code(img), int(H), int(W), \
            int(img.stride(0) * img.element_size())

    def detect(self, img, stream=None):
        """Enqueue a detection of the CUDA image on the stream (asynchronous)."""
        ptr, code, H, W, pitch = self._img_args(img)
        self._img_ref = img
        _n.check(_n.lib().mhfd_detect(self._h, ptr, code, H, W, pitch, _stream_handle(stream)))

    def detect_plain(self, img, stream=None):
        """Same detection through the unfused per-scale pipeline (baseline)."""
        ptr, code, H, W, pitch = self._img_args(img)
        self._img_ref = img
        _n.check(_n.lib().mhfd_detect_plain(self._h, ptr, code, H, W, pitch,
                                            _stream_handle(stream)))

    def detect_batch(self, imgs, stream=None):
        """Enqueue a batch of CUDA images (uneven sizes, mixed dtypes): one
        persistent fused launch over all their tiles, replayed from a CUDA
        graph for repeated batch shapes."""
        n = len(imgs)
        args = [self._img_args(t) for t in imgs]
        ptrs = (ctypes.c_void_p * n)(*[a[0].value for a in args])
        dts = (ctypes.c_int32 * n)(*[a[1] for a in args])
        Hs = (ctypes.c_int32 * n)(*[a[2] for a in args])
        Ws = (ctypes.c_int32 * n)(*[a[3] for a in args])
        ps = (ctypes.c_size_t * n)(*[a[4] for a in args])
        self._img_ref = list(imgs)
        self._batch_n = n
        _n.check(_n.lib().mhfd_detect_batch(self._h, n, ptrs, dts, Hs, Ws, ps,
                                            _stream_handle(stream)))

    def wait_batch(self):
        n = self._batch_n
        rs = (_n.Result * n)()
        _n.check(_n.lib().mhfd_result_wait_batch(self._h, rs, n))
        return [_to_result(rs[j], self.n) for j in range(n)]

    def ready(self) -> bool:
        """Non-blocking: has the last enqueued detection finished?"""
        r = _n.lib().mhfd_result_ready(self._h)
        if r < 0:
            _n.check(r)
        return r == 1

    def batch_uses_graph(self) -> bool:
        return _n.lib().mhfd_batch_uses_graph(self._h) == 1

    def wait(self) -> DetectionResult:
        r = _n.Result()
        _n.check(_n.lib().mhfd_result_wait(self._h, ctypes.byref(r)))
        return _to_result(r, self.n)

    def __call__(self, img, stream=None) -> DetectionResult:
        self.detect(img, stream)
        return self.wait()

    def detect_host(self, img: np.ndarray, stream=None, wait=True):
        """End to end from a host (numpy) image: copy in, detect, results out.
        With ``wait=False`` the copy and the detection are only enqueued
        (``img`` must stay alive and unchanged until ``wait()``); use pinned
        host memory for the copy to overlap other streams' work."""
        img = np.ascontiguousarray(img)
        code = {np.dtype(np.uint8): _n.U8, np.dtype(np.uint16): _n.U16,
                np.dtype(np.float32): _n.F32}.get(img.dtype)
        if code is None:
            raise TypeError("image must be uint8, uint16 or float32")
        H, W = img.shape
        if not wait:
            self._img_ref = img
            _n.check(_n.lib().mhfd_detect_host_async(self._h, img.ctypes.data_as(ctypes.c_void_p),
                                                     code, H, W, img.strides[0],
                                                     _stream_handle(stream)))
            return None
        r = _n.Result()
        _n.check(_n.lib().mhfd_detect_host(self._h, img.ctypes.data_as(ctypes.c_void_p), code,
                                           H, W, img.strides[0], _stream_handle(stream),
                                           ctypes.byref(r)))
        return _to_result(r, self.n)

    def debug_stack(self, img, stream=None, want=("D", "M", "A")):
        """Run the stack-storing variant: returns (D[n,H,W], M[H,W], argmax[H,W])."""
        import torch
        ptr, code, H, W, pitch = self._img_args(img)
        dev = img.device
        D = torch.empty((self.n, H, W), dtype=torch.float32, device=dev) if "D" in want else None
        M = torch.empty((H, W), dtype=torch.float32, device=dev) if "M" in want else None
        A = torch.empty((H, W), dtype=torch.int32, device=dev) if "A" in want else None
        vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        _n.check(_n.lib().mhfd_debug_stack(self._h, ptr, code, H, W, pitch,
                                           _stream_handle(stream), vp(D), vp(M), vp(A)))
        res = self.wait()
        return D, M, A, res

    def prune(self, x, y, i, resp, H, W, stream=None):
        """Overlap prune of a caller-supplied CUDA candidate list -> uint8 keep mask."""
        import torch
        x = x.to(torch.int32).contiguous(); y = y.to(torch.int32).contiguous()
        i = i.to(torch.int32).contiguous(); resp = resp.to(torch.float32).contiguous()
        keep = torch.zeros(x.numel(), dtype=torch.uint8, device=x.device)
        vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        _n.check(_n.lib().mhfd_prune(self._h, vp(x), vp(y), vp(i), vp(resp), int(x.numel()),
                                     int(H), int(W), vp(keep), _stream_handle(stream)))
        return keep

    def last_timing(self):
        """(ms of the fused/plain compute kernels, ms of the whole detection)."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _n.check(_n.lib().mhfd_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value


def probe_ffma_peak(stream=None) -> float:
    """Measured FP32 FFMA lane-operations per second of the current GPU."""
    v = ctypes.c_double()
    _n.check(_n.lib().mhfd_probe_ffma_peak(_stream_handle(stream), ctypes.byref(v)))
    return v.value
