"""Differentiable soft focus score (autograd wrapper of mhfd_soft_score).

    S(I, w) = sum_i w_i mean_{x,y} sigmoid((D_i(x,y) - tau) / T)

where D_i are the DoG responses (Eq. 2) of the stretched image (§3; the
stretch bounds are held fixed).  The hard detector counts features above the
threshold; this score replaces the count by a smooth per-scale occupancy so
that per-scale weights can be calibrated against known defocus by gradient
descent.  Forward and backward both run in the library's CUDA kernels; the
backward recomputes the Gaussian levels instead of keeping them.
"""
from __future__ import annotations

import ctypes

import torch

from . import Detector, _native as _n, _stream_handle, _dtype_code


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def soft_score(det: Detector, img: torch.Tensor, w: torch.Tensor, tau: float, T: float = 0.01,
               grad_s: float = 0.0, want_grad: bool = False, stream=None):
    """Returns (S, mean_sig, dS/dI * grad_s or None, dS/dw * grad_s or None)."""
    ptr, code, H, W, pitch = det._img_args(img)
    w = w.detach().to(device=img.device, dtype=torch.float32).contiguous()
    S = torch.empty(1, dtype=torch.float32, device=img.device)
    ms = torch.empty(det.n, dtype=torch.float32, device=img.device)
    dimg = torch.empty((H, W), dtype=torch.float32, device=img.device) if want_grad else None
    dw = torch.empty(det.n, dtype=torch.float32, device=img.device) if want_grad else None
    _n.check(_n.lib().mhfd_soft_score(det._h, ptr, code, H, W, pitch, _vp(w), ctypes.c_float(tau),
                                      ctypes.c_float(T), ctypes.c_float(grad_s),
                                      _stream_handle(stream), _vp(S), _vp(ms), _vp(dimg),
                                      _vp(dw)))
    return S[0], ms, dimg, dw


class SoftFocus(torch.autograd.Function):
    """S = soft focus score of `img` (float32, CUDA) with per-scale weights
    `w` (n,); differentiable in both."""

    @staticmethod
    def forward(ctx, img, w, det, tau, T):
        S, ms, _, _ = soft_score(det, img, w, tau, T)
        ctx.save_for_backward(img, w)
        ctx.det, ctx.tau, ctx.T = det, tau, T
        ctx.ms = ms
        return S

    @staticmethod
    def backward(ctx, gS):
        img, w = ctx.saved_tensors
        g = float(gS)
        need_img = ctx.needs_input_grad[0]
        if need_img:
            _, _, dimg, dw = soft_score(ctx.det, img, w, ctx.tau, ctx.T, grad_s=g,
                                        want_grad=True)
        else:
            dimg, dw = None, ctx.ms * g
        return dimg, dw, None, None, None


def features(det, imgs, tau, T=0.01):
    """Per-image mean sigmoid of every layer (S is linear in w: S = w . f)."""
    n = det.n
    ones = torch.ones(n, device=imgs[0].device)
    return torch.stack([soft_score(det, im, ones, tau, T)[1] for im in imgs])


def fit_weights(det, imgs, targets, tau, T=0.01, steps=200, lr=0.05, seed=0, timings=None):
    """Calibrate per-scale weights w and bias b so that S(I, w) + b regresses
    `targets` (e.g. the known defocus sigma_d) by Adam.

    S is linear in w, S(I, w) = w . f(I) with f the per-layer occupancies,
    so f is computed once per image by the CUDA forward and every Adam step
    evaluates w . f exactly (SoftFocus is for losses that also need dS/dI).
    The occupancies differ in spread by an order of magnitude and are small
    (mean sigmoids), so the optimiser works on standardised features:
    w = v / s and b = c - (m / s) . v with m, s the per-layer mean and spread
    over the calibration images, which leaves S(I, w) + b = sum_i v_i
    (f_i - m_i) / s_i + c.  The 17-parameter least-squares loss and its
    gradient are written out and Adam (default moments 0.9 / 0.999, eps 1e-8,
    bias-corrected) runs on the host in float64.  Returns (w, b, losses);
    `timings`, if a dict, receives the seconds spent on the features and on
    the optimiser."""
    import time
    import numpy as np
    t0 = time.perf_counter()
    dev = imgs[0].device
    f = features(det, imgs, tau, T).double().cpu().numpy()
    t1 = time.perf_counter()
    y = np.asarray(targets, dtype=np.float64)
    N = f.shape[0]
    m = f.mean(0)
    sd = f.std(0, ddof=1) + 1e-6 if N > 1 else np.ones_like(m)
    fz = (f - m) / sd
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = 0.1 * torch.randn(det.n, generator=g, dtype=torch.float64).numpy()
    c = float(y.mean())
    b1, b2, eps = 0.9, 0.999, 1e-8
    mv, sv = np.zeros_like(v), np.zeros_like(v)
    mc = sc = 0.0
    losses = []
    for k in range(1, steps + 1):
        r = fz @ v + c - y
        losses.append(float(np.mean(r * r)))
        gv = (2.0 / N) * (fz.T @ r)
        gc = (2.0 / N) * float(r.sum())
        mv = b1 * mv + (1 - b1) * gv
        sv = b2 * sv + (1 - b2) * gv * gv
        mc = b1 * mc + (1 - b1) * gc
        sc = b2 * sc + (1 - b2) * gc * gc
        h1, h2 = 1 - b1 ** k, 1 - b2 ** k
        v = v - lr * (mv / h1) / (np.sqrt(sv / h2) + eps)
        c = c - lr * (mc / h1) / (np.sqrt(sc / h2) + eps)
    w = torch.as_tensor(v / sd, dtype=torch.float32, device=dev)
    b = torch.tensor(c - float(np.dot(m / sd, v)), dtype=torch.float32, device=dev)
    if timings is not None:
        timings["features_s"] = t1 - t0
        timings["optimizer_s"] = time.perf_counter() - t1
    return w, b, losses


def evaluate(det, imgs, targets, w, b, tau, T=0.01):
    """Predictions S(I, w) + b of the calibrated score on `imgs` (CUDA
    forward) and their agreement with `targets`: returns (predictions, mean
    squared error, Spearman rank correlation)."""
    import numpy as np
    pred = np.array([float(soft_score(det, im, w, tau, T)[0]) for im in imgs]) + float(b)
    y = np.asarray(targets, dtype=np.float64)
    mse = float(np.mean((pred - y) ** 2))

    def ranks(a):
        r = np.empty(len(a))
        r[np.argsort(a, kind="stable")] = np.arange(len(a))
        return r

    rp, ry = ranks(pred), ranks(y)
    rp -= rp.mean()
    ry -= ry.mean()
    den = float(np.sqrt((rp * rp).sum() * (ry * ry).sum()))
    return pred, mse, float((rp * ry).sum() / den) if den > 0 else 0.0
