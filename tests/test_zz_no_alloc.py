"""The allocation-free prune (mhfd_prune_noalloc) against the regular one.

mhfd_prune_noalloc serves callers that must not allocate device memory, for
instance code running in a host callback or on a real-time thread (where the
allocator's implicit synchronisation is not allowed) or inside a framework
that owns every device allocation.  Its working memory is a fixed device
array inside the library, shared by all calls.  This test calls it twice in
a row through the C ABI, on two different candidate lists, and checks that
each result equals the detector-based mhfd_prune on the same input (the
prune is exact, so equality is bit for bit) and to the FP64 oracle's prune -
i.e. nothing left in the shared array by the first call leaks into the
second.  It also checks that a list larger than the fixed limit is refused,
and that a settle loop whose bounded wait runs out marks the candidates it
left unresolved (keep = 2) instead of silently dropping them, after which
the next call gives the usual result.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _ladder_radii(n, tmin, tmax):
    dt = (tmax - tmin) / n
    return [math.sqrt(2.0) * (tmin + i * dt) for i in range(n)]


def test_noalloc_prune_matches_regular_prune_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2108_12050_gb300 as mhfd
    from paper_2108_12050_gb300 import _native

    torch.cuda.set_device(0)
    lib = _native.lib()
    n, tmin, tmax, overlap = 10, 1.0, 10.0, 0.5
    radius = (ctypes.c_double * n)(*_ladder_radii(n, tmin, tmax))
    det = mhfd.Detector(n, tmin, tmax, threshold=0.1, overlap=overlap)
    stream = torch.cuda.current_stream()
    H, W = 900, 1100
    for seed, count, cluster in ((11, 6000, 0.85), (12, 3500, 0.5)):
        x, y, i, resp = synth.random_candidates(seed, count, H, W, n, cluster=cluster)
        dx, dy, di, dr = (torch.from_numpy(a).cuda() for a in (x, y, i, resp))
        keep_ref = det.prune(dx, dy, di, dr, H, W)
        keep = torch.full((x.size,), 7, dtype=torch.uint8, device="cuda")
        rc = lib.mhfd_prune_noalloc(radius, n, ctypes.c_float(overlap), _ptr(dx), _ptr(dy),
                                    _ptr(di), _ptr(dr), x.size, H, W, _ptr(keep),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.mhfd_last_error()
        torch.cuda.synchronize()
        assert torch.equal(keep, keep_ref)
        assert 0 < int(keep.sum()) < x.size
        want = oracle.prune(x, y, i, resp.astype(np.float64), list(radius), overlap, W)
        assert np.array_equal(keep.cpu().numpy(), want)
    det.close()


def test_noalloc_prune_reports_an_expired_wait(monkeypatch):
    """The settle loop's wait is bounded; with the bound set to zero sweeps
    it gives up at once and every candidate with a higher-priority
    conflicting neighbour stays unresolved (keep = 2, never a silent 0).
    The next call, with the default bound, gives the oracle's result."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_12050_gb300 import _native

    torch.cuda.set_device(0)
    lib = _native.lib()
    n, tmin, tmax, overlap = 10, 1.0, 10.0, 0.5
    radius = (ctypes.c_double * n)(*_ladder_radii(n, tmin, tmax))
    H, W = 600, 700
    x, y, i, resp = synth.random_candidates(14, 2000, H, W, n, cluster=0.8)
    dx, dy, di, dr = (torch.from_numpy(a).cuda() for a in (x, y, i, resp))
    want = oracle.prune(x, y, i, resp.astype(np.float64), list(radius), overlap, W)
    stream = torch.cuda.current_stream()

    def call():
        keep = torch.full((x.size,), 7, dtype=torch.uint8, device="cuda")
        rc = lib.mhfd_prune_noalloc(radius, n, ctypes.c_float(overlap), _ptr(dx), _ptr(dy),
                                    _ptr(di), _ptr(dr), x.size, H, W, _ptr(keep),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.mhfd_last_error()
        torch.cuda.synchronize()
        return keep.cpu().numpy()

    monkeypatch.setenv("MHFD_PRUNE_MAX_SWEEPS", "0")
    k0 = call()
    assert set(np.unique(k0).tolist()) <= {0, 1, 2}
    assert (k0 == 2).sum() > 0
    # what was decided before the loop (no higher-priority conflict) is kept
    assert np.all(want[k0 == 1] == 1)
    monkeypatch.delenv("MHFD_PRUNE_MAX_SWEEPS")
    assert np.array_equal(call(), want)


def test_noalloc_prune_rejects_lists_beyond_its_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_12050_gb300 import _native

    lib = _native.lib()
    radius = (ctypes.c_double * 2)(1.5, 2.5)
    big = 65537
    buf = torch.zeros(big, dtype=torch.int32, device="cuda")
    resp = torch.zeros(big, dtype=torch.float32, device="cuda")
    keep = torch.zeros(big, dtype=torch.uint8, device="cuda")
    rc = lib.mhfd_prune_noalloc(radius, 2, ctypes.c_float(0.5), _ptr(buf), _ptr(buf), _ptr(buf),
                                _ptr(resp), big, 100, 100, _ptr(keep), None)
    assert rc == _native.MHFD_ERR_INVALID_ARG
    assert b"65536" in lib.mhfd_last_error()
