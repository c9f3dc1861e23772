"""Continuous-batching server: each tile detected alone is held to the FP64
oracle (ambiguity rules of ``parity_util``), each served result equals the
tile detected alone bit for bit, requests overlap on the device, and the
HBM budget gates admission."""
import numpy as np
import pytest

import synth
from parity_util import check_detection, oracle_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARAMS = dict(n=16, t_min=1.0, t_max=12.0, threshold=0.05, overlap=0.5)


def _tiles():
    out = []
    for j, (H, W, dt) in enumerate([(512, 512, "u16"), (300, 700, "u8"), (1024, 256, "u16"),
                                    (256, 256, "u8"), (640, 480, "f32"), (128, 900, "u16"),
                                    (700, 300, "u8"), (512, 384, "u16")]):
        out.append(synth.make_scene(900 + j, synth.scene12bit_spec(0.5 * j, H, W, dt)))
    return out


def _alone(tiles, against_oracle=False):
    import paper_2108_12050_gb300 as mhfd
    det = mhfd.Detector(keep_candidates=True, **PARAMS)
    res = []
    for t in tiles:
        dev = torch.from_numpy(t.view(np.int16) if t.dtype == np.uint16 else t).cuda()
        r = det(dev)
        if against_oracle:
            ref, D, tol, lad, _ = oracle_reference(t, 16, 1.0, 12.0, 0.05, 0.5)
            assert (r.lo, r.hi) == (np.float32(ref.lo), np.float32(ref.hi))
            check_detection(r, ref, D, tol, 0.05, 0.5, "paper", lad)
        res.append(r)
    det.close()
    return res


def test_results_in_the_mix_equal_results_alone():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_12050_gb300 import serve
    torch.cuda.set_device(0)
    tiles = _tiles() * 3
    ref = _alone(tiles[:8], against_oracle=True)
    srv = serve.Server(n_slots=4, hbm_budget=8 << 30, **PARAMS)
    futs = [srv.submit(t) for t in tiles]
    got = [f.result(timeout=120) for f in futs]
    stats = dict(srv.stats)
    srv.close()
    for j, r in enumerate(got):
        want = ref[j % 8]
        assert (r.lo, r.hi) == (want.lo, want.hi)
        assert r.n_blobs == want.n_blobs and r.n_candidates_true == want.n_candidates_true
        assert np.array_equal(r.blobs, want.blobs)
        assert np.array_equal(r.per_scale, want.per_scale)
        assert r.mean_response == want.mean_response
    assert stats["completed"] == len(tiles)
    assert stats["peak_in_flight"] > 1          # requests overlapped on the device


def test_budget_limits_concurrency():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_12050_gb300 import serve
    import paper_2108_12050_gb300 as mhfd
    tiles = _tiles()[:4]
    ref = _alone(tiles)
    # room for the slots' fixed state plus exactly one 1024x256 uint16 tile
    probe = mhfd.Detector(**PARAMS)
    fixed, scratch = probe.device_bytes(1024, 256)
    probe.close()
    budget = 4 * fixed + serve.image_bytes((1024, 256), np.uint16) + scratch
    srv = serve.Server(n_slots=4, hbm_budget=budget, **PARAMS)
    assert srv.fixed == fixed
    got = [f.result(timeout=120) for f in [srv.submit(t) for t in tiles]]
    stats = dict(srv.stats)
    srv.close()
    assert stats["peak_bytes"] <= budget
    for r, want in zip(got, ref):
        assert np.array_equal(r.blobs, want.blobs)


def test_reported_device_bytes_match_the_allocations():
    """What the library reports (and the server charges) against what the
    device actually lost, read with cudaMemGetInfo: the detector's fixed
    state at creation, and the per-image scratch of a first detection of an
    8192 x 8192 uint8 tile.  The driver rounds allocations up to its page
    size, so each side may differ by a few pages per allocation."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2108_12050_gb300 as mhfd
    torch.cuda.set_device(0)
    warm = mhfd.Detector(**PARAMS)          # loads the compiled kernels once
    warm.close()
    img = torch.zeros((8192, 8192), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    det = mhfd.Detector(**PARAMS)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    fixed, scratch = det.device_bytes(8192, 8192)
    first = det(img)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    # trim gives the per-image scratch back; the next detection grows it again
    det.trim()
    torch.cuda.synchronize()
    free3 = torch.cuda.mem_get_info()[0]
    again = det(img)
    det.close()
    got_fixed, got_scratch = free0 - free1, free1 - free2
    print("device bytes: fixed %d reported / %d measured; image scratch %d / %d; "
          "trim returned %d" % (fixed, got_fixed, scratch, got_scratch, free3 - free2))
    slack = 32 << 20
    assert abs(got_fixed - fixed) <= slack
    assert abs(got_scratch - scratch) <= slack
    assert scratch > 2 * 8192 * 8192 * 0.9        # the 2 B/px candidate staging
    assert abs((free3 - free2) - scratch) <= slack
    assert again.n_blobs == first.n_blobs and np.array_equal(again.blobs, first.blobs)
