"""Batched detection (persistent launches, CUDA graph) vs the oracle and vs
single detections.

Each image's detection alone is held to the FP64 oracle (candidates, kept
set, counts, mean response, under the ambiguity rules of ``parity_util``),
and its result in a batch of uneven sizes and mixed dtypes must be
bit-identical to detecting it alone (the fused kernel is deterministic per
tile and the per-image post-processing runs in the same order), so every
batched result is held to the oracle too.  With the
tensor-core pass a batch runs two gated persistent launches: the
tensor-core kernel takes the images whose stretch range it holds exactly,
the FFMA kernel the others (float images, wide uint16 ranges) - the same
kernel each image gets alone."""
import numpy as np
import pytest

import synth
from parity_util import check_detection, oracle_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(img):
    if img.dtype == np.uint16:
        return torch.from_numpy(img.view(np.int16)).cuda()
    return torch.from_numpy(img).cuda()


def _held_to_oracle(img, res, **kw):
    """The detection of ``img`` alone (candidates kept) against the oracle."""
    p = dict(thr=0.05, nms="paper", response="dog", boundary="reflect")
    p.update(kw)
    ref, D, tol, t, _ = oracle_reference(img, 16, 1.0, 12.0, p["thr"], 0.5, p["nms"],
                                         p["response"], p["boundary"])
    assert (res.lo, res.hi) == (np.float32(ref.lo), np.float32(ref.hi))
    check_detection(res, ref, D, tol, p["thr"], 0.5, p["nms"], t)


def _same(o, s):
    assert (o.lo, o.hi) == (s.lo, s.hi)
    assert o.n_blobs == s.n_blobs and o.n_candidates_true == s.n_candidates_true
    assert np.array_equal(o.blobs, s.blobs)
    assert np.array_equal(o.per_scale, s.per_scale)
    assert o.mean_response == s.mean_response


def _batch_images():
    imgs = []
    for j, (H, W, dt) in enumerate([(300, 410, "u16"), (256, 256, "u8"), (517, 130, "u16"),
                                    (64, 900, "u8"), (401, 333, "u16"), (97, 97, "f32")]):
        imgs.append(synth.make_scene(700 + j, synth.scene12bit_spec(1.0 + j, H, W, dt)))
    # a uint16 image whose stretch range exceeds 4095 (FFMA kernel)
    wide = synth.make_scene(720, synth.scene12bit_spec(0.0, 200, 240, "u16"))
    imgs.insert(3, (wide.astype(np.uint32) * 9).clip(0, 65535).astype(np.uint16))
    return imgs


@pytest.mark.parametrize("tc", [True, 2, False], ids=["tc", "vtc", "ffma"])
def test_batch_equals_single_detections(tc):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2108_12050_gb300 as mhfd
    torch.cuda.set_device(0)
    imgs = _batch_images()
    devs = [_dev(i) for i in imgs]
    det = mhfd.Detector(16, 1.0, 12.0, threshold=0.05, overlap=0.5, tensor_cores=tc,
                        keep_candidates=True)
    assert det.uses_tensor_cores == bool(tc)
    singles = [det(d) for d in devs]
    for img, s in zip(imgs, singles):
        _held_to_oracle(img, s)
    for rep in range(3):          # capture, then replays of the graph
        det.detect_batch(devs)
        outs = det.wait_batch()
        assert len(outs) == len(imgs)
        for s, o in zip(singles, outs):
            _same(o, s)
    # new image contents with the same shapes replay the graph
    devs2 = [d.flip(0).contiguous() for d in devs]
    det.detect_batch(devs2)
    outs2 = det.wait_batch()
    for d, o in zip(devs2, outs2):
        assert np.array_equal(det(d).blobs, o.blobs)
    det.close()


@pytest.mark.parametrize("kw", [{"response": "log", "threshold": 0.05 / 0.6875},
                                {"boundary": "periodic"},
                                {"nms": "local26", "boundary": "periodic"}])
def test_batch_equals_single_detections_for_variants(kw):
    """The same identity for the compiled variants (LoG response, periodic
    boundary, 26-neighbour rule)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2108_12050_gb300 as mhfd
    torch.cuda.set_device(0)
    imgs = _batch_images()[:4]
    devs = [_dev(i) for i in imgs]
    params = dict(threshold=0.05, overlap=0.5)
    params.update(kw)
    det = mhfd.Detector(16, 1.0, 12.0, keep_candidates=True, **params)
    singles = [det(d) for d in devs]
    for img, s in zip(imgs, singles):
        _held_to_oracle(img, s, thr=params["threshold"], nms=params.get("nms", "paper"),
                        response=params.get("response", "dog"),
                        boundary=params.get("boundary", "reflect"))
    for rep in range(2):
        det.detect_batch(devs)
        outs = det.wait_batch()
        for s, o in zip(singles, outs):
            _same(o, s)
    det.close()


def test_batch_is_replayed_from_a_graph_and_matches_direct_launches():
    """Where capture is permitted (a detector without per-kernel timing) the
    batch is captured once and replayed as a CUDA graph; a detector with
    timing events runs the same batch as direct launches.  Both give the
    same bits."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2108_12050_gb300 as mhfd
    imgs = _batch_images()[:5]
    devs = [_dev(i) for i in imgs]
    graphed = mhfd.Detector(16, 1.0, 12.0, threshold=0.05, overlap=0.5)
    direct = mhfd.Detector(16, 1.0, 12.0, threshold=0.05, overlap=0.5, timing=True)
    for rep in range(2):
        graphed.detect_batch(devs)
        g = graphed.wait_batch()
        assert graphed.batch_uses_graph()
        direct.detect_batch(devs)
        d = direct.wait_batch()
        assert not direct.batch_uses_graph()
        for a, b in zip(g, d):
            _same(a, b)
    graphed.close()
    direct.close()
