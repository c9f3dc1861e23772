"""The debug build of the fused kernel (environment MHFD_DEBUG_CHECKS=1).

With compute-sanitizer unavailable, the fused kernel has a build whose
shared-memory and global indices are checked against their buffers (input
window rows and columns, the tensor-core window and the rows its MMAs read,
V rows, the maxima ring, candidate slots and tile counters, stored stack
planes, reflected image indices).  A failed check is recorded in the
kernel's flag word and reported as MHFD_ERR_CHECK; the access is skipped, so
nothing faults.  Here every kernel kind and the edge shapes of the parity
tests run through that build: each must report no failed check and give the
regular build's results bit for bit (the checks change no arithmetic).
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L16 = dict(n=16, t_min=1.0, t_max=12.0, threshold=0.05)
L10 = dict(n=10, t_min=1.0, t_max=10.0, threshold=0.1)
L4 = dict(n=4, t_min=1.0, t_max=4.0, threshold=0.1)

# (name, detector parameters, image (seed, H, W, dtype))
CASES = [
    ("tc_default", dict(L16), (91, 300, 420, "u16")),          # the two-pass kernel
    ("vtc", dict(L16, tensor_cores=2), (91, 300, 420, "u16")),  # the vertical-pass kernel
    ("ffma", dict(L16, tensor_cores=False), (91, 300, 420, "u16")),
    ("local26", dict(L16, nms="local26"), (92, 260, 333, "u8")),              # two-pass
    ("local26_vtc", dict(L16, nms="local26", tensor_cores=2), (92, 260, 333, "u8")),
    ("log_tc", dict(L10, threshold=0.1 / 0.9, response="log"), (93, 200, 270, "u16")),
    ("periodic", dict(L10, boundary="periodic"), (94, 70, 45, "u16")),
    ("two_row_tc", dict(L16, tensor_cores=2, tile_shape=[256, 18, 8, 288, 4, 2]),
     (95, 300, 620, "u16")),
    ("two_row_ffma", dict(L16, tensor_cores=False, tile_shape=[320, 18, 4, 448, 4, 2]),
     (95, 300, 620, "u16")),
    ("two_output_local26_ffma", dict(L16, nms="local26", tensor_cores=False,
                                     tile_shape=[192, 18, 4, 384, 2, 3]), (92, 260, 333, "u8")),
    ("narrower_than_halo", dict(L16), (96, 90, 40, "u16")),
    ("one_pixel_wide", dict(L4), (97, 40, 1, "u8")),
    ("wide_uint16_range", dict(L16), (98, 180, 260, "u16x9")),
]


def _image(seed, H, W, dtype):
    if dtype == "u8":
        return synth.make_scene(seed, synth.scene512_u8_spec(0.0, H, W))
    img = synth.make_scene(seed, synth.scene12bit_spec(0.0, H, W, "u16"))
    if dtype == "u16x9":   # stretch range beyond 4095: the FFMA companion
        img = (img.astype(np.uint32) * 9).clip(0, 65535).astype(np.uint16)
    return img


def _dev(img):
    return torch.from_numpy(img.view(np.int16) if img.dtype == np.uint16 else img).cuda()


def _precompile(args):
    kw, store, checks = args
    os.environ["MHFD_DEBUG_CHECKS"] = checks
    from paper_2108_12050_gb300 import _native
    try:
        return _native.precompile(store=store, **kw)
    except _native.MhfdError as e:
        return str(e)


@pytest.fixture(scope="module")
def checked_env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.set_device(0)
    old = os.environ.get("MHFD_DEBUG_CHECKS")
    # compile the regular and the checked variants (detection and
    # stack-storing) in parallel processes; detectors then load them from
    # the kernel cache
    from paper_2108_12050_gb300 import tune
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    kws = []
    for _, kw, _ in CASES:
        kw = dict(kw, nms=kw.get("nms", "paper"))
        # the two-pass kernel (the default for detection with the DoG
        # response; the 26-neighbour rule up to 16 layers) takes no tuned shape
        two_pass = (kw.get("tensor_cores", True) in (True, 1) and kw.get("response", "dog") == "dog"
                    and (kw["nms"] == "paper" or kw["n"] <= 16))
        if "tile_shape" not in kw and not two_pass:  # the shape a Detector takes from the table
            tc = kw.get("tensor_cores", True) and (kw["nms"] == "paper" or
                                                   kw.get("response", "dog") == "dog")
            kw["tile_shape"] = tune.lookup(kw["n"], kw["t_min"], kw["t_max"], kw["nms"], sms,
                                           4.0, kw.get("response", "dog"), tensor_cores=tc)
        kws.append(kw)
    jobs = [(kw, store, checks) for kw in kws for store in (0, 1) for checks in ("0", "1")]
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        rcs = list(ex.map(_precompile, jobs))
    assert all(rc == 0 for rc in rcs), rcs
    yield
    if old is None:
        os.environ.pop("MHFD_DEBUG_CHECKS", None)
    else:
        os.environ["MHFD_DEBUG_CHECKS"] = old


def _run(kw, dev):
    import paper_2108_12050_gb300 as mhfd
    # the stack-storing variant writes M and the argmax under the paper rule
    want = ("D",) if kw.get("nms") == "local26" else ("D", "M", "A")
    with mhfd.Detector(keep_candidates=True, **kw) as det:
        res = det(dev)
        D, M, A, _ = det.debug_stack(dev, want=want)
    return res, D, M, A


def _same(a, b):
    return (a is None and b is None) or torch.equal(a, b)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_checked_build_reports_nothing_and_matches_the_regular_build(checked_env, case):
    _, kw, spec = case
    dev = _dev(_image(*spec))
    os.environ["MHFD_DEBUG_CHECKS"] = "0"
    want, D0, M0, A0 = _run(kw, dev)
    os.environ["MHFD_DEBUG_CHECKS"] = "1"
    got, D1, M1, A1 = _run(kw, dev)       # raises MhfdError(-7) on a failed check
    assert got.status in (0, 1)
    assert (got.lo, got.hi) == (want.lo, want.hi)
    assert got.n_candidates_true == want.n_candidates_true
    assert np.array_equal(got.candidates, want.candidates)
    assert np.array_equal(got.blobs, want.blobs)
    assert _same(D0, D1) and _same(M0, M1) and _same(A0, A1)


def test_checked_build_in_a_batch(checked_env):
    import paper_2108_12050_gb300 as mhfd
    os.environ["MHFD_DEBUG_CHECKS"] = "1"
    imgs = [_image(*spec) for _, _, spec in CASES[:3]] + [_image(99, 517, 130, "u16")]
    devs = [_dev(i) for i in imgs]
    with mhfd.Detector(**L16) as det:
        det.detect_batch(devs)
        outs = det.wait_batch()
        singles = [det(d) for d in devs]
    for o, s in zip(outs, singles):
        assert o.status in (0, 1) and np.array_equal(o.blobs, s.blobs)
