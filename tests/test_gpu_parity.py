"""CUDA path vs FP64 oracle on seeded synthetic images (through the C ABI).

Sizes span several fused-kernel tiles and ragged tails; edge cases cover
1-pixel-wide images, images narrower than the kernel radius, pitched rows,
all three dtypes and a constant image.  The paper rule runs on both fused
kernels: the tensor-core vertical pass (the default) and the FFMA one."""
import math
import zlib

import numpy as np
import pytest

import oracle
import synth
from parity_util import (ambiguous_paper, assert_stack_close, check_detection, features,
                         log_eps, oracle_reference)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.set_device(0)


_DETS = {}


def detector(**kw):
    import paper_2108_12050_gb300 as mhfd
    key = tuple(sorted((k, tuple(v) if isinstance(v, list) else v) for k, v in kw.items()))
    if key not in _DETS:
        _DETS[key] = mhfd.Detector(**kw)
    return _DETS[key]


def to_dev(img):
    if img.dtype == np.uint16:
        return torch.from_numpy(img.view(np.int16)).cuda()
    return torch.from_numpy(img).cuda()


def scene(seed, H, W, dtype="u8", sigma_d=0.0):
    if dtype == "u8":
        return synth.make_scene(seed, synth.scene512_u8_spec(sigma_d, H, W))
    return synth.make_scene(seed, synth.scene12bit_spec(sigma_d, H, W, dtype))


def ref_stack(img, n, tmin, tmax):
    lo, hi = oracle.stretch_bounds(img)
    t = oracle.ladder(n, tmin, tmax)
    return oracle.dog_stack(oracle.stretch(img, lo, hi), t), (lo, hi), t


# ----------------------------------------------------------------- stretch

@pytest.mark.parametrize("dtype,shape", [("u8", (96, 80)), ("u16", (130, 257)),
                                         ("f32", (77, 61)), ("u8", (1, 1)), ("u16", (1, 300)),
                                         ("u8", (300, 1)), ("u16", (512, 512))])
def test_stretch_bounds_bit_exact(dtype, shape):
    rng = np.random.default_rng(zlib.crc32(repr((dtype, shape)).encode()))
    if dtype == "f32":
        img = rng.normal(3.0, 2.0, shape).astype(np.float32)
    elif dtype == "u8":
        img = rng.integers(0, 256, shape).astype(np.uint8)
    else:
        img = rng.integers(0, 4096, shape).astype(np.uint16)
    det = detector(n=4, t_min=1.0, t_max=4.0, threshold=0.1)
    res = det(to_dev(img))
    lo, hi = oracle.stretch_bounds(img)
    assert (res.lo, res.hi) == (np.float32(lo), np.float32(hi))


# ------------------------------------------------------------------- stack

STACK_CASES = [
    # (name, seed, H, W, dtype, n, tmin, tmax)
    ("c1_ladder_multi_tile", 31, 150, 390, "u8", 10, 1.0, 10.0),
    ("small_ladder_ragged", 32, 101, 203, "u8", 4, 1.0, 4.0),
    ("u16_scene", 33, 140, 170, "u16", 4, 1.0, 4.0),
    ("f32_scene", 34, 90, 100, "f32", 4, 1.0, 4.0),
    ("narrower_than_radius", 35, 7, 30, "u8", 4, 1.0, 4.0),
    ("one_pixel_wide", 36, 40, 1, "u8", 4, 1.0, 4.0),
    ("one_pixel_high", 37, 1, 57, "u8", 4, 1.0, 4.0),
    # the benchmark ladder (n = 16, t = 1..12: three level groups, R up to 48)
    ("c2_ladder_u16", 51, 300, 420, "u16", 16, 1.0, 12.0),
    ("c2_ladder_u8", 52, 260, 333, "u8", 16, 1.0, 12.0),
    ("c2_ladder_narrower_than_halo", 53, 90, 40, "u16", 16, 1.0, 12.0),
]


@pytest.mark.parametrize("tc", [True, 2, False], ids=["tc", "vtc", "ffma"])
@pytest.mark.parametrize("case", STACK_CASES, ids=lambda c: c[0])
def test_response_stack_within_tolerance(case, tc):
    name, seed, H, W, dtype, n, tmin, tmax = case
    img = scene(seed, H, W, dtype)
    det = detector(n=n, t_min=tmin, t_max=tmax, threshold=0.1, tensor_cores=tc)
    D, M, A, res = det.debug_stack(to_dev(img))
    D_ref, (lo, hi), t = ref_stack(img, n, tmin, tmax)
    assert (res.lo, res.hi) == (np.float32(lo), np.float32(hi))
    assert_stack_close(D.cpu().numpy(), D_ref, name)
    M_ref = D_ref.max(axis=0)
    _, amb_scale, e = ambiguous_paper(D_ref, 0.1)
    assert np.all(np.abs(M.cpu().numpy() - M_ref) <= e)
    A_ref = D_ref.argmax(axis=0)
    A_gpu = A.cpu().numpy()
    assert np.all((A_gpu == A_ref) | amb_scale)


def test_pitched_rows_match_contiguous():
    img = scene(38, 100, 120, "u8")
    padded = np.zeros((100, 160), np.uint8)
    padded[:, :120] = img
    det = detector(n=4, t_min=1.0, t_max=4.0, threshold=0.1)
    dev = to_dev(padded)[:, :120]
    assert dev.stride(0) == 160
    D1, _, _, r1 = det.debug_stack(dev)
    D2, _, _, r2 = det.debug_stack(to_dev(img))
    assert torch.equal(D1, D2)
    assert np.array_equal(r1.blobs, r2.blobs)


# ------------------------------------------------------------- detections

def _check_detection(img, n, tmin, tmax, thr, overlap, nms, response="dog",
                     boundary="reflect", plain=False, tc=True, **kw):
    """One detection through the C ABI against the oracle's, under the
    ambiguity rules with per-layer tolerances (the 5-point LoG stencil of
    the plain path gets its derived, wider tolerance).  Further keywords go
    to the detector (a tile shape)."""
    det = detector(n=n, t_min=tmin, t_max=tmax, threshold=thr, overlap=overlap, nms=nms,
                   keep_candidates=True, response=response, boundary=boundary,
                   tensor_cores=tc, **kw)
    if plain:
        det.detect_plain(to_dev(img))
        res = det.wait()
    else:
        res = det(to_dev(img))
    ref, D_ref, tol, t, Ip = oracle_reference(img, n, tmin, tmax, thr, overlap, nms, response,
                                              boundary)
    if response == "log" and plain:
        R = [oracle.kernel_radius(ti) for ti in t[:n]]
        tol = log_eps(D_ref, t, R, float(np.abs(Ip).max()))
    assert (res.lo, res.hi) == (np.float32(ref.lo), np.float32(ref.hi))
    check_detection(res, ref, D_ref, tol, thr, overlap, nms, t)
    return res, ref


@pytest.mark.parametrize("tc", [True, 2, False], ids=["tc", "vtc", "ffma"])
@pytest.mark.parametrize("which", ["A", "B"])
def test_pair_512_uint8_end_to_end(which, tc):
    a, b = synth.pair512_u8(seed=1)
    img = a if which == "A" else b
    _check_detection(img, 10, 1.0, 10.0, 0.1, 0.5, "paper", tc=tc)


@pytest.mark.parametrize("tc", [True, 2, False], ids=["tc", "vtc", "ffma"])
def test_pair_512_uint8_local26_end_to_end(tc):
    a, _ = synth.pair512_u8(seed=1, H=256, W=300)
    _check_detection(a, 10, 1.0, 10.0, 0.1, 0.5, "local26", tc=tc)


@pytest.mark.parametrize("tc", [True, 2, False], ids=["tc", "vtc", "ffma"])
def test_local26_plateau_keeps_every_item(tc):
    """A constant image has D = 0 in every layer: with a negative threshold
    every (pixel, layer) item is a 26-neighbour maximum (ties count), so the
    candidate list is the whole stack in row-major order, layers ascending
    within a pixel (several kept layers per pixel, one tile's worth)."""
    img = np.full((40, 37), 9, np.uint8)
    det = detector(n=2, t_min=1.0, t_max=2.0, threshold=-0.5, overlap=1.0, nms="local26",
                   keep_candidates=True, tensor_cores=tc)
    res = det(to_dev(img))
    assert res.n_candidates_true == 2 * 40 * 37 and not res.overflow
    c = res.candidates
    yy, xx, ii = np.meshgrid(np.arange(40), np.arange(37), np.arange(2), indexing="ij")
    assert np.array_equal(c["x"], xx.ravel()) and np.array_equal(c["y"], yy.ravel())
    assert np.array_equal(c["scale_idx"], ii.ravel()) and np.all(c["response"] == 0.0)


@pytest.mark.parametrize("shape,dtype", [((257, 383), "u16"), ((64, 64), "u8"),
                                         ((33, 500), "u8"), ((120, 90), "f32")])
def test_small_ladder_end_to_end(shape, dtype):
    img = scene(40 + shape[0], shape[0], shape[1], dtype)
    _check_detection(img, 4, 1.0, 4.0, 0.05, 0.5, "paper")
    _check_detection(img, 4, 1.0, 4.0, 0.05, 0.5, "paper", tc=False)
    _check_detection(img, 4, 1.0, 4.0, 0.05, 0.5, "local26")
    _check_detection(img, 4, 1.0, 4.0, 0.05, 0.5, "local26", tc=2)


@pytest.mark.parametrize("shape,dtype,sigma_d", [((300, 420), "u16", 0.0),
                                                 ((300, 420), "u16", 4.0),
                                                 ((260, 333), "u8", 1.0),
                                                 ((90, 40), "u16", 0.0)])
def test_headline_ladder_end_to_end(shape, dtype, sigma_d):
    """The benchmark's detector (n = 16, t = 1..12, tau = 0.05, overlap 0.5)
    on crops of its scene model, on both fused kernels and both rules; the
    90 x 40 image is narrower than the largest halo (48)."""
    img = scene(60 + shape[1], shape[0], shape[1], dtype, sigma_d)
    _check_detection(img, 16, 1.0, 12.0, 0.05, 0.5, "paper")
    _check_detection(img, 16, 1.0, 12.0, 0.05, 0.5, "paper", tc=False)
    _check_detection(img, 16, 1.0, 12.0, 0.05, 0.5, "local26")
    _check_detection(img, 16, 1.0, 12.0, 0.05, 0.5, "local26", tc=2)


@pytest.mark.parametrize("nms", ["paper", "local26"])
def test_two_pass_48_column_strips_match_oracle(nms):
    """The two-pass kernel at 48-column strips (24 columns a worker thread,
    the chooser's fallback for wide halos) on the benchmark ladder, both
    rules, and its response stack."""
    img = scene(64, 300, 333, "u16")
    kw = dict(tile_shape=[48, 0, 0, 0, 1])
    _check_detection(img, 16, 1.0, 12.0, 0.05, 0.5, nms, **kw)
    det = detector(n=16, t_min=1.0, t_max=12.0, threshold=0.05, nms=nms, **kw)
    assert det.tensor_core_kernel == 2
    D, _, _, _ = det.debug_stack(to_dev(img), want=("D",))
    D_ref, _, _ = ref_stack(img, 16, 1.0, 12.0)
    assert_stack_close(D.cpu().numpy(), D_ref, "48-column strips " + nms)


# ------------------------------------------------ tensor-core vertical pass

def test_tensor_core_pass_is_used_where_it_applies():
    # both passes for detection with the DoG response (the 26-neighbour rule
    # up to 16 layers), the vertical pass for the other tensor-core modes and
    # on request
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1).tensor_core_kernel == 2
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1,
                    tensor_cores=2).tensor_core_kernel == 1
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1,
                    nms="local26").tensor_core_kernel == 2
    assert detector(n=17, t_min=1.0, t_max=10.0, threshold=0.1,
                    nms="local26").tensor_core_kernel == 1
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1 / 0.9,
                    response="log").tensor_core_kernel == 1
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1).uses_tensor_cores
    assert not detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1,
                        tensor_cores=False).uses_tensor_cores
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1,
                    nms="local26").uses_tensor_cores
    assert not detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1 / 0.9, nms="local26",
                        response="log").uses_tensor_cores
    assert detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1 / 0.9,
                    response="log").uses_tensor_cores
    assert not detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1 / 0.9, response="log",
                        tensor_cores=False).uses_tensor_cores


@pytest.mark.parametrize("scale,kernel", [(1, "tensor cores"), (9, "FFMA companion")])
def test_uint16_stretch_range_decides_the_kernel(scale, kernel):
    """A uint16 image whose stretch range exceeds 4095 cannot be held exactly
    as fp16 integers: the FFMA companion takes it (gated on the device).
    Both ranges match the oracle's stack, and the two kernels agree on the
    same image within the stack tolerance."""
    base = scene(45, 180, 260, "u16")
    img = (base.astype(np.uint32) * scale).clip(0, 65535).astype(np.uint16)
    lo, hi = oracle.stretch_bounds(img)
    assert (hi - lo > 4095) == (scale > 1)
    det = detector(n=6, t_min=1.0, t_max=5.0, threshold=0.05)
    D, _, _, res = det.debug_stack(to_dev(img))
    D_ref, _, _ = ref_stack(img, 6, 1.0, 5.0)
    assert_stack_close(D.cpu().numpy(), D_ref, kernel)
    D2, _, _, _ = detector(n=6, t_min=1.0, t_max=5.0, threshold=0.05,
                           tensor_cores=False).debug_stack(to_dev(img))
    assert_stack_close(D.cpu().numpy(), D2.cpu().numpy().astype(np.float64), kernel + " vs FFMA")
    _check_detection(img, 6, 1.0, 5.0, 0.05, 0.5, "paper")


@pytest.mark.parametrize("overlap", [0.0, 0.3, 1.0])
def test_prune_overlap_settings(overlap):
    a, _ = synth.pair512_u8(seed=2, H=200, W=200)
    _check_detection(a, 10, 1.0, 10.0, 0.1, overlap, "paper")


def test_constant_image_has_no_features():
    img = np.full((70, 90), 77, np.uint8)
    det = detector(n=4, t_min=1.0, t_max=4.0, threshold=0.1)
    res = det(to_dev(img))
    assert res.lo == res.hi == 77.0
    assert res.n_blobs == 0 and res.n_candidates_true == 0


def test_overflow_reports_true_count():
    a, _ = synth.pair512_u8(seed=1)
    full = detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1)(to_dev(a))
    small = detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1, max_candidates=100)
    res = small(to_dev(a))
    assert res.overflow
    assert res.n_candidates == 100
    assert res.n_candidates_true == full.n_candidates_true > 100


def test_results_are_deterministic():
    img = scene(41, 300, 420, "u16")
    det = detector(n=4, t_min=1.0, t_max=4.0, threshold=0.05)
    r1 = det(to_dev(img))
    r2 = det(to_dev(img))
    assert np.array_equal(r1.blobs, r2.blobs)


def test_host_entry_point_matches_device_entry_point():
    a, _ = synth.pair512_u8(seed=3, H=200, W=180)
    det = detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1)
    r_dev = det(to_dev(a))
    r_host = det.detect_host(a)
    assert np.array_equal(r_dev.blobs, r_host.blobs)


def test_async_host_entry_point_on_several_streams():
    """Enqueued host detections on separate detectors and streams (copies
    overlapping other detections) give the results of the blocking call."""
    import paper_2108_12050_gb300 as mhfd
    imgs = [scene(90 + k, 300, 260, "u16", sigma_d=float(k)) for k in range(3)]
    pinned = []
    for im in imgs:
        t = torch.empty(im.shape, dtype=torch.int16, pin_memory=True)
        t.numpy()[:] = im.view(np.int16)
        pinned.append(t.numpy().view(np.uint16))
    dets = [mhfd.Detector(n=6, t_min=1.0, t_max=5.0, threshold=0.05) for _ in imgs]
    want = [d.detect_host(im) for d, im in zip(dets, imgs)]
    streams = [torch.cuda.Stream() for _ in imgs]
    for _ in range(2):
        for d, im, st in zip(dets, pinned, streams):
            assert d.detect_host(im, st, wait=False) is None
        for d, w in zip(dets, want):
            r = d.wait()
            assert r.n_blobs == w.n_blobs and np.array_equal(r.blobs, w.blobs)
    for d in dets:
        d.close()


# -------------------------------------------------------------------- prune

def test_settle_wait_limit_reports_timeout_and_detector_recovers(monkeypatch):
    """The prune's settle loop is bounded; when the bound runs out (here set
    to zero sweeps, so it gives up before the first) the detection reports
    MHFD_ERR_TIMEOUT, and the next detection on the same detector, with the
    default bound, gives the usual result (the context stays usable)."""
    import paper_2108_12050_gb300 as mhfd
    a, _ = synth.pair512_u8(seed=2, H=200, W=200)
    det = detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1, overlap=0.5)
    want = det(to_dev(a))
    assert want.n_candidates > 0
    monkeypatch.setenv("MHFD_PRUNE_MAX_SWEEPS", "0")
    with pytest.raises(mhfd.MhfdError) as e:
        det(to_dev(a))
    assert e.value.code == -5
    monkeypatch.delenv("MHFD_PRUNE_MAX_SWEEPS")
    again = det(to_dev(a))
    assert again.n_blobs == want.n_blobs and np.array_equal(again.blobs, want.blobs)


@pytest.mark.parametrize("seed,n,cluster,overlap", [(0, 3000, 0.0, 0.5), (1, 4000, 0.9, 0.5),
                                                    (2, 2500, 0.95, 0.1), (3, 1, 0.0, 0.5),
                                                    (4, 5000, 0.8, 0.0)])
def test_prune_bit_exact_on_identical_inputs(seed, n, cluster, overlap):
    H, W = 700, 900
    x, y, i, resp = synth.random_candidates(seed, n, H, W, 10, cluster=cluster)
    t = oracle.ladder(10, 1.0, 10.0)
    radius = math.sqrt(2.0) * t[:10]
    want = oracle.prune(x, y, i, resp.astype(np.float64), radius, overlap, W)
    det = detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1, overlap=overlap)
    keep = det.prune(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                     torch.from_numpy(i).cuda(), torch.from_numpy(resp).cuda(), H, W)
    torch.cuda.synchronize()
    assert np.array_equal(keep.cpu().numpy(), want)


# -------------------------------------------------------------- plain path

def test_plain_path_matches_oracle():
    """The unfused path's candidates, kept set, counts and mean response
    against the oracle under the same rules as the fused path."""
    a, _ = synth.pair512_u8(seed=4, H=260, W=300)
    _check_detection(a, 10, 1.0, 10.0, 0.1, 0.5, "paper", plain=True)
    img = scene(66, 300, 420, "u16")
    _check_detection(img, 16, 1.0, 12.0, 0.05, 0.5, "paper", plain=True)


# -------------------------------------------------- variants (plain path)

@pytest.mark.parametrize("response,boundary,nms,plain,tc", [
    ("dog", "periodic", "paper", False, False), ("dog", "reflect", "paper", False, False),
    ("log", "reflect", "paper", False, False), ("log", "periodic", "paper", False, False)] + [
    p + (True,) for p in [
    ("dog", "reflect", "paper", True), ("log", "reflect", "paper", True),
    ("dog", "periodic", "paper", True), ("log", "periodic", "paper", True),
    ("log", "reflect", "local26", True), ("dog", "periodic", "local26", True),
    ("dog", "periodic", "paper", False), ("dog", "periodic", "local26", False),
    ("log", "reflect", "paper", False), ("log", "periodic", "paper", False),
    ("log", "reflect", "local26", False)]])
def test_variants_match_oracle(response, boundary, nms, plain, tc):
    a, _ = synth.pair512_u8(seed=6, H=200, W=270)
    # the LoG response lacks the DoG's factor dt (0.9 here): threshold scaled
    thr = 0.1 / 0.9 if response == "log" else 0.1
    _check_detection(a, 10, 1.0, 10.0, thr, 0.5, nms, response=response, boundary=boundary,
                     plain=plain, tc=tc)


def test_fused_periodic_stack_within_tolerance():
    """The fused kernel's periodic variant against the oracle's periodic
    stack, on an image narrower than the largest kernel (wrap-around reads
    several periods away)."""
    img = scene(61, 70, 45, "u16")
    det = detector(n=10, t_min=1.0, t_max=10.0, threshold=0.1, boundary="periodic")
    D, _, _, _ = det.debug_stack(to_dev(img), want=("D",))
    lo, hi = oracle.stretch_bounds(img)
    t = oracle.ladder(10, 1.0, 10.0)
    D_ref = oracle.dog_stack(oracle.stretch(img, lo, hi), t, boundary=oracle.PERIODIC)
    assert_stack_close(D.cpu().numpy(), D_ref, "periodic")


def test_periodic_plain_commutes_with_circular_shift():
    import paper_2108_12050_gb300 as mhfd  # noqa: F401
    a = scene(77, 128, 160, "u16")
    det = detector(n=6, t_min=1.0, t_max=5.0, threshold=0.05, keep_candidates=True,
                   boundary="periodic")
    dy, dx = 37, 51
    det.detect_plain(to_dev(a))
    r0 = det.wait()
    det.detect_plain(to_dev(np.ascontiguousarray(np.roll(a, (dy, dx), axis=(0, 1)))))
    r1 = det.wait()
    H, W = a.shape
    inner = lambda x, y: 0 < x < W - 1 and 0 < y < H - 1  # noqa: E731
    f0 = {((x + dx) % W, (y + dy) % H, i) for x, y, i in features(r0.candidates)}
    f0 = {f for f in f0 if inner(f[0], f[1])}
    f1 = {f for f in features(r1.candidates) if inner(f[0], f[1])}
    # the 3x3 comparison window does not wrap: features whose window crosses
    # the image edge in either frame may differ
    edge0 = lambda x, y: x in (0, W - 1) or y in (0, H - 1)  # noqa: E731
    near = lambda f: any(edge0((f[0] - dx + ex) % W, (f[1] - dy + ey) % H)  # noqa: E731
                         for ex in (-1, 0, 1) for ey in (-1, 0, 1))
    diff = [f for f in f0 ^ f1 if not near(f)]
    assert not diff, diff[:10]


@pytest.mark.parametrize("tc", [True, False], ids=["tc", "ffma"])
@pytest.mark.parametrize("boundary,shape", [("reflect", (150, 230)), ("periodic", (70, 45))])
def test_fused_log_stack_within_tolerance(boundary, shape, tc):
    """The fused kernel's scale-normalised Laplacian (second differences
    folded into derived taps) against the oracle's 5-point stencil on its
    FP64 levels, including an image narrower than the largest kernel; on the
    tensor-core kernel (g and g'' vertical rows from the MMAs) and the FFMA
    one."""
    img = scene(71, shape[0], shape[1], "u16")
    n, tmin, tmax = 10, 1.0, 10.0
    det = detector(n=n, t_min=tmin, t_max=tmax, threshold=0.1, response="log",
                   boundary=boundary, tensor_cores=tc)
    assert det.uses_tensor_cores == tc
    D, _, _, _ = det.debug_stack(to_dev(img), want=("D",))
    lo, hi = oracle.stretch_bounds(img)
    t = oracle.ladder(n, tmin, tmax)
    Ip = oracle.stretch(img, lo, hi)
    bnd = oracle.PERIODIC if boundary == "periodic" else oracle.REFLECT
    D_ref = oracle.log_stack(Ip, t, boundary=bnd)
    # the derived taps leave no stencil cancellation: the DoG's 1e-4 bound
    assert_stack_close(D.cpu().numpy(), D_ref, "fused LoG %s" % boundary)


def test_soft_score_rejects_the_log_response():
    import paper_2108_12050_gb300 as mhfd
    from paper_2108_12050_gb300 import soft
    a, _ = synth.pair512_u8(seed=6, H=64, W=64)
    det = detector(n=4, t_min=1.0, t_max=4.0, threshold=0.1, response="log")
    with pytest.raises(mhfd.MhfdError) as e:
        soft.soft_score(det, to_dev(a.astype(np.float32)), torch.ones(4), 0.1)
    assert e.value.code == -2


# ------------------------------------------- two-row horizontal items (packed)

@pytest.mark.parametrize("shape,tc", [((256, 18, 8, 288, 4, 2), 2),
                                      ((284, 18, 8, 320, 4, 2), 2),
                                      ((320, 18, 4, 448, 3, 2), False)],
                         ids=["tc-256x8", "tc-284x8", "ffma-320x4"])
def test_two_row_items_match_oracle(shape, tc):
    """Shapes whose horizontal items cover two rows (packed two-lane FMAs
    over the row pair) on the benchmark ladder: the response stack within
    the tolerance and the detection under the parity rules."""
    img = scene(81, 300, 620, "u16")
    n, tmin, tmax = 16, 1.0, 12.0
    det = detector(n=n, t_min=tmin, t_max=tmax, threshold=0.05, tile_shape=list(shape),
                   tensor_cores=tc, keep_candidates=True)
    assert det.uses_tensor_cores == bool(tc)
    D, _, _, _ = det.debug_stack(to_dev(img), want=("D",))
    ref, D_ref, tol, t, _ = oracle_reference(img, n, tmin, tmax, 0.05, 0.5)
    assert_stack_close(D.cpu().numpy(), D_ref, str(shape))
    res = det(to_dev(img))
    check_detection(res, ref, D_ref, tol, 0.05, 0.5, "paper", t)


@pytest.mark.parametrize("response", ["dog", "log"])
def test_two_row_items_sum_like_one_row_items(response):
    """The packed two-row pass takes each lane's taps in the order of the
    one-row pass, so with the same geometry the FFMA kernel's stack is
    bit-identical."""
    img = scene(82, 200, 500, "u16")
    thr = 0.05 if response == "dog" else 0.05 / 0.6875
    kw = dict(n=16, t_min=1.0, t_max=12.0, threshold=thr, tensor_cores=False, response=response)
    one = detector(tile_shape=[320, 18, 4, 448, 4, 1], **kw)
    two = detector(tile_shape=[320, 18, 4, 448, 4, 2], **kw)
    D1, M1, A1, r1 = one.debug_stack(to_dev(img))
    D2, M2, A2, r2 = two.debug_stack(to_dev(img))
    assert torch.equal(D1, D2) and torch.equal(M1, M2) and torch.equal(A1, A2)
    assert np.array_equal(r1.blobs, r2.blobs)


@pytest.mark.parametrize("shape,nms,response", [
    ((192, 18, 4, 384, 2, 3), "local26", "dog"),
    ((192, 18, 4, 384, 2, 3), "paper", "dog"),
    ((160, 18, 4, 352, 3, 3), "paper", "log")], ids=["local26", "paper", "log"])
def test_two_output_items_match_oracle(shape, nms, response):
    """Shapes whose horizontal items cover one row of two outputs (twice the
    items per step, for strips too narrow to give every thread a four-output
    item) on the benchmark ladder: the stack within the tolerance and the
    detection under the parity rules, on the FFMA kernel."""
    img = scene(83, 300, 620, "u16")
    n, tmin, tmax = 16, 1.0, 12.0
    thr = 0.05 if response == "dog" else 0.05 / 0.6875
    det = detector(n=n, t_min=tmin, t_max=tmax, threshold=thr, tile_shape=list(shape),
                   tensor_cores=False, keep_candidates=True, nms=nms, response=response)
    D, _, _, _ = det.debug_stack(to_dev(img), want=("D",))
    ref, D_ref, tol, t, _ = oracle_reference(img, n, tmin, tmax, thr, 0.5, nms, response)
    assert_stack_close(D.cpu().numpy(), D_ref, str(shape))
    res = det(to_dev(img))
    check_detection(res, ref, D_ref, tol, thr, 0.5, nms, t)
