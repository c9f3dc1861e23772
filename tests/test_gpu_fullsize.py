"""Full-size parity in the launch configuration the benchmark times: the
4096x4096 uint16 tile of the defocus sweep, n = 16 scales (t = 1..12),
tau = 0.05, overlap 0.5, the autotuned tile shape.

The FP64 oracle builds the whole 17-level stack of the tile (about 2 GB of
FP64, a few seconds on the host's cores with its OpenMP loops) and the
detection from it, and every GPU path is held to it element by element:

* the response stack of the stack-storing variant of both fused kernels
  (tensor-core vertical pass, FFMA) within 1e-4 ||D_ref,i||_inf per layer;
* the whole candidate set (x, y, scale) of the fused kernels and of the
  plain path, the kept set after the prune, the counts per scale, the focus
  score and the mean response, up to the ambiguity rules of
  ``parity_util`` with per-layer tolerances;
* at sigma_d = 0 (dense maxima) and sigma_d = 4 (sparse, flat maxima), and
  for the scale-normalised Laplacian response at sigma_d = 0.

Each check prints one ``FULLSIZE {...}`` line with its counts (run with
``-s`` to see them).  The 8192^2 uint8 tile (the largest the service
takes) is checked on a sample of its candidates; the soft focus score at
its full size (2048^2 float32).
"""
import json
import math
import os
import time

import numpy as np
import pytest

import oracle
import synth
from parity_util import (ambiguous_paper, assert_stack_close, check_detection, log_eps,
                         oracle_reference, stack_rel_err)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, TMIN, TMAX, THR, OVERLAP = 16, 1.0, 12.0, 0.05, 0.5
DT = (TMAX - TMIN) / N


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.set_device(0)
    oracle.set_threads(os.cpu_count() or 1)


@pytest.fixture(scope="module", params=[("dog", 0.0), ("dog", 4.0), ("log", 0.0)],
                ids=["dog-sd0", "dog-sd4", "log-sd0"])
def reference(request):
    """The tile and the oracle's stack and detection of it (one at a time:
    each stack is 2.1 GB of FP64)."""
    response, sigma_d = request.param
    img = synth.sweep_tile_4096_u16(sigma_d)
    # the Laplacian lacks the DoG's factor dt: threshold scaled to match
    thr = THR / DT if response == "log" else THR
    t0 = time.time()
    ref, D, tol, t, Ip = oracle_reference(img, N, TMIN, TMAX, thr, OVERLAP, "paper", response)
    secs = time.time() - t0
    amb = ambiguous_paper(D, thr, tol)
    yield dict(img=img, ref=ref, D=D, tol=tol, t=t, Ip=Ip, thr=thr, amb=amb,
               response=response, sigma_d=sigma_d, oracle_s=secs)
    del D, amb


def _detector(response, tc, thr):
    import paper_2108_12050_gb300 as mhfd
    return mhfd.Detector(N, TMIN, TMAX, threshold=thr, overlap=OVERLAP, keep_candidates=True,
                         tensor_cores=tc, response=response)


# tc: the default (the two-pass kernel for the DoG, the vertical-pass kernel
# for the LoG); vtc: the vertical-pass kernel; ffma; plain
_TC = {"tc": True, "vtc": 2, "ffma": False, "plain": False}


@pytest.mark.parametrize("path", ["tc", "vtc", "ffma", "plain"])
def test_full_tile_detection_against_oracle(reference, path):
    r = reference
    img, ref, D_ref, t, thr = r["img"], r["ref"], r["D"], r["t"], r["thr"]
    det = _detector(r["response"], _TC[path], thr)
    assert det.uses_tensor_cores == bool(_TC[path])
    dev = torch.from_numpy(img.view(np.int16)).cuda()
    if path == "plain":
        det.detect_plain(dev)
        res = det.wait()
    else:
        res = det(dev)
    det.close()
    assert (res.lo, res.hi) == (ref.lo, ref.hi)
    assert res.n_candidates == res.n_candidates_true > 10000
    tol, amb = r["tol"], r["amb"]
    if r["response"] == "log" and path == "plain":
        # the plain path's 5-point stencil: its derived, wider tolerance
        R = [oracle.kernel_radius(ti) for ti in t[:N]]
        tol = log_eps(D_ref, t, R, float(np.abs(r["Ip"]).max()))
        amb = None
    stats = check_detection(res, ref, D_ref, tol, thr, OVERLAP, "paper", t, amb_maps=amb)
    stats.update(path=path, response=r["response"], sigma_d=r["sigma_d"],
                 score_gpu=res.n_blobs, score_ref=ref.score,
                 mean_response_gpu=res.mean_response, mean_response_ref=ref.mean_response,
                 oracle_s=round(r["oracle_s"], 1))
    print("FULLSIZE " + json.dumps(stats))


@pytest.mark.parametrize("tc", [True, 2], ids=["tc", "vtc"])
def test_full_tile_local26_against_oracle(reference, tc):
    """The 26-neighbour rule on the in-focus tile (the two-pass kernel by
    default, the vertical-pass kernel on request): the whole candidate set
    against the oracle's 3x3x3 maxima of the same stack, then the prune."""
    r = reference
    if r["response"] != "dog" or r["sigma_d"] != 0.0:
        pytest.skip("the 26-neighbour rule on the in-focus DoG tile")
    import paper_2108_12050_gb300 as mhfd
    if "ref26" not in r:
        ref26 = oracle.detect_from_stack(r["D"], r["t"], r["thr"], OVERLAP, mode=1)
        ref26["lo"], ref26["hi"] = r["ref"].lo, r["ref"].hi
        r["ref26"] = ref26
    ref26 = r["ref26"]
    det = mhfd.Detector(N, TMIN, TMAX, threshold=r["thr"], overlap=OVERLAP, nms="local26",
                        keep_candidates=True, tensor_cores=tc)
    assert det.tensor_core_kernel == (2 if tc is True else 1)
    res = det(torch.from_numpy(r["img"].view(np.int16)).cuda())
    det.close()
    assert (res.lo, res.hi) == (ref26.lo, ref26.hi)
    assert res.n_candidates == res.n_candidates_true > 10000
    stats = check_detection(res, ref26, r["D"], r["tol"], r["thr"], OVERLAP, "local26", r["t"])
    stats.update(path="local26", tc=tc)
    print("FULLSIZE " + json.dumps(stats))


@pytest.mark.parametrize("tc", [True, 2, False], ids=["tc", "vtc", "ffma"])
def test_full_tile_stack_within_tolerance(reference, tc):
    r = reference
    if r["sigma_d"] != 0.0:
        pytest.skip("stack compared on the in-focus tile")
    det = _detector(r["response"], tc, r["thr"])
    dev = torch.from_numpy(r["img"].view(np.int16)).cuda()
    D, _, _, res = det.debug_stack(dev, want=("D",))
    det.close()
    assert (res.lo, res.hi) == (r["ref"].lo, r["ref"].hi)
    Dh = D.cpu().numpy()
    del D
    rel = stack_rel_err(Dh, r["D"])
    print("FULLSIZE " + json.dumps({"stack": r["response"], "tc": tc,
                                    "max_rel_err_per_layer": [float("%.3g" % v) for v in rel]}))
    assert_stack_close(Dh, r["D"], "%s tc=%s" % (r["response"], tc))


def test_maximum_size_8192_uint8_sampled_against_oracle():
    """The largest tiles the service takes (8192^2, uint8): stretch bounds
    bit-exact, sampled candidates' responses and scales against the oracle
    (Eq. 2 at single pixels), counts consistent, and the prune of the GPU's
    list equal to the oracle's."""
    import paper_2108_12050_gb300 as mhfd
    img = synth.sweep_tile_4096_u16(0.0, seed=8192, H=8192, W=8192, dtype="u8")
    det = mhfd.Detector(N, TMIN, TMAX, threshold=THR, overlap=OVERLAP, keep_candidates=True)
    res = det(torch.from_numpy(img).cuda())
    det.close()
    lo, hi = oracle.stretch_bounds(img)
    assert (res.lo, res.hi) == (lo, hi)
    cands = res.candidates
    assert res.n_candidates == res.n_candidates_true == len(cands) > 10000
    rng = np.random.default_rng(13)
    pick = rng.choice(len(cands), 200, replace=False)
    t = oracle.ladder(N, TMIN, TMAX)
    D = oracle.dog_at(img, lo, hi, t, cands["x"][pick].astype(int), cands["y"][pick].astype(int))
    eps_i = 1e-4 * np.abs(D).max(axis=0)
    for k, j in enumerate(pick):
        i = int(cands["scale_idx"][j])
        assert abs(float(cands["response"][j]) - D[k, i]) <= eps_i[i], (k, i)
        srt = np.sort(D[k])
        assert i == int(D[k].argmax()) or srt[-1] - srt[-2] <= eps_i.max()
    radius = math.sqrt(2.0) * t[:N]
    keep = oracle.prune(cands["x"], cands["y"], cands["scale_idx"],
                        cands["response"].astype(np.float64), radius, OVERLAP, img.shape[1])
    assert res.n_blobs == res.focus_score == int(keep.sum())


def test_soft_score_full_size_2048_float32():
    import paper_2108_12050_gb300 as mhfd
    from paper_2108_12050_gb300 import soft
    img, _ = synth.soft_tile_f32(0)
    det = mhfd.Detector(N, TMIN, TMAX, threshold=THR)
    w = np.linspace(-0.5, 1.5, N)
    S, ms, _, _ = soft.soft_score(det, torch.from_numpy(img).cuda(),
                                  torch.tensor(w, dtype=torch.float32), THR, 0.01)
    lo, hi = oracle.stretch_bounds(img)
    S_ref, ms_ref, _ = oracle.soft_score(img, N, TMIN, TMAX, w, tau=THR, T=0.01, lo=lo, hi=hi,
                                         grad=False)
    np.testing.assert_allclose(ms.cpu().numpy(), ms_ref, rtol=0, atol=1e-4)
    assert abs(float(S) - S_ref) <= 1e-4 * np.abs(w).sum()
    det.close()
