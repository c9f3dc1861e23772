"""The two-pass kernel restates the 26-neighbour rule (§3's 3x3x3 test on
the layers of Eq. 2) as a pass over the layers in order, keeping per pixel
only the previous layer's 3x3 maximum and one pending flag.  This is that
restatement in numpy, step for step as the kernel takes it, held to the
oracle's brute-force rule on stacks with ties, plateaus, image edges,
negative thresholds and one- or two-layer stacks.  It shows that the
decomposition itself (not its CUDA) keeps exactly the oracle's items."""
import numpy as np
import pytest

import oracle


def _max3x3(a):
    """3x3 maximum around each pixel, neighbours outside the image left out."""
    H, W = a.shape
    p = np.full((H + 2, W + 2), -np.inf)
    p[1:-1, 1:-1] = a
    return np.max([p[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
                   for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)


def layerwise_local26(D, thr):
    """Per layer I: S_I = 3x3 max of D_I; an item of layer I - 1 flagged one
    layer earlier is kept when its response (the stored maximum there) is not
    below S_I; the items of layer I with D_I >= max(S_I, S_{I-1}, next float
    above thr) are flagged (kept at once in the top layer); the stored
    maximum becomes max(S_I, next float above thr)."""
    n = D.shape[0]
    thrp = np.nextafter(thr, np.inf)
    mx = np.full(D.shape[1:], thrp)
    fl = np.zeros(D.shape[1:], bool)
    kept = []
    for I in range(n):
        x = D[I]
        S = _max3x3(x)
        ge = ~(S > mx)
        for y, xx in zip(*np.nonzero(fl & ge)):
            kept.append((int(xx), int(y), I - 1))
        flag = ~(np.maximum(S, mx) > x)
        mx = np.maximum(S, thrp)
        if I == n - 1:
            for y, xx in zip(*np.nonzero(flag)):
                kept.append((int(xx), int(y), I))
        fl = flag
    return kept


def _stack(rng, n, H, W, levels):
    return np.round(rng.uniform(-0.2, 1.0, (n, H, W)) * levels) / levels


@pytest.mark.parametrize("seed,shape,levels,thr", [
    (0, (6, 16, 16), 8, 0.1), (1, (1, 9, 13), 8, 0.1), (2, (4, 1, 12), 8, 0.1),
    (3, (2, 7, 7), 4, 0.1), (4, (5, 12, 1), 3, -0.5), (5, (3, 20, 17), 2, 0.0),
    (6, (16, 24, 31), 16, 0.3), (7, (8, 11, 9), 1000, 0.05)])
def test_layerwise_restatement_keeps_the_oracles_items(seed, shape, levels, thr):
    rng = np.random.default_rng(seed)
    D = _stack(rng, *shape, levels)
    x, y, i, r, cnt = oracle.nms_local26(D, thr)
    want = sorted(zip(x.tolist(), y.tolist(), i.tolist()), key=lambda f: (f[1], f[0], f[2]))
    got = sorted(layerwise_local26(D, thr), key=lambda f: (f[1], f[0], f[2]))
    assert got == want and cnt == len(want)
    assert 0 < cnt < D.size or thr < 0


def test_layerwise_restatement_keeps_plateaus_whole():
    """A constant stack with a negative threshold keeps every item; a flat
    plateau above the threshold in two adjacent layers keeps both layers."""
    D = np.zeros((3, 5, 6))
    assert len(layerwise_local26(D, -0.5)) == D.size
    D[1:3, 1:4, 2:5] = 0.7
    got = set(layerwise_local26(D, 0.5))
    x, y, i, r, cnt = oracle.nms_local26(D, 0.5)
    assert got == set(zip(x.tolist(), y.tolist(), i.tolist())) and len(got) == 18
