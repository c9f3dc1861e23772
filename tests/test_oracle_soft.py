"""Pins of the oracle's soft focus score and its gradient.

* the blur adjoint satisfies <B x, y> = <x, B^T y> (dot-product test), with
  the reflect boundary and windows wider than the image;
* dS/dI matches FP64 central differences (h = 1e-3 input units) on 64x64
  crops with the stretch bounds held fixed, away from pixels within h of
  lo/hi (where the clamp is not differentiable);
* S is linear in the weights with dS/dw_i = mean sigmoid of layer i.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.usefixtures("oracle_mod")


@pytest.mark.parametrize("shape,t", [((23, 31), 1.9), ((7, 40), 3.1), ((64, 64), 12.0)])
def test_blur_adjoint_dot_product(shape, t):
    rng = np.random.default_rng(3)
    x = rng.normal(size=shape)
    y = rng.normal(size=shape)
    g = oracle.kernel(t, 4.0)
    lhs = np.sum(oracle.blur(x, g) * y)
    rhs = np.sum(x * oracle.blur_adjoint(y, g))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def _crop():
    img, _ = synth.soft_tile_f32(0, H=256, W=256)
    return np.ascontiguousarray(img[40:104, 80:144])


@pytest.mark.parametrize("n,tmin,tmax", [(4, 1.0, 4.0), (16, 1.0, 12.0)])
def test_gradient_matches_central_differences(n, tmin, tmax):
    img = _crop().astype(np.float32)
    lo, hi = oracle.stretch_bounds(img)
    w = np.linspace(0.5, 1.5, n)
    tau, T = 0.05, 0.01
    S, ms, g = oracle.soft_score(img, n, tmin, tmax, w, tau=tau, T=T, lo=lo, hi=hi)
    h = 1e-3
    rng = np.random.default_rng(4)
    inside = np.argwhere((img > lo + 2 * h) & (img < hi - 2 * h))
    pick = inside[rng.choice(len(inside), 24, replace=False)]
    # include the pixels with the largest gradients
    big = np.dstack(np.unravel_index(np.argsort(-np.abs(g).ravel())[:8], g.shape))[0]
    scale = np.abs(g).max()
    for y, x in list(pick) + list(big):
        if not (lo + 2 * h < img[y, x] < hi - 2 * h):
            continue
        a = img.astype(np.float64)
        # perturb in float64 precision through a float32 image: use exact
        # representable steps by evaluating on float64-converted copies
        ap = a.copy(); ap[y, x] += h
        am = a.copy(); am[y, x] -= h
        Sp = oracle.soft_score(ap.astype(np.float32), n, tmin, tmax, w, tau=tau, T=T, lo=lo,
                               hi=hi, grad=False)[0]
        Sm = oracle.soft_score(am.astype(np.float32), n, tmin, tmax, w, tau=tau, T=T, lo=lo,
                               hi=hi, grad=False)[0]
        hp = float(np.float32(a[y, x] + h)) - float(np.float32(a[y, x]))
        hm = float(np.float32(a[y, x])) - float(np.float32(a[y, x] - h))
        fd = (Sp - Sm) / (hp + hm)
        assert abs(fd - g[y, x]) <= 1e-6 * scale + 1e-4 * abs(g[y, x]), (y, x, fd, g[y, x])


def test_score_is_linear_in_weights():
    img = _crop().astype(np.float32)
    n = 4
    w = np.array([0.3, -0.2, 1.1, 0.7])
    S, ms, _ = oracle.soft_score(img, n, 1.0, 4.0, w, tau=0.05, grad=False)
    assert abs(S - np.dot(w, ms)) < 1e-12
    for i in range(n):
        w2 = w.copy(); w2[i] += 0.25
        S2, _, _ = oracle.soft_score(img, n, 1.0, 4.0, w2, tau=0.05, grad=False)
        assert abs((S2 - S) - 0.25 * ms[i]) < 1e-12
    assert np.all((ms > 0) & (ms < 1))


@pytest.mark.parametrize("H,W,t", [(40, 50, 3.0), (20, 9, 4.0), (7, 5, 6.0)])
def test_reflect_blur_is_self_adjoint(H, W, t):
    """Symmetric taps with the half-sample symmetric (reflect) extension give
    a symmetric operator, also when the kernel is wider than the image: the
    adjoint written from the mirror families equals the blur itself."""
    rng = np.random.default_rng(int(H * W))
    y = rng.standard_normal((H, W))
    g = oracle.kernel(t)
    np.testing.assert_allclose(oracle.blur_adjoint(y, g), oracle.blur(y, g), rtol=0, atol=1e-13)
