"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test ties one oracle step to something other than the oracle itself:
closed forms (the Gaussian of §2.2, Gaussians convolving by adding variances,
the lens area), invariances, a library routine (numpy FFT for the paper's
Fourier formulation of §3, ``np.partition`` for order statistics, numerical
quadrature for overlaps) or brute force written differently on tiny inputs.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.usefixtures("oracle_mod")


# ----------------------------------------------------------------- ladder, taps

def test_ladder_matches_section_2_2():
    # §2.2: dt = (max_t - min_t)/n, t_i = min_t + (i-1) dt, i = 1..n+1
    t = oracle.ladder(10, 1.0, 10.0)
    np.testing.assert_allclose(t, 1.0 + 0.9 * np.arange(11), rtol=0, atol=1e-12)
    t = oracle.ladder(16, 1.0, 12.0)
    assert t.size == 17 and t[0] == 1.0 and abs(t[-1] - 12.0) < 1e-12
    np.testing.assert_allclose(np.diff(t), 11.0 / 16.0, atol=1e-12)


def test_kernel_radii_of_both_ladders():
    r10 = [oracle.kernel_radius(x) for x in oracle.ladder(10, 1, 10)]
    r16 = [oracle.kernel_radius(x) for x in oracle.ladder(16, 1, 12)]
    assert r10 == [4, 8, 12, 15, 19, 22, 26, 30, 33, 37, 40]
    assert r16 == [4, 7, 10, 13, 15, 18, 21, 24, 26, 29, 32, 35, 37, 40, 43, 46, 48]


@pytest.mark.parametrize("t", [1.0, 1.9, 3.7, 12.0])
def test_kernel_is_normalised_sampled_gaussian(t):
    g = oracle.kernel(t, 4.0)
    R = (g.size - 1) // 2
    assert R == math.ceil(4 * t)
    assert abs(g.sum() - 1.0) < 1e-14
    k = np.arange(-R, R + 1)
    ratio = g / g[R]
    np.testing.assert_allclose(ratio, np.exp(-k * k / (2 * t * t)), rtol=1e-13)
    np.testing.assert_array_equal(g, g[::-1])


# ------------------------------------------------------------- impulse response

@pytest.mark.parametrize("t", [1.0, 2.5])
def test_impulse_gives_outer_product(t):
    N = 101
    img = np.zeros((N, N)); img[50, 50] = 1.0
    g = oracle.kernel(t, 4.0)
    R = (g.size - 1) // 2
    L = oracle.blur(img, g)
    ref = np.zeros((N, N))
    ref[50 - R:51 + R, 50 - R:51 + R] = np.outer(g, g)
    np.testing.assert_allclose(L, ref, rtol=0, atol=1e-17)


@pytest.mark.parametrize("t", [1.0, 1.9, 4.6])
def test_impulse_matches_continuous_gaussian(t):
    # §2.2: G(x, y, t) = exp(-(x^2 + y^2)/(2 t^2)) / (2 pi t^2).  With the
    # truncation pushed to 8 t the sampled, normalised kernel matches the
    # density at integer points to ~2 exp(-2 pi^2 t^2) relative (Poisson sum).
    N = 2 * math.ceil(8 * t) + 11
    c = N // 2
    img = np.zeros((N, N)); img[c, c] = 1.0
    L = oracle.blur(img, oracle.kernel(t, 8.0))
    y, x = np.mgrid[0:N, 0:N]
    G = np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2 * t * t)) / (2 * math.pi * t * t)
    np.testing.assert_allclose(L, G, rtol=0, atol=1e-8)


# -------------------------------------------------- DoG of a planted Gaussian

def _gauss_image(N, s, A, c=None):
    c = N // 2 if c is None else c
    y, x = np.mgrid[0:N, 0:N]
    return A * np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2 * s * s))


def _dog_closed_form(t, s, A):
    # Gaussians convolve by adding variances, so L(centre, t) = A s^2/(s^2+t^2)
    L = A * s * s / (s * s + t * t)
    return t[:-1] * (L[1:] - L[:-1])


@pytest.mark.parametrize("s", [2.0, 3.5, 6.0])
@pytest.mark.parametrize("truncate,tol", [(4.0, 1e-3), (8.0, 1e-8)])
def test_dog_of_gaussian_blob_closed_form(s, truncate, tol):
    A = -0.6
    t = oracle.ladder(10, 1.0, 10.0)
    N = 241
    D = oracle.dog_stack(_gauss_image(N, s, A), t, truncate=truncate)
    got = D[:, N // 2, N // 2]
    want = _dog_closed_form(t, s, A)
    # Sampling both Gaussians on the pixel grid adds an aliasing term of
    # relative size ~2 exp(-2 pi^2 t^2 s^2 / (t^2 + s^2)) per level (Poisson
    # summation); for each DoG layer it enters twice, scaled by t_i.
    v = t * t * s * s / (t * t + s * s)
    alias = 4.0 * t[:-1] * np.exp(-2 * math.pi ** 2 * np.minimum(v[:-1], v[1:]))
    np.testing.assert_allclose(got, want, rtol=0, atol=tol * abs(A) + alias.max() * abs(A))
    assert int(np.argmax(got)) == int(np.argmax(want))


def test_dark_blob_response_is_positive_and_peaks_near_its_scale():
    # Eq. 2 with L_{i+1} - L_i: a dark blob (A < 0) gives a positive response;
    # the continuous scale-normalised Laplacian peaks at t = s.
    s, A = 4.6, -0.6
    t = oracle.ladder(10, 1.0, 10.0)
    D = oracle.dog_stack(_gauss_image(201, s, A), t)[:, 100, 100]
    assert D.max() > 0.1
    # the discrete DoG over [t_i, t_{i+1}] brackets the continuous optimum
    i = int(np.argmax(D))
    assert t[i] <= s + 1e-9 <= t[i + 1] + 1.0


# ------------------------------------------------------------------ invariances

def test_affine_invariance():
    rng = np.random.default_rng(5)
    I = rng.uniform(0, 1, (40, 37))
    t = oracle.ladder(4, 1.0, 3.0)
    D1 = oracle.dog_stack(I, t)
    D2 = oracle.dog_stack(2.5 * I + 0.3, t)
    np.testing.assert_allclose(D2, 2.5 * D1, rtol=0, atol=1e-12)


def test_periodic_shift_commutes_bit_exactly():
    rng = np.random.default_rng(6)
    I = rng.uniform(0, 1, (32, 29))
    t = oracle.ladder(3, 1.0, 2.5)
    D = oracle.dog_stack(I, t, boundary=oracle.PERIODIC)
    Ds = oracle.dog_stack(np.roll(I, (5, -7), axis=(0, 1)), t, boundary=oracle.PERIODIC)
    np.testing.assert_array_equal(Ds, np.roll(D, (5, -7), axis=(1, 2)))


def test_reflect_interior_shift_invariance():
    rng = np.random.default_rng(7)
    big = rng.uniform(0, 1, (90, 90))
    t = oracle.ladder(3, 1.0, 2.5)
    Rm = oracle.kernel_radius(t[-1])
    D1 = oracle.dog_stack(big[0:70, 0:70], t)
    D2 = oracle.dog_stack(big[9:79, 4:74], t)
    m = Rm + 1
    # pixel (y, x) of crop 2 is pixel (y+9, x+4) of crop 1
    a = D1[:, 9 + m:70 - m, 4 + m:70 - m]
    b = D2[:, m:70 - 9 - m, m:70 - 4 - m]
    np.testing.assert_array_equal(a, b)


def test_transpose_symmetry():
    rng = np.random.default_rng(8)
    I = rng.uniform(0, 1, (23, 31))
    t = oracle.ladder(4, 1.0, 4.0)
    D = oracle.dog_stack(I, t)
    DT = oracle.dog_stack(I.T.copy(), t)
    np.testing.assert_allclose(DT, np.transpose(D, (0, 2, 1)), rtol=0, atol=1e-14)


# ------------------------------------------------------------ boundary, 2-D sum

@pytest.mark.parametrize("shape", [(9, 7), (3, 20), (1, 5), (30, 2)])
def test_reflect_blur_equals_2d_direct_sum(shape):
    # brute force: pad by reflection (numpy's half-sample "symmetric" mode) and
    # sum the full 2-D kernel g g^T over the window; windows wider than the
    # image reflect more than once.
    rng = np.random.default_rng(9)
    I = rng.uniform(0, 1, shape)
    g = oracle.kernel(1.7, 4.0)
    R = (g.size - 1) // 2
    P = np.pad(I, R, mode="symmetric")
    K = np.outer(g, g)
    H, W = shape
    ref = np.empty(shape)
    for y in range(H):
        for x in range(W):
            ref[y, x] = np.sum(K * P[y:y + 2 * R + 1, x:x + 2 * R + 1])
    np.testing.assert_allclose(oracle.blur(I, g), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("boundary,pad", [(oracle.REFLECT, "symmetric"),
                                          (oracle.PERIODIC, "wrap")])
def test_log_stencil_equals_separable_second_difference_taps(boundary, pad):
    # the 5-point Laplacian of L = g (*)_x g (*)_y I, with L extended through
    # the blur's boundary, equals the sum of the two separable blurs with one
    # factor replaced by its second difference g''[k] = g[k-1] - 2 g[k] + g[k+1]
    # (radius R + 1): the formulation the fused LoG kernel computes.  Numpy
    # padding and explicit window sums, independent of the oracle's loops.
    rng = np.random.default_rng(21)
    I = rng.uniform(-0.5, 0.5, (23, 17))
    t = oracle.ladder(3, 1.0, 2.5)
    D = oracle.log_stack(I, t, boundary=boundary)

    def conv(img, taps, axis):
        K = (taps.size - 1) // 2
        widths = [(K, K) if a == axis else (0, 0) for a in range(2)]
        P = np.pad(img, widths, mode=pad)
        n = img.shape[axis]
        return sum(taps[j] * np.take(P, np.arange(j, j + n), axis=axis)
                   for j in range(taps.size))

    for i, ti in enumerate(t[:3]):
        g = oracle.kernel(float(ti))
        ge = np.concatenate(([0.0, 0.0], g, [0.0, 0.0]))
        d2 = ge[:-2] - 2 * ge[1:-1] + ge[2:]             # g''[-R-1..R+1]
        g1 = np.concatenate(([0.0], g, [0.0]))           # g on the same support
        ref = ti * ti * (conv(conv(I, g1, 0), d2, 1) + conv(conv(I, d2, 0), g1, 1))
        np.testing.assert_allclose(D[i], ref, rtol=0, atol=1e-13)


def test_dog_at_matches_separable_stack():
    img = synth.pair512_u8(seed=3, H=64, W=72)[0]
    lo, hi = oracle.stretch_bounds(img)
    t = oracle.ladder(10, 1.0, 10.0)
    D = oracle.dog_stack(oracle.stretch(img, lo, hi), t)
    xs = np.array([0, 5, 71, 33, 70, 1]); ys = np.array([0, 63, 10, 31, 62, 2])
    Dp = oracle.dog_at(img, lo, hi, t, xs, ys)
    np.testing.assert_allclose(Dp, D[:, ys, xs].T, rtol=0, atol=1e-13)


# ------------------------------------------------ the paper's FFT formulation

def test_periodic_mode_equals_fourier_product():
    # §3: L = F^-1{ F{G} . F{I} } is a circular convolution.  numpy's FFT of
    # the periodised sampled kernel must reproduce the periodic-mode blur.
    rng = np.random.default_rng(10)
    N = 64
    I = rng.uniform(0, 1, (N, N))
    t = 2.3
    g = oracle.kernel(t, 12.0)              # wide enough to wrap several times
    R = (g.size - 1) // 2
    k1 = np.zeros(N)
    for k in range(-R, R + 1):
        k1[k % N] += g[k + R]
    K = np.outer(k1, k1)
    ref = np.real(np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(I)))
    got = oracle.blur(I, g, boundary=oracle.PERIODIC)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------- NMS

def _stack_with_ties(rng, n, H, W):
    D = np.round(rng.uniform(-0.2, 1.0, (n, H, W)) * 8) / 8   # coarse -> ties
    D[:, 3:6, 3:6] = 0.75                                      # a plateau
    return D


def _brute_paper(D, thr):
    # "value is the maximum of the 3x3 x all-scales window, scale = first argmax"
    n, H, W = D.shape
    out = set()
    for y in range(H):
        for x in range(W):
            v = D[:, y, x].max()
            if not v > thr:
                continue
            win = D[:, max(0, y - 1):y + 2, max(0, x - 1):x + 2]
            if v >= win.max():
                out.add((x, y, int(np.flatnonzero(D[:, y, x] == v)[0])))
    return out


def _brute_26(D, thr):
    n, H, W = D.shape
    out = set()
    for i in range(n):
        for y in range(H):
            for x in range(W):
                v = D[i, y, x]
                if not v > thr:
                    continue
                ok = True
                for di in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            ii, yy, xx = i + di, y + dy, x + dx
                            if 0 <= ii < n and 0 <= yy < H and 0 <= xx < W and D[ii, yy, xx] > v:
                                ok = False
                if ok:
                    out.add((x, y, i))
    return out


@pytest.mark.parametrize("seed,shape", [(0, (6, 16, 16)), (1, (1, 9, 13)), (2, (4, 1, 12)),
                                        (3, (5, 11, 1)), (4, (3, 2, 2))])
def test_nms_paper_bruteforce(seed, shape):
    rng = np.random.default_rng(seed)
    D = _stack_with_ties(rng, *shape) if min(shape[1:]) > 6 else \
        np.round(rng.uniform(-0.2, 1.0, shape) * 8) / 8
    x, y, i, r, cnt = oracle.nms_paper(D, 0.1)
    got = set(zip(x.tolist(), y.tolist(), i.tolist()))
    assert got == _brute_paper(D, 0.1) and cnt == len(got)
    for xx, yy, ii, rr in zip(x, y, i, r):
        assert rr == D[ii, yy, xx]


@pytest.mark.parametrize("seed,shape", [(0, (6, 16, 16)), (1, (1, 9, 13)), (2, (4, 1, 12)),
                                        (5, (2, 7, 7))])
def test_nms_local26_bruteforce(seed, shape):
    rng = np.random.default_rng(seed)
    D = _stack_with_ties(rng, *shape) if min(shape[1:]) > 6 else \
        np.round(rng.uniform(-0.2, 1.0, shape) * 8) / 8
    x, y, i, r, cnt = oracle.nms_local26(D, 0.1)
    got = set(zip(x.tolist(), y.tolist(), i.tolist()))
    assert got == _brute_26(D, 0.1) and cnt == len(got)


def test_nms_threshold_is_strict_and_plateaus_are_kept():
    D = np.zeros((2, 5, 5)); D[1, 1:4, 1:4] = 0.5
    x, y, i, r, cnt = oracle.nms_paper(D, 0.5)
    assert cnt == 0
    x, y, i, r, cnt = oracle.nms_paper(D, 0.4999)
    assert cnt == 9 and set(i.tolist()) == {1}


# --------------------------------------------------------------- lens overlap

def test_lens_overlap_closed_forms():
    assert oracle.lens_overlap(2.0, 3.0, 0.0) == 1.0
    assert oracle.lens_overlap(2.0, 3.0, 5.0) == 0.0
    assert oracle.lens_overlap(2.0, 3.0, 6.0) == 0.0
    assert oracle.lens_overlap(1.0, 3.0, 1.5) == 1.0        # contained
    r = 2.7
    want = (2 * math.pi / 3 - math.sqrt(3) / 2) / math.pi   # r1 = r2 = d
    assert abs(oracle.lens_overlap(r, r, r) - want) < 1e-14


@pytest.mark.parametrize("r1,r2,d", [(1.4, 2.2, 2.0), (3.0, 3.0, 4.5), (5.1, 1.9, 4.0),
                                     (2.0, 2.5, 0.8)])
def test_lens_overlap_by_quadrature(r1, r2, d):
    from scipy import integrate
    # area of {|p| <= r1} & {|p - (d,0)| <= r2} by integrating chord lengths
    def chord(x):
        h1 = math.sqrt(max(r1 * r1 - x * x, 0.0))
        h2 = math.sqrt(max(r2 * r2 - (x - d) ** 2, 0.0))
        return 2 * min(h1, h2)
    lo, hi = max(-r1, d - r2), min(r1, d + r2)
    area, _ = integrate.quad(chord, lo, hi, epsabs=1e-13, epsrel=1e-12, limit=200)
    want = area / (math.pi * min(r1, r2) ** 2)
    assert abs(oracle.lens_overlap(r1, r2, d) - want) < 1e-9


# ----------------------------------------------------------------------- prune

def _brute_prune(x, y, i, resp, radius, overlap, W):
    order = sorted(range(len(x)), key=lambda j: (-i[j], -resp[j], y[j] * W + x[j]))
    kept = []
    keep = np.zeros(len(x), np.uint8)
    for j in order:
        ok = True
        for k in kept:
            d = math.hypot(x[j] - x[k], y[j] - y[k])
            if oracle.lens_overlap(radius[i[k]], radius[i[j]], d) > overlap:
                ok = False
                break
        if ok:
            kept.append(j)
            keep[j] = 1
    return keep


@pytest.mark.parametrize("seed,n,cluster,overlap", [(0, 300, 0.0, 0.5), (1, 400, 0.8, 0.5),
                                                    (2, 250, 0.9, 0.1), (3, 200, 0.9, 1.0),
                                                    (4, 1, 0.0, 0.5)])
def test_prune_bruteforce(seed, n, cluster, overlap):
    H, W = 120, 150
    x, y, i, resp = synth.random_candidates(seed, n, H, W, 10, cluster=cluster)
    radius = math.sqrt(2) * oracle.ladder(10, 1.0, 10.0)[:10]
    keep = oracle.prune(x, y, i, resp.astype(np.float64), radius, overlap, W)
    want = _brute_prune(x.tolist(), y.tolist(), i.tolist(), resp.tolist(), radius, overlap, W)
    np.testing.assert_array_equal(keep, want)
    if overlap >= 1.0:
        assert keep.all()


# --------------------------------------------------------------------- stretch

@pytest.mark.parametrize("dtype,shape", [(np.uint8, (37, 53)), (np.uint16, (64, 64)),
                                         (np.float32, (17, 19)), (np.uint8, (1, 1)),
                                         (np.uint16, (1, 600))])
def test_stretch_bounds_are_order_statistics(dtype, shape):
    rng = np.random.default_rng(11)
    if dtype == np.float32:
        img = rng.normal(0, 3, shape).astype(np.float32)
    else:
        img = rng.integers(0, np.iinfo(dtype).max + 1, shape).astype(dtype)
    N = img.size
    k = int(math.floor(0.00175 * N))
    flat = np.sort(img.ravel().astype(np.float64))
    lo, hi = oracle.stretch_bounds(img)
    assert lo == np.partition(img.ravel(), k)[k] == flat[k]
    assert hi == flat[N - 1 - k]


def test_stretch_saturates_and_maps_to_unit_interval():
    img = np.arange(2000, dtype=np.uint16).reshape(40, 50)
    lo, hi = oracle.stretch_bounds(img)
    assert (lo, hi) == (3.0, 1996.0)           # k = floor(0.00175 * 2000) = 3
    S = oracle.stretch(img, lo, hi)
    assert S.min() == 0.0 and S.max() == 1.0
    assert (S == 0).sum() == 4 and (S == 1).sum() == 4
    const = np.full((8, 8), 7, np.uint8)
    lo, hi = oracle.stretch_bounds(const)
    assert lo == hi == 7 and not oracle.stretch(const, lo, hi).any()


# -------------------------------------------------------------------- recovery

def test_noise_free_blob_recovery():
    # well separated dark Gaussian blobs on a flat background, no noise: each
    # blob is found within 1 px, at the scale that maximises the closed form
    N = 320
    cs = [(60, 60), (160, 60), (260, 60), (60, 200), (160, 200), (260, 200)]
    ss = [1.6, 2.4, 3.3, 4.2, 5.1, 6.0]
    img = np.full((N, N), 180.0)
    y, x = np.mgrid[0:N, 0:N]
    for (cx, cy), s in zip(cs, ss):
        img += -100.0 * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
    img8 = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    r = oracle.detect(img8, 10, 1.0, 10.0, threshold=0.1, overlap=0.5)
    t = r.t
    kx, ky, ki = r.x[r.keep], r.y[r.keep], r.i[r.keep]
    for (cx, cy), s in zip(cs, ss):
        d = np.hypot(kx - cx, ky - cy)
        j = int(np.argmin(d))
        assert d[j] <= 1.0
        want = int(np.argmax(_dog_closed_form(t, s, -1.0)))
        assert abs(int(ki[j]) - want) <= 1


def test_defocus_lowers_the_feature_count():
    a, b = synth.pair512_u8(seed=1, H=256, W=256)
    ra = oracle.detect(a, 10, 1.0, 10.0, threshold=0.1, overlap=0.5)
    rb = oracle.detect(b, 10, 1.0, 10.0, threshold=0.1, overlap=0.5)
    assert rb.score < ra.score


# ------------------------------------------------------- variants of §2.2 / §3

@pytest.mark.parametrize("s", [2.5, 4.0])
def test_log_response_of_gaussian_blob_closed_form(s):
    # L of a sampled Gaussian blob is (up to exp(-2 pi^2 v) aliasing) the
    # Gaussian of variance v = s^2 + t^2 and amplitude A s^2 / v; its 5-point
    # Laplacian at the centre is 4 L0 (exp(-1/(2v)) - 1) exactly.
    A = -0.6
    t = oracle.ladder(6, 1.0, 6.0)
    N = 181
    D = oracle.log_stack(_gauss_image(N, s, A), t, truncate=8.0)[:, N // 2, N // 2]
    v = s * s + t[:-1] ** 2
    L0 = A * s * s / v
    want = t[:-1] ** 2 * 4.0 * L0 * (np.exp(-1.0 / (2.0 * v)) - 1.0)
    np.testing.assert_allclose(D, want, rtol=0, atol=1e-7)
    assert np.all(D > 0)                      # dark blob -> positive, like the DoG


def test_log_and_dog_agree_in_sign_and_peak():
    # the DoG of Eq. 2 is the delta-t discretisation of t^2 grad^2 L
    s, A = 4.0, -0.6
    t = oracle.ladder(10, 1.0, 10.0)
    img = _gauss_image(201, s, A)
    dog = oracle.dog_stack(img, t)[:, 100, 100]
    log = oracle.log_stack(img, t)[:, 100, 100]
    assert abs(int(np.argmax(dog)) - int(np.argmax(log))) <= 1
    assert np.all(np.sign(dog) == np.sign(log))


def test_periodic_detection_commutes_with_circular_shift():
    # the blur wraps around; the 3x3 max-pool of Eq. 3 pads with -inf and
    # does not, so features on the outermost pixel ring are excluded
    H, W, dy, dx = 96, 128, 17, -30
    img = synth.pair512_u8(seed=5, H=H, W=W)[0]
    r0 = oracle.detect(img, 4, 1.0, 4.0, threshold=0.1, overlap=1.0, boundary=oracle.PERIODIC)
    sh = np.roll(img, (dy, dx), axis=(0, 1))
    r1 = oracle.detect(sh, 4, 1.0, 4.0, threshold=0.1, overlap=1.0, boundary=oracle.PERIODIC)

    def inner(x, y):
        return 0 < x < W - 1 and 0 < y < H - 1

    a = set()
    for x, y, i in zip(r0.x.tolist(), r0.y.tolist(), r0.i.tolist()):
        xs, ys = (x + dx) % W, (y + dy) % H
        if inner(x, y) and inner(xs, ys):
            a.add((xs, ys, i))
    b = set()
    for x, y, i in zip(r1.x.tolist(), r1.y.tolist(), r1.i.tolist()):
        x0, y0 = (x - dx) % W, (y - dy) % H
        if inner(x, y) and inner(x0, y0):
            b.add((x, y, i))
    assert a == b and len(a) > 10


# ------------------------------------------------- per-image statistics (a9)

def test_mean_response_of_identical_blobs_is_the_closed_form_peak():
    # Six identical noise-free dark Gaussian blobs at integer centres, far
    # apart, on a flat float image.  With no saturation (clip 0) the stretch
    # is affine, mapping the background to 1 and each blob's centre to 0, so
    # every blob has amplitude -1 after stretching.  Each is kept once, at
    # the scale maximising the closed-form DoG of its centre, and the mean
    # response of the kept features is that peak value.
    N, s = 360, 3.0
    cs = [(60, 60), (180, 60), (300, 60), (60, 240), (180, 240), (300, 240)]
    img = np.full((N, N), 180.0)
    y, x = np.mgrid[0:N, 0:N]
    for cx, cy in cs:
        img += -100.0 * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
    r = oracle.detect(img.astype(np.float32), 10, 1.0, 10.0, threshold=0.1, overlap=0.5,
                      clip=0.0)
    assert r.score == len(cs)
    t = r.t
    want = _dog_closed_form(t, s, -1.0)
    v = t * t * s * s / (t * t + s * s)
    alias = 4.0 * t[:-1] * np.exp(-2 * math.pi ** 2 * np.minimum(v[:-1], v[1:]))
    # float32 rounding of the image (relative 6e-8 of 180 over a range of 100)
    assert abs(r.mean_response - want.max()) <= 1e-3 + alias.max() + 1e-6
    assert set(r.i[r.keep].tolist()) == {int(np.argmax(want))}
    assert r.per_scale.sum() == r.score


def test_mean_response_is_zero_without_features():
    r = oracle.detect(np.full((40, 50), 9, np.uint8), 4, 1.0, 4.0, threshold=0.1)
    assert r.score == 0 and r.mean_response == 0.0


def test_detect_from_stack_equals_detect():
    a, _ = synth.pair512_u8(seed=3, H=150, W=170)
    for mode in (oracle.MODE_PAPER, oracle.MODE_LOCAL26):
        want = oracle.detect(a, 6, 1.0, 5.0, threshold=0.05, overlap=0.3, mode=mode)
        lo, hi = oracle.stretch_bounds(a)
        t = oracle.ladder(6, 1.0, 5.0)
        D = oracle.dog_stack(oracle.stretch(a, lo, hi), t)
        got = oracle.detect_from_stack(D, t, 0.05, 0.3, mode=mode)
        for k in ("x", "y", "i", "resp", "keep"):
            assert np.array_equal(got[k], want[k]), k
        assert got.score == want.score and got.mean_response == want.mean_response


def test_lens_overlap_many_equals_the_scalar_form():
    rng = np.random.default_rng(9)
    r1, r2 = rng.uniform(0.5, 5, 200), rng.uniform(0.5, 5, 200)
    d = rng.uniform(0, 11, 200)
    got = oracle.lens_overlap_many(r1, r2, d)
    want = [oracle.lens_overlap(a, b, c) for a, b, c in zip(r1, r2, d)]
    assert np.array_equal(got, np.array(want))
