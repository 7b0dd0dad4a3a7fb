"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check ties the oracle to something other than itself: a brute-force
sum written independently in Python, closed forms (constant image, box mean,
window area, step edge of height T), invariants (convexity of the weighted
mean, range-shift equivariance, transpose/flip symmetry) and the Gaussian
limit of q_N (Eq. approx2). The gradient is pinned by central differences of
the oracle's own forward and by the closed form of the linear N = 0 case.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1107_4617_gb300 import synth

GAMMA1 = math.pi / 2.0  # T = 1


def brute_force(f, r, gamma, N):
    """Independent Python restatement of Eq. filter2 on a tiny image:
    quadruple loop, math.cos ** N, truncated box window."""
    H, W = f.shape
    out = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            num = eta = 0.0
            for yy in range(max(0, y - r), min(H, y + r + 1)):
                for xx in range(max(0, x - r), min(W, x + r + 1)):
                    w = math.cos(gamma * (float(f[yy, xx]) - float(f[y, x]))) ** N
                    num += w * float(f[yy, xx])
                    eta += w
            out[y, x] = num / eta
    return out


def box_sum(a, r):
    """Truncated box sum via 2-D cumulative sums (a textbook summed-area table)."""
    H, W = a.shape
    S = np.zeros((H + 1, W + 1))
    S[1:, 1:] = np.cumsum(np.cumsum(a, 0), 1)
    y0 = np.clip(np.arange(H) - r, 0, H)
    y1 = np.clip(np.arange(H) + r + 1, 0, H)
    x0 = np.clip(np.arange(W) - r, 0, W)
    x1 = np.clip(np.arange(W) + r + 1, 0, W)
    return (S[y1][:, x1] - S[y0][:, x1] - S[y1][:, x0] + S[y0][:, x0])


@pytest.mark.parametrize("r", [1, 3, 8])
@pytest.mark.parametrize("N", [0, 1, 2, 5, 11])
def test_brute_force_8x8(r, N):
    f = np.random.default_rng(10 * r + N).uniform(0, 1, (8, 8))
    got = oracle.bilateral(f, r, GAMMA1, N)
    ref = brute_force(f, r, GAMMA1, N)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_brute_force_nonsquare_odd():
    f = synth.rectangles(5, 9, seed=3).astype(np.float64)
    for r, N in [(2, 3), (4, 8)]:
        np.testing.assert_allclose(oracle.bilateral(f, r, GAMMA1, N),
                                   brute_force(f, r, GAMMA1, N), rtol=0, atol=1e-13)


def test_constant_image_unchanged():
    f = np.full((17, 23), 0.37)
    out, den = oracle.bilateral(f, 5, GAMMA1, 11, return_den=True)
    np.testing.assert_allclose(out, 0.37, rtol=0, atol=1e-14)
    np.testing.assert_allclose(den, box_sum(np.ones_like(f), 5), rtol=0, atol=1e-12)


def test_window_area_closed_form():
    """N = 0: every weight is 1, so den is the clipped window area
    (min(x+r, W-1) - max(x-r, 0) + 1) * (same in y)."""
    H, W, r = 13, 29, 4
    f = np.random.default_rng(1).uniform(0, 1, (H, W))
    _, den = oracle.bilateral(f, r, GAMMA1, 0, return_den=True)
    ys, xs = np.arange(H), np.arange(W)
    cy = np.minimum(ys + r, H - 1) - np.maximum(ys - r, 0) + 1
    cx = np.minimum(xs + r, W - 1) - np.maximum(xs - r, 0) + 1
    np.testing.assert_array_equal(den, np.outer(cy, cx).astype(np.float64))
    assert den[H // 2, W // 2] == (2 * r + 1) ** 2


@pytest.mark.parametrize("r", [0, 2, 7])
def test_N0_is_box_mean(r):
    f = synth.sinusoids(31, 40, seed=2).astype(np.float64)
    ref = box_sum(f, r) / box_sum(np.ones_like(f), r)
    np.testing.assert_allclose(oracle.bilateral(f, r, GAMMA1, 0), ref, rtol=0, atol=1e-13)


def test_r0_identity():
    f = synth.rectangles(19, 21, seed=4).astype(np.float64)
    np.testing.assert_array_equal(oracle.bilateral(f, 0, GAMMA1, 11), f)


def test_convexity():
    """Weights are >= 0 on [-T, T], so out(x) lies between the window's min
    and max (a kernel is non-negative, Sec. 2)."""
    from scipy.ndimage import maximum_filter, minimum_filter
    f = synth.rectangles(40, 33, seed=5).astype(np.float64)
    for r, N in [(3, 11), (6, 41), (2, 1)]:
        out = oracle.bilateral(f, r, GAMMA1, N)
        lo = minimum_filter(f, size=2 * r + 1, mode="nearest")
        hi = maximum_filter(f, size=2 * r + 1, mode="nearest")
        assert np.all(out >= lo - 1e-12) and np.all(out <= hi + 1e-12)


def test_range_shift_equivariance():
    f = 0.5 * synth.rectangles(24, 24, seed=6).astype(np.float64)
    a = oracle.bilateral(f, 4, GAMMA1, 11)
    b = oracle.bilateral(f + 0.3, 4, GAMMA1, 11)
    np.testing.assert_allclose(b, a + 0.3, rtol=0, atol=1e-13)


def test_transpose_and_flip_symmetry():
    f = synth.rectangles(18, 27, seed=8).astype(np.float64)
    out = oracle.bilateral(f, 3, GAMMA1, 5)
    np.testing.assert_allclose(oracle.bilateral(f.T, 3, GAMMA1, 5), out.T, atol=1e-14, rtol=0)
    np.testing.assert_allclose(oracle.bilateral(f[::-1, ::-1], 3, GAMMA1, 5),
                               out[::-1, ::-1], atol=1e-14, rtol=0)


def test_step_of_height_T_is_preserved():
    """Across a step of height exactly T, cos^N(pi/2) = 0 for N >= 1, so no
    weight crosses the edge and each side is returned unchanged."""
    f = np.zeros((12, 16))
    f[:, 8:] = 1.0
    for N in (1, 2, 11):
        np.testing.assert_allclose(oracle.bilateral(f, 5, GAMMA1, N), f, rtol=0, atol=1e-15)


def test_gaussian_limit_of_kernel():
    """Eq. approx2: with gamma sqrt(N) = 1/sigma, cos^N(gamma t) ->
    exp(-t^2 / (2 sigma^2)); the sup error over [-1,1] shrinks as N grows."""
    sigma = 0.2
    ts = np.linspace(-1, 1, 401)
    errs = []
    for N in (11, 25, 50, 100, 400):
        g = oracle.gamma_from_sigma(sigma, N)
        w = np.array([oracle.weight(t, g, N) for t in ts])
        errs.append(np.max(np.abs(w - np.exp(-ts ** 2 / (2 * sigma ** 2)))))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-3
    # roughly O(1/N): quadrupling N cuts the error by at least 3x
    assert errs[-2] / errs[-1] > 3.0


def test_gaussian_limit_of_filter():
    f = synth.rectangles(24, 24, seed=9).astype(np.float64)
    ref = oracle.bilateral_gauss(f, 3, 0.2)
    errs = []
    for N in (11, 50, 400):
        errs.append(np.max(np.abs(oracle.bilateral(f, 3, oracle.gamma_from_sigma(0.2, N), N) - ref)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


def test_order_rule():
    assert [oracle.resolve_N(s, 1.0) for s in (0.1, 0.15, 0.2, 0.3)] == [41, 19, 11, 5]
    assert oracle.resolve_N(0.4, 1.0) == 3
    assert oracle.resolve_N(0.08, 1.0) == 64


def _loss(f, g, r, gamma, N):
    return float(np.sum(g * oracle.bilateral(f, r, gamma, N)))


@pytest.mark.parametrize("N", [1, 4, 11])
def test_gradient_vs_central_differences(N):
    rng = np.random.default_rng(N)
    f = 0.2 + 0.6 * rng.uniform(0, 1, (9, 11))
    g = rng.normal(0, 1, f.shape)
    r, gamma, h = 2, GAMMA1, 1e-4
    gf, gg = oracle.bilateral_grad(f, g, r, gamma, N)
    for (y, x) in [(0, 0), (4, 5), (8, 10), (3, 0), (6, 9)]:
        fp = f.copy(); fp[y, x] += h
        fm = f.copy(); fm[y, x] -= h
        fd = (_loss(fp, g, r, gamma, N) - _loss(fm, g, r, gamma, N)) / (2 * h)
        assert abs(fd - gf[y, x]) <= 1e-7 * max(1.0, abs(fd)), (y, x, fd, gf[y, x])
    fd = (_loss(f, g, r, gamma + h, N) - _loss(f, g, r, gamma - h, N)) / (2 * h)
    assert abs(fd - gg) <= 1e-7 * max(1.0, abs(fd)), (fd, gg)


@pytest.mark.parametrize("N", [4, 11])
def test_gradient_range_shift_invariance(N):
    """out(f + c) = out(f) + c (the weights depend on differences of f only),
    so L(f + c) = L(f) + c sum(g): dL/df and dL/dgamma do not change when the
    whole range moves by a constant. The GPU engine relies on this when it
    runs on f - T/2."""
    rng = np.random.default_rng(20 + N)
    f = 0.7 * rng.uniform(0, 1, (12, 15))
    g = rng.normal(0, 1, f.shape)
    gf, gg = oracle.bilateral_grad(f, g, 3, GAMMA1, N)
    gf2, gg2 = oracle.bilateral_grad(f + 0.3, g, 3, GAMMA1, N)
    np.testing.assert_allclose(gf2, gf, rtol=0, atol=1e-12 * np.abs(gf).max())
    assert abs(gg2 - gg) <= 1e-11 * max(1.0, abs(gg)), (gg, gg2)


def test_gradient_N0_closed_form():
    """N = 0 is the linear box mean, whose adjoint is Box[g / count]."""
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, (10, 13))
    g = rng.normal(0, 1, f.shape)
    r = 3
    gf, gg = oracle.bilateral_grad(f, g, r, GAMMA1, 0)
    cnt = box_sum(np.ones_like(f), r)
    np.testing.assert_allclose(gf, box_sum(g / cnt, r), rtol=0, atol=1e-13)
    assert gg == 0.0


def test_points_match_full():
    f = synth.rectangles(30, 37, seed=11).astype(np.float64)
    full = oracle.bilateral(f, 4, GAMMA1, 11)
    idx = np.array([0, 5, 36, 37 * 15 + 20, 30 * 37 - 1])
    np.testing.assert_array_equal(oracle.bilateral_points(f, 4, GAMMA1, 11, idx), full.ravel()[idx])
    part = oracle.bilateral(f, 4, GAMMA1, 11, rows=(10, 17))
    np.testing.assert_array_equal(part, full[10:17])


# ---- truncated expansion (end of Sec. 3) ------------------------------------

def binom_coeffs(N):
    ks = list(range(N % 2, N + 1, 2))
    a = [math.comb(N, (N - k) // 2) / 2.0 ** (N - 1) for k in ks]
    if N % 2 == 0:
        a[0] /= 2
    return ks, a


@pytest.mark.parametrize("N", [0, 1, 4, 11, 41])
def test_truncated_kernel_full_expansion_is_cos_power(N):
    """All N/2 + 1 harmonics: the expansion is cos^N exactly (binomial
    theorem), so the truncated-kernel filter reproduces the q_N filter."""
    K = N // 2 + 1
    for t in np.linspace(-1, 1, 41):
        assert abs(oracle.trunc_weight(t, GAMMA1, N, K) - math.cos(GAMMA1 * t) ** N) <= 1e-14
    f = synth.rectangles(14, 17, seed=N).astype(np.float64)
    np.testing.assert_allclose(
        oracle.bilateral_general(f, 3, range_kind=oracle.RANGE_TRUNC, gamma=GAMMA1, N=N,
                                 K_keep=K),
        oracle.bilateral(f, 3, GAMMA1, N), rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,K", [(11, 3), (41, 11), (41, 15), (20, 4)])
def test_truncated_kernel_error_closed_form(N, K):
    """Dropping the harmonics from index K on changes the kernel by at most
    the dropped coefficients' sum, reached at t = 0 (all cosines 1); the
    kept kernel equals an independent sum of math.cos terms."""
    ks, a = binom_coeffs(N)
    tail = sum(a[K:])
    ts = np.linspace(-1, 1, 801)
    dev = [abs(oracle.trunc_weight(t, GAMMA1, N, K) - math.cos(GAMMA1 * t) ** N) for t in ts]
    assert max(dev) <= tail + 1e-14
    assert abs(oracle.trunc_weight(0.0, GAMMA1, N, K) - (1.0 - tail)) <= 1e-14
    for t in (-0.7, 0.13, 0.9):
        ref = sum(ai * math.cos(k * GAMMA1 * t) for ai, k in zip(a[:K], ks[:K]))
        assert abs(oracle.trunc_weight(t, GAMMA1, N, K) - ref) <= 1e-14


def test_truncated_filter_brute_force_and_bound():
    """Truncated-kernel filter against a Python quadruple loop, and its
    distance to the exact q_N filter within the bound
    |out_t - out| <= n * tail * max|f - out_t| / den (den of the exact q_N)."""
    N, K, r = 41, 11, 2
    ks, a = binom_coeffs(N)
    f = np.random.default_rng(3).uniform(0, 1, (7, 9))
    H, W = f.shape
    ref = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            num = eta = 0.0
            for yy in range(max(0, y - r), min(H, y + r + 1)):
                for xx in range(max(0, x - r), min(W, x + r + 1)):
                    t = f[yy, xx] - f[y, x]
                    w = sum(ai * math.cos(k * GAMMA1 * t) for ai, k in zip(a[:K], ks[:K]))
                    num += w * f[yy, xx]
                    eta += w
            ref[y, x] = num / eta
    got = oracle.bilateral_general(f, r, range_kind=oracle.RANGE_TRUNC, gamma=GAMMA1, N=N,
                                   K_keep=K)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    # out - out_t = sum (w - w_t)(f - out_t) / sum w, |w - w_t| <= tail, |f - out_t| <= 1
    exact, den = oracle.bilateral(f, r, GAMMA1, N, return_den=True)
    tail = sum(a[K:])
    n = (2 * r + 1) ** 2
    assert np.all(np.abs(got - exact) <= n * tail / den + 1e-12)


# ---- shiftable spatial kernel (Algorithm 1; Algorithm 2 with M > 0) ---------

def test_spatial_kernel_closed_form():
    """q_M(d) = cos^M(pi d / (2 Ts)) with Ts = r + 1/2 (Sec. 3): unimodal,
    1 at d = 0, positive on the window |d| <= r."""
    for r, M in [(1, 1), (5, 2), (10, 4), (3, 8)]:
        vals = [oracle.spatial_weight(d, r, M) for d in range(-r, r + 1)]
        for d, v in zip(range(-r, r + 1), vals):
            assert abs(v - math.cos(math.pi * d / (2 * r + 1)) ** M) <= 1e-15
        assert vals[r] == 1.0 and min(vals) > 0
        assert all(vals[i] <= vals[i + 1] for i in range(r))


@pytest.mark.parametrize("r,M", [(1, 1), (3, 2), (5, 4), (7, 6)])
def test_algorithm1_is_normalised_separable_correlation(r, M):
    """Without a range kernel the filter is the linear spatial filter of
    Eq. filter1 normalised over the in-image part of the window: a separable
    correlation of f and of the all-ones image with the 1-D q_M taps
    (scipy.ndimage, zero padding), divided."""
    ndimage = pytest.importorskip("scipy.ndimage")
    f = synth.sinusoids(23, 31, seed=r + M).astype(np.float64)
    taps = np.array([math.cos(math.pi * d / (2 * r + 1)) ** M for d in range(-r, r + 1)])

    def sep(a):
        a = ndimage.correlate1d(a, taps, axis=0, mode="constant", cval=0.0)
        return ndimage.correlate1d(a, taps, axis=1, mode="constant", cval=0.0)
    ref = sep(f) / sep(np.ones_like(f))
    got = oracle.bilateral_general(f, r, spatial=oracle.SPATIAL_QM, M=M,
                                   range_kind=oracle.RANGE_NONE)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_spatial_M0_is_box():
    f = synth.rectangles(12, 15, seed=2).astype(np.float64)
    np.testing.assert_allclose(
        oracle.bilateral_general(f, 3, spatial=oracle.SPATIAL_QM, M=0, gamma=GAMMA1, N=11),
        oracle.bilateral(f, 3, GAMMA1, 11), rtol=0, atol=1e-15)


@pytest.mark.parametrize("r,M,N", [(2, 2, 4), (3, 1, 3), (1, 2, 0)])
def test_spatial_range_brute_force(r, M, N):
    """Algorithm 2's target, Eq. filter2 with phi = q_M x q_M and phi_range = q_N,
    against an independent Python quadruple loop."""
    f = np.random.default_rng(r * 7 + M + N).uniform(0, 1, (7, 8))
    H, W = f.shape
    ref = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            num = eta = 0.0
            for yy in range(max(0, y - r), min(H, y + r + 1)):
                for xx in range(max(0, x - r), min(W, x + r + 1)):
                    ws = (math.cos(math.pi * (yy - y) / (2 * r + 1)) ** M *
                          math.cos(math.pi * (xx - x) / (2 * r + 1)) ** M)
                    wr = math.cos(GAMMA1 * (f[yy, xx] - f[y, x])) ** N
                    num += ws * wr * f[yy, xx]
                    eta += ws * wr
            ref[y, x] = num / eta
    got = oracle.bilateral_general(f, r, spatial=oracle.SPATIAL_QM, M=M,
                                   range_kind=oracle.RANGE_COSN if N else oracle.RANGE_NONE,
                                   gamma=GAMMA1, N=N)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_spatial_constant_image_and_convexity():
    c = np.full((9, 13), 0.37)
    np.testing.assert_allclose(
        oracle.bilateral_general(c, 4, spatial=oracle.SPATIAL_QM, M=2, gamma=GAMMA1, N=4), c,
        rtol=0, atol=1e-15)
    f = synth.rectangles(20, 20, seed=9).astype(np.float64)
    out = oracle.bilateral_general(f, 3, spatial=oracle.SPATIAL_QM, M=2, gamma=GAMMA1, N=4)
    assert out.min() >= f.min() - 1e-15 and out.max() <= f.max() + 1e-15


# ---- polynomial range kernel p_N (Sec. 3) -----------------------------------

def test_poly_kernel_gaussian_limit():
    """Eq. approx1: p_N(t / sqrt(N)) -> exp(-t^2 / T^2), monotonically in N on
    [-T, T] (T = 1 here), with the direct oracle filter converging to the
    exact-Gaussian filter of variance T^2 / 2."""
    t = np.linspace(-1, 1, 201)
    gaps = []
    for N in (1, 2, 4, 8, 16, 64, 256):
        pn = (1 - (t / math.sqrt(N)) ** 2) ** N
        gaps.append(np.max(np.abs(pn - np.exp(-t ** 2))))
    assert all(a > b for a, b in zip(gaps, gaps[1:])) and gaps[-1] < 2e-3
    f = synth.rectangles(24, 24, seed=4).astype(np.float64)
    # p_N with T_r = sqrt(N) T: kernel (1 - t^2/(N T^2))^N -> exp(-t^2/T^2) = Gaussian sigma^2 = 1/2
    g = oracle.bilateral_gauss(f, 3, math.sqrt(0.5))
    errs = [np.abs(oracle.bilateral_general(f, 3, range_kind=oracle.RANGE_POLY, N=N,
                                            Tr=math.sqrt(N)) - g).max() for N in (2, 8, 32)]
    assert errs[0] > errs[1] > errs[2]


def test_poly_filter_brute_force_and_N0():
    N, r = 3, 2
    f = np.random.default_rng(8).uniform(0, 1, (6, 9))
    H, W = f.shape
    ref = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            num = eta = 0.0
            for yy in range(max(0, y - r), min(H, y + r + 1)):
                for xx in range(max(0, x - r), min(W, x + r + 1)):
                    w = (1.0 - (f[yy, xx] - f[y, x]) ** 2) ** N
                    num += w * f[yy, xx]
                    eta += w
            ref[y, x] = num / eta
    got = oracle.bilateral_general(f, r, range_kind=oracle.RANGE_POLY, N=N, Tr=1.0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    # p_0 = 1: the box mean
    np.testing.assert_allclose(oracle.bilateral_general(f, r, range_kind=oracle.RANGE_POLY, N=0),
                               box_sum(f, r) / box_sum(np.ones_like(f), r), rtol=0, atol=1e-14)


def test_gauss_points_match_full():
    f = synth.rectangles(20, 23, seed=6).astype(np.float64)
    full = oracle.bilateral_gauss(f, 3, 0.2)
    idx = np.array([0, 5, 77, 199, 459])
    np.testing.assert_allclose(oracle.bilateral_gauss_points(f, 3, 0.2, idx), full.ravel()[idx],
                               rtol=0, atol=1e-15)


def test_gauss_filter_brute_force():
    """The exact-Gaussian bilateral filter (the kernel q_N approximates, Eq.
    approx2) against an independent Python quadruple loop with math.exp."""
    f = np.random.default_rng(21).uniform(0, 1, (7, 8))
    r, sig = 2, 0.15
    H, W = f.shape
    ref = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            num = eta = 0.0
            for yy in range(max(0, y - r), min(H, y + r + 1)):
                for xx in range(max(0, x - r), min(W, x + r + 1)):
                    wgt = math.exp(-(f[yy, xx] - f[y, x]) ** 2 / (2 * sig * sig))
                    num += wgt * f[yy, xx]
                    eta += wgt
            ref[y, x] = num / eta
    np.testing.assert_allclose(oracle.bilateral_gauss(f, r, sig), ref, rtol=0, atol=1e-13)


# ---- stored fixtures (tests/golden) ----------------------------------------

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(_GOLDEN, name), comments="#")


def _golden_fp32(name):
    """Stored FP32 values (9 significant digits round-trip through FP32 only)."""
    return _golden(name).astype(np.float32).astype(np.float64)


def _golden_header(name, key):
    for line in open(os.path.join(_GOLDEN, name)):
        if line.startswith("# " + key):
            return float(line.split("=")[1])
    raise KeyError(key)


@pytest.mark.parametrize("r,N", [(2, 3), (1, 4), (3, 41), (2, 50)])
def test_golden_outputs_reproduce(r, N):
    """The oracle on the stored 24 x 20 image gives the stored outputs (written
    by tests/golden/make_golden.py): a change to the oracle's arithmetic shows
    here. The stored values also match the Python brute force of Eq. filter2."""
    f = _golden_fp32("img_24x20.txt")
    want = _golden("out_r%d_N%d.txt" % (r, N))
    assert f.shape == want.shape == (24, 20)
    np.testing.assert_allclose(oracle.bilateral(f, r, GAMMA1, N), want, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(brute_force(f, r, GAMMA1, N), want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("r,N", [(2, 3), (3, 41)])
def test_golden_gradients_reproduce(r, N):
    """The oracle's direct-form dL/df and dL/dgamma on the stored image and
    weights give the stored values; dL/dgamma also against FP64 central
    differences of the brute force in gamma."""
    f = _golden_fp32("img_24x20.txt")
    g = _golden_fp32("weights_24x20.txt")
    name = "grad_r%d_N%d.txt" % (r, N)
    gf, gg = oracle.bilateral_grad(f, g, r, GAMMA1, N)
    np.testing.assert_allclose(gf, _golden(name), rtol=1e-12, atol=1e-14)
    want_gg = _golden_header(name, "dL/dgamma")
    assert abs(gg - want_gg) <= 1e-12 * max(1.0, abs(want_gg))
    h = 1e-6
    fd = (np.sum(g * brute_force(f, r, GAMMA1 + h, N))
          - np.sum(g * brute_force(f, r, GAMMA1 - h, N))) / (2 * h)
    assert abs(fd - want_gg) <= 1e-6 * max(1.0, abs(want_gg)), (fd, want_gg)
