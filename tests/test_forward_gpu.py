"""GPU parity of bf_forward against the FP64 oracle (element by element).

Tolerance: |gpu - oracle| / max(|oracle|, 1e-2 T) <= 1e-4 for every pixel
(relative error with a floor at 1% of the range bound T, so pixels near 0 do
not divide by ~0). The oracle is the direct O(r^2) definition; the GPU runs
the O(1) moving-sum method, so agreement tests the whole method.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from _quads import rowmajor
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_err(got, ref, T=1.0):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2 * T)


def run_fwd(bf, img_np, r, sigma_r=0.2, T=1.0, N=0, kahan=False, dtype=torch.float32,
            tile_h=0, tile_w=0, saved=False, guard=0):
    dev = torch.device("cuda:0")
    img = torch.from_numpy(np.ascontiguousarray(img_np)).to(dev).to(dtype)
    H, W = img_np.shape
    opts = bf._opts(kahan=kahan, in_dtype=bf.BF16 if dtype == torch.bfloat16 else bf.F32,
                    tile_h=tile_h, tile_w=tile_w, save=saved)
    buf = torch.full((H * W + 2 * guard,), 12345.0, dtype=torch.float32, device=dev)
    out = buf[guard:guard + H * W].view(H, W)
    sv = torch.empty((H, W, 4), dtype=torch.float32, device=dev) if saved else None
    bf.bf_forward(img, r, sigma_r, T, N, out=out, opts=opts, saved=sv)
    torch.cuda.synchronize()
    if guard:
        b = buf.cpu().numpy()
        assert np.all(b[:guard] == 12345.0) and np.all(b[guard + H * W:] == 12345.0), "guard band written"
    res = out.cpu().numpy()
    # saved quads as planes: (f - T/2, 1/den, out - T/2, dnum_s - out dden_s)
    return (res, np.moveaxis(rowmajor(sv), 2, 0)) if saved else res


def oracle_ref(img_np, r, sigma_r, T, N, gamma=None):
    if N <= 0:
        N = oracle.resolve_N(sigma_r, T)
    g = oracle.gamma_fixed(T) if gamma is None else gamma
    return oracle.bilateral(img_np.astype(np.float64), r, g, N, return_den=True)


def test_config1_plain_forward(cuda_lib):
    """256x256 rectangles+noise, r=5, sigma_r=0.2 -> N=11, T=1 (full image)."""
    f = synth.rectangles(256, 256, seed=0)
    got = run_fwd(cuda_lib, f, 5, 0.2, 1.0, 0, guard=4096)
    ref, den = oracle_ref(f, 5, 0.2, 1.0, 0)
    e = rel_err(got, ref)
    assert e.max() <= TOL, e.max()


@pytest.mark.parametrize("kind", ["rect", "sin"])
@pytest.mark.parametrize("r,sigma", [(3, 0.1), (10, 0.2), (30, 0.3)])
def test_sweep_small(cuda_lib, kind, r, sigma):
    """Forward-sweep parameters (r, sigma_r -> N = 41/11/5) on 160x203 images
    (several strips and bands, ragged tails)."""
    f = synth.image(kind, 160, 203, seed=1)
    got = run_fwd(cuda_lib, f, r, sigma, 1.0, 0, tile_h=48)
    ref, _ = oracle_ref(f, r, sigma, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (29, 1), (5, 300), (300, 7), (33, 65)])
@pytest.mark.parametrize("r", [0, 1, 32])
def test_degenerate_shapes(cuda_lib, H, W, r):
    f = synth.rectangles(H, W, seed=H * 1000 + W)
    got = run_fwd(cuda_lib, f, r, 0.2, 1.0, 0, guard=256)
    ref, _ = oracle_ref(f, r, 0.2, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


@pytest.mark.parametrize("N", [0, 1, 2, 3, 40, 41, 64])
def test_orders(cuda_lib, N):
    f = synth.rectangles(97, 131, seed=N)
    got = run_fwd(cuda_lib, f, 4, 0.2, 1.0, N)
    ref, _ = oracle_ref(f, 4, 0.2, 1.0, N)
    assert rel_err(got, ref).max() <= TOL


def test_r0_identity_and_constant(cuda_lib):
    f = synth.rectangles(64, 70, seed=3)
    got = run_fwd(cuda_lib, f, 0, 0.1, 1.0, 0)
    np.testing.assert_allclose(got, f, rtol=0, atol=2e-6)
    c = np.full((50, 77), 0.625, np.float32)
    got = run_fwd(cuda_lib, c, 7, 0.1, 1.0, 0)
    np.testing.assert_allclose(got, 0.625, rtol=0, atol=1e-5)


def test_range_bound_T(cuda_lib):
    """T != 1: an image in [0, 4] filtered with T = 4 equals 4x the [0, 1]
    image filtered with T = 1."""
    f = synth.rectangles(80, 90, seed=5)
    a = run_fwd(cuda_lib, f, 5, 0.2, 1.0, 0)
    b = run_fwd(cuda_lib, 4.0 * f, 5, 0.8, 4.0, 0)
    ref, _ = oracle_ref(4.0 * f, 5, 0.8, 4.0, 0)
    assert rel_err(b, ref, T=4.0).max() <= TOL
    np.testing.assert_allclose(b, 4.0 * a, rtol=0, atol=4e-5)


@pytest.mark.parametrize("tile_w,tile_h", [(64, 16), (128, 40), (256, 300)])
def test_tile_overrides(cuda_lib, tile_w, tile_h):
    f = synth.sinusoids(120, 250, seed=9)
    got = run_fwd(cuda_lib, f, 9, 0.15, 1.0, 0, tile_h=tile_h, tile_w=tile_w)
    ref, _ = oracle_ref(f, 9, 0.15, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


def test_kahan_forward(cuda_lib):
    f = synth.rectangles(300, 180, seed=11)
    got = run_fwd(cuda_lib, f, 30, 0.1, 1.0, 0, kahan=True)
    ref, _ = oracle_ref(f, 30, 0.1, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


def test_bf16_input(cuda_lib):
    """BF16-stored input: parity against the oracle on the BF16-decoded image."""
    f = synth.rectangles(200, 150, seed=12)
    fb = torch.from_numpy(f).to(torch.bfloat16).float().numpy()
    got = run_fwd(cuda_lib, f, 6, 0.1, 1.0, 0, dtype=torch.bfloat16)
    ref, _ = oracle_ref(fb, 6, 0.1, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


def test_saved_buffers(cuda_lib):
    """The saved quads: f and out shifted by the range midpoint T/2 (exactly
    as read and written, in FP32), 1/den equal to the oracle's normaliser's
    reciprocal; den >= 1."""
    f = synth.rectangles(90, 110, seed=13)
    got, sv = run_fwd(cuda_lib, f, 5, 0.2, 1.0, 0, saved=True)
    ref, den = oracle_ref(f, 5, 0.2, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL
    np.testing.assert_array_equal(sv[0], f - np.float32(0.5))
    np.testing.assert_array_equal(sv[2] + np.float32(0.5), got)
    np.testing.assert_allclose(1.0 / sv[1], den, rtol=2e-5, atol=0)
    assert (1.0 / sv[1]).min() >= 1.0 - 1e-5


def test_full_size_sampled_n40(cuda_lib):
    """4096x4096, r=10, N=40 (even order: the constant harmonic runs apart from
    the pairs) in the default launch configuration, with saved quads as in the
    fwd+bwd step: 1200 sampled pixels plus corners and edge midpoints."""
    H = W = 4096
    f = synth.rectangles(H, W, seed=0)
    got, sv = run_fwd(cuda_lib, f, 10, 0.1, 1.0, 40, saved=True)
    rng = np.random.default_rng(40)
    idx = np.concatenate([rng.integers(0, H * W, 1200),
                          [0, W - 1, (H - 1) * W, H * W - 1, W // 2, (H // 2) * W, (H // 2) * W + W - 1,
                           (H - 1) * W + W // 2]])
    ref, den = oracle.bilateral_points(f.astype(np.float64), 10, math.pi / 2, 40, idx,
                                       return_den=True)
    assert rel_err(got.ravel()[idx], ref).max() <= TOL
    np.testing.assert_allclose(1.0 / sv[1].ravel()[idx], den, rtol=2e-5, atol=0)


def test_full_size_sampled_headline(cuda_lib):
    """4096x4096, r=10, sigma_r=0.1 -> N=41 in the default launch
    configuration: 3000 sampled pixels (plus the four corners and edge
    midpoints) against the oracle, and den >= 1 everywhere."""
    H = W = 4096
    f = synth.rectangles(H, W, seed=0)
    got, sv = run_fwd(cuda_lib, f, 10, 0.1, 1.0, 0, saved=True)
    rng = np.random.default_rng(42)
    idx = np.concatenate([rng.integers(0, H * W, 3000),
                          [0, W - 1, (H - 1) * W, H * W - 1, W // 2, (H // 2) * W, (H // 2) * W + W - 1,
                           (H - 1) * W + W // 2]])
    ref = oracle.bilateral_points(f.astype(np.float64), 10, math.pi / 2, 41, idx)
    assert rel_err(got.ravel()[idx], ref).max() <= TOL
    assert (1.0 / sv[1]).min() >= 1.0 - 1e-4
    assert np.isfinite(got).all()



@pytest.mark.parametrize("N", [44, 50, 64])
def test_chunked_harmonics_with_saved(cuda_lib, N):
    """N > 43 runs the harmonics in chunks that accumulate in the saved
    buffers; result, den and the centre derivatives match a single pass."""
    f = synth.rectangles(150, 170, seed=N)
    got, sv = run_fwd(cuda_lib, f, 6, 0.2, 1.0, N, saved=True)
    ref, den = oracle_ref(f, 6, 0.2, 1.0, N)
    assert rel_err(got, ref).max() <= TOL
    np.testing.assert_array_equal(sv[0], f - np.float32(0.5))
    np.testing.assert_array_equal(sv[2] + np.float32(0.5), got)
    np.testing.assert_allclose(1.0 / sv[1], den, rtol=2e-5, atol=0)


@pytest.mark.parametrize("r", [21, 30, 45, 56, 57, 64])
def test_wide_strips_large_r(cuda_lib, r):
    """Large r: 128-thread strips up to r = 40, 256-thread strips above, up to
    BF_R_MAX = 64 (256 - 2 * 64 = 128 output columns per strip)."""
    f = synth.sinusoids(260, 333, seed=r)
    got = run_fwd(cuda_lib, f, r, 0.1, 1.0, 0)
    ref, _ = oracle_ref(f, r, 0.1, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


@pytest.mark.parametrize("saved", [False, True])
def test_kahan_precision_form(cuda_lib, saved):
    """Kahan-compensated running sums at r=30, N=41 (the precision workload's
    parameters) on a tall image: with saved buffers the compensated skewed-strip
    engine (harmonic chunks), without them the single-pass kernel."""
    f = synth.rectangles(900, 140, seed=21)
    res = run_fwd(cuda_lib, f, 30, 0.1, 1.0, 0, kahan=True, saved=saved, tile_h=900)
    got = res[0] if saved else res
    ref, _ = oracle_ref(f, 30, 0.1, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


def _noise_case(cuda_lib, r, N, tile_h):
    """Independent U[0, 1] pixels on 8192 x 300 (den near 1: the hardest case
    for cancellation), forward with plain and with Kahan-compensated running
    sums, relative error on 3000 pixels of the bottom 200 rows (where the
    vertical running sums of a tall band have run longest) and 1000 others."""
    H, W = 8192, 300
    f = synth.noise(H, W, seed=3)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.integers((H - 200) * W, H * W, 3000), rng.integers(0, H * W, 1000)])
    ref = oracle.bilateral_points(f.astype(np.float64), r, math.pi / 2, N, idx)
    errs = {}
    for kahan in (False, True):
        got, _ = run_fwd(cuda_lib, f, r, 0.1, 1.0, N, kahan=kahan, saved=True, tile_h=tile_h)
        errs[kahan] = rel_err(got.ravel()[idx], ref).max()
    return errs[False], errs[True]


def test_kahan_bounds_the_drift_of_a_tall_band(cuda_lib):
    """A case where plain FP32 running sums drift past the parity bar and the
    Kahan form keeps them inside it: white noise, r = 2, N = 64, one band of
    all 8192 rows per strip (tile_h = H). Each step adds the planes of a pixel
    entering the window and of one leaving it 2r+1 rows after it entered; the
    rounding of those adds random-walks down the band. Kahan-compensated adds
    of every stream's (bit-identical) products let a pixel's entering and
    leaving contributions cancel."""
    plain, kahan = _noise_case(cuda_lib, 2, 64, 8192)
    assert kahan <= TOL, kahan
    assert plain > TOL, plain  # measured 5.1e-4 on a GB300


@pytest.mark.parametrize("r", [0, 1])
def test_smallest_windows_on_white_noise(cuda_lib, r):
    """The worst case of the error growth along a strip: white noise, r <= 1
    (den close to 1 at most pixels), N = 64, in the default launch
    configuration. The Kahan form stays inside the parity bar; the plain form
    reaches about 1.4 times it (measured 1.4e-4 at r = 1: 7e-6 absolute, at
    pixels whose value is near 0, where the relative metric's floor is 1e-2),
    the bound recorded here."""
    plain, kahan = _noise_case(cuda_lib, r, 64, 0)
    assert kahan <= TOL, kahan
    assert plain <= 3 * TOL, plain


@pytest.mark.parametrize("kp_max", [1, 3, 6])
def test_kp_max_chunks(cuda_lib, kp_max):
    """Fewer harmonic pairs per launch (chunks accumulating in the saved
    buffers) give the same filter and den."""
    bf = cuda_lib
    f = synth.rectangles(120, 200, seed=kp_max)
    dev = torch.device("cuda:0")
    img = torch.from_numpy(f).to(dev)
    sv1 = torch.empty((120, 200, 4), device=dev)
    sv2 = torch.empty((120, 200, 4), device=dev)
    a = bf.bf_forward(img, 8, 0.1, 1.0, 0, opts=bf._opts(save=True, kp_max=kp_max), saved=sv1)
    b = bf.bf_forward(img, 8, 0.1, 1.0, 0, opts=bf._opts(save=True), saved=sv2)
    torch.cuda.synchronize()
    ref, den = oracle_ref(f, 8, 0.1, 1.0, 0)
    assert rel_err(a.cpu().numpy(), ref).max() <= TOL
    assert torch.max(torch.abs(a - b)).item() <= 1e-5
    # den and the centre derivatives: same sums in another order (the
    # derivative planes cancel heavily, so compare against each plane's scale)
    s1, s2 = np.moveaxis(sv1.cpu().numpy(), 2, 0), np.moveaxis(sv2.cpu().numpy(), 2, 0)
    scale = np.abs(s2).max(axis=(1, 2), keepdims=True)
    assert np.all(np.abs(s1 - s2) <= 1e-4 * scale)


@pytest.mark.parametrize("H,W,r", [(300, 333, 0), (300, 333, 1), (64, 1000, 2), (512, 700, 1)])
def test_small_r_wide_images(cuda_lib, H, W, r):
    """Small windows (den close to 1 where neighbours differ) on wide images,
    where the horizontal chain runs through all 128 lanes of a strip."""
    f = synth.rectangles(H, W, seed=H + r)
    got = run_fwd(cuda_lib, f, r, 0.1, 1.0, 0)
    ref, _ = oracle_ref(f, r, 0.1, 1.0, 0)
    assert rel_err(got, ref).max() <= TOL


_SWEEP_IMAGES = {}


@pytest.mark.parametrize("size", [1024, 4096])
@pytest.mark.parametrize("kind", ["rect", "sin"])
@pytest.mark.parametrize("r", [3, 10, 30])
@pytest.mark.parametrize("sigma", [0.1, 0.2, 0.3])
def test_sweep_full_size_sampled(cuda_lib, size, kind, r, sigma):
    """The forward sweep at its own sizes, all 36 runs crossed: 1024^2 and
    4096^2, rectangles+noise and the sinusoid field, r in {3, 10, 30}, sigma_r
    in {0.1, 0.2, 0.3} -> N = 41/11/5, in the default launch configuration:
    400 sampled pixels plus the corners and edge midpoints against the
    oracle, evaluated one by one."""
    key = (kind, size)
    if key not in _SWEEP_IMAGES:
        _SWEEP_IMAGES[key] = synth.image(kind, size, size, seed=2)
    f = _SWEEP_IMAGES[key]
    got = run_fwd(cuda_lib, f, r, sigma, 1.0, 0)
    rng = np.random.default_rng(size + r)
    n = size * size
    idx = np.concatenate([rng.integers(0, n, 400),
                          [0, size - 1, n - size, n - 1, size // 2, (size // 2) * size,
                           (size // 2) * size + size - 1, n - size + size // 2]])
    ref = oracle.bilateral_points(f.astype(np.float64), r, math.pi / 2,
                                  oracle.resolve_N(sigma, 1.0), idx)
    assert rel_err(got.ravel()[idx], ref).max() <= TOL
    assert np.isfinite(got).all()


@pytest.mark.parametrize("H,W", [(1, 1), (7, 3), (512, 700), (2048, 2048)])
def test_check_range(cuda_lib, H, W):
    """bf_check_range reports the image's min and max (the precondition
    max - min <= T of the range kernels), FP32 and BF16."""
    bf = cuda_lib
    rng = np.random.default_rng(H + W)
    f = rng.normal(0.3, 2.0, (H, W)).astype(np.float32)
    t = torch.from_numpy(f).cuda()
    mm = bf.bf_check_range(t).cpu().numpy()
    assert mm[0] == f.min() and mm[1] == f.max()
    tb = t.to(torch.bfloat16)
    mb = bf.bf_check_range(tb).cpu().numpy()
    fb = tb.float().cpu().numpy()
    assert mb[0] == fb.min() and mb[1] == fb.max()


@pytest.mark.parametrize("H,W,r,sigma,N", [(300, 500, 10, 0.1, 40), (257, 390, 3, 0.1, 41),
                                           (200, 333, 24, 0.2, 11), (1024, 1024, 3, 0.1, 41)])
def test_narrow_strips_on_small_images(cuda_lib, H, W, r, sigma, N):
    """Small images take 64-thread strips (four CTAs per SM) where the launch
    model says they finish sooner; r = 24 is the widest window they hold
    (64 - 2r = 16 output columns). The default launch against the oracle
    (whole image, or 2000 sampled pixels at 1024^2) and against explicit
    128-thread strips, with and without the saved quads."""
    f = synth.rectangles(H, W, seed=H + r)
    got, sv = run_fwd(cuda_lib, f, r, sigma, 1.0, N, saved=True)
    wide, sv_w = run_fwd(cuda_lib, f, r, sigma, 1.0, N, saved=True, tile_w=128)
    plain = run_fwd(cuda_lib, f, r, sigma, 1.0, N)
    if H * W <= 200000:
        ref, den = oracle_ref(f, r, sigma, 1.0, N)
        assert rel_err(got, ref).max() <= TOL
        np.testing.assert_allclose(1.0 / sv[1], den, rtol=2e-5, atol=0)
    else:
        idx = np.random.default_rng(H).integers(0, H * W, 2000)
        ref = oracle.bilateral_points(f.astype(np.float64), r, math.pi / 2, N, idx)
        assert rel_err(got.ravel()[idx], ref).max() <= TOL
    assert np.abs(got - wide).max() <= 1e-5
    assert np.abs(plain - got).max() <= 1e-5
    np.testing.assert_array_equal(sv[0], sv_w[0])
