"""GPU adjoint (bf_backward and the autograd wrapper) against the oracle's
direct-form reference gradient and FP64 central differences.

Gradient tolerance: max |gpu - ref| / max |ref| <= 1e-3 over the image, and
elementwise |gpu - ref| <= 1e-3 max(|ref|, 1e-2 max|ref|).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from _quads import rowmajor
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

GTOL = 1e-3


def check_grad(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= GTOL * scale, (np.abs(got - ref).max(), scale)
    assert np.all(np.abs(got - ref) <= GTOL * np.maximum(np.abs(ref), 1e-2 * scale))


@pytest.mark.parametrize("H,W,r,sigma", [(64, 80, 3, 0.2), (96, 70, 7, 0.15), (40, 300, 12, 0.1),
                                         (33, 17, 2, 0.3)])
def test_grad_image_fixed_gamma(cuda_lib, H, W, r, sigma):
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=H + W)
    w = synth.weights((H, W), seed=1)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    s = torch.tensor(sigma, requires_grad=True)
    out = bf.bilateral(ft, r, s, 1.0)
    L = (torch.from_numpy(w).cuda() * out).sum()
    L.backward()
    N = oracle.resolve_N(sigma, 1.0)
    gref, _ = oracle.bilateral_grad(f.astype(np.float64), w.astype(np.float64), r, math.pi / 2, N)
    check_grad(ft.grad.cpu().numpy(), gref)
    assert s.grad is not None and float(s.grad) == 0.0  # gamma fixed: dL/dsigma = 0


@pytest.mark.parametrize("sigma,r", [(0.15, 7), (0.3, 4)])
def test_grad_sigma_from_sigma(cuda_lib, sigma, r):
    """BF_GAMMA_FROM_SIGMA: gamma = 1/(sigma sqrt N), N frozen by the rule.
    dL/dsigma against the oracle's dL/dgamma * dgamma/dsigma and against
    central differences of the oracle forward in sigma."""
    bf = cuda_lib
    H, W = 72, 88
    f = synth.rectangles(H, W, seed=7)
    w = synth.weights((H, W), seed=1)
    N = oracle.resolve_N(sigma, 1.0)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    s = torch.tensor(sigma, requires_grad=True)
    out = bf.bilateral(ft, r, s, 1.0, N=N, gamma_mode=bf.GAMMA_FROM_SIGMA)
    (torch.from_numpy(w).cuda() * out).sum().backward()
    g = oracle.gamma_from_sigma(sigma, N)
    gref, dgam = oracle.bilateral_grad(f.astype(np.float64), w.astype(np.float64), r, g, N)
    check_grad(ft.grad.cpu().numpy(), gref)
    dsig_ref = -(g / sigma) * dgam
    h = 1e-4
    Lp = np.sum(w * oracle.bilateral(f, r, oracle.gamma_from_sigma(sigma + h, N), N))
    Lm = np.sum(w * oracle.bilateral(f, r, oracle.gamma_from_sigma(sigma - h, N), N))
    fd = (Lp - Lm) / (2 * h)
    assert abs(dsig_ref - fd) <= 1e-6 * max(1.0, abs(fd))
    assert abs(float(s.grad) - dsig_ref) <= GTOL * max(1.0, abs(dsig_ref)), (float(s.grad), dsig_ref)


def test_adjoint_range_shift_invariance(cuda_lib):
    """The engine runs on f - T/2 and out - T/2 (the saved quads hold the
    shifted values). Shifting the input by a constant inside [0, T] must then
    shift out by the same constant and leave dL/df and dL/dsigma_r unchanged,
    as the oracle's pins fix; both runs are also checked against the oracle."""
    bf = cuda_lib
    H, W, r, sigma = 80, 150, 6, 0.15
    f = 0.75 * synth.rectangles(H, W, seed=31)
    w = synth.weights((H, W), seed=3)
    N = oracle.resolve_N(sigma, 1.0)
    g = oracle.gamma_from_sigma(sigma, N)
    res = []
    for c in (0.0, 0.25):
        fc = (f + np.float32(c)).astype(np.float32)
        ft = torch.from_numpy(fc).cuda().requires_grad_(True)
        s = torch.tensor(sigma, requires_grad=True)
        out = bf.bilateral(ft, r, s, 1.0, N=N, gamma_mode=bf.GAMMA_FROM_SIGMA)
        (torch.from_numpy(w).cuda() * out).sum().backward()
        gref, dgam = oracle.bilateral_grad(fc.astype(np.float64), w.astype(np.float64), r, g, N)
        check_grad(ft.grad.cpu().numpy(), gref)
        dsig = -(g / sigma) * dgam
        assert abs(float(s.grad) - dsig) <= 3e-4 * max(1.0, abs(dsig)), (c, float(s.grad), dsig)
        res.append((out.detach().cpu().numpy().astype(np.float64), ft.grad.cpu().numpy(),
                    float(s.grad)))
    (o0, g0, s0), (o1, g1, s1) = res
    assert np.abs(o1 - 0.25 - o0).max() <= 1e-4
    assert np.abs(g1 - g0).max() <= GTOL * np.abs(g0).max()
    assert abs(s1 - s0) <= 3e-4 * max(1.0, abs(s0)), (s0, s1)


@pytest.mark.parametrize("H,W,r,sigma", [(160, 230, 10, 0.1), (120, 333, 24, 0.2)])
def test_adjoint_narrow_strips(cuda_lib, H, W, r, sigma):
    """The adjoint on 64-thread strips (small images): dL/df against the
    oracle's direct-form gradient, and against explicit 128-thread strips."""
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=H + W + r)
    w = synth.weights((H, W), seed=5)
    N = oracle.resolve_N(sigma, 1.0)
    ft = torch.from_numpy(f).cuda()
    wt = torch.from_numpy(w).cuda()
    res = []
    for tw in (0, 128):
        o = bf._opts(save=True, tile_w=tw)
        sv = torch.empty((H, W, 4), device="cuda")
        out = bf.bf_forward(ft, r, sigma, 1.0, N, opts=o, saved=sv)
        gi = torch.empty_like(ft)
        bf.bf_backward(ft, out, wt, sv, r, sigma, 1.0, N, grad_img=gi, opts=o)
        torch.cuda.synchronize()
        res.append(gi.cpu().numpy())
    gref, _ = oracle.bilateral_grad(f.astype(np.float64), w.astype(np.float64), r, math.pi / 2, N)
    check_grad(res[0], gref)
    assert np.abs(res[0] - res[1]).max() <= 1e-4 * np.abs(gref).max()


def test_grad_batch_differentiation_config(cuda_lib):
    """Differentiation workload shape: a batch of 512x512 images, r=7,
    sigma_r=0.15 (N=19); image gradient checked on 2 images against the
    reference gradient of the oracle at sampled pixels via central
    differences of the oracle forward."""
    bf = cuda_lib
    B, H, W, r, sigma = 2, 512, 512, 7, 0.15
    f = np.stack([synth.rectangles(H, W, seed=100 + b) for b in range(B)])
    w = synth.weights((B, H, W), seed=1)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    out = bf.bilateral(ft, r, sigma, 1.0)
    (torch.from_numpy(w).cuda() * out).sum().backward()
    gg = ft.grad.cpu().numpy()
    N = 19
    rng = np.random.default_rng(5)
    for b in range(B):
        for _ in range(6):
            y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
            y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
            x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
            # outputs affected by f[y, x] lie within r of it; their windows within 2r
            sub = f[b, y0:y1, x0:x1].astype(np.float64)
            wsub = w[b, y0:y1, x0:x1].astype(np.float64)
            mask = np.zeros_like(sub)
            yy0, yy1 = max(0, y - r) - y0, min(H, y + r + 1) - y0
            xx0, xx1 = max(0, x - r) - x0, min(W, x + r + 1) - x0
            mask[yy0:yy1, xx0:xx1] = 1.0
            # interior outputs of the crop see the true window only if the crop
            # holds their full window: true when the crop edge is the image edge
            # or at distance >= r from them, which holds for the masked region.
            h = 1e-4
            sp = sub.copy(); sp[y - y0, x - x0] += h
            sm = sub.copy(); sm[y - y0, x - x0] -= h
            Lp = np.sum(mask * wsub * oracle.bilateral(sp, r, math.pi / 2, N))
            Lm = np.sum(mask * wsub * oracle.bilateral(sm, r, math.pi / 2, N))
            fd = (Lp - Lm) / (2 * h)
            assert abs(gg[b, y, x] - fd) <= GTOL * max(1.0, abs(fd)), (b, y, x, gg[b, y, x], fd)


def test_backward_raw_abi_grad_sigma_fixed_is_zero(cuda_lib):
    bf = cuda_lib
    H, W = 40, 50
    f = torch.from_numpy(synth.rectangles(H, W, seed=2)).cuda()
    opts = bf._opts(save=True)
    sv = torch.empty((H, W, 4), device="cuda")
    out = bf.bf_forward(f, 3, 0.2, 1.0, 0, opts=opts, saved=sv)
    g = torch.ones_like(out)
    gs = torch.full((1,), 7.0, device="cuda")
    ws = torch.empty((bf.bf_backward_workspace_bytes(H, W, 3, 0.2, 1.0, 0) // 4 + 1,), device="cuda")
    bf.bf_backward(f, out, g, sv, 3, 0.2, 1.0, 0, grad_img=None, grad_sigma=gs, workspace=ws)
    torch.cuda.synchronize()
    assert float(gs) == 0.0


@pytest.mark.parametrize("H,W,r,sigma", [(70, 90, 5, 0.085), (50, 300, 30, 0.2)])
def test_grad_chunked_and_wide(cuda_lib, H, W, r, sigma):
    """N > 43 (harmonic chunks with workspace accumulators) and r = 30
    (256-thread strips) through the autograd wrapper."""
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=H * 7 + W)
    w = synth.weights((H, W), seed=3)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    out = bf.bilateral(ft, r, sigma, 1.0)
    (torch.from_numpy(w).cuda() * out).sum().backward()
    N = oracle.resolve_N(sigma, 1.0)
    gref, _ = oracle.bilateral_grad(f.astype(np.float64), w.astype(np.float64), r, math.pi / 2, N)
    check_grad(ft.grad.cpu().numpy(), gref)


@pytest.mark.parametrize("kahan_fallback", [False, True])
def test_3d_launch_matches_per_image(cuda_lib, kahan_fallback):
    """bf_forward3d / bf_backward3d over [B, H, W] equal B single-image calls
    (skewed-strip engine with grid.z, and the per-image single-pass fallback)."""
    bf = cuda_lib
    B, H, W, r, sigma = 3, 70, 130, 6, 0.15
    f = torch.from_numpy(np.stack([synth.rectangles(H, W, seed=40 + b) for b in range(B)])).cuda()
    g = torch.from_numpy(synth.weights((B, H, W), seed=2)).cuda()
    N = oracle.resolve_N(sigma, 1.0)
    opts = bf._opts(save=not kahan_fallback, kahan=kahan_fallback, gamma_mode=bf.GAMMA_FROM_SIGMA)
    sv = torch.empty((B, H, W, 4), device="cuda")
    out3 = bf.bf_forward3d(f, r, sigma, 1.0, N, opts=opts, saved=None if kahan_fallback else sv)
    for b in range(B):
        o1 = bf.bf_forward(f[b], r, sigma, 1.0, N, opts=opts, saved=None if kahan_fallback else sv[b])
        torch.cuda.synchronize()
        assert torch.max(torch.abs(o1 - out3[b])).item() <= 1e-6
    if kahan_fallback:
        return
    bf.bf_forward3d(f, r, sigma, 1.0, N, out=out3, opts=opts, saved=sv)
    gi = torch.empty_like(f)
    gs = torch.zeros((1,), device="cuda")
    ws = torch.empty((bf.bf_backward3d_workspace_bytes(B, H, W, r, sigma, 1.0, N, opts) // 4 + 1,),
                     device="cuda")
    bf.bf_backward3d(f, out3, g, sv, r, sigma, 1.0, N, grad_img=gi, grad_sigma=gs, workspace=ws,
                     opts=opts)
    total = 0.0
    for b in range(B):
        gi1 = torch.empty_like(f[b])
        gs1 = torch.zeros((1,), device="cuda")
        ws1 = torch.empty((bf.bf_backward_workspace_bytes(H, W, r, sigma, 1.0, N, opts) // 4 + 1,),
                          device="cuda")
        bf.bf_backward(f[b], out3[b], g[b], sv[b], r, sigma, 1.0, N, grad_img=gi1, grad_sigma=gs1,
                       workspace=ws1, opts=opts)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(gi1 - gi[b])).item() <= 1e-6 * max(1.0, gi1.abs().max().item())
        total += float(gs1)
    assert abs(float(gs) - total) <= 1e-4 * max(1.0, abs(total))


@pytest.mark.parametrize("N", [41, 40])
def test_headline_adjoint_full_size_sampled(cuda_lib, N):
    """The headline workload (4096^2, r=10, sigma_r=0.1 -> N=41, and the
    metric's N=40) in the bench's launch configuration: dL/df at 12 sampled
    pixels (corners included) against FP64 central differences of the oracle
    on a crop around each."""
    bf = cuda_lib
    H = W = 4096
    r = 10
    f = synth.rectangles(H, W, seed=0)
    w = synth.weights((H, W), seed=1)
    img = torch.from_numpy(f).cuda()
    g = torch.from_numpy(w).cuda()
    opts = bf._opts(save=True)
    sv = torch.empty((H, W, 4), device="cuda")
    out = bf.bf_forward(img, r, 0.1, 1.0, N, opts=opts, saved=sv)
    gi = torch.empty_like(img)
    bf.bf_backward(img, out, g, sv, r, 0.1, 1.0, N, grad_img=gi, opts=opts)
    gg = gi.cpu().numpy()
    rng = np.random.default_rng(17 + N)
    pts = [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0)] + \
        [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(8)]
    for y, x in pts:
        y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
        x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
        sub = f[y0:y1, x0:x1].astype(np.float64)
        mask = np.zeros_like(sub)
        mask[max(0, y - r) - y0:min(H, y + r + 1) - y0, max(0, x - r) - x0:min(W, x + r + 1) - x0] = 1
        wsub = w[y0:y1, x0:x1].astype(np.float64) * mask
        h = 1e-4
        sp = sub.copy(); sp[y - y0, x - x0] += h
        sm = sub.copy(); sm[y - y0, x - x0] -= h
        fd = (np.sum(wsub * oracle.bilateral(sp, r, math.pi / 2, N)) -
              np.sum(wsub * oracle.bilateral(sm, r, math.pi / 2, N))) / (2 * h)
        assert abs(gg[y, x] - fd) <= GTOL * max(1.0, abs(fd)), (y, x, gg[y, x], fd)


@pytest.mark.parametrize("r", [57, 64])
def test_adjoint_largest_windows(cuda_lib, r):
    """The adjoint at r = 57 and at BF_R_MAX = 64 (256-thread strips) against
    the oracle's direct-form gradient on the whole image."""
    bf = cuda_lib
    H, W = 180, 300
    f = synth.sinusoids(H, W, seed=r)
    w = synth.weights((H, W), seed=2)
    img = torch.from_numpy(f).cuda()
    g = torch.from_numpy(w).cuda()
    opts = bf._opts(save=True)
    sv = torch.empty((H, W, 4), device="cuda")
    out = bf.bf_forward(img, r, 0.2, 1.0, 0, opts=opts, saved=sv)
    gi = torch.empty_like(img)
    bf.bf_backward(img, out, g, sv, r, 0.2, 1.0, 0, grad_img=gi, opts=opts)
    torch.cuda.synchronize()
    N = oracle.resolve_N(0.2, 1.0)
    ref, _ = oracle.bilateral_grad(f.astype(np.float64), w.astype(np.float64), r, math.pi / 2, N)
    got = gi.cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= GTOL * scale


@pytest.mark.parametrize("H,W,r,sigma,N", [(150, 260, 6, 0.1, 41), (120, 200, 4, 0.2, 40),
                                           (90, 140, 3, 0.3, 5), (100, 130, 5, 0.085, 50)])
def test_bf16_input_forward_and_adjoint(cuda_lib, H, W, r, sigma, N):
    """BF16-stored input through the forward with saved quads (the BF16
    first-chunk kernels, and the general ones for N > 43) and the adjoint
    (which reads only the quads): against the oracle on the BF16-decoded
    image, and the quads' f - T/2 exactly as decoded."""
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=H + N)
    w = synth.weights((H, W), seed=7)
    fb = torch.from_numpy(f).cuda().to(torch.bfloat16)
    f16 = fb.float().cpu().numpy()
    o = bf._opts(save=True, in_dtype=bf.BF16)
    sv = torch.empty((H, W, 4), device="cuda")
    out = bf.bf_forward(fb, r, sigma, 1.0, N, opts=o, saved=sv)
    gi = torch.empty((H, W), device="cuda")
    ws = torch.empty((bf.bf_backward_workspace_bytes(H, W, r, sigma, 1.0, N, o) // 4 + 1,),
                     device="cuda")
    bf.bf_backward(fb, out, torch.from_numpy(w).cuda(), sv, r, sigma, 1.0, N, grad_img=gi,
                   workspace=ws, opts=o)
    torch.cuda.synchronize()
    ref = oracle.bilateral(f16.astype(np.float64), r, math.pi / 2, N)
    got = out.cpu().numpy()
    assert (np.abs(got - ref) / np.maximum(np.abs(ref), 1e-2)).max() <= 1e-4
    np.testing.assert_array_equal(rowmajor(sv)[..., 0], f16 - np.float32(0.5))
    gref, _ = oracle.bilateral_grad(f16.astype(np.float64), w.astype(np.float64), r, math.pi / 2, N)
    check_grad(gi.cpu().numpy(), gref)
