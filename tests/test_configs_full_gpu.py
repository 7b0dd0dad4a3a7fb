"""The precision, batching and differentiation configurations at their own
sizes, in the launch configurations the benchmark times, checked on sampled
outputs the oracle computes one by one:

- precision: 8192^2 rectangles+noise, r=30, sigma_r=0.1 (N=41), FP32 with
  plain and Kahan-compensated running sums, and the BF16-stored image;
- batching: 256 uneven images (sides 64..2048, r 2..32, sigma_r 0.08..0.4)
  in one persistent launch;
- differentiation: 16 x 512^2, r=7, sigma_r=0.15 (N=19), gamma from sigma_r,
  one [B,H,W] forward and one adjoint launch, dL/dsigma_r and dL/df against
  FP64 central differences and the direct-form gradient.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
G1 = math.pi / 2


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1e-2)


def test_precision_config_8192sq(cuda_lib):
    bf = cuda_lib
    H = W = 8192
    r = 30
    f = synth.rectangles(H, W, seed=0)
    img = torch.from_numpy(f).cuda()
    N = bf.bf_resolve_N(0.1, 1.0)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.integers(0, H * W, 200), [0, W - 1, H * W - W, H * W - 1]])
    ref = oracle.bilateral_points(f.astype(np.float64), r, G1, N, idx)
    out = torch.empty_like(img)
    sv = torch.empty((H, W, 4), device="cuda")
    bf.bf_forward(img, r, 0.1, 1.0, N, out=out)
    assert rel_err(out.cpu().numpy().ravel()[idx], ref).max() <= TOL
    bf.bf_forward(img, r, 0.1, 1.0, N, out=out, opts=bf._opts(kahan=True, save=True), saved=sv)
    assert rel_err(out.cpu().numpy().ravel()[idx], ref).max() <= TOL
    del sv
    i16 = img.to(torch.bfloat16)
    f16 = i16.float().cpu().numpy()
    ref16 = oracle.bilateral_points(f16.astype(np.float64), r, G1, N, idx)
    bf.bf_forward(i16, r, 0.1, 1.0, N, out=out, opts=bf._opts(in_dtype=bf.BF16))
    assert rel_err(out.cpu().numpy().ravel()[idx], ref16).max() <= TOL


def test_batching_config_256_images(cuda_lib):
    bf = cuda_lib
    specs = synth.batch_specs(256, seed=7)
    imgs = [torch.from_numpy(synth.rectangles(s["H"], s["W"], seed=s["seed"])).cuda()
            for s in specs]
    outs = [torch.full_like(im, -7.0) for im in imgs]
    descs = bf.make_descs(imgs, outs, [s["r"] for s in specs], [s["sigma_r"] for s in specs])
    ws = torch.empty(((bf.bf_batch_workspace_bytes(descs) + 3) // 4,), device="cuda")
    bf.bf_batch(descs, ws)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    for k in range(0, 256, 8):  # every eighth image, 40 sampled pixels each
        s = specs[k]
        n = s["H"] * s["W"]
        idx = np.concatenate([rng.integers(0, n, 36), [0, s["W"] - 1, n - s["W"], n - 1]])
        ref = oracle.bilateral_points(imgs[k].cpu().numpy().astype(np.float64), s["r"], G1,
                                      oracle.resolve_N(s["sigma_r"], 1.0), idx)
        got = outs[k].cpu().numpy().ravel()[idx]
        assert rel_err(got, ref).max() <= TOL, (k, s)
    assert all(float(o.min()) > -7.0 for o in outs)  # every image written


def _loss(f, w, r, gamma, N):
    """L = sum(w * out) over a [B, H, W] batch, from the FP64 oracle."""
    return sum(float(np.sum(w[b].astype(np.float64) * oracle.bilateral(f[b], r, gamma, N)))
               for b in range(f.shape[0]))


def test_differentiation_config_16x512sq(cuda_lib):
    """16 x 512^2, r=7, sigma_r=0.15 (N=19) with gamma = 1/(sigma_r sqrt N) (the
    variance control of Sec. 3, N frozen by the rule), so dL/dsigma_r is live:
    one [B,H,W] forward and one adjoint launch, as the benchmark runs them.
    dL/dsigma_r (summed over the batch) against FP64 central differences of the
    oracle in sigma_r (h = 1e-4, N frozen) and against the oracle's direct-form
    derivative; dL/df against the direct-form gradient at every pixel and
    against FP64 central differences at 256 sampled pixels per image."""
    bf = cuda_lib
    B, H, W, r, sigma = 16, 512, 512, 7, 0.15
    N = bf.bf_resolve_N(sigma, 1.0)
    f = np.stack([synth.rectangles(H, W, seed=100 + b) for b in range(B)])
    w = synth.weights((B, H, W), seed=1)
    ft = torch.from_numpy(f).cuda()
    wt = torch.from_numpy(w).cuda()
    opts = bf._opts(save=True, gamma_mode=bf.GAMMA_FROM_SIGMA)
    sv = torch.empty((B, H, W, 4), device="cuda")
    out = bf.bf_forward3d(ft, r, sigma, 1.0, N, opts=opts, saved=sv)
    gi = torch.empty_like(ft)
    gs = torch.zeros((1,), device="cuda")
    ws = torch.empty((bf.bf_backward3d_workspace_bytes(B, H, W, r, sigma, 1.0, N, opts) // 4 + 1,),
                     device="cuda")
    bf.bf_backward3d(ft, out, wt, sv, r, sigma, 1.0, N, grad_img=gi, grad_sigma=gs, workspace=ws,
                     opts=opts)
    torch.cuda.synchronize()
    gamma = oracle.gamma_from_sigma(sigma, N)
    o = out.cpu().numpy()
    gg = gi.cpu().numpy()
    f64 = f.astype(np.float64)
    # forward on sampled pixels and dL/df on every pixel (direct form)
    rng = np.random.default_rng(13)
    dgamma = 0.0
    for b in range(B):
        idx = rng.integers(0, H * W, 64)
        ref = oracle.bilateral_points(f64[b], r, gamma, N, idx)
        assert rel_err(o[b].ravel()[idx], ref).max() <= TOL
        gref, dg = oracle.bilateral_grad(f64[b], w[b].astype(np.float64), r, gamma, N)
        dgamma += dg
        assert np.abs(gg[b] - gref).max() <= 1e-3 * np.abs(gref).max(), b
    # dL/dsigma_r: gamma = 1/(sigma sqrt N), so dL/dsigma = -(gamma / sigma) dL/dgamma
    dsig_direct = -(gamma / sigma) * dgamma
    h = 1e-4
    fd = (_loss(f64, w, r, oracle.gamma_from_sigma(sigma + h, N), N) -
          _loss(f64, w, r, oracle.gamma_from_sigma(sigma - h, N), N)) / (2 * h)
    assert abs(dsig_direct - fd) <= 1e-5 * max(1.0, abs(fd)), (dsig_direct, fd)
    # the gradient bar (1e-3); measured 5.6e-4 with the 171-row bands of one
    # wave over the batch (1.0e-4 with 32-row bands: the running sums' rounding
    # drifts with the band height)
    assert abs(float(gs) - fd) <= 1e-3 * max(1.0, abs(fd)), (float(gs), fd)
    # dL/df: FP64 central differences at 256 pixels of each image, on a crop
    for b in range(B):
        for _ in range(256):
            y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
            y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
            x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
            sub = f64[b, y0:y1, x0:x1]
            mask = np.zeros_like(sub)
            mask[max(0, y - r) - y0:min(H, y + r + 1) - y0,
                 max(0, x - r) - x0:min(W, x + r + 1) - x0] = 1
            wsub = w[b, y0:y1, x0:x1].astype(np.float64) * mask
            sp = sub.copy(); sp[y - y0, x - x0] += h
            sm = sub.copy(); sm[y - y0, x - x0] -= h
            fdf = (np.sum(wsub * oracle.bilateral(sp, r, gamma, N)) -
                   np.sum(wsub * oracle.bilateral(sm, r, gamma, N))) / (2 * h)
            assert abs(gg[b, y, x] - fdf) <= 1e-3 * max(1.0, abs(fdf)), (b, y, x, gg[b, y, x], fdf)
