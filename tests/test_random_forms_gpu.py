"""Seeded random cases of the other forms, each against the oracle:

- batches of 1..10 uneven images (sizes 1..300, r 0..64, N by the order rule
  or given up to 64, row-pitched images, the optional den output, FP32 or
  BF16 input), the three persistent launch groups mixed in one batch, with the
  built-in band height or a given one;
- Kahan-compensated forward, with and without saved quads (the engine's
  chunked pass and the single-pass kernel);
- gamma from sigma_r: dL/dsigma_r against the oracle's direct form;
- the variant filters (shiftable spatial kernel, Algorithm 1, p_N, truncated
  q_N) against the oracle's general direct form;
- explicit launch shapes (strip widths, band heights) and the Kahan batch.
The cases are drawn from fixed seeds, so every run checks the same ones."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
SENT = -7.0


def _rel(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1e-2)


def _batches(n=8, seed=41):
    g = np.random.default_rng(seed)
    out = []
    for k in range(n):
        imgs = []
        for _ in range(int(g.integers(1, 11))):
            H = int(g.choice([1, 5, 40, 97, 160, 257, 300]))
            W = int(g.choice([1, 7, 64, 130, 211, 300]))
            r = int(g.choice([0, 1, 3, 8, 20, 33, 41, 50, 64]))
            sigma = float(g.uniform(0.08, 0.4))
            N = int(g.choice([0, 0, 0, 2, 9, 40, 47, 64]))
            pad = int(g.choice([0, 0, 3]))
            den = bool(g.random() < 0.5)
            imgs.append((H, W, r, sigma, N, pad, den))
        bf16 = bool(g.random() < 0.3)
        tile_h = int(g.choice([0, 0, 64, 256]))
        out.append((k, bf16, tile_h, imgs))
    return out


@pytest.mark.parametrize("case", _batches(), ids=lambda c: "batch%d" % c[0])
def test_random_batch(cuda_lib, case):
    bf = cuda_lib
    k, bf16, tile_h, specs = case
    dt = torch.bfloat16 if bf16 else torch.float32
    imgs, outs, dens, bigs, fds = [], [], [], [], []
    for i, (H, W, r, sigma, N, pad, den) in enumerate(specs):
        f = synth.rectangles(H, W, seed=100 * k + i)
        P = W + pad
        big = torch.zeros((H, P), dtype=dt, device="cuda")
        big[:, :W] = torch.from_numpy(f).to(dt)
        fds.append(big[:, :W].float().cpu().numpy().astype(np.float64))
        ob = torch.full((H, P), SENT, device="cuda")
        db = torch.full((H, P), SENT, device="cuda") if den else None
        imgs.append(big[:, :W])
        outs.append(ob[:, :W])
        dens.append(db[:, :W] if den else None)
        bigs.append((ob, db, W))
    o = bf._opts(in_dtype=bf.BF16 if bf16 else bf.F32, tile_h=tile_h)
    descs = bf.make_descs(imgs, outs, [s[2] for s in specs], [s[3] for s in specs],
                          Ns=[s[4] for s in specs], dens=dens)
    ws = torch.empty(((bf.bf_batch_workspace_bytes(descs, o) + 3) // 4,), device="cuda")
    bf.bf_batch(descs, ws, opts=o)
    torch.cuda.synchronize()
    for i, (H, W, r, sigma, N, pad, den) in enumerate(specs):
        Nr = N if N > 0 else oracle.resolve_N(sigma, 1.0)
        ref, rden = oracle.bilateral(fds[i], r, math.pi / 2, Nr, return_den=True)
        got = outs[i].cpu().numpy()
        assert _rel(got, ref).max() <= TOL, (k, i, specs[i])
        ob, db, _ = bigs[i]
        assert np.all(ob[:, W:].cpu().numpy() == SENT), (k, i, "padding written")
        if den:
            np.testing.assert_allclose(dens[i].cpu().numpy(), rden, rtol=2e-5, atol=1e-6)
            assert np.all(db[:, W:].cpu().numpy() == SENT), (k, i, "den padding written")


def _kahan_cases(n=8, seed=43):
    g = np.random.default_rng(seed)
    return [(i, int(g.choice([1, 33, 150, 260])), int(g.choice([2, 45, 129, 300])),
             int(g.choice([0, 1, 4, 12, 30, 64])), int(g.choice([3, 11, 24, 41, 64])),
             bool(g.random() < 0.5), bool(g.random() < 0.3)) for i in range(n)]


@pytest.mark.parametrize("case", _kahan_cases(), ids=lambda c: "kahan%d" % c[0])
def test_random_kahan(cuda_lib, case):
    bf = cuda_lib
    i, H, W, r, N, saved, bf16 = case
    f = synth.rectangles(H, W, seed=7000 + i)
    dt = torch.bfloat16 if bf16 else torch.float32
    img = torch.from_numpy(f).cuda().to(dt)
    fd = img.float().cpu().numpy().astype(np.float64)
    o = bf._opts(kahan=True, save=saved, in_dtype=bf.BF16 if bf16 else bf.F32)
    sv = torch.empty((H, W, 4), device="cuda") if saved else None
    out = bf.bf_forward(img, r, 0.2, 1.0, N, opts=o, saved=sv)
    torch.cuda.synchronize()
    ref = oracle.bilateral(fd, r, math.pi / 2, N)
    assert _rel(out.cpu().numpy(), ref).max() <= TOL, case


def _sigma_cases(n=6, seed=47):
    g = np.random.default_rng(seed)
    return [(i, int(g.choice([20, 64, 130])), int(g.choice([17, 90, 200])),
             int(g.choice([1, 3, 9, 24])), float(g.uniform(0.09, 0.35)), int(g.choice([1, 2])))
            for i in range(n)]


@pytest.mark.parametrize("case", _sigma_cases(), ids=lambda c: "sigma%d" % c[0])
def test_random_sigma_gradient(cuda_lib, case):
    bf = cuda_lib
    i, H, W, r, sigma, B = case
    N = oracle.resolve_N(sigma, 1.0)
    f = np.stack([synth.rectangles(H, W, seed=8000 + 10 * i + b) for b in range(B)])
    w = synth.weights((B, H, W), seed=i)
    ft = torch.from_numpy(f).cuda()
    opts = bf._opts(save=True, gamma_mode=bf.GAMMA_FROM_SIGMA)
    sv = torch.empty((B, H, W, 4), device="cuda")
    out = bf.bf_forward3d(ft, r, sigma, 1.0, N, opts=opts, saved=sv)
    gs = torch.zeros((1,), device="cuda")
    gi = torch.empty_like(ft)
    ws = torch.empty((bf.bf_backward3d_workspace_bytes(B, H, W, r, sigma, 1.0, N, opts) // 4 + 1,),
                     device="cuda")
    bf.bf_backward3d(ft, out, torch.from_numpy(w).cuda(), sv, r, sigma, 1.0, N, grad_img=gi,
                     grad_sigma=gs, workspace=ws, opts=opts)
    torch.cuda.synchronize()
    gamma = oracle.gamma_from_sigma(sigma, N)
    dg = sum(oracle.bilateral_grad(f[b].astype(np.float64), w[b].astype(np.float64), r, gamma,
                                   N)[1] for b in range(B))
    ref = -(gamma / sigma) * dg
    assert abs(float(gs) - ref) <= 1e-3 * max(1.0, abs(ref)), (case, float(gs), ref)


def _variant_cases(n=16, seed=53):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = ["spatial", "alg1", "poly", "trunc"][i % 4]
        H = int(g.choice([1, 9, 64, 131, 200]))
        W = int(g.choice([2, 33, 100, 170, 256]))
        r = int(g.choice([0, 1, 4, 11, 25, 40, 56]))
        if kind == "spatial":
            M, N = int(g.choice([1, 2])), int(g.choice([1, 2, 3, 4]))
        elif kind == "alg1":
            M, N = int(g.choice([1, 2, 3, 4, 6, 8])), 0
        elif kind == "poly":
            M, N = 0, int(g.choice([1, 2, 4, 6, 8]))
        else:
            M, N = int(g.choice([0, 1, 2])), int(g.choice([11, 19, 41, 64]))   # M: tolerance index
        out.append((i, kind, H, W, r, M, N))
    return out


@pytest.mark.parametrize("case", _variant_cases(), ids=lambda c: "%s%d" % (c[1], c[0]))
def test_random_variant(cuda_lib, case):
    """The variant filters (shiftable spatial kernel q_M x q_M with q_N,
    Algorithm 1, p_N, truncated q_N) on random shapes against the oracle's
    general direct form."""
    bf = cuda_lib
    i, kind, H, W, r, M, N = case
    f = synth.rectangles(H, W, seed=9000 + i)
    ft = torch.from_numpy(f).cuda()
    f64 = f.astype(np.float64)
    if kind in ("spatial", "alg1"):
        got = bf.bf_spatial_forward(ft, r, M, 0.0, 1.0, N)
        ref = oracle.bilateral_general(f64, r, spatial=oracle.SPATIAL_QM, M=M,
                                       range_kind=oracle.RANGE_COSN if N else oracle.RANGE_NONE,
                                       gamma=math.pi / 2, N=N)
    elif kind == "poly":
        got = bf.bf_poly_forward(ft, r, 0.0, 1.0, N)
        ref = oracle.bilateral_general(f64, r, range_kind=oracle.RANGE_POLY, N=N)
    else:
        tol = [1e-6, 1e-3, 1e-2][M]
        K = bf.bf_trunc_harmonics(N, r, tol)
        got = bf.bf_forward(ft, r, 0.0, 1.0, N, opts=bf._opts(trunc_tol=tol))
        ref = oracle.bilateral_general(f64, r, range_kind=oracle.RANGE_TRUNC, gamma=math.pi / 2,
                                       N=N, K_keep=K)
    torch.cuda.synchronize()
    assert _rel(got.cpu().numpy(), ref).max() <= TOL, case


def _shape_cases(n=12, seed=59):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        tw = int(g.choice([64, 96, 128, 160, 224, 256]))
        r = int(g.integers(0, min((tw - 16) // 2, 64) + 1))   # r <= BF_R_MAX
        out.append((i, int(g.choice([5, 60, 150, 233])), int(g.choice([9, 100, 190, 300])), r,
                    int(g.choice([4, 11, 25, 41, 52])), tw, int(g.choice([16, 32, 77, 300]))))
    return out


@pytest.mark.parametrize("case", _shape_cases(), ids=lambda c: "shape%d" % c[0])
def test_random_launch_shapes(cuda_lib, case):
    """Explicit strip widths (multiples of 32 up to 256, the tuner's knobs)
    and band heights: forward with saved quads and the adjoint against the
    oracle."""
    bf = cuda_lib
    i, H, W, r, N, tw, th = case
    f = synth.rectangles(H, W, seed=9500 + i)
    w = synth.weights((H, W), seed=i)
    ft = torch.from_numpy(f).cuda()
    o = bf._opts(save=True, tile_w=tw, tile_h=th)
    sv = torch.empty((H, W, 4), device="cuda")
    out = bf.bf_forward(ft, r, 0.0, 1.0, N, opts=o, saved=sv)
    gi = torch.empty_like(ft)
    ws = torch.empty((bf.bf_backward_workspace_bytes(H, W, r, 0.0, 1.0, N, o) // 4 + 1,),
                     device="cuda")
    bf.bf_backward(ft, out, torch.from_numpy(w).cuda(), sv, r, 0.0, 1.0, N, grad_img=gi,
                   workspace=ws, opts=o)
    torch.cuda.synchronize()
    f64 = f.astype(np.float64)
    assert _rel(out.cpu().numpy(), oracle.bilateral(f64, r, math.pi / 2, N)).max() <= TOL, case
    gref, _ = oracle.bilateral_grad(f64, w.astype(np.float64), r, math.pi / 2, N)
    assert np.abs(gi.cpu().numpy() - gref).max() <= 1e-3 * np.abs(gref).max(), case


@pytest.mark.parametrize("seed", [61, 67])
def test_random_kahan_batch(cuda_lib, seed):
    """The Kahan batch (single-pass kernel over a tile queue) on random uneven
    images against the oracle."""
    bf = cuda_lib
    g = np.random.default_rng(seed)
    specs = [(int(g.choice([1, 30, 120, 200])), int(g.choice([3, 64, 150, 280])),
              int(g.choice([0, 2, 7, 20])), float(g.uniform(0.08, 0.4))) for _ in range(6)]
    imgs = [torch.from_numpy(synth.rectangles(H, W, seed=seed + k)).cuda()
            for k, (H, W, r, s) in enumerate(specs)]
    outs = [torch.full_like(im, SENT) for im in imgs]
    descs = bf.make_descs(imgs, outs, [s[2] for s in specs], [s[3] for s in specs])
    o = bf._opts(kahan=True)
    ws = torch.empty(((bf.bf_batch_workspace_bytes(descs, o) + 3) // 4,), device="cuda")
    bf.bf_batch(descs, ws, opts=o)
    torch.cuda.synchronize()
    for k, (H, W, r, s) in enumerate(specs):
        ref = oracle.bilateral(imgs[k].cpu().numpy().astype(np.float64), r, math.pi / 2,
                               oracle.resolve_N(s, 1.0))
        assert _rel(outs[k].cpu().numpy(), ref).max() <= TOL, (seed, k, specs[k])
