"""Persistent batched filter: uneven images, each with its own r, sigma_r and
N, in one launch (and replayed from a CUDA graph), checked against the
single-image launch and the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu


def make_batch(bf, n, seed, side_hi=300):
    specs = synth.batch_specs(n, seed=seed, side_lo=1, side_hi=side_hi)
    imgs = [torch.from_numpy(synth.rectangles(s["H"], s["W"], seed=s["seed"])).cuda() for s in specs]
    outs = [torch.full_like(im, -7.0) for im in imgs]
    descs = bf.make_descs(imgs, outs, [s["r"] for s in specs], [s["sigma_r"] for s in specs])
    return specs, imgs, outs, descs


def test_batch_matches_single_and_oracle(cuda_lib):
    bf = cuda_lib
    specs, imgs, outs, descs = make_batch(bf, 24, seed=3)
    ws = torch.empty((bf.bf_batch_workspace_bytes(descs) // 4 + 1,), dtype=torch.float32,
                     device="cuda")
    bf.bf_batch(descs, ws)
    torch.cuda.synchronize()
    for s, im, o in zip(specs, imgs, outs):
        hb = max(128, 4 * s["r"])
        single = bf.bf_forward(im, s["r"], s["sigma_r"], 1.0, 0, opts=bf._opts(tile_h=hb))
        torch.cuda.synchronize()
        # same filter, possibly a different tile engine: agree to FP32 rounding
        assert torch.max(torch.abs(single - o)).item() <= 1e-5
        N = oracle.resolve_N(s["sigma_r"], 1.0)
        ref = oracle.bilateral(im.cpu().numpy().astype(np.float64), s["r"], math.pi / 2, N)
        e = np.abs(o.cpu().numpy() - ref) / np.maximum(np.abs(ref), 1e-2)
        assert e.max() <= 1e-4, (s, e.max())


def test_batch_graph_replay(cuda_lib):
    bf = cuda_lib
    specs, imgs, outs, descs = make_batch(bf, 16, seed=4, side_hi=200)
    ws = torch.empty((bf.bf_batch_workspace_bytes(descs) // 4 + 1,), dtype=torch.float32,
                     device="cuda")
    opts = bf._opts()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bf.bf_batch_prepare(descs, ws, opts, stream=s)
        bf.bf_batch_launch(ws, opts, stream=s)  # warm-up (sets kernel attributes)
    s.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bf.bf_batch_launch(ws, opts, stream=s)
    for _ in range(2):
        for o in outs:
            o.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(first, outs):
            assert torch.equal(a, b)


def test_batch_validation_rejects_bad_descriptor(cuda_lib):
    bf = cuda_lib
    specs, imgs, outs, descs = make_batch(bf, 4, seed=5, side_hi=64)
    descs[2].T = 0.0
    ws = torch.empty((bf.bf_batch_workspace_bytes(descs) // 4 + 1,), device="cuda")
    with pytest.raises(bf.BfError):
        bf.bf_batch(descs, ws)
    descs[2].T = 1.0
    small = torch.empty((4,), device="cuda")
    with pytest.raises(bf.BfError):
        bf.bf_batch(descs, small)


def test_batch_kahan_and_bf16(cuda_lib):
    """Kahan-compensated batch (single-pass kernel queue) and a BF16-input
    batch (skewed-strip engine) against the oracle."""
    bf = cuda_lib
    specs = synth.batch_specs(6, seed=9, side_lo=20, side_hi=160)
    for opts, dt in [(bf._opts(kahan=True), torch.float32), (bf._opts(in_dtype=bf.BF16), torch.bfloat16)]:
        imgs = [torch.from_numpy(synth.rectangles(s["H"], s["W"], seed=s["seed"])).cuda().to(dt)
                for s in specs]
        outs = [torch.full(im.shape, -7.0, device="cuda") for im in imgs]
        descs = bf.make_descs(imgs, outs, [s["r"] for s in specs], [s["sigma_r"] for s in specs])
        ws = torch.empty((bf.bf_batch_workspace_bytes(descs, opts) // 4 + 1,), device="cuda")
        bf.bf_batch(descs, ws, opts)
        torch.cuda.synchronize()
        for s, im, o in zip(specs, imgs, outs):
            N = oracle.resolve_N(s["sigma_r"], 1.0)
            ref = oracle.bilateral(im.float().cpu().numpy().astype(np.float64), s["r"], math.pi / 2, N)
            e = np.abs(o.cpu().numpy() - ref) / np.maximum(np.abs(ref), 1e-2)
            assert e.max() <= 1e-4, (s, e.max())


def test_batch_launch_needs_a_prepared_table(cuda_lib):
    """A table whose tag was overwritten launches no work (outputs keep their
    sentinel); preparing it again restores the filter."""
    bf = cuda_lib
    specs = synth.batch_specs(6, seed=13, side_lo=40, side_hi=300)
    imgs = [torch.from_numpy(synth.rectangles(s["H"], s["W"], seed=s["seed"])).cuda()
            for s in specs]
    outs = [torch.full_like(im, -7.0) for im in imgs]
    descs = bf.make_descs(imgs, outs, [s["r"] for s in specs], [s["sigma_r"] for s in specs])
    opts = bf._opts()
    ws = torch.empty(((bf.bf_batch_workspace_bytes(descs, opts) + 3) // 4,), device="cuda")
    bf.bf_batch_prepare(descs, ws, opts)
    ws.view(torch.int32)[4] = 0  # the tag follows the four work counters
    bf.bf_batch_launch(ws, opts)
    torch.cuda.synchronize()
    assert all(bool(torch.all(o == -7.0)) for o in outs)
    bf.bf_batch_prepare(descs, ws, opts)
    bf.bf_batch_launch(ws, opts)
    torch.cuda.synchronize()
    for s, im, o in zip(specs, imgs, outs):
        ref = bf.bf_forward(im, s["r"], s["sigma_r"])
        assert torch.max(torch.abs(o - ref)).item() <= 2e-4


@pytest.mark.parametrize("H,W,r,N", [(300, 410, 10, 41), (96, 128, 4, 50), (700, 900, 45, 11)])
def test_step_graph_replay(cuda_lib, H, W, r, N):
    """The forward with saved quads and the adjoint (dL/df and dL/dsigma_r)
    captured into one CUDA graph and replayed equal the eager calls bit for
    bit: one harmonic chunk, two chunks with their workspace accumulators,
    and 256-thread strips."""
    bf = cuda_lib
    f = torch.from_numpy(synth.rectangles(H, W, seed=H)).cuda()
    g = torch.from_numpy(synth.weights((H, W), seed=2)).cuda()
    sigma = 0.15
    opts = bf._opts(save=True, gamma_mode=bf.GAMMA_FROM_SIGMA)
    out = torch.empty_like(f)
    sv = torch.empty((H, W, 4), device="cuda")
    gi = torch.empty_like(f)
    gs = torch.zeros((1,), device="cuda")
    ws = torch.empty((bf.bf_backward_workspace_bytes(H, W, r, sigma, 1.0, N, opts) // 4 + 1,),
                     device="cuda")
    s = torch.cuda.Stream()

    def step():
        bf.bf_forward(f, r, sigma, 1.0, N, out=out, opts=opts, saved=sv, stream=s)
        bf.bf_backward(f, out, g, sv, r, sigma, 1.0, N, grad_img=gi, grad_sigma=gs,
                       workspace=ws, opts=opts, stream=s)
    with torch.cuda.stream(s):
        step()  # eager (also sets the kernels' attributes)
    s.synchronize()
    ref = (out.clone(), gi.clone(), gs.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step()
    for _ in range(2):
        out.fill_(-1.0); gi.fill_(-1.0); gs.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref[0]) and torch.equal(gi, ref[1]) and torch.equal(gs, ref[2])
