"""GPU parity of bf_spatial_forward (Algorithm 2 with a shiftable spatial
kernel q_M x q_M, and Algorithm 1 without a range kernel) against the
oracle's direct O(r^2) definition, element by element. Same tolerance as the
box filter: |gpu - oracle| / max(|oracle|, 1e-2) <= 1e-4."""
import math

import numpy as np
import pytest
import torch

import oracle
from _quads import rowmajor
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
G1 = math.pi / 2


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1e-2)


def run(bf, f, r, M, N, guard=0):
    H, W = f.shape
    buf = torch.full((H * W + 2 * guard,), -5.0, device="cuda")
    out = buf[guard:guard + H * W].view(H, W)
    bf.bf_spatial_forward(torch.from_numpy(np.ascontiguousarray(f)).cuda(), r, M, 0.0, 1.0, N,
                          out=out)
    torch.cuda.synchronize()
    if guard:
        b = buf.cpu().numpy()
        assert np.all(b[:guard] == -5.0) and np.all(b[guard + H * W:] == -5.0)
    return out.cpu().numpy()


def ref(f, r, M, N):
    return oracle.bilateral_general(f.astype(np.float64), r, spatial=oracle.SPATIAL_QM, M=M,
                                    range_kind=oracle.RANGE_COSN if N else oracle.RANGE_NONE,
                                    gamma=G1, N=N)


def test_paper_timing_workload_512sq(cuda_lib):
    """The paper's timing instance (Sec. 2): 512 x 512, T = 5 (r = 5),
    M x N = 3^2 x 5 basis functions, i.e. q_2 x q_2 spatial and q_4 range."""
    f = synth.rectangles(512, 512, seed=0)
    got = run(cuda_lib, f, 5, 2, 4, guard=1024)
    assert rel_err(got, ref(f, 5, 2, 4)).max() <= TOL


@pytest.mark.parametrize("M,N", [(1, 1), (1, 2), (1, 3), (1, 4), (2, 1), (2, 2), (2, 3), (2, 4)])
def test_algorithm2_orders(cuda_lib, M, N):
    f = synth.rectangles(150, 233, seed=10 * M + N)
    got = run(cuda_lib, f, 4, M, N)
    assert rel_err(got, ref(f, 4, M, N)).max() <= TOL


@pytest.mark.parametrize("M", [1, 2, 3, 4, 6, 8])
def test_algorithm1_linear_filter(cuda_lib, M):
    f = synth.sinusoids(130, 270, seed=M)
    got = run(cuda_lib, f, 9, M, 0)
    assert rel_err(got, ref(f, 9, M, 0)).max() <= TOL


@pytest.mark.parametrize("H,W,r", [(1, 1, 3), (1, 200, 4), (200, 1, 2), (7, 5, 20), (300, 333, 0),
                                   (97, 500, 30), (260, 140, 56)])
def test_edges_and_ragged_tiles(cuda_lib, H, W, r):
    f = synth.rectangles(H, W, seed=H + W + r)
    got = run(cuda_lib, f, r, 2, 4)
    assert rel_err(got, ref(f, r, 2, 4)).max() <= TOL


@pytest.mark.parametrize("M,N,r", [(8, 0, 1), (6, 0, 1), (8, 0, 2), (4, 0, 0), (2, 4, 0),
                                   (2, 4, 1), (1, 3, 1)])
def test_short_phase_period(cuda_lib, M, N, r):
    """Small windows, whose phase period 2 (2r + 1) can be shorter than the
    spatial harmonic b. r = 0: a 1 x 1 window weighs the centre alone, so out =
    f, the saved quad is (f, 1, f, 0) and the adjoint returns dL/dout. 130
    rows, so the saved quads are sheared."""
    bf = cuda_lib
    f = synth.sinusoids(130, 300, seed=M + r)
    ft = torch.from_numpy(f).cuda()
    sv = torch.empty((130, 300, 4), device="cuda")
    got = bf.bf_spatial_forward(ft, r, M, 0.0, 1.0, N, saved=sv)
    torch.cuda.synchronize()
    want = ref(f, r, M, N)
    assert rel_err(got.cpu().numpy(), want).max() <= TOL
    s = rowmajor(sv)
    assert np.array_equal(s[..., 0], f) and np.allclose(s[..., 2], got.cpu().numpy())
    if r == 0:
        assert np.array_equal(got.cpu().numpy(), f)
        assert np.array_equal(s, np.stack([f, np.ones_like(f), f, np.zeros_like(f)], -1))
        g = torch.from_numpy(synth.weights((130, 300), seed=3)).cuda()
        gi = bf.bf_spatial_backward(g, sv, r, M, 0.0, 1.0, N)
        torch.cuda.synchronize()
        assert torch.equal(gi, g)


def test_rejects_unbuilt_orders(cuda_lib):
    bf = cuda_lib
    f = torch.zeros((8, 8), device="cuda")
    for M, N in [(3, 2), (5, 0), (2, 6), (0, 4)]:
        with pytest.raises(bf.BfError):
            bf.bf_spatial_forward(f, 2, M, 0.0, 1.0, N)
    with pytest.raises(bf.BfError):
        bf.bf_spatial_forward(f, 57, 2, 0.0, 1.0, 4)


def fd_grad(f, w, r, M, N, y, x, h=1e-4):
    """Central difference of L = sum(w * out) in f[y, x] on the FP64 oracle,
    re-evaluating only the outputs within r of (y, x) (on a crop holding their
    windows)."""
    H, W = f.shape
    y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
    x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
    sub = f[y0:y1, x0:x1].astype(np.float64)
    mask = np.zeros_like(sub)
    mask[max(0, y - r) - y0:min(H, y + r + 1) - y0, max(0, x - r) - x0:min(W, x + r + 1) - x0] = 1
    wsub = w[y0:y1, x0:x1].astype(np.float64) * mask
    sp = sub.copy(); sp[y - y0, x - x0] += h
    sm = sub.copy(); sm[y - y0, x - x0] -= h
    return (np.sum(wsub * ref(sp, r, M, N)) - np.sum(wsub * ref(sm, r, M, N))) / (2 * h)


@pytest.mark.parametrize("H,W,r,M,N", [(64, 90, 3, 2, 4), (80, 70, 5, 1, 3), (50, 140, 4, 2, 0),
                                       (33, 41, 2, 4, 0), (96, 200, 5, 2, 2), (150, 170, 4, 2, 4)])
def test_spatial_adjoint_vs_central_differences(cuda_lib, H, W, r, M, N):
    """dL/df of Algorithm 2 with the spatial kernel (and of Algorithm 1 for
    N = 0), through the autograd wrapper, against FP64 central differences
    of the oracle at sampled pixels: |gpu - fd| <= 1e-3 max(1, |fd|)."""
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=H + M + N)
    w = synth.weights((H, W), seed=1)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    out = bf.bilateral_spatial(ft, r, M, 0.0, 1.0, N)
    assert rel_err(out.detach().cpu().numpy(), ref(f, r, M, N)).max() <= TOL
    (torch.from_numpy(w).cuda() * out).sum().backward()
    gg = ft.grad.cpu().numpy()
    rng = np.random.default_rng(H * W + r)
    pts = [(0, 0), (H - 1, W - 1)] + [(int(rng.integers(0, H)), int(rng.integers(0, W)))
                                      for _ in range(8)]
    for y, x in pts:
        fd = fd_grad(f, w, r, M, N, y, x)
        assert abs(gg[y, x] - fd) <= 1e-3 * max(1.0, abs(fd)), (y, x, gg[y, x], fd)


def test_spatial_saved_quads(cuda_lib):
    """The forward's saved quads: f and out exactly as read and written, 1/den
    equal to the oracle's normaliser's reciprocal. 150 rows: pixel (y, x)'s
    quad sits at ((y + (x mod 128)) mod H) W + x."""
    bf = cuda_lib
    f = synth.rectangles(150, 90, seed=4)
    sv = torch.empty((150, 90, 4), device="cuda")
    out = bf.bf_spatial_forward(torch.from_numpy(f).cuda(), 3, 2, 0.0, 1.0, 4, saved=sv)
    q = rowmajor(sv)
    got = out.cpu().numpy()
    r_, den = oracle.bilateral_general(f.astype(np.float64), 3, spatial=oracle.SPATIAL_QM, M=2,
                                       range_kind=oracle.RANGE_COSN, gamma=G1, N=4,
                                       return_den=True)
    np.testing.assert_array_equal(q[..., 0], f)
    np.testing.assert_array_equal(q[..., 2], got)
    np.testing.assert_allclose(1.0 / q[..., 1], den, rtol=2e-5, atol=0)


def test_batched_autograd_matches_per_image(cuda_lib):
    """bilateral_spatial on [B, H, W]: each image's output and dL/df equal those
    of the image on its own (the same kernels on the same data)."""
    bf = cuda_lib
    fs = np.stack([synth.rectangles(90, 140, seed=30 + b) for b in range(3)])
    w = torch.from_numpy(synth.weights((3, 90, 140), seed=4)).cuda()
    ft = torch.from_numpy(fs).cuda().requires_grad_(True)
    out = bf.bilateral_spatial(ft, 4, 2, 0.0, 1.0, 4)
    (w * out).sum().backward()
    for b in range(3):
        fb = torch.from_numpy(fs[b]).cuda().requires_grad_(True)
        ob = bf.bilateral_spatial(fb, 4, 2, 0.0, 1.0, 4)
        (w[b] * ob).sum().backward()
        assert torch.equal(out[b].detach(), ob.detach())
        assert torch.equal(ft.grad[b], fb.grad)
