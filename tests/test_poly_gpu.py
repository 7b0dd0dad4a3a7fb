"""GPU parity of bf_poly_forward (polynomial range kernel p_N of Sec. 3,
box window) against the oracle's direct definition, element by element:
|gpu - oracle| / max(|oracle|, 1e-2) <= 1e-4."""
import numpy as np
import pytest
import torch

import oracle
from _quads import rowmajor
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1e-2)


def run(bf, f, r, N, T=1.0):
    out = bf.bf_poly_forward(torch.from_numpy(np.ascontiguousarray(f)).cuda(), r, 0.0, T, N)
    return out.cpu().numpy()


def ref(f, r, N, T=1.0):
    return oracle.bilateral_general(f.astype(np.float64), r, range_kind=oracle.RANGE_POLY, N=N,
                                    Tr=T)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_poly_orders(cuda_lib, N):
    f = synth.rectangles(200, 250, seed=N)
    assert rel_err(run(cuda_lib, f, 5, N), ref(f, 5, N)).max() <= TOL


@pytest.mark.parametrize("H,W,r,N", [(1, 1, 2, 6), (1, 300, 3, 6), (300, 1, 3, 6), (512, 512, 10, 6),
                                     (97, 333, 30, 8), (140, 260, 56, 4), (64, 64, 0, 6)])
def test_poly_shapes_and_windows(cuda_lib, H, W, r, N):
    f = synth.sinusoids(H, W, seed=H + W)
    assert rel_err(run(cuda_lib, f, r, N), ref(f, r, N)).max() <= TOL


def test_poly_range_bound_T(cuda_lib):
    """Values in [0, T] with T = 2: the kernel is p_N(t) = (1 - t^2/4)^N."""
    f = 2.0 * synth.rectangles(150, 180, seed=3)
    assert rel_err(run(cuda_lib, f, 6, 5, T=2.0), ref(f, 6, 5, T=2.0)).max() <= TOL


def test_poly_order_from_sigma(cuda_lib):
    bf = cuda_lib
    f = torch.from_numpy(synth.rectangles(64, 80, seed=1)).cuda()
    a = bf.bf_poly_forward(f, 4, 0.3, 1.0, 0)
    b = bf.bf_poly_forward(f, 4, 0.0, 1.0, bf.bf_poly_resolve_N(0.3, 1.0))
    assert torch.equal(a, b)
    with pytest.raises(bf.BfError):
        bf.bf_poly_forward(f, 4, 0.0, 1.0, 9)


@pytest.mark.parametrize("H,W,r,N,T", [(60, 80, 3, 3, 1.0), (70, 90, 5, 6, 1.0), (50, 140, 4, 8, 1.0),
                                       (64, 64, 6, 5, 2.0), (150, 170, 5, 6, 1.0)])
def test_poly_adjoint_vs_central_differences(cuda_lib, H, W, r, N, T):
    """dL/df of the p_N filter through the autograd wrapper against FP64
    central differences of the oracle at sampled pixels (within 1e-3)."""
    bf = cuda_lib
    f = T * synth.rectangles(H, W, seed=H + N)
    w = synth.weights((H, W), seed=1)
    ft = torch.from_numpy(f.astype(np.float32)).cuda().requires_grad_(True)
    out = bf.bilateral_poly(ft, r, 0.0, T, N)
    assert rel_err(out.detach().cpu().numpy(), ref(f, r, N, T)).max() <= TOL
    (torch.from_numpy(w).cuda() * out).sum().backward()
    gg = ft.grad.cpu().numpy()
    rng = np.random.default_rng(H * W + r)
    f64 = f.astype(np.float32).astype(np.float64)
    pts = [(0, 0), (H - 1, W - 1)] + [(int(rng.integers(0, H)), int(rng.integers(0, W)))
                                      for _ in range(8)]
    for y, x in pts:
        y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
        x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
        sub = f64[y0:y1, x0:x1]
        mask = np.zeros_like(sub)
        mask[max(0, y - r) - y0:min(H, y + r + 1) - y0, max(0, x - r) - x0:min(W, x + r + 1) - x0] = 1
        wsub = w[y0:y1, x0:x1].astype(np.float64) * mask
        h = 1e-4 * T
        sp = sub.copy(); sp[y - y0, x - x0] += h
        sm = sub.copy(); sm[y - y0, x - x0] -= h
        fd = (np.sum(wsub * ref(sp, r, N, T)) - np.sum(wsub * ref(sm, r, N, T))) / (2 * h)
        assert abs(gg[y, x] - fd) <= 1e-3 * max(1.0, abs(fd)), (y, x, gg[y, x], fd)


def test_unit_window_closed_form(cuda_lib):
    """r = 0 (a 1 x 1 window): out = f, saved quads (f, 1, f, 0), dL/df = dL/dout,
    on an image wider than one strip and taller than 128 rows (sheared quads)."""
    bf = cuda_lib
    f = synth.sinusoids(140, 300, seed=11)
    ft = torch.from_numpy(f).cuda()
    sv = torch.empty((140, 300, 4), device="cuda")
    out = bf.bf_poly_forward(ft, 0, 0.0, 1.0, 6, saved=sv)
    g = torch.from_numpy(synth.weights((140, 300), seed=2)).cuda()
    gi = bf.bf_poly_backward(g, sv, 0, 0.0, 1.0, 6)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), f)
    assert np.array_equal(rowmajor(sv), np.stack([f, np.ones_like(f), f, np.zeros_like(f)], -1))
    assert torch.equal(gi, g)


def test_batched_autograd_matches_per_image(cuda_lib):
    """bilateral_poly on [B, H, W]: each image's output and dL/df equal those of
    the image on its own."""
    bf = cuda_lib
    fs = np.stack([synth.rectangles(90, 140, seed=40 + b) for b in range(3)])
    w = torch.from_numpy(synth.weights((3, 90, 140), seed=5)).cuda()
    ft = torch.from_numpy(fs).cuda().requires_grad_(True)
    out = bf.bilateral_poly(ft, 4, 0.0, 1.0, 5)
    (w * out).sum().backward()
    for b in range(3):
        fb = torch.from_numpy(fs[b]).cuda().requires_grad_(True)
        ob = bf.bilateral_poly(fb, 4, 0.0, 1.0, 5)
        (w[b] * ob).sum().backward()
        assert torch.equal(out[b].detach(), ob.detach())
        assert torch.equal(ft.grad[b], fb.grad)
