"""Guard bands around every buffer the library writes (saved quads,
gradients, the [B, H, W] forms, the spatial-kernel and p_N variants, the
range check): each buffer is a view into a larger allocation filled with a
sentinel, and the sentinel outside the view must survive the call. This
stands in for a memory checker on this GPU pool."""
import numpy as np
import pytest
import torch

from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

SENT = -12345.0
G = 4096  # guard floats on each side


def guarded(n):
    buf = torch.full((n + 2 * G,), SENT, device="cuda")
    return buf, buf[G:G + n]


def intact(buf, n):
    b = buf.cpu().numpy()
    return np.all(b[:G] == SENT) and np.all(b[G + n:] == SENT)


@pytest.mark.parametrize("H,W,r,N", [(97, 131, 5, 11), (64, 300, 10, 41), (50, 70, 3, 50)])
def test_box_forward_saved_and_adjoint(cuda_lib, H, W, r, N):
    bf = cuda_lib
    img = torch.from_numpy(synth.rectangles(H, W, seed=H)).cuda()
    g = torch.from_numpy(synth.weights((H, W), seed=1)).cuda()
    bo, out = guarded(H * W)
    bs, sv = guarded(H * W * 4)
    opts = bf._opts(save=True)
    bf.bf_forward(img, r, 0.2, 1.0, N, out=out.view(H, W), opts=opts, saved=sv)
    bg, gi = guarded(H * W)
    nb = bf.bf_backward_workspace_bytes(H, W, r, 0.2, 1.0, N, opts)
    bw, ws = guarded(max(1, (nb + 3) // 4))
    bf.bf_backward(img, out.view(H, W), g, sv, r, 0.2, 1.0, N, grad_img=gi.view(H, W),
                   workspace=ws, opts=opts)
    torch.cuda.synchronize()
    assert intact(bo, H * W) and intact(bs, H * W * 4) and intact(bg, H * W)
    assert intact(bw, max(1, (nb + 3) // 4))


def test_3d_forms(cuda_lib):
    bf = cuda_lib
    B, H, W, r = 3, 80, 90, 4
    img = torch.from_numpy(np.stack([synth.rectangles(H, W, seed=b) for b in range(B)])).cuda()
    g = torch.from_numpy(synth.weights((B, H, W), seed=1)).cuda()
    opts = bf._opts(save=True)
    bo, out = guarded(B * H * W)
    bs, sv = guarded(B * H * W * 4)
    bf.bf_forward3d(img, r, 0.15, 1.0, 0, out=out.view(B, H, W), opts=opts, saved=sv)
    bg, gi = guarded(B * H * W)
    bf.bf_backward3d(img, out.view(B, H, W), g, sv, r, 0.15, 1.0, 0, grad_img=gi.view(B, H, W),
                     opts=opts)
    torch.cuda.synchronize()
    assert intact(bo, B * H * W) and intact(bs, B * H * W * 4) and intact(bg, B * H * W)


@pytest.mark.parametrize("M,N", [(2, 4), (1, 0), (4, 0)])
def test_spatial_variant(cuda_lib, M, N):
    bf = cuda_lib
    H, W, r = 90, 150, 5
    img = torch.from_numpy(synth.rectangles(H, W, seed=M + N)).cuda()
    g = torch.from_numpy(synth.weights((H, W), seed=1)).cuda()
    bo, out = guarded(H * W)
    bs, sv = guarded(H * W * 4)
    bf.bf_spatial_forward(img, r, M, 0.0, 1.0, N, out=out.view(H, W), saved=sv)
    bg, gi = guarded(H * W)
    bf.bf_spatial_backward(g, sv, r, M, 0.0, 1.0, N, grad_img=gi.view(H, W))
    torch.cuda.synchronize()
    assert intact(bo, H * W) and intact(bs, H * W * 4) and intact(bg, H * W)


@pytest.mark.parametrize("N", [1, 6, 8])
def test_poly_variant(cuda_lib, N):
    bf = cuda_lib
    H, W, r = 77, 140, 6
    img = torch.from_numpy(synth.rectangles(H, W, seed=N)).cuda()
    g = torch.from_numpy(synth.weights((H, W), seed=1)).cuda()
    bo, out = guarded(H * W)
    bs, sv = guarded(H * W * 4)
    bf.bf_poly_forward(img, r, 0.0, 1.0, N, out=out.view(H, W), saved=sv)
    bg, gi = guarded(H * W)
    bf.bf_poly_backward(g, sv, r, 0.0, 1.0, N, grad_img=gi.view(H, W))
    torch.cuda.synchronize()
    assert intact(bo, H * W) and intact(bs, H * W * 4) and intact(bg, H * W)


def test_check_range_writes_two_floats(cuda_lib):
    bf = cuda_lib
    img = torch.from_numpy(synth.rectangles(33, 45, seed=2)).cuda()
    bm, mm = guarded(2)
    st = bf.load().bf_check_range(bf._dptr(img, "img"), 33, 45, bf.F32, bf._dptr(mm, "mm"),
                                  bf._stream_handle(None))
    assert st == 0
    torch.cuda.synchronize()
    assert intact(bm, 2)
    assert mm.cpu().numpy()[0] == img.min().item() and mm.cpu().numpy()[1] == img.max().item()
