"""Row-pitched images through the C ABI: the filter of a region of a wider
image (a column slice of a wider tensor, rows `pitch` elements apart)
matches the FP64 oracle and the filter of the same region copied into a
compact buffer, and never touches the columns between W and pitch (guard
columns filled with a sentinel). Pitched images run the general engine
kernels, compact ones the kernels specialised per harmonic count, so the two
agree to rounding (1e-4 of the largest value), not bit for bit; within one
kernel family (the batch, pitched or not) results are compared exactly. The batch call's optional
den output is checked against the oracle's normaliser eta(x) of Eq. filter2."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

SENT = -777.0
TOL = 1e-4


def rel_err(got, ref, T=1.0):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1e-2 * T)


def close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    assert np.abs(a - b).max() <= 1e-4 * max(np.abs(b).max(), 1e-30), np.abs(a - b).max()


def wide(H, P, fill=SENT):
    return torch.full((H, P), fill, dtype=torch.float32, device="cuda")


def view(t, x0, W):
    return t[..., x0:x0 + W]


@pytest.mark.parametrize("H,W,r,N,pad", [(97, 131, 5, 11, 37), (64, 300, 10, 41, 5),
                                         (80, 90, 12, 40, 64), (50, 70, 3, 50, 9)])
def test_forward_and_adjoint_on_a_pitched_view(cuda_lib, H, W, r, N, pad):
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=H + N)
    g = synth.weights((H, W), seed=2)
    P, x0 = W + pad, pad // 2
    big = wide(H, P)                       # input: sentinel outside the region
    view(big, x0, W).copy_(torch.from_numpy(f))
    obig = wide(H, P)                      # output: guard columns must survive
    gbig = wide(H, P)
    view(gbig, x0, W).copy_(torch.from_numpy(g))
    gibig = wide(H, P)
    img, out, gout, gimg = view(big, x0, W), view(obig, x0, W), view(gbig, x0, W), view(gibig, x0, W)
    opts = bf._opts(save=True)
    sv = torch.empty((H, W, 4), device="cuda")
    bf.bf_forward(img, r, 0.2, 1.0, N, out=out, opts=opts, saved=sv)
    ws = torch.empty(max(1, bf.bf_backward_workspace_bytes(H, W, r, 0.2, 1.0, N, opts) // 4),
                     device="cuda")
    bf.bf_backward(img, out, gout, sv, r, 0.2, 1.0, N, grad_img=gimg, workspace=ws, opts=opts)
    # the same region, compact
    ci = torch.from_numpy(f).cuda()
    co = torch.empty_like(ci)
    csv = torch.empty_like(sv)
    bf.bf_forward(ci, r, 0.2, 1.0, N, out=co, opts=opts, saved=csv)
    cg = torch.empty_like(ci)
    bf.bf_backward(ci, co, torch.from_numpy(g).cuda(), csv, r, 0.2, 1.0, N, grad_img=cg,
                   workspace=ws, opts=opts)
    torch.cuda.synchronize()
    ob, gib = obig.cpu().numpy(), gibig.cpu().numpy()
    for b in (ob, gib):
        assert np.all(b[:, :x0] == SENT) and np.all(b[:, x0 + W:] == SENT), "guard column written"
    close(ob[:, x0:x0 + W], co.cpu().numpy())
    close(gib[:, x0:x0 + W], cg.cpu().numpy())
    close(sv.cpu().numpy(), csv.cpu().numpy())
    ref = oracle.bilateral(f.astype(np.float64), r, oracle.gamma_fixed(1.0), N)
    assert rel_err(ob[:, x0:x0 + W], ref).max() <= TOL


def test_plain_forward_fallback_kernel_on_a_pitched_view(cuda_lib):
    """N > 43 without saved buffers runs the single-pass kernel."""
    bf = cuda_lib
    H, W, r, N, P = 70, 96, 4, 50, 130
    f = synth.sinusoids(H, W, seed=4)
    big = wide(H, P)
    view(big, 11, W).copy_(torch.from_numpy(f))
    obig = wide(H, P)
    bf.bf_forward(view(big, 11, W), r, 0.2, 1.0, N, out=view(obig, 11, W))
    torch.cuda.synchronize()
    ob = obig.cpu().numpy()
    assert np.all(ob[:, :11] == SENT) and np.all(ob[:, 11 + W:] == SENT)
    ref = oracle.bilateral(f.astype(np.float64), r, oracle.gamma_fixed(1.0), N)
    assert rel_err(ob[:, 11:11 + W], ref).max() <= TOL


def test_3d_forms_with_pitch(cuda_lib):
    """[B, H, W] launches with rows `pitch` apart (images H * pitch apart)."""
    bf = cuda_lib
    lib = bf.load()
    B, H, W, P, r = 3, 60, 75, 90, 6
    f = np.stack([synth.rectangles(H, W, seed=b) for b in range(B)])
    g = synth.weights((B, H, W), seed=1)
    big = torch.full((B, H, P), SENT, device="cuda")
    big[:, :, :W] = torch.from_numpy(f)
    gbig = torch.full((B, H, P), SENT, device="cuda")
    gbig[:, :, :W] = torch.from_numpy(g)
    obig = torch.full((B, H, P), SENT, device="cuda")
    gibig = torch.full((B, H, P), SENT, device="cuda")
    sv = torch.empty((B, H, W, 4), device="cuda")
    o = bf._opts(save=True, pitch=P)
    st = lib.bf_forward3d(ctypes.c_void_p(big.data_ptr()), B, H, W, r, 0.15, 1.0, 0,
                          ctypes.c_void_p(obig.data_ptr()), ctypes.byref(o),
                          ctypes.c_void_p(sv.data_ptr()), bf._stream_handle(None))
    assert st == 0
    st = lib.bf_backward3d(ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(obig.data_ptr()),
                           ctypes.c_void_p(gbig.data_ptr()), ctypes.c_void_p(sv.data_ptr()),
                           B, H, W, r, 0.15, 1.0, 0, ctypes.c_void_p(gibig.data_ptr()), None,
                           None, 0, ctypes.byref(o), bf._stream_handle(None))
    assert st == 0
    ci = torch.from_numpy(f).cuda()
    co = bf.bf_forward3d(ci, r, 0.15, 1.0, 0, opts=bf._opts(save=True),
                         saved=(csv := torch.empty_like(sv)))
    cg = torch.empty_like(ci)
    bf.bf_backward3d(ci, co, torch.from_numpy(g).cuda(), csv, r, 0.15, 1.0, 0, grad_img=cg,
                     opts=bf._opts(save=True))
    torch.cuda.synchronize()
    ob, gib = obig.cpu().numpy(), gibig.cpu().numpy()
    assert np.all(ob[:, :, W:] == SENT) and np.all(gib[:, :, W:] == SENT)
    close(ob[:, :, :W], co.cpu().numpy())
    close(gib[:, :, :W], cg.cpu().numpy())


def test_batch_pitch_and_den_output(cuda_lib):
    """bf_desc.pitch and bf_desc.den: pitched and compact images in one batch;
    outputs equal the compact batch, den equals the oracle's normaliser."""
    bf = cuda_lib
    specs = [(90, 120, 5, 0.2, 30), (64, 200, 10, 0.1, 0), (40, 33, 2, 0.3, 7)]
    imgs, outs, dens, fs, bigs = [], [], [], [], []
    for i, (H, W, r, s, pad) in enumerate(specs):
        f = synth.rectangles(H, W, seed=30 + i)
        fs.append(f)
        P = W + pad
        big, obig, dbig = wide(H, P), wide(H, P), wide(H, P)
        view(big, 0, W).copy_(torch.from_numpy(f))
        bigs.append((obig, dbig, W))
        imgs.append(view(big, 0, W))
        outs.append(view(obig, 0, W))
        dens.append(view(dbig, 0, W))
    rs = [s[2] for s in specs]
    sig = [s[3] for s in specs]
    descs = bf.make_descs(imgs, outs, rs, sig, dens=dens)
    ws = torch.empty(bf.bf_batch_workspace_bytes(descs) // 4 + 64, device="cuda")
    bf.bf_batch(descs, ws)
    cimgs = [torch.from_numpy(f).cuda() for f in fs]
    couts = [torch.empty_like(c) for c in cimgs]
    cdescs = bf.make_descs(cimgs, couts, rs, sig)
    bf.bf_batch(cdescs, ws)
    torch.cuda.synchronize()
    for i, (H, W, r, s, pad) in enumerate(specs):
        obig, dbig, _ = bigs[i]
        ob, db = obig.cpu().numpy(), dbig.cpu().numpy()
        assert np.all(ob[:, W:] == SENT) and np.all(db[:, W:] == SENT)
        # both batches run the general kernels: equal bit for bit
        assert np.array_equal(ob[:, :W], couts[i].cpu().numpy())
        N = oracle.resolve_N(s, 1.0)
        ref, den = oracle.bilateral(fs[i].astype(np.float64), r, oracle.gamma_fixed(1.0), N,
                                    return_den=True)
        assert rel_err(ob[:, :W], ref).max() <= TOL
        np.testing.assert_allclose(db[:, :W], den, rtol=1e-4, atol=0)
