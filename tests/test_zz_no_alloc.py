"""bf_backward_noalloc against bf_backward.

The allocation-free adjoint is for callers that cannot allocate device
memory (a plugin whose host application owns the GPU's memory pool, a loop
that cannot afford an allocation's device synchronisation). It keeps its
dL/dsigma_r partial sums in a fixed array inside the library instead of a
caller workspace. Both run the same kernels with the same launch shape and
sum the partials in the same fixed order, so dL/dimg and dL/dsigma_r must
equal the workspace version's bit for bit. Calls in a row on different
images check that the array's leftover contents from one call do not leak
into the next, also when the harmonics run in chunks (N > 43) and the
array holds the chunks' image-sized accumulators too. This file is
collected last, so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu


def _case(bf, H, W, r, sigma, seed, N=0):
    dev = torch.device("cuda:0")
    f = torch.from_numpy(synth.rectangles(H, W, seed=seed)).to(dev)
    g = torch.from_numpy(synth.weights((H, W), seed=seed + 1)).to(dev)
    N = N or bf.bf_resolve_N(sigma, 1.0)
    opts = bf._opts(save=True, gamma_mode=bf.GAMMA_FROM_SIGMA)
    sv = torch.empty((H, W, 4), device=dev)
    out = bf.bf_forward(f, r, sigma, 1.0, N, opts=opts, saved=sv)
    return f, g, out, sv, N, opts


def _reference(bf, f, g, out, sv, r, sigma, N, opts):
    H, W = f.shape
    gi = torch.empty_like(f)
    gs = torch.zeros((1,), device=f.device)
    ws = torch.empty((bf.bf_backward_workspace_bytes(H, W, r, sigma, 1.0, N, opts) // 4 + 1,), device=f.device)
    bf.bf_backward(f, out, g, sv, r, sigma, 1.0, N, grad_img=gi, grad_sigma=gs, workspace=ws,
                   opts=opts)
    return gi, gs


def _noalloc_raw(bf, f, g, out, sv, r, sigma, N, opts):
    """Direct call through the C ABI (ctypes), no Python wrapper logic."""
    lib = bf.load()
    fn = lib.bf_backward_noalloc
    vp = ctypes.c_void_p
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                   ctypes.c_float, ctypes.c_int, vp, vp, ctypes.POINTER(bf.BfOpts), vp]
    H, W = f.shape
    gi = torch.full_like(f, -9.0)
    gs = torch.full((1,), -9.0, device=f.device)
    st = fn(vp(f.data_ptr()), vp(out.data_ptr()), vp(g.data_ptr()), vp(sv.data_ptr()), H, W, r,
            sigma, 1.0, N, vp(gi.data_ptr()), vp(gs.data_ptr()), ctypes.byref(opts),
            vp(torch.cuda.current_stream().cuda_stream))
    assert st == 0, bf.bf_status_string(st)
    return gi, gs


def _equal(a, b):
    a = a.detach().cpu().numpy()
    b = b.detach().cpu().numpy()
    assert np.array_equal(a, b), float(np.abs(a.astype(np.float64) - b).max())


@pytest.mark.parametrize("cases", [
    # whole harmonics in one launch, two images in a row
    [(300, 410, 7, 0.15, 3, 0), (257, 129, 4, 0.3, 11, 0)],
    # harmonic chunks (N = 50): the accumulators live in the array too; the
    # larger image first leaves its contents behind for the smaller one
    [(88, 90, 6, 0.1, 5, 50), (48, 64, 5, 0.1, 7, 50)],
])
def test_noalloc_matches_workspace_version_bit_for_bit(cuda_lib, cases):
    bf = cuda_lib
    for (H, W, r, sigma, seed, N) in cases:
        f, g, out, sv, N, opts = _case(bf, H, W, r, sigma, seed, N)
        gi_ref, gs_ref = _reference(bf, f, g, out, sv, r, sigma, N, opts)
        gi, gs = _noalloc_raw(bf, f, g, out, sv, r, sigma, N, opts)
        torch.cuda.synchronize()
        _equal(gi, gi_ref)
        _equal(gs, gs_ref)


def test_noalloc_rejects_oversize(cuda_lib):
    bf = cuda_lib
    lib = bf.load()
    # a grid with more CTAs than the fixed array holds partial slots (checked
    # before any launch: the pointers are never dereferenced)
    o = bf._opts(gamma_mode=bf.GAMMA_FROM_SIGMA, tile_h=16, tile_w=64)
    need = bf.bf_backward_workspace_bytes(1 << 20, 4096, 10, 0.2, 1.0, 0, o)
    assert need > 4 * 16384
    vp = ctypes.c_void_p
    fn = lib.bf_backward_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                   ctypes.c_float, ctypes.c_int, vp, vp, ctypes.POINTER(bf.BfOpts), vp]
    bogus = vp(0x1000)
    st = fn(bogus, bogus, bogus, bogus, 1 << 20, 4096, 10, 0.2, 1.0, 0, bogus, bogus,
            ctypes.byref(o), None)
    assert st == 2  # BF_ERR_UNSUPPORTED
