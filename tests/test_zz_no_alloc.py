"""bf_backward_noalloc against bf_backward.

The allocation-free adjoint is for callers that cannot allocate device
memory (a plugin whose host application owns the GPU's memory pool, a loop
that cannot afford an allocation's device synchronisation). It keeps its
dL/dsigma_r partial sums in a fixed array inside the library instead of a
caller workspace; its results must equal the workspace version's. Two calls
in a row on different images check that the array's leftover contents from
the first call do not leak into the second. This file is collected last, so
a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

GTOL = 1e-3  # gradient tolerance used by the adjoint tests


def _case(bf, H, W, r, sigma, seed):
    dev = torch.device("cuda:0")
    f = torch.from_numpy(synth.rectangles(H, W, seed=seed)).to(dev)
    g = torch.from_numpy(synth.weights((H, W), seed=seed + 1)).to(dev)
    N = bf.bf_resolve_N(sigma, 1.0)
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


def _close(a, b):
    a = a.detach().cpu().numpy().astype(np.float64)
    b = b.detach().cpu().numpy().astype(np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    assert np.abs(a - b).max() <= GTOL * scale, (np.abs(a - b).max(), scale)


def test_noalloc_matches_workspace_version_twice(cuda_lib):
    bf = cuda_lib
    for (H, W, r, sigma, seed) in [(300, 410, 7, 0.15, 3), (257, 129, 4, 0.3, 11)]:
        f, g, out, sv, N, opts = _case(bf, H, W, r, sigma, seed)
        gi_ref, gs_ref = _reference(bf, f, g, out, sv, r, sigma, N, opts)
        gi, gs = _noalloc_raw(bf, f, g, out, sv, r, sigma, N, opts)
        torch.cuda.synchronize()
        _close(gi, gi_ref)
        assert abs(float(gs) - float(gs_ref)) <= GTOL * max(1.0, abs(float(gs_ref)))


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
