"""The CUDA path against the stored oracle fixtures of tests/golden (a 24 x 20
FP32 image; outputs at (r, N) = (2, 3), (1, 4), (3, 41), (2, 50); dL/df at two
of them), element by element, through the C ABI: the same bar as the other
parity tests (1e-4 relative with a floor at 1e-2 T; gradients 1e-3 of their
maximum)."""
import math
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-4
GTOL = 1e-3


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _image(name):
    return torch.from_numpy(_load(name).astype(np.float32)).cuda()


@pytest.mark.parametrize("r,N", [(2, 3), (1, 4), (3, 41), (2, 50)])
def test_forward_matches_stored_oracle(cuda_lib, r, N):
    bf = cuda_lib
    f = _image("img_24x20.txt")
    want = _load("out_r%d_N%d.txt" % (r, N))
    out = torch.full_like(f, -5.0)
    bf.bf_forward(f, r, 0.2, 1.0, N, out=out)
    torch.cuda.synchronize()
    rel = np.abs(out.cpu().numpy().astype(np.float64) - want) / np.maximum(np.abs(want), 1e-2)
    assert rel.max() <= TOL, rel.max()


@pytest.mark.parametrize("r,N", [(2, 3), (3, 41)])
def test_adjoint_matches_stored_oracle(cuda_lib, r, N):
    bf = cuda_lib
    H, W = 24, 20
    f = _image("img_24x20.txt")
    g = _image("weights_24x20.txt")
    want = _load("grad_r%d_N%d.txt" % (r, N))
    opts = bf._opts(save=True)
    out = torch.empty_like(f)
    sv = torch.empty((H, W, 4), device="cuda")
    bf.bf_forward(f, r, 0.2, 1.0, N, out=out, opts=opts, saved=sv)
    gi = torch.full_like(f, -5.0)
    ws = torch.empty((bf.bf_backward_workspace_bytes(H, W, r, 0.2, 1.0, N, opts) // 4 + 1,),
                     device="cuda")
    bf.bf_backward(f, out, g, sv, r, 0.2, 1.0, N, grad_img=gi, workspace=ws, opts=opts)
    torch.cuda.synchronize()
    err = np.abs(gi.cpu().numpy().astype(np.float64) - want).max()
    assert err <= GTOL * np.abs(want).max(), (err, np.abs(want).max())
