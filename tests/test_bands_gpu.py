"""One image in row bands on the GPU (the multi-GPU split, its ranks run one
after another in one process): the CUDA filter on each band's haloed frame,
restricted to the band's rows, reproduces the whole-image output and dL/df
(r halo for the forward; 2r on f and r on dL/dout for the adjoint)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import dist as bdist
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

H, W, R, SIGMA = 300, 500, 10, 0.1


def _frame(a, y0, y1, halo):
    lo, hi = max(0, y0 - halo), min(a.shape[0], y1 + halo)
    return a[lo:hi], y0 - lo


def _fwd(bf, f):
    return bf.bf_forward(torch.from_numpy(np.ascontiguousarray(f)).cuda(), R, SIGMA, 1.0, 0)


def _grad(bf, f, g):
    t = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    o = bf._opts(save=True)
    sv = torch.empty((*f.shape, 4), device="cuda")
    out = bf.bf_forward(t, R, SIGMA, 1.0, 0, opts=o, saved=sv)
    gi = torch.empty_like(t)
    bf.bf_backward(t, out, torch.from_numpy(np.ascontiguousarray(g)).cuda(), sv, R, SIGMA, 1.0, 0,
                   grad_img=gi, opts=o)
    return gi


@pytest.mark.parametrize("world", [2, 3])
def test_bands_reproduce_whole_image(cuda_lib, world):
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=8)
    g = synth.weights((H, W), seed=9)
    full_out = _fwd(bf, f).cpu().numpy()
    full_gi = _grad(bf, f, g).cpu().numpy()
    outs, gis = [], []
    for k in range(world):
        y0, y1 = bdist.band(H, k, world)
        fr, top = _frame(f, y0, y1, R)
        outs.append(_fwd(bf, fr).cpu().numpy()[top:top + y1 - y0])
        fr2, top2 = _frame(f, y0, y1, 2 * R)
        gr, top1 = _frame(g, y0, y1, R)
        gframe = np.zeros_like(fr2)
        gframe[top2 - top1:top2 - top1 + gr.shape[0]] = gr
        gis.append(_grad(bf, fr2, gframe).cpu().numpy()[top2:top2 + y1 - y0])
    out = np.concatenate(outs)
    gi = np.concatenate(gis)
    # bands change only the summation order of the running sums
    assert np.max(np.abs(out - full_out)) <= 2e-6
    assert np.max(np.abs(gi - full_gi)) <= 1e-5 * np.max(np.abs(full_gi))
    N = oracle.resolve_N(SIGMA, 1.0)
    ref = oracle.bilateral(f.astype(np.float64), R, math.pi / 2, N)
    assert np.max(np.abs(out - ref) / np.maximum(np.abs(ref), 1e-2)) <= 1e-4
