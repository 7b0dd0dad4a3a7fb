"""GPU parity of bf_spatial_forward (Algorithm 2 with a shiftable spatial
kernel q_M x q_M, and Algorithm 1 without a range kernel) against the
oracle's direct O(r^2) definition, element by element. Same tolerance as the
box filter: |gpu - oracle| / max(|oracle|, 1e-2) <= 1e-4."""
import math

import numpy as np
import pytest
import torch

import oracle
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


def test_rejects_unbuilt_orders(cuda_lib):
    bf = cuda_lib
    f = torch.zeros((8, 8), device="cuda")
    for M, N in [(3, 2), (5, 0), (2, 6), (0, 4)]:
        with pytest.raises(bf.BfError):
            bf.bf_spatial_forward(f, 2, M, 0.0, 1.0, N)
    with pytest.raises(bf.BfError):
        bf.bf_spatial_forward(f, 57, 2, 0.0, 1.0, 4)
