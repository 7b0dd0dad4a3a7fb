"""GPU parity of the truncated-basis option (bf_opts.trunc_tol: keep only the
lowest harmonics of q_N's expansion, end of Sec. 3) against the oracle's
plain definition of the truncated-kernel filter, element by element, and of
its adjoint against central differences of that oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
GTOL = 1e-3
G1 = math.pi / 2


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1e-2)


@pytest.mark.parametrize("H,W,r,N,tol", [(160, 300, 10, 41, 1e-3), (97, 131, 5, 41, 1e-6),
                                         (120, 77, 3, 19, 1e-2), (140, 150, 30, 64, 1e-4),
                                         (64, 64, 2, 11, 1e-3)])
def test_truncated_forward_matches_truncated_oracle(cuda_lib, H, W, r, N, tol):
    bf = cuda_lib
    f = synth.rectangles(H, W, seed=r + N)
    K = bf.bf_trunc_harmonics(N, r, tol)
    out = bf.bf_forward(torch.from_numpy(f).cuda(), r, 0.0, 1.0, N,
                        opts=bf._opts(trunc_tol=tol)).cpu().numpy()
    ref = oracle.bilateral_general(f.astype(np.float64), r, range_kind=oracle.RANGE_TRUNC,
                                   gamma=G1, N=N, K_keep=K)
    assert rel_err(out, ref).max() <= TOL
    # and within the analytic distance of the exact q_N filter
    exact, den = oracle.bilateral(f.astype(np.float64), r, G1, N, return_den=True)
    tail = sum(bf.bf_coeffs(N)[K:])
    assert np.all(np.abs(out - exact) <= (2 * r + 1) ** 2 * tail / den + 2e-5)


def test_truncated_saved_and_adjoint(cuda_lib):
    """Forward with saved quads and the adjoint with the same truncation:
    dL/df at sampled pixels against central differences of the truncated
    oracle (only the outputs a pixel reaches are re-evaluated)."""
    bf = cuda_lib
    H, W, r, N, tol = 96, 120, 6, 41, 1e-3
    K = bf.bf_trunc_harmonics(N, r, tol)
    f = synth.rectangles(H, W, seed=5)
    w = synth.weights((H, W), seed=1)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    out = bf.bilateral(ft, r, 0.1, 1.0, N, trunc_tol=tol)
    (torch.from_numpy(w).cuda() * out).sum().backward()
    gg = ft.grad.cpu().numpy()
    ref = oracle.bilateral_general(f.astype(np.float64), r, range_kind=oracle.RANGE_TRUNC,
                                   gamma=G1, N=N, K_keep=K)
    assert rel_err(out.detach().cpu().numpy(), ref).max() <= TOL
    rng = np.random.default_rng(11)
    for _ in range(8):
        y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
        y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
        x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
        sub = f[y0:y1, x0:x1].astype(np.float64)
        mask = np.zeros_like(sub)
        mask[max(0, y - r) - y0:min(H, y + r + 1) - y0, max(0, x - r) - x0:min(W, x + r + 1) - x0] = 1
        wsub = w[y0:y1, x0:x1].astype(np.float64) * mask
        h = 1e-4
        sp = sub.copy(); sp[y - y0, x - x0] += h
        sm = sub.copy(); sm[y - y0, x - x0] -= h
        Lp = np.sum(wsub * oracle.bilateral_general(sp, r, range_kind=oracle.RANGE_TRUNC,
                                                    gamma=G1, N=N, K_keep=K))
        Lm = np.sum(wsub * oracle.bilateral_general(sm, r, range_kind=oracle.RANGE_TRUNC,
                                                    gamma=G1, N=N, K_keep=K))
        fd = (Lp - Lm) / (2 * h)
        assert abs(gg[y, x] - fd) <= GTOL * max(1.0, abs(fd)), (y, x, gg[y, x], fd)
