"""Full-size sampled parity of the variant filters in the launch configuration
the benchmark times (4096^2, r=10):
- Algorithm 2 with the q_2 x q_2 spatial kernel and the q_4 range kernel;
- Algorithm 1 (q_2 x q_2, no range kernel);
- the p_6 range kernel with the box window.

Forward outputs on sampled rows (borders and interior) are checked against the
FP64 oracle: relative error with a floor at 1e-2 T. dL/df at sampled pixels
(corners included) is checked against FP64 central differences of the oracle
on a crop around each pixel."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_4617_gb300 import synth

pytestmark = pytest.mark.gpu

TOL, GTOL = 1e-4, 1e-3
H = W = 4096
R = 10
CASES = {
    "alg2_M2_N4": dict(kind="spatial", M=2, N=4),
    "alg1_M2": dict(kind="spatial", M=2, N=0),
    "poly_N6": dict(kind="poly", N=6),
}
ROWS = (0, 511, 512, 2731, 4095)


def oracle_filter(f, case, rows=None):
    if case["kind"] == "spatial":
        return oracle.bilateral_general(
            f, R, spatial=oracle.SPATIAL_QM, M=case["M"],
            range_kind=oracle.RANGE_COSN if case["N"] else oracle.RANGE_NONE,
            gamma=math.pi / 2, N=case["N"], rows=rows)
    return oracle.bilateral_general(f, R, range_kind=oracle.RANGE_POLY, N=case["N"], Tr=1.0,
                                    rows=rows)


def gpu_forward_backward(bf, case, img, g):
    sv = torch.empty((H, W, 4), device="cuda")
    if case["kind"] == "spatial":
        out = bf.bf_spatial_forward(img, R, case["M"], 0.0, 1.0, case["N"], saved=sv)
        gi = bf.bf_spatial_backward(g, sv, R, case["M"], 0.0, 1.0, case["N"])
    else:
        out = bf.bf_poly_forward(img, R, 0.0, 1.0, case["N"], saved=sv)
        gi = bf.bf_poly_backward(g, sv, R, 0.0, 1.0, case["N"])
    torch.cuda.synchronize()
    return out.cpu().numpy(), gi.cpu().numpy()


@pytest.mark.parametrize("name", sorted(CASES))
def test_variant_full_size_sampled(cuda_lib, name):
    case = CASES[name]
    f = synth.rectangles(H, W, seed=0)
    w = synth.weights((H, W), seed=1)
    out, gg = gpu_forward_backward(cuda_lib, case, torch.from_numpy(f).cuda(),
                                   torch.from_numpy(w).cuda())
    f64 = f.astype(np.float64)
    for y in ROWS:
        ref = oracle_filter(f64, case, rows=(y, y + 1))[0]
        err = np.abs(out[y].astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-2)
        assert err.max() <= TOL, (name, y, err.max())
    rng = np.random.default_rng(23)
    pts = [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0)] + \
        [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(6)]
    h = 1e-4
    for y, x in pts:
        # outputs that see pixel (y, x) lie within r of it; their windows
        # within 2r, so the crop reproduces their border truncation exactly
        y0, y1 = max(0, y - 2 * R), min(H, y + 2 * R + 1)
        x0, x1 = max(0, x - 2 * R), min(W, x + 2 * R + 1)
        sub = f64[y0:y1, x0:x1]
        mask = np.zeros_like(sub)
        mask[max(0, y - R) - y0:min(H, y + R + 1) - y0,
             max(0, x - R) - x0:min(W, x + R + 1) - x0] = 1
        wsub = w[y0:y1, x0:x1].astype(np.float64) * mask
        sp = sub.copy()
        sp[y - y0, x - x0] += h
        sm = sub.copy()
        sm[y - y0, x - x0] -= h
        fd = (np.sum(wsub * oracle_filter(sp, case)) - np.sum(wsub * oracle_filter(sm, case))) / (2 * h)
        assert abs(gg[y, x] - fd) <= GTOL * max(1.0, abs(fd)), (name, y, x, gg[y, x], fd)
