"""CPU-side checks of the C-ABI library: it loads, exports every symbol
include/bf.h declares, and its host-only parameter rules match the
mathematics (no GPU compute is called here)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_1107_4617_gb300 as bf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(bf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = bf.load()
    names = declared_functions()
    assert "bf_forward" in names and "bf_backward" in names and "bf_batch" in names
    for n in names:
        assert hasattr(lib, n), n


def test_no_oracle_in_product_sources():
    """The product path never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1107_4617_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "bf_oracle" not in txt, fn


@pytest.mark.parametrize("N", list(range(0, 65)))
def test_coefficients_reproduce_cos_power(N):
    """sum_k a_k cos(k theta) == cos(theta)^N (binomial expansion of q_N, Sec. 3,
    written with the shift identity of Sec. 1)."""
    a = bf.bf_coeffs(N)
    assert len(a) == N // 2 + 1
    th = np.linspace(-math.pi, math.pi, 1001)
    ks = (N % 2) + 2 * np.arange(len(a))
    series = sum(ai * np.cos(k * th) for ai, k in zip(a, ks))
    np.testing.assert_allclose(series, np.cos(th) ** N, rtol=0, atol=1e-14)
    assert abs(sum(a) - 1.0) < 1e-14  # q_N(0) = 1
    assert all(ai > 0 for ai in a)


def test_coefficients_shift_identity():
    """cos^N(s - t) = sum_k a_k [C_k(s)C_k(t) + S_k(s)S_k(t)] (Eq. def)."""
    rng = np.random.default_rng(0)
    s, t = rng.uniform(0, math.pi / 2, 200), rng.uniform(0, math.pi / 2, 200)
    for N in (1, 2, 11, 40, 41, 64):
        a = bf.bf_coeffs(N)
        ks = (N % 2) + 2 * np.arange(len(a))
        lhs = np.cos(s - t) ** N
        rhs = sum(ai * (np.cos(k * s) * np.cos(k * t) + np.sin(k * s) * np.sin(k * t))
                  for ai, k in zip(a, ks))
        np.testing.assert_allclose(rhs, lhs, rtol=0, atol=1e-13)


def test_invalid_coefficients():
    with pytest.raises(ValueError):
        bf.bf_coeffs(-1)
    with pytest.raises(ValueError):
        bf.bf_coeffs(65)


def test_order_rule_and_gamma():
    assert [bf.bf_resolve_N(s, 1.0) for s in (0.1, 0.15, 0.2, 0.3, 0.4, 0.08)] == [41, 19, 11, 5, 3, 64]
    assert bf.bf_resolve_N(0.2, 2.0) == bf.bf_resolve_N(0.1, 1.0)  # scale invariance sigma/T
    assert bf.bf_resolve_N(0.0, 1.0) == -1
    assert bf.bf_resolve_N(0.1, 0.0) == -1
    assert bf.bf_gamma(0.1, 1.0, 41, bf.GAMMA_FIXED) == pytest.approx(math.pi / 2)
    assert bf.bf_gamma(0.15, 1.0, 19, bf.GAMMA_FROM_SIGMA) == pytest.approx(1 / (0.15 * math.sqrt(19)))
    # variance control keeps gamma below pi/(2T), so the kernel stays >= 0 on [-T, T]
    for s in (0.08, 0.1, 0.15, 0.2, 0.3, 0.4):
        N = bf.bf_resolve_N(s, 1.0)
        assert bf.bf_gamma(s, 1.0, N, bf.GAMMA_FROM_SIGMA) <= math.pi / 2 + 1e-12


def test_sizes():
    assert bf.bf_saved_bytes(4, 5) == 4 * 4 * 5 * 4
    assert bf.bf_saved_bytes(0, 5) == 0


def _sheared(H, W):
    """The saved-quad layout as include/bf.h states it, written out."""
    ys, xs = np.meshgrid(np.arange(H, dtype=np.int64), np.arange(W, dtype=np.int64),
                         indexing="ij")
    if H >= 128:
        return ((ys + (xs % 128)) % H) * W + xs
    return ys * W + xs


@pytest.mark.parametrize("H,W", [(1, 1), (5, 300), (127, 130), (128, 1), (128, 129), (200, 64),
                                 (300, 257), (1000, 3)])
def test_saved_index_is_the_documented_layout(H, W):
    """bf_saved_index gives the header's formula at every pixel, and the map is
    one-to-one onto [0, H W): every quad slot belongs to exactly one pixel."""
    got = np.array([[bf.bf_saved_index(y, x, H, W) for x in range(W)] for y in range(H)],
                   dtype=np.int64)
    np.testing.assert_array_equal(got, _sheared(H, W))
    assert np.array_equal(np.sort(got.ravel()), np.arange(H * W))


def test_saved_index_past_2_31_pixels_and_bad_arguments():
    H, W = 50000, 50000  # 2.5e9 pixels: the index needs 64 bits
    for y, x in [(H - 1, W - 1), (H - 100, 127), (H - 100, 99), (0, W - 1), (H // 2, 12345)]:
        want = ((y + (x % 128)) % H) * W + x
        assert bf.bf_saved_index(y, x, H, W) == want
    assert bf.bf_saved_index(H - 1, 0, H, W) == (H - 1) * W > 2 ** 31  # column 0: no shear
    for args in [(-1, 0, 4, 4), (0, -1, 4, 4), (4, 0, 4, 4), (0, 4, 4, 4), (0, 0, 0, 4),
                 (0, 0, 4, 0)]:
        assert bf.bf_saved_index(*args) == -1


def test_rowmajor_helper_inverts_the_library_layout():
    """The GPU tests read saved quads through tests/_quads.rowmajor; placing each
    pixel's coordinates at bf_saved_index and un-shearing returns them in place."""
    from _quads import rowmajor
    for H, W in [(70, 90), (150, 170), (300, 257)]:
        sv = np.zeros((H * W, 4), np.float32)
        for y in range(H):
            for x in range(W):
                sv[bf.bf_saved_index(y, x, H, W)] = (y, x, 1, 0)
        back = rowmajor(sv.reshape(H, W, 4))
        ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        assert np.array_equal(back[..., 0], ys) and np.array_equal(back[..., 1], xs)


def test_variants_reject_images_of_2_31_pixels_first():
    """bf_spatial_* and bf_poly_* index their saved quads in 32 bits: an image of
    2^31 or more pixels is BF_ERR_UNSUPPORTED (2), checked before any other
    argument (the pointers here are null and never read)."""
    lib = bf.load()
    H = W = 46341  # 46341^2 > 2^31 - 1
    assert lib.bf_spatial_forward(None, H, W, 1, 2, 0.0, 1.0, 4, None, None, None, None) == 2
    assert lib.bf_spatial_backward(None, None, H, W, 1, 2, 0.0, 1.0, 4, None, None, None) == 2
    assert lib.bf_poly_forward(None, H, W, 1, 0.0, 1.0, 3, None, None, None, None) == 2
    assert lib.bf_poly_backward(None, None, H, W, 1, 0.0, 1.0, 3, None, None, None) == 2
    # one pixel row fewer fits: the null pointers are then the error (1)
    assert lib.bf_spatial_forward(None, 46340, 46340, 1, 2, 0.0, 1.0, 4, None, None, None,
                                  None) == 1
    assert lib.bf_poly_forward(None, 46340, 46340, 1, 0.0, 1.0, 3, None, None, None, None) == 1


def test_argument_checks_return_before_any_launch():
    lib = bf.load()
    o = bf.BfOpts()
    lib.bf_default_opts(ctypes.byref(o))
    p = ctypes.c_void_p(0x1000)
    q = ctypes.c_void_p(0x2000)
    # null image / output, bad sizes, bad r, bad T, bad sigma: BF_ERR_INVALID_ARG (1)
    assert lib.bf_forward(None, 4, 4, 1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    assert lib.bf_forward(p, 0, 4, 1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    assert lib.bf_forward(p, 4, 4, -1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    assert lib.bf_forward(p, 4, 4, 1, 0.2, 0.0, 0, q, ctypes.byref(o), None, None) == 1
    assert lib.bf_forward(p, 4, 4, 1, 0.0, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    assert lib.bf_forward(p, 4, 4, 1, 0.2, 1.0, 0, p, ctypes.byref(o), None, None) == 1  # aliasing
    # out of the built range: BF_ERR_UNSUPPORTED (2)
    assert lib.bf_forward(p, 4, 4, 1, 0.2, 1.0, 65, q, ctypes.byref(o), None, None) == 2
    assert lib.bf_forward(p, 4, 4, 65, 0.2, 1.0, 3, q, ctypes.byref(o), None, None) == 2
    assert lib.bf_forward(p, 4, 4, 1, 0.05, 1.0, 0, q, ctypes.byref(o), None, None) == 2  # N=163
    # bad opts
    o.in_dtype = 7
    assert lib.bf_forward(p, 4, 4, 1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    lib.bf_default_opts(ctypes.byref(o))
    o.tile_w = 48
    assert lib.bf_forward(p, 4, 4, 1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    # backward: missing saved buffer; grad_sigma without workspace -> NOMEM (6)
    assert lib.bf_backward(p, q, q, None, 4, 4, 1, 0.2, 1.0, 0, q, None, None, 0, None, None) == 1
    lib.bf_default_opts(ctypes.byref(o))
    o.gamma_mode = bf.GAMMA_FROM_SIGMA
    assert lib.bf_backward(p, q, q, q, 4, 4, 1, 0.2, 1.0, 0, None, q, None, 0,
                           ctypes.byref(o), None) == 6
    # adjoint: dL/dimg aliasing an input
    s16 = ctypes.c_void_p(0x3000)
    for gi in (p, q, s16):
        assert lib.bf_backward(p, q, q, s16, 4, 4, 1, 0.2, 1.0, 0, gi, None, None, 0, None,
                               None) == 1
    # variant adjoints: dL/dimg aliasing dL/dout or the saved quads
    for gi in (p, s16):
        assert lib.bf_spatial_backward(p, s16, 4, 4, 1, 2, 0.0, 1.0, 4, gi, None, None) == 1
        assert lib.bf_poly_backward(p, s16, 4, 4, 1, 0.0, 1.0, 3, gi, None, None) == 1
    # batch: empty list
    assert lib.bf_batch(None, 0, None, p, 64, None) == 1
    # truncation tolerance outside [0, 1)
    for bad in (-1e-3, 1.0, float("nan")):
        lib.bf_default_opts(ctypes.byref(o))
        o.trunc_tol = bad
        assert lib.bf_forward(p, 4, 4, 1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
    # row pitch: negative or shorter than a row is rejected; the variant filters
    # accept only a compact image (pitch 0 or W)
    for bad in (-1, 3):
        lib.bf_default_opts(ctypes.byref(o))
        o.pitch = bad
        assert lib.bf_forward(p, 4, 4, 1, 0.2, 1.0, 0, q, ctypes.byref(o), None, None) == 1
        assert lib.bf_backward(p, q, q, s16, 4, 4, 1, 0.2, 1.0, 0, ctypes.c_void_p(0x4000),
                               None, None, 0, ctypes.byref(o), None) == 1
    lib.bf_default_opts(ctypes.byref(o))
    o.pitch = 8
    assert lib.bf_spatial_forward(p, 4, 4, 1, 2, 0.0, 1.0, 4, q, ctypes.byref(o), None, None) == 2
    assert lib.bf_poly_forward(p, 4, 4, 1, 0.0, 1.0, 3, q, ctypes.byref(o), None, None) == 2
    # batch descriptor: pitch below W, den aliasing the output
    d = bf.BfDesc()
    d.img, d.out, d.den = 0x1000, 0x2000, None
    d.H, d.W, d.pitch, d.r, d.N, d.sigma_r, d.T = 4, 4, 3, 1, 3, 0.2, 1.0
    arr = (bf.BfDesc * 1)(d)
    assert lib.bf_batch_workspace_bytes(arr, 1, None) == 0
    d.pitch, d.den = 0, 0x2000
    arr = (bf.BfDesc * 1)(d)
    assert lib.bf_batch_workspace_bytes(arr, 1, None) == 0
    # the persistent batch launches run 128- or 256-thread strips only
    d.den = None
    arr = (bf.BfDesc * 1)(d)
    assert lib.bf_batch_workspace_bytes(arr, 1, None) > 0
    for tw, ok in ((96, False), (64, False), (128, True), (256, True)):
        lib.bf_default_opts(ctypes.byref(o))
        o.tile_w = tw
        assert (lib.bf_batch_workspace_bytes(arr, 1, ctypes.byref(o)) > 0) == ok, tw


def test_status_strings():
    for s in range(7):
        assert isinstance(bf.bf_status_string(s), str) and bf.bf_status_string(s)


def truncation_rule(N, r, tol):
    """Independent restatement of the truncated-basis rule: drop the highest
    harmonics of cos^N's expansion (smallest a_k, end of Sec. 3) while their
    coefficients sum to at most min(tol, 1/(2 (2r+1)^2))."""
    ks = list(range(N % 2, N + 1, 2))
    a = [math.comb(N, (N - k) // 2) / 2.0 ** (N - 1) for k in ks]
    if N % 2 == 0:
        a[0] /= 2
    if tol <= 0:
        return len(a)
    cap = min(tol, 0.5 / (2 * r + 1) ** 2)
    keep, tail = len(a), 0.0
    while keep > 1 and tail + a[keep - 1] <= cap:
        keep -= 1
        tail += a[keep]
    return keep


@pytest.mark.parametrize("N", [1, 2, 5, 11, 19, 40, 41, 64])
@pytest.mark.parametrize("r", [1, 10, 30])
@pytest.mark.parametrize("tol", [0.0, 1e-6, 1e-4, 1e-3, 1e-2, 0.5])
def test_truncated_basis_rule(N, r, tol):
    K = bf.bf_trunc_harmonics(N, r, tol)
    assert K == truncation_rule(N, r, tol)
    assert 1 <= K <= N // 2 + 1
    # the kept expansion differs from cos^N by at most the dropped coefficients,
    # and by exactly that at t = 0
    a = bf.bf_coeffs(N)
    dropped = sum(a[K:])
    assert dropped <= min(tol, 0.5 / (2 * r + 1) ** 2) + 1e-15 if tol > 0 else dropped == 0
    th = np.linspace(0, math.pi / 2, 2001)
    ks = (N % 2) + 2 * np.arange(K)
    w = sum(ai * np.cos(k * th) for ai, k in zip(a[:K], ks))
    assert np.max(np.abs(w - np.cos(th) ** N)) <= dropped + 1e-14
    assert abs((1.0 - w[0]) - dropped) <= 1e-14


def test_truncated_basis_rule_rejects_bad_arguments():
    assert bf.bf_trunc_harmonics(-1, 3, 0.0) == -1
    assert bf.bf_trunc_harmonics(65, 3, 0.0) == -1
    assert bf.bf_trunc_harmonics(11, -1, 0.0) == -1
    assert bf.bf_trunc_harmonics(11, 3, 1.0) == -1
    assert bf.bf_trunc_harmonics(11, 3, -0.5) == -1


def test_poly_order_rule():
    """N = ceil(T^2 / (2 sigma_r^2)) from Eq. approx1."""
    for sigma, T, N in [(0.3, 1.0, 6), (0.25, 1.0, 8), (0.5, 1.0, 2), (0.4, 1.0, 4), (1.0, 2.0, 2)]:
        assert bf.bf_poly_resolve_N(sigma, T) == N
        assert N == max(1, math.ceil(T * T / (2 * sigma * sigma) - 1e-9))
    assert bf.bf_poly_resolve_N(0.0, 1.0) == -1


def test_binding_rejects_undersized_saved_buffer():
    """The binding checks buffer sizes the C ABI cannot see (a raw pointer):
    a saved buffer of the old three-plane size is refused before any call."""
    import torch
    img = torch.zeros((8, 9))
    small = torch.zeros((3, 8, 9))
    with pytest.raises(ValueError, match="saved"):
        bf._check_bytes(small, bf.bf_saved_bytes(8, 9), "saved")
    bf._check_bytes(torch.zeros((8, 9, 4)), bf.bf_saved_bytes(8, 9), "saved")
    assert img.numel() * 16 == bf.bf_saved_bytes(8, 9)
