"""Constant-time raised-cosine bilateral filter for one NVIDIA GB300 (sm_103a).

Python binding of the C ABI in ``include/bf.h`` (library ``libbf.so`` built
from ``csrc/``). The functions named ``bf_*`` mirror the C entry points one to
one and only marshal arguments: torch supplies device memory and the CUDA
stream, every step of the filter runs in the library's kernels. There is no
CPU or PyTorch fallback: if the library cannot be loaded, or a tensor is not
on a CUDA device, the call raises.

``bilateral(f, r, sigma_r, ...)`` wraps forward and adjoint kernels in a
``torch.autograd.Function`` (gradients with respect to the image and to
sigma_r).
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "BfError", "BfOpts", "BfDesc", "load", "lib_path",
    "bf_forward", "bf_backward", "bf_forward3d", "bf_backward3d", "bf_batch", "bf_batch_prepare",
    "bf_batch_launch", "bf_backward3d_workspace_bytes",
    "bf_resolve_N", "bf_coeffs", "bf_trunc_harmonics", "bf_gamma", "bf_saved_bytes", "bf_saved_index", "bf_backward_workspace_bytes",
    "bf_batch_workspace_bytes", "bf_status_string", "bf_last_cuda_error", "bilateral",
    "bf_spatial_forward", "bf_spatial_backward", "bilateral_spatial", "bf_poly_forward", "bf_poly_backward", "bilateral_poly", "bf_poly_resolve_N", "bf_check_range",
    "GAMMA_FIXED", "GAMMA_FROM_SIGMA", "F32", "BF16", "N_MAX", "R_MAX",
]

GAMMA_FIXED, GAMMA_FROM_SIGMA = 0, 1
F32, BF16 = 0, 1
N_MAX, R_MAX = 64, 64

_lock = threading.Lock()
_lib = None


class BfError(RuntimeError):
    """A C-ABI call returned a status other than BF_OK."""

    def __init__(self, fn: str, status: int, cuda_code: int = 0):
        msg = f"{fn}: {_status_string(status)} (status {status})"
        if cuda_code:
            msg += f", cudaError {cuda_code}"
        super().__init__(msg)
        self.status = status
        self.cuda_code = cuda_code


class BfOpts(ctypes.Structure):
    _fields_ = [("kahan", ctypes.c_int), ("gamma_mode", ctypes.c_int),
                ("in_dtype", ctypes.c_int), ("save_for_backward", ctypes.c_int),
                ("tile_h", ctypes.c_int), ("tile_w", ctypes.c_int), ("kp_max", ctypes.c_int),
                ("trunc_tol", ctypes.c_float), ("pitch", ctypes.c_int)]


class BfDesc(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("out", ctypes.c_void_p), ("den", ctypes.c_void_p),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int),
                ("r", ctypes.c_int), ("N", ctypes.c_int),
                ("sigma_r", ctypes.c_float), ("T", ctypes.c_float)]


def lib_path() -> str:
    from . import build as _b
    return _b.LIB


def load():
    """Load libbf.so, compiling it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        path = _b.LIB
        if not _b.up_to_date():
            try:
                path = _b.build()
            except Exception as e:  # no silent fallback: the product needs the library
                raise RuntimeError(f"libbf.so is missing and could not be built: {e}") from e
        lib = ctypes.CDLL(path)
        c_int, c_float, c_size, vp = ctypes.c_int, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p
        P_opts = ctypes.POINTER(BfOpts)
        P_desc = ctypes.POINTER(BfDesc)
        sig = {
            "bf_default_opts": (None, [P_opts]),
            "bf_resolve_N": (c_int, [c_float, c_float]),
            "bf_coeffs": (c_int, [c_int, ctypes.POINTER(ctypes.c_double), c_int]),
            "bf_trunc_harmonics": (c_int, [c_int, c_int, c_float]),
            "bf_gamma": (ctypes.c_double, [c_float, c_float, c_int, c_int]),
            "bf_saved_bytes": (c_size, [c_int, c_int]),
            "bf_saved_index": (c_size, [c_int, c_int, c_int, c_int]),
            "bf_forward": (c_int, [vp, c_int, c_int, c_int, c_float, c_float, c_int, vp, P_opts,
                                   vp, vp]),
            "bf_backward_workspace_bytes": (c_size, [c_int, c_int, c_int, c_float, c_float, c_int,
                                                     P_opts]),
            "bf_backward3d_workspace_bytes": (c_size, [c_int, c_int, c_int, c_int, c_float,
                                                       c_float, c_int, P_opts]),
            "bf_forward3d": (c_int, [vp, c_int, c_int, c_int, c_int, c_float, c_float, c_int, vp,
                                     P_opts, vp, vp]),
            "bf_backward3d": (c_int, [vp, vp, vp, vp, c_int, c_int, c_int, c_int, c_float, c_float,
                                      c_int, vp, vp, vp, c_size, P_opts, vp]),
            "bf_backward": (c_int, [vp, vp, vp, vp, c_int, c_int, c_int, c_float, c_float, c_int,
                                    vp, vp, vp, c_size, P_opts, vp]),
            "bf_spatial_forward": (c_int, [vp, c_int, c_int, c_int, c_int, c_float, c_float,
                                           c_int, vp, P_opts, vp, vp]),
            "bf_spatial_backward": (c_int, [vp, vp, c_int, c_int, c_int, c_int, c_float, c_float,
                                            c_int, vp, P_opts, vp]),
            "bf_poly_resolve_N": (c_int, [c_float, c_float]),
            "bf_poly_forward": (c_int, [vp, c_int, c_int, c_int, c_float, c_float, c_int, vp,
                                        P_opts, vp, vp]),
            "bf_poly_backward": (c_int, [vp, vp, c_int, c_int, c_int, c_float, c_float, c_int,
                                         vp, P_opts, vp]),
            "bf_check_range": (c_int, [vp, c_int, c_int, c_int, vp, vp]),
            "bf_batch_workspace_bytes": (c_size, [P_desc, c_int, P_opts]),
            "bf_batch": (c_int, [P_desc, c_int, P_opts, vp, c_size, vp]),
            "bf_batch_prepare": (c_int, [P_desc, c_int, P_opts, vp, c_size, vp]),
            "bf_batch_launch": (c_int, [vp, c_size, P_opts, vp]),
            "bf_status_string": (ctypes.c_char_p, [c_int]),
            "bf_last_cuda_error": (c_int, [ctypes.POINTER(c_int)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _status_string(s: int) -> str:
    try:
        return load().bf_status_string(int(s)).decode()
    except Exception:
        return "unknown"


def bf_status_string(s: int) -> str:
    return _status_string(s)


def bf_last_cuda_error() -> int:
    code = ctypes.c_int(0)
    load().bf_last_cuda_error(ctypes.byref(code))
    return int(code.value)


def _check(fn: str, status: int):
    if status != 0:
        raise BfError(fn, status, bf_last_cuda_error() if status == 3 else 0)


def _opts(kahan=False, gamma_mode=GAMMA_FIXED, in_dtype=F32, save=False, tile_h=0, tile_w=0,
          kp_max=0, trunc_tol=0.0, pitch=0):
    o = BfOpts()
    o.kahan, o.gamma_mode, o.in_dtype = int(bool(kahan)), int(gamma_mode), int(in_dtype)
    o.save_for_backward, o.tile_h, o.tile_w = int(bool(save)), int(tile_h), int(tile_w)
    o.kp_max = int(kp_max)
    o.trunc_tol = float(trunc_tol)
    o.pitch = int(pitch)
    return o


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _rows(t, name):
    """Device pointer and row pitch (elements) of a CUDA tensor whose rows are
    contiguous: [H, W] with strides (pitch, 1), or [B, H, W] with strides
    (H * pitch, pitch, 1); pitch >= W. A compact tensor has pitch W."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() not in (2, 3) or t.stride(-1) != 1:
        raise ValueError(f"{name} must be 2-D or 3-D with contiguous rows")
    H, W = t.shape[-2], t.shape[-1]
    pitch = t.stride(-2) if H > 1 else W
    if pitch < W:
        raise ValueError(f"{name}: rows overlap (pitch {pitch} < W {W})")
    if t.dim() == 3 and t.shape[0] > 1 and t.stride(0) != H * pitch:
        raise ValueError(f"{name}: images must be H * pitch elements apart")
    return ctypes.c_void_p(t.data_ptr()), int(pitch)


def _pitch_opts(opts, pitch):
    """A copy of opts with its row pitch set."""
    o = BfOpts()
    ctypes.pointer(o)[0] = opts
    o.pitch = int(pitch)
    return o


def _like_rows(t, pitch, dtype=None):
    """An uninitialised tensor shaped like t whose rows lie pitch elements apart."""
    import torch
    dtype = dtype or torch.float32
    if t.dim() == 2:
        return torch.empty((t.shape[0], pitch), dtype=dtype, device=t.device)[:, :t.shape[1]]
    B, H, W = t.shape
    return torch.empty((B, H, pitch), dtype=dtype, device=t.device)[:, :, :W]


def _check_bytes(t, need: int, name: str):
    """Raise if tensor t holds fewer than `need` bytes (the library cannot
    check the size of a raw device pointer)."""
    have = t.numel() * t.element_size()
    if have < need:
        raise ValueError(f"{name} holds {have} bytes, needs {need}")


def _in_dtype(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise ValueError("image must be float32 or bfloat16")


# ---- host-only helpers (no GPU needed) -------------------------------------

def bf_resolve_N(sigma_r: float, T: float = 1.0) -> int:
    return int(load().bf_resolve_N(float(sigma_r), float(T)))


def bf_coeffs(N: int):
    """a_k (FP64) for k = N mod 2, N mod 2 + 2, ..., N."""
    buf = (ctypes.c_double * 64)()
    K = load().bf_coeffs(int(N), buf, 64)
    if K < 0:
        raise ValueError(f"bf_coeffs: invalid N={N}")
    return [buf[i] for i in range(K)]


def bf_trunc_harmonics(N: int, r: int, trunc_tol: float) -> int:
    """Harmonics of q_N's expansion kept under trunc_tol (see bf_opts)."""
    return int(load().bf_trunc_harmonics(int(N), int(r), float(trunc_tol)))


def bf_gamma(sigma_r: float, T: float, N: int, gamma_mode: int = GAMMA_FIXED) -> float:
    return float(load().bf_gamma(float(sigma_r), float(T), int(N), int(gamma_mode)))


def bf_saved_bytes(H: int, W: int) -> int:
    return int(load().bf_saved_bytes(int(H), int(W)))


def bf_saved_index(y: int, x: int, H: int, W: int) -> int:
    """Index, in quads, of pixel (y, x)'s quad in a saved buffer; -1 outside the image."""
    i = int(load().bf_saved_index(int(y), int(x), int(H), int(W)))
    return -1 if i == ctypes.c_size_t(-1).value else i


def bf_backward_workspace_bytes(H: int, W: int, r: int, sigma_r: float = 0.2, T: float = 1.0,
                                N: int = 0, opts: BfOpts | None = None) -> int:
    return int(load().bf_backward_workspace_bytes(int(H), int(W), int(r), float(sigma_r),
                                                  float(T), int(N),
                                                  ctypes.byref(opts) if opts else None))


def bf_batch_workspace_bytes(descs, opts: BfOpts | None = None) -> int:
    arr = (BfDesc * len(descs))(*descs)
    return int(load().bf_batch_workspace_bytes(arr, len(descs), ctypes.byref(opts) if opts else None))


# ---- device entry points ----------------------------------------------------

def bf_forward(img, r: int, sigma_r: float, T: float = 1.0, N: int = 0, out=None,
               opts: BfOpts | None = None, saved=None, stream=None):
    """Forward filter of a 2-D CUDA tensor (float32 or bfloat16) -> float32.
    img and out may be row-pitched views (e.g. a column slice of a wider
    tensor); they must share one row pitch, which goes to the C ABI as
    bf_opts.pitch."""
    if img.dim() != 2:
        raise ValueError("img must be 2-D (H, W)")
    H, W = img.shape
    if opts is None:
        opts = _opts(in_dtype=_in_dtype(img))
    elif opts.in_dtype != _in_dtype(img):
        raise ValueError("opts.in_dtype does not match img.dtype")
    pimg, pitch = _rows(img, "img")
    if out is None:
        out = _like_rows(img, pitch)
    pout, opitch = _rows(out, "out")
    if tuple(out.shape) != (H, W) or opitch != pitch:
        raise ValueError("out must be (H, W) with the row pitch of img")
    if saved is not None:
        _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    o = _pitch_opts(opts, pitch if pitch != W else 0)
    st = load().bf_forward(pimg, H, W, int(r), float(sigma_r), float(T), int(N), pout,
                           ctypes.byref(o),
                           _dptr(saved, "saved") if saved is not None else None,
                           _stream_handle(stream))
    _check("bf_forward", st)
    return out


def bf_backward(img, out, grad_out, saved, r: int, sigma_r: float, T: float = 1.0, N: int = 0,
                grad_img=None, grad_sigma=None, workspace=None, opts: BfOpts | None = None,
                stream=None):
    """Adjoint pass; writes grad_img (H, W) and/or grad_sigma (1,) if given.
    grad_out and grad_img may be row-pitched views sharing one row pitch
    (bf_opts.pitch); the saved quads are compact."""
    H, W = img.shape
    if opts is None:
        opts = _opts(in_dtype=_in_dtype(img))
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    pg, pitch = _rows(grad_out, "grad_out")
    if tuple(grad_out.shape) != (H, W):
        raise ValueError("grad_out must be (H, W)")
    pgi = None
    if grad_img is not None:
        pgi, gpitch = _rows(grad_img, "grad_img")
        if tuple(grad_img.shape) != (H, W) or gpitch != pitch:
            raise ValueError("grad_img must be (H, W) with the row pitch of grad_out")
    o = _pitch_opts(opts, pitch if pitch != W else 0)
    st = load().bf_backward(ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(out.data_ptr()), pg,
                            _dptr(saved, "saved"), H, W, int(r), float(sigma_r), float(T), int(N),
                            pgi,
                            _dptr(grad_sigma, "grad_sigma") if grad_sigma is not None else None,
                            _dptr(workspace, "workspace") if workspace is not None else None,
                            ws_bytes, ctypes.byref(o), _stream_handle(stream))
    _check("bf_backward", st)


def bf_spatial_forward(img, r: int, M: int, sigma_r: float = 0.0, T: float = 1.0, N: int = 0,
                       out=None, opts: BfOpts | None = None, saved=None, stream=None):
    """Neighbourhood filter with the separable spatial kernel q_M(d1) q_M(d2)
    (q_M on [-(r+1/2), r+1/2]) and range kernel q_N (N = 0: none, i.e.
    Algorithm 1; N < 0: from sigma_r): Algorithm 2 with a shiftable spatial
    kernel. 2-D float32 CUDA tensor -> float32."""
    import torch
    if img.dim() != 2 or img.dtype != torch.float32:
        raise ValueError("img must be a 2-D float32 tensor")
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    _check_bytes(out, 4 * H * W, "out")
    if saved is not None:
        _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    st = load().bf_spatial_forward(_dptr(img, "img"), H, W, int(r), int(M), float(sigma_r),
                                   float(T), int(N), _dptr(out, "out"),
                                   ctypes.byref(opts) if opts is not None else None,
                                   _dptr(saved, "saved") if saved is not None else None,
                                   _stream_handle(stream))
    _check("bf_spatial_forward", st)
    return out


def bf_spatial_backward(grad_out, saved, r: int, M: int, sigma_r: float = 0.0, T: float = 1.0,
                        N: int = 0, grad_img=None, opts: BfOpts | None = None, stream=None):
    """Adjoint of bf_spatial_forward (saved = its quads); returns dL/dimg."""
    import torch
    H, W = grad_out.shape
    if grad_img is None:
        grad_img = torch.empty((H, W), dtype=torch.float32, device=grad_out.device)
    _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    _check_bytes(grad_img, 4 * H * W, "grad_img")
    st = load().bf_spatial_backward(_dptr(grad_out, "grad_out"), _dptr(saved, "saved"), H, W,
                                    int(r), int(M), float(sigma_r), float(T), int(N),
                                    _dptr(grad_img, "grad_img"),
                                    ctypes.byref(opts) if opts is not None else None,
                                    _stream_handle(stream))
    _check("bf_spatial_backward", st)
    return grad_img


def bf_poly_resolve_N(sigma_r: float, T: float = 1.0) -> int:
    return int(load().bf_poly_resolve_N(float(sigma_r), float(T)))


def bf_poly_forward(img, r: int, sigma_r: float = 0.0, T: float = 1.0, N: int = 0, out=None,
                    opts: BfOpts | None = None, saved=None, stream=None):
    """Bilateral filter with the polynomial range kernel p_N(t) = (1 -
    t^2/T^2)^N (Sec. 3) and the box window. 2-D float32 CUDA tensor."""
    import torch
    if img.dim() != 2 or img.dtype != torch.float32:
        raise ValueError("img must be a 2-D float32 tensor")
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    _check_bytes(out, 4 * H * W, "out")
    if saved is not None:
        _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    st = load().bf_poly_forward(_dptr(img, "img"), H, W, int(r), float(sigma_r), float(T),
                                int(N), _dptr(out, "out"),
                                ctypes.byref(opts) if opts is not None else None,
                                _dptr(saved, "saved") if saved is not None else None,
                                _stream_handle(stream))
    _check("bf_poly_forward", st)
    return out


def bf_poly_backward(grad_out, saved, r: int, sigma_r: float = 0.0, T: float = 1.0, N: int = 0,
                     grad_img=None, opts: BfOpts | None = None, stream=None):
    """Adjoint of bf_poly_forward (saved = its quads); returns dL/dimg."""
    import torch
    H, W = grad_out.shape
    if grad_img is None:
        grad_img = torch.empty((H, W), dtype=torch.float32, device=grad_out.device)
    _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    _check_bytes(grad_img, 4 * H * W, "grad_img")
    st = load().bf_poly_backward(_dptr(grad_out, "grad_out"), _dptr(saved, "saved"), H, W,
                                 int(r), float(sigma_r), float(T), int(N),
                                 _dptr(grad_img, "grad_img"),
                                 ctypes.byref(opts) if opts is not None else None,
                                 _stream_handle(stream))
    _check("bf_poly_backward", st)
    return grad_img


def bf_check_range(img, stream=None):
    """(min, max) of a 2-D float32/bfloat16 CUDA tensor as a device tensor of 2
    floats (the filters need max - min <= T)."""
    import torch
    if img.dim() != 2:
        raise ValueError("img must be 2-D")
    H, W = img.shape
    mm = torch.empty((2,), dtype=torch.float32, device=img.device)
    st = load().bf_check_range(_dptr(img, "img"), H, W, _in_dtype(img), _dptr(mm, "minmax"),
                               _stream_handle(stream))
    _check("bf_check_range", st)
    return mm


def bf_backward3d_workspace_bytes(B: int, H: int, W: int, r: int, sigma_r: float = 0.2,
                                  T: float = 1.0, N: int = 0, opts: BfOpts | None = None) -> int:
    return int(load().bf_backward3d_workspace_bytes(int(B), int(H), int(W), int(r),
                                                    float(sigma_r), float(T), int(N),
                                                    ctypes.byref(opts) if opts else None))


def bf_forward3d(img, r: int, sigma_r: float, T: float = 1.0, N: int = 0, out=None,
                 opts: BfOpts | None = None, saved=None, stream=None):
    """Forward filter of a [B, H, W] CUDA tensor in one launch -> float32."""
    import torch
    if img.dim() != 3:
        raise ValueError("img must be 3-D (B, H, W)")
    B, H, W = img.shape
    if opts is None:
        opts = _opts(in_dtype=_in_dtype(img))
    elif opts.in_dtype != _in_dtype(img):
        raise ValueError("opts.in_dtype does not match img.dtype")
    if out is None:
        out = torch.empty((B, H, W), dtype=torch.float32, device=img.device)
    _check_bytes(out, 4 * B * H * W, "out")
    if saved is not None:
        _check_bytes(saved, B * bf_saved_bytes(H, W), "saved")
    st = load().bf_forward3d(_dptr(img, "img"), B, H, W, int(r), float(sigma_r), float(T), int(N),
                             _dptr(out, "out"), ctypes.byref(opts),
                             _dptr(saved, "saved") if saved is not None else None,
                             _stream_handle(stream))
    _check("bf_forward3d", st)
    return out


def bf_backward3d(img, out, grad_out, saved, r: int, sigma_r: float, T: float = 1.0, N: int = 0,
                  grad_img=None, grad_sigma=None, workspace=None, opts: BfOpts | None = None,
                  stream=None):
    """Adjoint of bf_forward3d; grad_sigma (1,) receives the sum over images."""
    B, H, W = img.shape
    if opts is None:
        opts = _opts(in_dtype=_in_dtype(img))
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check_bytes(saved, B * bf_saved_bytes(H, W), "saved")
    _check_bytes(grad_out, 4 * B * H * W, "grad_out")
    if grad_img is not None:
        _check_bytes(grad_img, 4 * B * H * W, "grad_img")
    st = load().bf_backward3d(_dptr(img, "img"), _dptr(out, "out"), _dptr(grad_out, "grad_out"),
                              _dptr(saved, "saved"), B, H, W, int(r), float(sigma_r), float(T),
                              int(N),
                              _dptr(grad_img, "grad_img") if grad_img is not None else None,
                              _dptr(grad_sigma, "grad_sigma") if grad_sigma is not None else None,
                              _dptr(workspace, "workspace") if workspace is not None else None,
                              ws_bytes, ctypes.byref(opts), _stream_handle(stream))
    _check("bf_backward3d", st)


def make_descs(imgs, outs, rs, sigmas, T=1.0, Ns=None, dens=None):
    """Batch descriptors; each image, output (and den, if given) may be a
    row-pitched view sharing one row pitch per image."""
    descs = []
    for i, (im, o) in enumerate(zip(imgs, outs)):
        d = BfDesc()
        pi, pitch = _rows(im, "img")
        po, opitch = _rows(o, "out")
        if opitch != pitch or tuple(o.shape) != tuple(im.shape):
            raise ValueError("out must match img in shape and row pitch")
        d.img, d.out = pi.value, po.value
        d.den = None
        if dens is not None and dens[i] is not None:
            pd, dpitch = _rows(dens[i], "den")
            if dpitch != pitch or tuple(dens[i].shape) != tuple(im.shape):
                raise ValueError("den must match img in shape and row pitch")
            d.den = pd.value
        d.H, d.W = int(im.shape[0]), int(im.shape[1])
        d.pitch = pitch if pitch != d.W else 0
        d.r, d.N = int(rs[i]), int(Ns[i]) if Ns is not None else 0
        d.sigma_r, d.T = float(sigmas[i]), float(T)
        descs.append(d)
    return descs


def bf_batch_prepare(descs, workspace, opts: BfOpts | None = None, stream=None):
    arr = (BfDesc * len(descs))(*descs)
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().bf_batch_prepare(arr, len(descs), ctypes.byref(opts) if opts else None,
                                 _dptr(workspace, "workspace"), ws_bytes, _stream_handle(stream))
    _check("bf_batch_prepare", st)


def bf_batch_launch(workspace, opts: BfOpts | None = None, stream=None):
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().bf_batch_launch(_dptr(workspace, "workspace"), ws_bytes,
                                ctypes.byref(opts) if opts else None, _stream_handle(stream))
    _check("bf_batch_launch", st)


def bf_batch(descs, workspace, opts: BfOpts | None = None, stream=None):
    arr = (BfDesc * len(descs))(*descs)
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().bf_batch(arr, len(descs), ctypes.byref(opts) if opts else None,
                         _dptr(workspace, "workspace"), ws_bytes, _stream_handle(stream))
    _check("bf_batch", st)


# ---- autograd ----------------------------------------------------------------

def _make_function():
    import torch

    class BilateralCosN(torch.autograd.Function):
        """out = bilateral(f) with range kernel cos^N; differentiable in f and
        sigma_r (a 0-d tensor). Forward saves per pixel (f, 1/den, out, centre
        derivative term); the adjoint kernel recomputes the stack from them."""

        @staticmethod
        def forward(ctx, f, sigma_r, r, T, N, kahan, gamma_mode, trunc_tol):
            s = float(sigma_r)
            if N <= 0:
                N = bf_resolve_N(s, T)
            squeeze = f.dim() == 2
            fb = f.unsqueeze(0) if squeeze else f
            fb = fb.contiguous()
            B, H, W = fb.shape
            opts = _opts(kahan=kahan, gamma_mode=gamma_mode, in_dtype=_in_dtype(fb), save=True,
                         trunc_tol=trunc_tol)
            out = torch.empty((B, H, W), dtype=torch.float32, device=f.device)
            saved = torch.empty((B, H, W, 4), dtype=torch.float32, device=f.device)
            bf_forward3d(fb, r, s, T, N, out=out, opts=opts, saved=saved)
            ctx.save_for_backward(fb, out, saved)
            ctx.cfg = (r, s, T, N, kahan, gamma_mode, trunc_tol, squeeze)
            return out[0] if squeeze else out

        @staticmethod
        def backward(ctx, g):
            fb, out, saved = ctx.saved_tensors
            r, s, T, N, kahan, gamma_mode, trunc_tol, squeeze = ctx.cfg
            g = g.unsqueeze(0) if squeeze else g
            g = g.contiguous().float()
            B, H, W = fb.shape
            opts = _opts(kahan=kahan, gamma_mode=gamma_mode, in_dtype=_in_dtype(fb),
                         trunc_tol=trunc_tol)
            need_f = ctx.needs_input_grad[0]
            need_s = ctx.needs_input_grad[1]
            gf = torch.empty((B, H, W), dtype=torch.float32, device=fb.device) if need_f else None
            gs = torch.zeros((1,), dtype=torch.float32, device=fb.device) if need_s else None
            ws = None
            nb = bf_backward3d_workspace_bytes(B, H, W, r, s, T, N, opts)
            if nb > 0:
                ws = torch.empty((max(1, (nb + 3) // 4),), dtype=torch.float32, device=fb.device)
            bf_backward3d(fb, out, g, saved, r, s, T, N, grad_img=gf, grad_sigma=gs,
                          workspace=ws, opts=opts)
            if gf is not None:
                gf = gf[0] if squeeze else gf
                gf = gf.to(fb.dtype)
            gsig = gs[0] if gs is not None else None
            return gf, gsig, None, None, None, None, None, None

    return BilateralCosN


_fn = None
_spatial_fn = None


def _as_batch(x):
    """[H, W] or [B, H, W] -> contiguous [B, H, W] (a view when possible)."""
    if x.dim() == 2:
        x = x.unsqueeze(0)
    if x.dim() != 3:
        raise ValueError("expected an [H, W] or [B, H, W] tensor")
    return x.contiguous()


def _make_spatial_function():
    import torch

    class BilateralSpatial(torch.autograd.Function):
        """Algorithm 2 with the q_M x q_M spatial kernel and range q_N (Algorithm
        1 for N = 0); differentiable in the image."""

        @staticmethod
        def forward(ctx, f, r, M, sigma_r, T, N):
            fb = _as_batch(f)
            B, H, W = fb.shape
            saved = torch.empty((B, H, W, 4), dtype=torch.float32, device=f.device)
            out = torch.empty((B, H, W), dtype=torch.float32, device=f.device)
            for b in range(B):  # one launch per image, in order on the current stream
                bf_spatial_forward(fb[b], r, M, sigma_r, T, N, out=out[b], saved=saved[b])
            ctx.save_for_backward(saved)
            ctx.cfg = (r, M, sigma_r, T, N, f.dim())
            return out[0] if f.dim() == 2 else out

        @staticmethod
        def backward(ctx, g):
            (saved,) = ctx.saved_tensors
            r, M, sigma_r, T, N, dim = ctx.cfg
            gb = _as_batch(g.float())
            gi = torch.empty_like(gb)
            for b in range(gb.shape[0]):
                bf_spatial_backward(gb[b], saved[b], r, M, sigma_r, T, N, grad_img=gi[b])
            return (gi[0] if dim == 2 else gi), None, None, None, None, None

    return BilateralSpatial


_poly_fn = None


def _make_poly_function():
    import torch

    class BilateralPoly(torch.autograd.Function):
        """Bilateral filter with the polynomial range kernel p_N; differentiable
        in the image."""

        @staticmethod
        def forward(ctx, f, r, sigma_r, T, N):
            fb = _as_batch(f)
            B, H, W = fb.shape
            saved = torch.empty((B, H, W, 4), dtype=torch.float32, device=f.device)
            out = torch.empty((B, H, W), dtype=torch.float32, device=f.device)
            for b in range(B):  # one launch per image, in order on the current stream
                bf_poly_forward(fb[b], r, sigma_r, T, N, out=out[b], saved=saved[b])
            ctx.save_for_backward(saved)
            ctx.cfg = (r, sigma_r, T, N, f.dim())
            return out[0] if f.dim() == 2 else out

        @staticmethod
        def backward(ctx, g):
            (saved,) = ctx.saved_tensors
            r, sigma_r, T, N, dim = ctx.cfg
            gb = _as_batch(g.float())
            gi = torch.empty_like(gb)
            for b in range(gb.shape[0]):
                bf_poly_backward(gb[b], saved[b], r, sigma_r, T, N, grad_img=gi[b])
            return (gi[0] if dim == 2 else gi), None, None, None, None

    return BilateralPoly


def bilateral_poly(f, r: int, sigma_r: float = 0.0, T: float = 1.0, N: int = 0):
    """Bilateral filter with range kernel p_N(t) = (1 - t^2/T^2)^N (N <= 0:
    from sigma_r) and the box window, of an [H, W] or [B, H, W] float32 CUDA
    tensor, differentiable in f."""
    global _poly_fn
    if _poly_fn is None:
        _poly_fn = _make_poly_function()
    return _poly_fn.apply(f, int(r), float(sigma_r), float(T), int(N))


def bilateral_spatial(f, r: int, M: int, sigma_r: float = 0.0, T: float = 1.0, N: int = 0):
    """Neighbourhood filter with the separable spatial kernel q_M x q_M and
    range kernel q_N (N = 0: the linear filter of Algorithm 1; N < 0: from
    sigma_r) of an [H, W] or [B, H, W] float32 CUDA tensor, differentiable in f."""
    global _spatial_fn
    if _spatial_fn is None:
        _spatial_fn = _make_spatial_function()
    return _spatial_fn.apply(f, int(r), int(M), float(sigma_r), float(T), int(N))


def bilateral(f, r: int, sigma_r, T: float = 1.0, N: int = 0, kahan: bool = False,
              gamma_mode: int = GAMMA_FIXED, trunc_tol: float = 0.0):
    """Raised-cosine bilateral filter of f ([H, W] or [B, H, W], CUDA, float32
    or bfloat16) with a (2r+1)^2 box window. sigma_r may be a float or a 0-d
    tensor (to get dL/dsigma_r); N <= 0 derives N from sigma_r. trunc_tol > 0
    keeps only the lowest harmonics of q_N's expansion (see bf_opts)."""
    import torch
    global _fn
    if _fn is None:
        _fn = _make_function()
    if not isinstance(sigma_r, torch.Tensor):
        sigma_r = torch.tensor(float(sigma_r), dtype=torch.float32)
    return _fn.apply(f, sigma_r, int(r), float(T), int(N), bool(kahan), int(gamma_mode),
                     float(trunc_tol))


def bf_backward_noalloc(img, out, grad_out, saved, r: int, sigma_r: float, T: float = 1.0,
                        N: int = 0, grad_img=None, grad_sigma=None, opts: BfOpts | None = None,
                        stream=None):
    """bf_backward for callers that cannot allocate device memory: the
    dL/dsigma_r partial sums use a fixed scratch array inside the library
    instead of a caller workspace. The first call on a device looks up that
    array's address; calls that overlap on the GPU share it and race."""
    lib = load()
    f = lib.bf_backward_noalloc
    vp, c_int, c_float = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    f.restype = c_int
    f.argtypes = [vp, vp, vp, vp, c_int, c_int, c_int, c_float, c_float, c_int, vp, vp,
                  ctypes.POINTER(BfOpts), vp]
    H, W = img.shape
    if opts is None:
        opts = _opts(in_dtype=_in_dtype(img))
    _check_bytes(saved, bf_saved_bytes(H, W), "saved")
    st = f(_dptr(img, "img"), _dptr(out, "out"), _dptr(grad_out, "grad_out"),
           _dptr(saved, "saved"), H, W, int(r), float(sigma_r), float(T), int(N),
           _dptr(grad_img, "grad_img") if grad_img is not None else None,
           _dptr(grad_sigma, "grad_sigma") if grad_sigma is not None else None,
           ctypes.byref(opts), _stream_handle(stream))
    _check("bf_backward_noalloc", st)
