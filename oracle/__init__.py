"""FP64 CPU oracle for the raised-cosine bilateral filter.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (the CUDA library and its Python binding) never
imports, links or calls it, and it shares no code with them.

The C file ``bf_oracle.c`` holds the arithmetic (plain definition of Eq.
filter2 with the box window of Sec. 2 and q_N of Sec. 3, the exact-Gaussian
filter, and the direct-form gradient); this module compiles it with gcc and
wraps it with ctypes. The helpers below restate the parameter rules (gamma of
q_N, the order rule from the Gaussian-approximation theorem) independently of
the product's host code.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbf_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP). Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_weight.restype = ctypes.c_double
            lib.oracle_weight.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
            lib.oracle_bf_cosn_rows.restype = ctypes.c_int
            lib.oracle_bf_cosn_rows.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, _dp, _dp]
            lib.oracle_bf_cosn_points.restype = ctypes.c_int
            lib.oracle_bf_cosn_points.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_double, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_longlong),
                                                  ctypes.c_longlong, _dp, _dp]
            lib.oracle_bf_gauss.restype = ctypes.c_int
            lib.oracle_bf_gauss.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, _dp]
            lib.oracle_bf_gauss_points.restype = ctypes.c_int
            lib.oracle_bf_gauss_points.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double,
                                                   ctypes.POINTER(ctypes.c_longlong),
                                                   ctypes.c_longlong, _dp]
            lib.oracle_bf_grad.restype = ctypes.c_int
            lib.oracle_bf_grad.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int, _dp, _dp]
            lib.oracle_bf_general_rows.restype = ctypes.c_int
            lib.oracle_bf_general_rows.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                   _dp, _dp]
            lib.oracle_trunc_weight.restype = ctypes.c_double
            lib.oracle_trunc_weight.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int]
            lib.oracle_spatial_weight.restype = ctypes.c_double
            lib.oracle_spatial_weight.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            _lib = lib
    return _lib


def _as_f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.ndim != 2:
        raise ValueError("image must be 2-D (H, W)")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().oracle_num_threads())


def gamma_fixed(T: float) -> float:
    """gamma of q_N(t) = cos^N(pi t / (2T)) (Sec. 3)."""
    return math.pi / (2.0 * T)


def resolve_N(sigma_r: float, T: float) -> int:
    """Order rule from the Gaussian-approximation theorem (Eq. approx2):
    cos^N(gamma t) ~ exp(-N gamma^2 t^2 / 2), so matching the variance
    sigma_r^2 gives N = 1/(gamma sigma_r)^2; round up so the effective width
    does not exceed sigma_r (and N is above the non-negativity threshold
    discussed at the end of Sec. 3)."""
    g = gamma_fixed(T)
    v = 1.0 / (g * sigma_r) ** 2
    return max(1, int(math.ceil(v - 1e-9)))


def gamma_from_sigma(sigma_r: float, N: int) -> float:
    """gamma with the Gaussian limit's variance equal to sigma_r^2:
    gamma sqrt(N) = 1/sigma_r (Eq. approx2 rescaled)."""
    return 1.0 / (sigma_r * math.sqrt(N))


def weight(t: float, gamma: float, N: int) -> float:
    """q_N range weight cos^N(gamma t), evaluated directly."""
    return float(_load().oracle_weight(float(t), float(gamma), int(N)))


def bilateral(f, r: int, gamma: float, N: int, rows=None, return_den=False):
    """Direct O(r^2) raised-cosine bilateral filter (Eq. filter2, box window,
    q_N), truncated at the border. ``rows=(row0, row1)`` limits the output
    rows computed (the whole image is still read)."""
    f = _as_f64(f)
    H, W = f.shape
    r0, r1 = (0, H) if rows is None else (max(0, rows[0]), min(H, rows[1]))
    out = np.empty((r1 - r0, W), np.float64)
    den = np.empty((r1 - r0, W), np.float64)
    rc = _load().oracle_bf_cosn_rows(_ptr(f), H, W, int(r), float(gamma), int(N), r0, r1,
                                     _ptr(out), _ptr(den))
    if rc != 0:
        raise ValueError(f"oracle_bf_cosn_rows failed ({rc})")
    return (out, den) if return_den else out


def bilateral_points(f, r: int, gamma: float, N: int, idx, return_den=False):
    """Direct filter at the flat pixel indices ``idx`` only."""
    f = _as_f64(f)
    H, W = f.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(idx.shape[0], np.float64)
    den = np.empty(idx.shape[0], np.float64)
    rc = _load().oracle_bf_cosn_points(_ptr(f), H, W, int(r), float(gamma), int(N),
                                       idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                       idx.shape[0], _ptr(out), _ptr(den))
    if rc != 0:
        raise ValueError(f"oracle_bf_cosn_points failed ({rc})")
    return (out, den) if return_den else out


def bilateral_gauss(f, r: int, sigma: float):
    """Exact-Gaussian bilateral filter over the same window (reported only)."""
    f = _as_f64(f)
    H, W = f.shape
    out = np.empty((H, W), np.float64)
    rc = _load().oracle_bf_gauss(_ptr(f), H, W, int(r), float(sigma), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_bf_gauss failed ({rc})")
    return out


def bilateral_gauss_points(f, r: int, sigma: float, idx):
    """Exact-Gaussian bilateral filter at the flat pixel indices ``idx`` only."""
    f = _as_f64(f)
    H, W = f.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(idx.shape[0], np.float64)
    rc = _load().oracle_bf_gauss_points(_ptr(f), H, W, int(r), float(sigma),
                                        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                        idx.shape[0], _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_bf_gauss_points failed ({rc})")
    return out


def bilateral_grad(f, g, r: int, gamma: float, N: int):
    """(dL/df, dL/dgamma) for L = sum(g * out), from the direct form."""
    f = _as_f64(f)
    g = _as_f64(g)
    if g.shape != f.shape:
        raise ValueError("g must match f")
    H, W = f.shape
    gf = np.empty((H, W), np.float64)
    gg = ctypes.c_double(0.0)
    rc = _load().oracle_bf_grad(_ptr(f), _ptr(g), H, W, int(r), float(gamma), int(N),
                                _ptr(gf), ctypes.byref(gg))
    if rc != 0:
        raise ValueError(f"oracle_bf_grad failed ({rc})")
    return gf, float(gg.value)


# ---- generalised filters (Algorithm 1, Algorithm 2 with a shiftable spatial
# kernel, truncated expansion, polynomial range kernel) ---------------------

SPATIAL_BOX, SPATIAL_QM = 0, 1
RANGE_NONE, RANGE_COSN, RANGE_TRUNC, RANGE_POLY = 0, 1, 2, 3


def trunc_weight(t: float, gamma: float, N: int, K_keep: int) -> float:
    """q_N's shift expansion cut to its K_keep lowest harmonics, evaluated
    term by term (end of Sec. 3: discarding the less significant basis
    functions)."""
    return float(_load().oracle_trunc_weight(float(t), float(gamma), int(N), int(K_keep)))


def spatial_weight(d: int, r: int, M: int) -> float:
    """1-D factor of the separable spatial kernel q_M(d) = cos^M(pi d / (2 Ts)),
    Ts = r + 1/2 (Sec. 3, separable kernels)."""
    return float(_load().oracle_spatial_weight(int(d), int(r), int(M)))


def bilateral_general(f, r: int, spatial: int = SPATIAL_BOX, M: int = 0,
                      range_kind: int = RANGE_COSN, gamma: float = math.pi / 2, N: int = 0,
                      K_keep: int = 0, Tr: float = 1.0, rows=None, return_den=False):
    """Direct O(r^2) neighbourhood filter with spatial kernel box or
    q_M(d1) q_M(d2) and range kernel none (Algorithm 1), q_N, truncated q_N or
    p_N (Algorithm 2); truncated window at the border."""
    f = _as_f64(f)
    H, W = f.shape
    r0, r1 = (0, H) if rows is None else (max(0, rows[0]), min(H, rows[1]))
    out = np.empty((r1 - r0, W), np.float64)
    den = np.empty((r1 - r0, W), np.float64)
    rc = _load().oracle_bf_general_rows(_ptr(f), H, W, int(r), int(spatial), int(M),
                                        int(range_kind), float(gamma), int(N), int(K_keep),
                                        float(Tr), r0, r1, _ptr(out), _ptr(den))
    if rc != 0:
        raise ValueError(f"oracle_bf_general_rows failed ({rc})")
    return (out, den) if return_den else out
