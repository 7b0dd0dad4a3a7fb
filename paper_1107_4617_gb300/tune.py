"""Autotuner for the filter's launch shape.

For a workload (image size, r, number of harmonics, input dtype, whether the
adjoint is run) it times the forward (and adjoint) for a set of candidate
launch shapes on the current GPU and keeps the fastest:

* tile_w: threads per strip (128 or 256; each thread owns one column, so a
  strip yields tile_w - 2r output columns),
* tile_h: rows per band (0 = the built-in one-wave choice, or fixed heights),
* kp_max: harmonic pairs per launch (fewer registers per thread, more
  resident warps, at the cost of repeating the per-row overhead per chunk;
  only tried when the saved buffers can hold the chunk partials).

For a batch of uneven images (``tune_batch``) the same holds for the one
launch shape that every tile of the persistent batch launch uses: the band
height and the strip width, tried only where every image admits the width.

Results go to a JSON cache (``$BF_TUNE_CACHE`` or
``~/.cache/paper_1107_4617_gb300/tune.json``) keyed by GPU name and a bucket
of the workload, so later calls reuse them without timing.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
import threading

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("BF_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1107_4617_gb300", "tune.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def bucket(H: int, W: int, r: int, K: int, dtype: str, adjoint: bool) -> str:
    """Workload bucket: image sides rounded to powers of two, r exact, the
    harmonic count rounded up to even."""
    def p2(x):
        return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))
    return f"{p2(H)}x{p2(W)}|r{r}|K{K + (K & 1)}|{dtype}|{'fb' if adjoint else 'f'}"


def candidates(r: int, K: int, allow_chunks: bool):
    out = []
    for tw in (128, 256):
        if tw - 2 * r < 16:
            continue
        for th in (0, 256, 512, 1024):
            out.append({"tile_w": tw, "tile_h": th, "kp_max": 0})
            if allow_chunks and K > 12:
                out.append({"tile_w": tw, "tile_h": th, "kp_max": 6})
    return out


def choose(timings):
    """The candidate with the smallest time; ties keep the earlier one."""
    best = None
    for cand, t in timings:
        if best is None or t < best[1]:
            best = (cand, t)
    return best


def tune(H: int, W: int, r: int, sigma_r: float, T: float = 1.0, N: int = 0,
         dtype=None, adjoint: bool = True, reps: int = 3, use_cache: bool = True,
         timer=None):
    """Best launch shape for the workload: dict(tile_w, tile_h, kp_max, ms).
    `timer(cand) -> ms` may replace the GPU timing (tests)."""
    import torch

    import paper_1107_4617_gb300 as bf
    dtype = dtype or torch.float32
    if N <= 0:
        N = bf.bf_resolve_N(sigma_r, T)
    K = N // 2 + 1
    dname = "bf16" if dtype == torch.bfloat16 else "f32"
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    key = f"{gpu}|{bucket(H, W, r, K, dname, adjoint)}"
    path = cache_path()
    if use_cache:
        with _lock:
            hit = _load(path).get(key)
        if hit:
            return hit
    cands = candidates(r, K, allow_chunks=adjoint)
    if timer is None:
        timer = _gpu_timer(H, W, r, sigma_r, T, N, dtype, adjoint, reps)
    timings = [(c, timer(c)) for c in cands]
    best, ms = choose(timings)
    res = dict(best, ms=ms)
    if use_cache:
        with _lock:
            data = _load(path)
            data[key] = res
            _store(path, data)
    return res


def _gpu_timer(H, W, r, sigma_r, T, N, dtype, adjoint, reps):
    import torch

    import paper_1107_4617_gb300 as bf
    from paper_1107_4617_gb300 import synth
    dev = torch.device("cuda")
    img = torch.from_numpy(synth.rectangles(H, W, seed=0)).to(dev).to(dtype)
    g = torch.from_numpy(synth.weights((H, W), seed=1)).to(dev)
    out = torch.empty((H, W), device=dev)
    sv = torch.empty((H, W, 4), device=dev)  # bf_saved_bytes(H, W): one 16-byte quad per pixel
    gi = torch.empty((H, W), device=dev)
    flush = torch.empty((64 << 20,), device=dev)
    in_dtype = bf.BF16 if dtype == torch.bfloat16 else bf.F32

    def run(c):
        o = bf._opts(in_dtype=in_dtype, save=adjoint, tile_w=c["tile_w"], tile_h=c["tile_h"],
                     kp_max=c["kp_max"])
        bf.bf_forward(img, r, sigma_r, T, N, out=out, opts=o, saved=sv if adjoint else None)
        if adjoint:
            nb = bf.bf_backward_workspace_bytes(H, W, r, sigma_r, T, N, o)
            ws = torch.empty((max(1, (nb + 3) // 4),), device=dev) if nb else None
            bf.bf_backward(img, out, g, sv, r, sigma_r, T, N, grad_img=gi, workspace=ws, opts=o)

    def timer(c):
        run(c)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run(c)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ts.sort()
        return ts[len(ts) // 2]

    return timer


def tuned_opts(H: int, W: int, r: int, sigma_r: float, T: float = 1.0, N: int = 0, dtype=None,
               adjoint: bool = True, **kw):
    """BfOpts carrying the tuned launch shape (tuning on a cache miss)."""
    import torch

    import paper_1107_4617_gb300 as bf
    dtype = dtype or torch.float32
    best = tune(H, W, r, sigma_r, T, N, dtype=dtype, adjoint=adjoint)
    return bf._opts(in_dtype=bf.BF16 if dtype == torch.bfloat16 else bf.F32, save=adjoint,
                    tile_w=best["tile_w"], tile_h=best["tile_h"], kp_max=best["kp_max"], **kw)


def batch_signature(descs) -> str:
    """Cache key of a batch: the image count and a digest of every image's
    (H, W, r, N, sigma_r, T), in order. Buffer addresses do not enter."""
    h = hashlib.sha1()
    for d in descs:
        h.update(f"{d.H},{d.W},{d.r},{d.N},{d.sigma_r:.6g},{d.T:.6g};".encode())
    return f"batch{len(descs)}|{h.hexdigest()[:16]}"


def batch_candidates(rs):
    """Launch shapes for a batch whose largest half-width is max(rs): strip
    width 0 (each image's own rule) or 256 where every strip keeps >= 16 output
    columns, and band heights 0 (the built-in rule) and fixed ones."""
    rmax = max(rs) if rs else 0
    out = []
    for tw in (0, 256):
        if tw and tw - 2 * rmax < 16:
            continue
        for th in (0, 256, 384, 768, 1024, 1536, 2048):
            out.append({"tile_w": tw, "tile_h": th})
    return out


def tune_batch(descs, reps: int = 3, use_cache: bool = True, timer=None):
    """Best launch shape for the persistent batch launch over `descs`:
    dict(tile_w, tile_h, ms). The GPU timing writes each image's filtered
    result into its `out` buffer. `timer(cand) -> ms` may replace it (tests)."""
    import torch
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    key = f"{gpu}|{batch_signature(descs)}"
    path = cache_path()
    if use_cache:
        with _lock:
            hit = _load(path).get(key)
        if hit:
            return hit
    cands = batch_candidates([d.r for d in descs])
    if timer is None:
        timer = _gpu_batch_timer(descs, reps)
    best, ms = choose([(c, timer(c)) for c in cands])
    res = dict(best, ms=ms)
    if use_cache:
        with _lock:
            data = _load(path)
            data[key] = res
            _store(path, data)
    return res


def _gpu_batch_timer(descs, reps):
    import torch

    import paper_1107_4617_gb300 as bf
    dev = torch.device("cuda")
    flush = torch.empty((64 << 20,), device=dev)

    def timer(c):
        o = bf._opts(tile_w=c["tile_w"], tile_h=c["tile_h"])
        nb = bf.bf_batch_workspace_bytes(descs, o)
        ws = torch.empty((max(1, (nb + 3) // 4),), device=dev)
        bf.bf_batch_prepare(descs, ws, o)
        bf.bf_batch_launch(ws, o)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bf.bf_batch_launch(ws, o)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ts.sort()
        return ts[len(ts) // 2]

    return timer


def tuned_batch_opts(descs, **kw):
    """BfOpts carrying the tuned batch launch shape (tuning on a cache miss)."""
    import paper_1107_4617_gb300 as bf
    best = tune_batch(descs)
    return bf._opts(tile_w=best["tile_w"], tile_h=best["tile_h"], **kw)
