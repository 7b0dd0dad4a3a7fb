"""Autotuner host logic (CPU, fake timer) and a GPU check that tuned launch
shapes give the same filter."""
import math

import numpy as np
import pytest
import torch

import paper_1107_4617_gb300 as bf
from paper_1107_4617_gb300 import synth, tune


def test_bucket_and_candidates():
    assert tune.bucket(4096, 4096, 10, 21, "f32", True) == "4096x4096|r10|K22|f32|fb"
    assert tune.bucket(3000, 1025, 7, 10, "bf16", False) == "4096x2048|r7|K10|bf16|f"
    c = tune.candidates(10, 21, allow_chunks=True)
    assert {x["tile_w"] for x in c} == {128, 256}
    assert any(x["kp_max"] == 6 for x in c)
    assert all(x["tile_w"] == 256 for x in tune.candidates(60, 5, allow_chunks=False))
    assert tune.choose([({"a": 1}, 3.0), ({"a": 2}, 1.0), ({"a": 3}, 1.0)])[0] == {"a": 2}


def test_tune_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("BF_TUNE_CACHE", str(tmp_path / "t.json"))
    calls = []

    def fake(c):
        calls.append(c)
        return 1.0 + (c["tile_w"] == 256) + c["tile_h"] / 1e4 + (c["kp_max"] > 0)

    best = tune.tune(512, 512, 5, 0.1, timer=fake)
    assert best["tile_w"] == 128 and best["tile_h"] == 0 and best["kp_max"] == 0
    n = len(calls)
    again = tune.tune(512, 500, 5, 0.1, timer=fake)  # same bucket: served from the cache
    assert again == best and len(calls) == n


def _descs(specs):
    out = []
    for sp in specs:
        d = bf.BfDesc()
        d.H, d.W, d.r, d.N, d.sigma_r, d.T = sp["H"], sp["W"], sp["r"], 0, sp["sigma_r"], 1.0
        out.append(d)
    return out


def test_batch_signature_and_candidates():
    specs = synth.batch_specs(6, seed=3)
    a, b = _descs(specs), _descs(specs)
    b[0].img = 12345  # addresses do not enter the key
    assert tune.batch_signature(a) == tune.batch_signature(b)
    b[2].r += 1
    assert tune.batch_signature(a) != tune.batch_signature(b)
    assert tune.batch_signature(a).startswith("batch6|")
    c = tune.batch_candidates([3, 30])
    assert {x["tile_w"] for x in c} == {0, 256} and {"tile_w": 0, "tile_h": 0} in c
    # a half-width too wide for a 256-column strip leaves only the per-image rule
    assert {x["tile_w"] for x in tune.batch_candidates([3, 121])} == {0}


def test_tune_batch_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("BF_TUNE_CACHE", str(tmp_path / "t.json"))
    descs = _descs(synth.batch_specs(5, seed=9))
    calls = []

    def fake(c):
        calls.append(c)
        return 2.0 - (c["tile_h"] == 768) + (c["tile_w"] == 256)

    best = tune.tune_batch(descs, timer=fake)
    assert best["tile_w"] == 0 and best["tile_h"] == 768 and best["ms"] == 1.0
    n = len(calls)
    assert tune.tune_batch(_descs(synth.batch_specs(5, seed=9)), timer=fake) == best
    assert len(calls) == n  # served from the cache
    other = tune.tune_batch(_descs(synth.batch_specs(5, seed=10)), timer=fake)
    assert len(calls) == 2 * n and other["tile_h"] == 768


@pytest.mark.gpu
def test_tuned_batch_same_filter(cuda_lib, tmp_path, monkeypatch):
    """Every tried batch launch shape gives the filter of the separate launches."""
    monkeypatch.setenv("BF_TUNE_CACHE", str(tmp_path / "t.json"))
    specs = synth.batch_specs(12, seed=5, side_lo=40, side_hi=700)
    imgs = [torch.from_numpy(synth.rectangles(sp["H"], sp["W"], seed=sp["seed"])).cuda()
            for sp in specs]
    outs = [torch.empty_like(im) for im in imgs]
    descs = bf.make_descs(imgs, outs, [sp["r"] for sp in specs], [sp["sigma_r"] for sp in specs])
    refs = [bf.bf_forward(im, sp["r"], sp["sigma_r"]) for sp, im in zip(specs, imgs)]
    for c in tune.batch_candidates([sp["r"] for sp in specs]):
        for o in outs:
            o.fill_(float("nan"))
        o = bf._opts(tile_w=c["tile_w"], tile_h=c["tile_h"])
        ws = torch.empty(((bf.bf_batch_workspace_bytes(descs, o) + 3) // 4,), device="cuda")
        bf.bf_batch(descs, ws, o)
        torch.cuda.synchronize()
        # different band / strip splits round differently: each side is within
        # the parity tolerance 1e-4 * max(|v|, 1e-2 T) of the exact filter
        for a, b in zip(outs, refs):
            tol = 2e-4 * torch.clamp(torch.abs(b), min=1e-2)
            assert bool(torch.all(torch.abs(a - b) <= tol)), c
    o = tune.tuned_batch_opts(descs)
    assert (o.tile_w, o.tile_h) in {(c["tile_w"], c["tile_h"]) for c in
                                    tune.batch_candidates([sp["r"] for sp in specs])}


@pytest.mark.gpu
def test_tuned_opts_same_filter(cuda_lib, tmp_path, monkeypatch):
    monkeypatch.setenv("BF_TUNE_CACHE", str(tmp_path / "t.json"))
    H, W, r, sigma = 600, 700, 10, 0.1
    o = tune.tuned_opts(H, W, r, sigma)
    f = torch.from_numpy(synth.rectangles(H, W, seed=4)).cuda()
    sv = torch.empty((H, W, 4), device="cuda")
    a = bf.bf_forward(f, r, sigma, 1.0, 0, opts=o, saved=sv)
    b = bf.bf_forward(f, r, sigma, 1.0, 0)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(a - b)).item() <= 1e-5
