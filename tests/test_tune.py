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
