"""Measured pipe throughputs of the GPU (FP32 FMA scalar and FP32x2, FP32 add,
shuffle, shared-memory loads, MUFU), from the small CUDA program peak.cu.

Used by the bench to report the measured FP32 FMA peak beside the peak
derived from unit counts and clocks.
"""
from __future__ import annotations

import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "peak.cu")
EXE = os.path.join(HERE, "_build", "peak")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def build(force: bool = False) -> str:
    if not force and os.path.exists(EXE) and os.path.getmtime(EXE) >= os.path.getmtime(SRC):
        return EXE
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", EXE, SRC],
                   check=True)
    return EXE


def measure() -> dict:
    """Run the micro-benchmarks on the current GPU (about a second)."""
    out = subprocess.run([build()], check=True, capture_output=True, text=True).stdout
    return json.loads(out.strip().splitlines()[-1])
