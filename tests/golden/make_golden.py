"""Writes the text fixtures in this folder. Run from the repository root:

    python tests/golden/make_golden.py

The paper prints no worked example of the filter's output (its only numbers
are the MATLAB timings of Sec. 2), so every expected value here is the FP64
oracle's: the direct definition of Eq. filter2 with the box window of Sec. 2
and the range kernel q_N(t) = cos^N(gamma t), gamma = pi / (2T), of Sec. 3,
and its direct-form gradient. This script calls only ``oracle`` for them; the
input image comes from the seeded generator ``synth`` and is stored too
(rounded to FP32, the type the filter takes), so the fixtures do not depend on
the generator staying the same.
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1107_4617_gb300 import synth  # noqa: E402

H, W = 24, 20
GAMMA = math.pi / 2  # T = 1
# (r, N): odd and even orders, the headline order 41, and 50 (above the
# 43 harmonics one pass of the fast path holds)
CASES = [(2, 3), (1, 4), (3, 41), (2, 50)]
GRAD_CASES = [(2, 3), (3, 41)]
SOURCE = ("# FP64 oracle values (oracle/bf_oracle.c: Eq. filter2, box window (Sec. 2), "
          "q_N of Sec. 3, gamma = pi/2, T = 1, border-truncated window), written by "
          "tests/golden/make_golden.py")


def write(name, a, fmt, extra=()):
    lines = [SOURCE] + ["# " + e for e in extra]
    np.savetxt(os.path.join(HERE, name), a, fmt=fmt, header="\n".join(l[2:] for l in lines),
               comments="# ")


def main():
    f = synth.rectangles(H, W, seed=7).astype(np.float32)
    w = synth.weights((H, W), seed=8).astype(np.float32)
    write("img_24x20.txt", f, "%.9g", ["input image, FP32 values (synth.rectangles, seed 7)"])
    write("weights_24x20.txt", w, "%.9g",
          ["loss weights g for L = sum(g * out), FP32 values (synth.weights, seed 8)"])
    fd, wd = f.astype(np.float64), w.astype(np.float64)
    for r, N in CASES:
        out = oracle.bilateral(fd, r, GAMMA, N)
        write("out_r%d_N%d.txt" % (r, N), out, "%.17g", ["filter output, r = %d, N = %d" % (r, N)])
    for r, N in GRAD_CASES:
        gf, gg = oracle.bilateral_grad(fd, wd, r, GAMMA, N)
        write("grad_r%d_N%d.txt" % (r, N), gf, "%.17g",
              ["dL/df for L = sum(g * out), r = %d, N = %d" % (r, N),
               "dL/dgamma = %.17g" % gg])


if __name__ == "__main__":
    main()
