"""Per-layer error study of the network's precision forms, oracle only.

TEST INFRASTRUCTURE: it calls the FP64 oracle and the seeded input generators,
nothing of the CUDA path.  For the 512^2 obstacle workload (128^3 plume with a
sphere obstacle, perspective camera, step 2 voxels; the oracle's guide) it
prints, per output plane, the error relative to the range max|o| of the FP64
network for:
  * every convolution in one form (BF16, FP16, FP8, split BF16);
  * one convolution at a time in BF16 (and in FP8), the others exact: how much
    of the error a single layer's rounding contributes, and which layers
    amplify it most.
Run:  python -m oracle.precision_study [--size 512] [--rows R]
(--rows limits the guide to a band of R rows centred on the image, for a
quicker run; the default marches the whole image).
"""
from __future__ import annotations

import argparse
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2604_03748_gb300 import inputs as I  # noqa: E402


def range_err(g, o):
    return [float(np.abs(g[c] - o[c]).max() / max(np.abs(o[c]).max(), 1e-30)) for c in range(o.shape[0])]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--rows", type=int, default=0)
    a = ap.parse_args(argv)
    oracle.build()
    pf = I.config_obstacle_128(width=a.size, height=a.size)
    H = pf.camera.height
    rows = None
    if a.rows:
        r0 = (H - a.rows) // 2 // 8 * 8
        rows = (r0, r0 + a.rows)
    g, _, _ = oracle.guide(pf.density, pf.mask, pf.camera, pf.step, rows=rows)
    if rows:
        g = g[:, rows[0]:rows[1]]
    params = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ds = 1.0 / math.sqrt(sum(float(v) ** 2 for v in pf.density.shape))
    ref = oracle.net_forward(g, params, 16, ds)
    print(f"workload {pf.meta['name']}, guide {g.shape[1]}x{g.shape[2]}, C0 = 16, Kaiming seed 0")
    print("error per plane relative to max|o| of the FP64 network (planes +X -X +Y -Y +Z -Z T E)")
    for name, code in (("all BF16", oracle.PREC_BF16), ("all FP16", oracle.PREC_F16),
                       ("all FP8", oracle.PREC_FP8), ("all split BF16", oracle.PREC_BF16X3)):
        e = range_err(oracle.net_forward_prec(g, params, 16, ds, code), ref)
        print(f"{name:16s} max {max(e):.4f}  " + " ".join(f"{v:.4f}" for v in e))
    for form, code in (("BF16", oracle.PREC_BF16), ("FP8", oracle.PREC_FP8)):
        print(f"one convolution in {form}, the others exact:")
        for l, lname in enumerate(oracle.NET_LAYERS):
            if l == 0 and code == oracle.PREC_FP8:
                continue   # the first convolution keeps exact operands in every form
            codes = [oracle.PREC_F64] * 17
            codes[l] = code
            e = range_err(oracle.net_forward_prec(g, params, 16, ds, codes), ref)
            print(f"  {lname:6s} max {max(e):.4f}")


if __name__ == "__main__":
    main()
