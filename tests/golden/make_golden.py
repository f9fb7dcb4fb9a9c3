"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Only the oracle (``oracle/``) and the seeded input generators
(``paper_2604_03748_gb300.inputs``) are called: no value here comes from the
CUDA path.  One chained case on a small masked plume, each stage stored with
its inputs' recipe:

  guide_small12_persp8.json      guiding map (Sec. 4.2, Alg. 1; Eq. approx)
  lightmaps_small12_persp8.json  network forward on that guide (Sec. 4.3)
  shade_small12_persp8.json      six-way shading of those lightmaps (Sec. 3)

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the recipe shared by the writer and the tests
CASE = dict(n=12, width=8, height=8, seed=21, step=1.5, c0=16, param_seed=0)
LIGHT_SEEDS = (21, 5)


def plume():
    from paper_2604_03748_gb300 import inputs as I
    return I.small_case(CASE["n"], CASE["width"], CASE["height"], seed=CASE["seed"], kind=I.PERSP,
                        step=CASE["step"])


def lights():
    from paper_2604_03748_gb300 import inputs as I
    return [I.random_light(s) for s in LIGHT_SEEDS]


def depth_scale():
    n = CASE["n"]
    return 1.0 / math.sqrt(3 * n * n)


def f32(a):
    """The float32 rounding a GPU input goes through, back in float64."""
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def compute(orc):
    from paper_2604_03748_gb300 import inputs as I
    pf = plume()
    g, s, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    flat = I.flat_params(I.make_params(CASE["c0"], CASE["param_seed"])).astype(np.float64)
    lm = orc.net_forward(f32(g), flat, CASE["c0"], depth_scale())
    rgba = orc.shade(f32(lm), pf.camera, lights())
    return dict(guide=g, samples=s, flags=f, lightmaps=lm, rgba=rgba)


def _vals(a):
    return [float(v) for v in np.asarray(a, np.float64).reshape(-1)]


def write(orc):
    r = compute(orc)
    recipe = dict(CASE, light_seeds=list(LIGHT_SEEDS),
                  generator="paper_2604_03748_gb300.inputs.small_case(n, width, height, seed, PERSP, step); "
                            "weights make_params(c0, param_seed); lights random_light(s)")
    files = {
        "guide_small12_persp8.json": dict(
            cite="Sec. 4.2, Alg. 1 and Eq. approx: the guiding map (L~, T, D) with the front/top/bottom "
                 "surrogate lights, default march options",
            recipe=recipe, shape=[3, CASE["height"], CASE["width"]], values=_vals(r["guide"]),
            flags=[int(v) for v in r["flags"].reshape(-1)], samples_total=int(r["samples"].sum())),
        "lightmaps_small12_persp8.json": dict(
            cite="Sec. 4.3: UNet encoder/decoder and four NAFBlock channel adapters, 8 output planes; "
                 "input = the stored guide rounded to float32, depth scaled by 1/sqrt(3 n^2)",
            recipe=recipe, shape=[8, CASE["height"], CASE["width"]], values=_vals(r["lightmaps"])),
        "shade_small12_persp8.json": dict(
            cite="Sec. 3, the six-way interpolation of the scattering term: shading of the stored lightmaps "
                 "rounded to float32 under two directional lights",
            recipe=recipe, shape=[4, CASE["height"], CASE["width"]], values=_vals(r["rgba"])),
    }
    for name, obj in files.items():
        with open(os.path.join(HERE, name), "w") as fh:
            json.dump(obj, fh, indent=0, separators=(",", ":"))
            fh.write("\n")


def load(name):
    with open(os.path.join(HERE, name)) as fh:
        obj = json.load(fh)
    obj["array"] = np.asarray(obj["values"], np.float64).reshape(obj["shape"])
    return obj


if __name__ == "__main__":
    import oracle
    oracle.build()
    write(oracle)
