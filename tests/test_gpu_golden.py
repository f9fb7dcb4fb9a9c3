"""GPU parity on the stored expected values under tests/golden/ (written from
the FP64 oracle by tests/golden/make_golden.py): guide, FP32 network and
shading, each stage fed the stored input of the previous one."""
import os
import sys

import numpy as np
import pytest

import parity as PT

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden as G  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


def test_golden_chain(lib):
    import torch
    pf = G.plume()
    ctx = PT.make_ctx(pf, c0=G.CASE["c0"], seed=G.CASE["param_seed"])
    want = G.load("guide_small12_persp8.json")
    got = PT.gpu_guide(ctx, pf)
    errs, bad = PT.compare_guide(got, want["array"], np.asarray(want["flags"]).reshape(got.shape[1:]))
    assert max(errs) <= PT.TOL_GUIDE and bad == 0, errs
    # density evaluations: a sample's box test may fall the other way in float32
    n = ctx.guide_sample_count(pf.camera, pf.step)
    assert abs(n - want["samples_total"]) <= max(2, 0.005 * want["samples_total"]), (n, want["samples_total"])

    lm = PT.gpu_net(ctx, want["array"], lib.NSL_PREC_F32)
    ref = G.load("lightmaps_small12_persp8.json")["array"]
    assert np.abs(lm - ref).max() <= PT.TOL_NET_F32_ABS, np.abs(lm - ref).max()

    H, W = pf.camera.height, pf.camera.width
    lm_dev = torch.from_numpy(ref.astype(np.float32)).cuda()
    out = torch.full((4, H, W), float("nan"), dtype=torch.float32, device="cuda")
    ctx.shade(lm_dev, W, H, pf.camera, G.lights(), out)
    torch.cuda.synchronize()
    rgba = out.cpu().numpy().astype(np.float64)
    assert max(PT.range_err(rgba, G.load("shade_small12_persp8.json")["array"])) <= PT.TOL_SHADE
    ctx.close()
