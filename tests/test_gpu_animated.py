"""The animated 256^3 FP16 workload: frames 0, 150 and 299 of the advected
sequence, 1024x1024, step 4.  Guide against the FP64 oracle on every pixel, the
FP16 tensor-core network against the oracle's network on the oracle's guide,
and shading of the frame's light."""
import math

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


@pytest.fixture(scope="module")
def seq(lib):
    return I.animated_sequence(256, 300, seed=3, width=1024, height=1024, step=4.0, device="cuda",
                               keep=[0, 150, 299])


@pytest.mark.parametrize("t", [0, 150, 299])
def test_animated_frame_guide(lib, orc, seq, t):
    import torch
    W = H = 1024
    blob = I.pack_blob(I.make_params(16, 0), 16)
    ctx = lib.Context((256, 256, 256), lib.NSL_F16, blob, W, H)
    g = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
    ctx.guiding_map(seq.frames[t], None, seq.cameras[t], seq.step, g)
    torch.cuda.synchronize()
    got = g.cpu().numpy().astype(np.float64)
    host = seq.frames[t].cpu().numpy()
    assert host.dtype == np.float16
    o, _, f = orc.guide(host, None, seq.cameras[t], seq.step)
    errs, bad = PT.compare_guide(got, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= PT.MAX_EXCUSED_FRAC * o[0].size
    if t == 150:
        lm = torch.empty((8, H, W), dtype=torch.float32, device="cuda")
        ctx.predict_lightmaps(torch.from_numpy(o.astype(np.float32)).cuda(), W, H, lib.NSL_PREC_F16, lm)
        torch.cuda.synchronize()
        flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
        ref = orc.net_forward(o.astype(np.float32).astype(np.float64), flat, 16, 1.0 / math.sqrt(3 * 256 * 256))
        assert max(PT.range_err(lm.cpu().numpy().astype(np.float64), ref)) <= PT.TOL_NET_F16
    ctx.close()


def test_animated_sequence_properties(seq):
    """The input recipe itself: FP16 frames in [0, 2], mass drifting slowly,
    the light turning 1 degree per frame about Y, the camera 2.5 n away at the
    spline's control points."""
    import torch
    for t, v in seq.frames.items():
        assert v.dtype == torch.float16 and float(v.min()) >= 0.0 and float(v.max()) <= 2.0
    m0, m1 = float(seq.frames[0].float().sum()), float(seq.frames[299].float().sum())
    assert 0.5 < m1 / m0 < 1.5
    a, b = np.array(seq.lights[0].dir), np.array(seq.lights[90].dir)
    assert abs(a[1] - b[1]) < 1e-12
    ang = math.degrees(math.atan2(a[0] * b[2] - a[2] * b[0], a[0] * b[0] + a[2] * b[2]))
    assert abs(abs(ang) - 90.0) < 1e-6
    ctr = np.array([128.0] * 3)
    r = np.linalg.norm(np.array(seq.cameras[0].eye) - ctr)
    assert abs(r - 2.5 * 256) < 1e-6
