"""The lightmap network at base width C0 = 32 (Sec. 4.3; the second width the
FP32 path runs) against the FP64 oracle through the C ABI: ragged and
several-tile sizes, the 512^2 workload on the oracle's guide, and the entry
points that run C0 = 16 only refusing a C0 = 32 blob.  Marked gpu."""
import math

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu

C0 = 32


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    return nsl


def _guide_input(H, W, seed):
    rng = np.random.default_rng(seed)
    g = np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 100, (H, W))])
    return g.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("H,W", [(8, 8), (16, 40), (64, 96), (128, 128)])
def test_net_f32_c0_32_parity(lib, orc, H, W):
    from paper_2604_03748_gb300 import nsl
    vol = np.zeros((64, 64, 64), np.float32)
    pf = I.PlumeFrame(vol, None, I.orbit_ortho_camera(64, 1, W, H), I.random_light(1), 4.0)
    ctx = PT.make_ctx(pf, c0=C0)
    guide = _guide_input(H, W, H * 5 + W)
    got = PT.gpu_net(ctx, guide, nsl.NSL_PREC_F32)
    flat = I.flat_params(I.make_params(C0, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, C0, 1.0 / math.sqrt(3 * 64 * 64))
    assert np.abs(got - ref).max() <= PT.TOL_NET_F32_ABS, np.abs(got - ref).max()
    ctx.close()


def test_net_f32_c0_32_parity_on_oracle_guide_512(lib, orc):
    """The 512^2 obstacle workload at C0 = 32, every output value."""
    from paper_2604_03748_gb300 import nsl
    pf = I.config_obstacle_128()
    o, _, _ = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    guide = o.astype(np.float32).astype(np.float64)
    ctx = PT.make_ctx(pf, c0=C0)
    got = PT.gpu_net(ctx, guide, nsl.NSL_PREC_F32)
    flat = I.flat_params(I.make_params(C0, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, C0, 1.0 / math.sqrt(3 * 128 * 128))
    assert np.abs(got - ref).max() <= PT.TOL_NET_F32_ABS, np.abs(got - ref).max()
    ctx.close()


def test_c0_32_runs_the_fp32_path_only(lib):
    """A C0 = 32 context marches, shades and runs the FP32 network; the
    tensor-core precisions, batches and the trainer refuse its blob."""
    import torch
    from paper_2604_03748_gb300 import nsl
    pf = I.small_case(24, 32, 24, seed=11, kind=I.PERSP, step=2.0)
    ctx = PT.make_ctx(pf, c0=C0)
    g = PT.gpu_guide(ctx, pf)
    assert np.isfinite(g).all()
    H, W = pf.camera.height, pf.camera.width
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    out = torch.empty((8, H, W), device="cuda")
    for prec in (nsl.NSL_PREC_F16, nsl.NSL_PREC_BF16, nsl.NSL_PREC_FP8):
        with pytest.raises(nsl.NslError) as e:
            ctx.predict_lightmaps(gd, W, H, prec, out)
        assert e.value.status == nsl.NSL_ERR_UNSUPPORTED
    blob = I.pack_blob(I.make_params(C0, 0), C0)
    with pytest.raises(nsl.NslError) as e:
        nsl.Batch(blob, 4)
    assert e.value.status == nsl.NSL_ERR_UNSUPPORTED
    with pytest.raises(nsl.NslError) as e:
        nsl.Trainer(blob, nsl.train_opts(batch=1, width=16, height=16))
    assert e.value.status == nsl.NSL_ERR_UNSUPPORTED
    ctx.close()
