"""FP8 E4M3 tensor-core network (tcgen05 kind::f8f6f4) against the oracle's
emulation of the same quantised network, on random guides of several sizes
(ragged ones included) and on the oracle's guide of the 512^2 obstacle scene;
batched FP8 equals the single-image path."""
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


def _check_fp8(got, emu):
    """Median, 99th percentile and maximum of |gpu - emulation| / range per plane."""
    rel = [np.abs(got[c] - emu[c]) / max(np.abs(emu[c]).max(), 1e-30) for c in range(8)]
    med = [float(np.median(r)) for r in rel]
    p99 = [float(np.percentile(r, 99)) for r in rel]
    mx = [float(r.max()) for r in rel]
    assert max(med) <= PT.TOL_NET_FP8_EMU_MEDIAN, (med, p99, mx)
    assert max(p99) <= PT.TOL_NET_FP8_EMU_P99, (med, p99, mx)
    assert max(mx) <= PT.TOL_NET_FP8_EMU_MAX, (med, p99, mx)


def _guide(H, W, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 60, (H, W))])


@pytest.mark.parametrize("H,W", [(64, 64), (24, 136), (128, 96)])
def test_net_fp8_matches_emulation(lib, orc, H, W):
    n = 64
    pf = I.PlumeFrame(np.zeros((n, n, n), np.float32), None, I.perspective_camera(n, 1, W, H),
                      I.random_light(1), 2.0)
    ctx = PT.make_ctx(pf)
    guide = _guide(H, W, H * 3 + W)
    got = PT.gpu_net(ctx, guide, lib.NSL_PREC_FP8)
    again = PT.gpu_net(ctx, guide, lib.NSL_PREC_FP8)
    assert np.array_equal(got, again)
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    g32 = guide.astype(np.float32).astype(np.float64)
    emu = orc.net_forward_q8(g32, flat, 16, 1.0 / math.sqrt(3 * n * n))
    _check_fp8(got, emu)
    ctx.close()


def test_net_fp8_on_oracle_guide_512(lib, orc):
    pf = I.config_obstacle_128()
    o, _, _ = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    guide = o.astype(np.float32).astype(np.float64)
    ctx = PT.make_ctx(pf)
    got = PT.gpu_net(ctx, guide, lib.NSL_PREC_FP8)
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    emu = orc.net_forward_q8(guide, flat, 16, 1.0 / math.sqrt(3 * 128 * 128))
    _check_fp8(got, emu)
    ctx.close()


def test_batched_fp8_equals_single(lib):
    import torch
    frames = [I.small_case(24, 32, 24, seed=61, kind=I.PERSP, step=2.0),
              I.small_case(32, 64, 48, seed=62, kind=I.ORTHO, step=2.0, with_mask=False)]
    b = lib.Batch(I.pack_blob(I.make_params(16, seed=0), 16), max_plumes=2)
    items = []
    for pf in frames:
        H, W = pf.camera.height, pf.camera.width
        items.append(dict(density=torch.from_numpy(np.ascontiguousarray(pf.density)).cuda(),
                          mask=None if pf.mask is None else torch.from_numpy(pf.mask).cuda(),
                          camera=pf.camera, step=pf.step, light=pf.light,
                          guide=torch.empty((3, H, W), device="cuda"),
                          lightmaps=torch.empty((8, H, W), device="cuda"),
                          rgba=torch.empty((4, H, W), device="cuda")))
    b.render(items, lib.NSL_PREC_FP8)
    torch.cuda.synchronize()
    for it, pf in zip(items, frames):
        ctx = PT.make_ctx(pf)
        g = PT.gpu_guide(ctx, pf)
        lm = PT.gpu_net(ctx, g, lib.NSL_PREC_FP8)
        assert np.array_equal(it["lightmaps"].cpu().numpy().astype(np.float64), lm)
        ctx.close()
    b.close()
