"""The split-BF16 network (NSL_PREC_BF16X3): every convolution after the first
takes the bfloat16 high part and the bfloat16 rounding of the remainder of
both operands and adds hi*hi + hi*lo + lo*hi in FP32 on the tensor cores, with
binary32 activations between layers; the adapters run as in the other
tensor-core networks (binary16 operands).  Held to the FP64 oracle at the
half-precision bound of 2e-2 of range, which no form with single bfloat16
operands reaches on these weights, and to the oracle's emulation of the split
form, which differs from it by the adapters' binary16 operands only."""
import math

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu
TOL_SPLIT = 2e-2            # of each plane's range, against FP64 (the half-precision bound)
TOL_SPLIT_EMU = 1e-2        # against the emulation of the split convolutions (FP64 adapters)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    return nsl.load()


def _guide_input(H, W, seed):
    rng = np.random.default_rng(seed)
    g = np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 100, (H, W))])
    return g.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("H,W", [(8, 8), (16, 40), (128, 128), (24, 136)])
def test_split_bf16_against_fp64_and_emulation(lib, orc, H, W):
    from paper_2604_03748_gb300 import nsl
    vol = np.zeros((64, 64, 64), np.float32)
    pf = I.PlumeFrame(vol, None, I.orbit_ortho_camera(64, 1, W, H), I.random_light(1), 4.0)
    ctx = PT.make_ctx(pf)
    guide = _guide_input(H, W, H * 11 + W)
    got = PT.gpu_net(ctx, guide, nsl.NSL_PREC_BF16X3)
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ds = 1.0 / math.sqrt(3 * 64 * 64)
    ref = orc.net_forward(guide, flat, 16, ds)
    emu = orc.net_forward_prec(guide, flat, 16, ds, orc.PREC_BF16X3)
    assert not np.isnan(got).any()
    errs = PT.range_err(got, ref)
    assert max(errs) <= TOL_SPLIT, errs
    assert max(PT.range_err(got, emu)) <= TOL_SPLIT_EMU
    ctx.close()


def test_split_bf16_on_oracle_guide_512(lib, orc):
    """The 512^2 obstacle workload on the oracle's guide: within 2e-2 of range of
    FP64, where the single-BF16 network is about 7% away."""
    from paper_2604_03748_gb300 import nsl
    pf = I.config_obstacle_128()
    o, _, _ = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    guide = o.astype(np.float32).astype(np.float64)
    ctx = PT.make_ctx(pf)
    got = PT.gpu_net(ctx, guide, nsl.NSL_PREC_BF16X3)
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, 16, 1.0 / math.sqrt(3 * 128 * 128))
    errs = PT.range_err(got, ref)
    assert max(errs) <= TOL_SPLIT, errs
    again = PT.gpu_net(ctx, guide, nsl.NSL_PREC_BF16X3)
    assert np.array_equal(got, again)               # deterministic
    ctx.close()
