"""Failure detection without a GPU fault: a bounded mbarrier wait that runs out
(nothing ever arrives at it) records a code in the context's error word and
returns; the next network call reports NSL_ERR_TIMEOUT, and the context keeps
working afterwards."""
import time

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


def test_wait_timeout_reported_and_context_survives(lib):
    import torch
    H = W = 64
    blob = I.pack_blob(I.make_params(16, 0), 16)
    ctx = lib.Context((32, 32, 32), lib.NSL_F32, blob, W, H)
    rng = np.random.default_rng(3)
    g = torch.from_numpy(np.stack([rng.uniform(0, .2, (H, W)), rng.uniform(0, 1, (H, W)),
                                   rng.uniform(0, 60, (H, W))]).astype(np.float32)).cuda()
    ref = torch.empty((8, H, W), device="cuda")
    ctx.predict_lightmaps(g, W, H, lib.NSL_PREC_F16, ref)
    torch.cuda.synchronize()
    # the probe's wait gives up after its bound (about 2 s) and returns
    t0 = time.perf_counter()
    lib.check(lib.load().nsl_selftest_wait_timeout(ctx.ctx, None), "nsl_selftest_wait_timeout")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert 0.3 < dt < 30.0, dt
    out = torch.empty((8, H, W), device="cuda")
    with pytest.raises(lib.NslError) as ei:
        ctx.predict_lightmaps(g, W, H, lib.NSL_PREC_F16, out)
    assert ei.value.status == lib.NSL_ERR_TIMEOUT
    assert "0x8000" in str(ei.value)
    # reported once; the context and the device are still usable
    ctx.predict_lightmaps(g, W, H, lib.NSL_PREC_F16, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    ctx.close()
