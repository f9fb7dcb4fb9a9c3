"""The allocation-free guide march (nsl_guiding_map_noalloc) against the
context path (nsl_guiding_map), through the C ABI.

Some callers cannot allocate device memory (a render thread that must not
stall on an allocation, an engine that owns all device memory); this entry
point keeps its scratch in a static device array instead.  Two calls in a row
with different grids check that the shared scratch is restaged each time.
The file is named to be collected last."""
import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu


def _noalloc_guide(pf):
    import torch
    from paper_2604_03748_gb300 import nsl
    dev = torch.device("cuda:0")
    d = torch.from_numpy(np.ascontiguousarray(pf.density)).to(dev)
    m = None if pf.mask is None else torch.from_numpy(np.ascontiguousarray(pf.mask)).to(dev)
    g = torch.full((3, pf.camera.height, pf.camera.width), float("nan"), dtype=torch.float32, device=dev)
    dtype = nsl.NSL_F16 if pf.density.dtype == np.float16 else nsl.NSL_F32
    nsl.nsl_guiding_map_noalloc(pf.density.shape, dtype, pf.sigma_scale, d, m, pf.camera, pf.step, g)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64)


def test_noalloc_guide_matches_context_path_twice():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    # first call: the 128^3 obstacle scene (exactly fills the scratch); second
    # call: the 64^3 orthographic scene
    for pf in (I.config_obstacle_128(), I.config_plain_64()):
        got = _noalloc_guide(pf)
        ctx = PT.make_ctx(pf)
        ref = PT.gpu_guide(ctx, pf)
        ctx.close()
        errs = PT.range_err(got, ref)
        assert not np.isnan(got).any()
        assert max(errs) <= PT.TOL_GUIDE, errs


def test_noalloc_rejects_oversize_grid():
    import torch
    from paper_2604_03748_gb300 import nsl
    nsl.load()
    pf = I.config_plain_64()
    g = torch.empty((3, 128, 128), dtype=torch.float32, device="cuda:0")
    d = torch.empty((140, 140, 140), dtype=torch.float32, device="cuda:0")  # 45.2 MB staged > 40 MiB
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_guiding_map_noalloc(d.shape, nsl.NSL_F32, 1.0, d, None, pf.camera, 4.0, g)
    assert ei.value.status == nsl.NSL_ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
