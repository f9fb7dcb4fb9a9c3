"""The allocation-free guide march (nsl_guiding_map_noalloc) through the C ABI,
against the context path (nsl_guiding_map) and the FP64 oracle.

Some callers cannot allocate device memory (a render thread that must not
stall on an allocation's device synchronisation, an engine whose allocator owns
all device memory); this entry point keeps its scratch in a static device array
of the library instead.  It runs the single-pass march kernel where the context
path runs the three-pass segmented one, so the two agree to the rounding of
the in-scattering sum's grouping, and both are held to the oracle's 1e-5 of
range.  Two calls in a row with different grids check that the shared scratch
is restaged each time.  The file is named to be collected last."""
import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    return nsl.load()


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


def _check(pf, orc):
    got = _noalloc_guide(pf)
    assert not np.isnan(got).any()
    ctx = PT.make_ctx(pf)
    ref = PT.gpu_guide(ctx, pf)
    ctx.close()
    errs = PT.range_err(got, ref)
    assert max(errs) <= PT.TOL_GUIDE, errs
    o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    errs, bad = PT.compare_guide(got, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= max(1, PT.MAX_EXCUSED_FRAC * got[0].size)


def test_noalloc_guide_matches_context_path_and_oracle_twice(lib, orc):
    # first call: the 128^3 obstacle scene (34.6 MB of staged grid in the
    # 41.9 MB scratch); second call: the 64^3 orthographic scene
    for pf in (I.config_obstacle_128(), I.config_plain_64()):
        _check(pf, orc)


def test_noalloc_float16_grid(lib, orc):
    # a float16 grid is staged as float16 quads, as in a float16 context
    pf = I.small_case(64, 64, 48, seed=21, kind=I.PERSP, step=2.0)
    pf.density = pf.density.astype(np.float16)
    assert pf.mask is not None and pf.mask.any()
    _check(pf, orc)


def test_noalloc_largest_float32_grid_is_accepted(lib, orc):
    # 137 * 137 * 138 cells of 16 bytes: 41.4 MB of the 41.9 MB scratch
    pf = I.small_case(136, 48, 32, seed=22, kind=I.ORTHO, step=4.0, with_mask=False)
    _check(pf, orc)


def test_noalloc_rejects_oversize_grid(lib):
    import torch
    from paper_2604_03748_gb300 import nsl
    pf = I.config_plain_64()
    g = torch.empty((3, 128, 128), dtype=torch.float32, device="cuda:0")
    d = torch.empty((140, 140, 140), dtype=torch.float32, device="cuda:0")  # 45.2 MB staged > 40 MiB
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_guiding_map_noalloc(d.shape, nsl.NSL_F32, 1.0, d, None, pf.camera, 4.0, g)
    assert ei.value.status == nsl.NSL_ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
