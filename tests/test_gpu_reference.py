"""The fine-step six-light reference renderer (nsl_reference_lightmaps: single
scattering of Sec. 3, the training target of Sec. 4.4) against the oracle's
nslo_reference_lightmaps, through the C ABI."""
import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu
TOL_REFERENCE = 1e-5      # of each plane's range


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    return nsl.load()


def _gpu_reference(pf, hf, g=0.0):
    import torch
    from paper_2604_03748_gb300 import nsl
    ctx = PT.make_ctx(pf)
    dev = torch.device("cuda:0")
    d = torch.from_numpy(np.ascontiguousarray(pf.density)).to(dev)
    m = None if pf.mask is None else torch.from_numpy(np.ascontiguousarray(pf.mask)).to(dev)
    out = torch.full((7, pf.camera.height, pf.camera.width), float("nan"), device=dev)
    nsl.nsl_reference_lightmaps(ctx.ctx, d, m, pf.camera, hf, out, phase_g=g)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kind,hf,g", [(I.PERSP, 0.25, 0.0), (I.ORTHO, 0.5, 0.0), (I.PERSP, 0.5, 0.4)])
def test_reference_matches_oracle(lib, orc, kind, hf, g):
    pf = I.small_case(24, 40, 24, seed=31, kind=kind, step=2.0)
    got = _gpu_reference(pf, hf, g)
    ref = orc.reference_lightmaps(pf.density, pf.mask, pf.camera, hf=hf, phase_g=g)
    assert not np.isnan(got).any()
    assert ref[:6].max() > 0
    errs = PT.range_err(got, ref)
    assert max(errs) <= TOL_REFERENCE, errs


def test_reference_float16_grid_and_ragged_box(lib, orc):
    vol = I.blob_fbm_volume(20, 33)[:, :17, :].astype(np.float16)
    mask = np.zeros(vol.shape, np.uint8)
    mask[5:9, 6:10, 4:12] = 1
    cam = I.perspective_camera(20, 33, 32, 16)
    pf = I.PlumeFrame(np.ascontiguousarray(vol), mask, cam, I.random_light(3), 2.0)
    got = _gpu_reference(pf, 0.25)
    ref = orc.reference_lightmaps(pf.density, pf.mask, pf.camera, hf=0.25)
    assert max(PT.range_err(got, ref)) <= TOL_REFERENCE


def test_reference_quad_staged_large_grid(lib, orc):
    """A float32 grid too large for octo cells in the L2 share (144^3) is staged
    as quad cells; the reference renderer reads those the same way."""
    vol = I.blob_fbm_volume(144, 35)
    cam = I.perspective_camera(144, 35, 8, 8)
    pf = I.PlumeFrame(vol, None, cam, I.random_light(35), 2.0)
    got = _gpu_reference(pf, 1.0)
    ref = orc.reference_lightmaps(pf.density, pf.mask, pf.camera, hf=1.0)
    assert ref[:6].max() > 0
    assert max(PT.range_err(got, ref)) <= TOL_REFERENCE


def test_reference_empty_volume(lib):
    pf = I.small_case(16, 16, 16, seed=34, kind=I.ORTHO, step=2.0, with_mask=False)
    pf.density = np.zeros_like(pf.density)
    got = _gpu_reference(pf, 0.5)
    assert np.all(got[:6] == 0.0) and np.all(got[6] == 1.0)
