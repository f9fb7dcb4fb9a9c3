"""GPU parity of the obstacle shadowing (Sec. 4.5) through the C ABI against
the oracle: the shadow map of the obstacle mask (bit-identical hit texels and
depths), and the shadowed six-way shading (bit-identical visibility decisions)."""
import math

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu

LIGHTS = [(0.0, 1.0, 0.0), (0.3, 1.0, 0.2), (-0.7, 0.2, 0.5), (0.0, 0.0, -1.0), (1.0, 1.0, 1.0),
          (0.0, 1.0, 1.0)]


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


def _gpu_map(lib, mask, d, R):
    import torch
    out = torch.full((R, R), float("nan"), dtype=torch.float32, device="cuda")
    lib.nsl_obstacle_shadow_map(torch.from_numpy(np.ascontiguousarray(mask)).cuda(), d, R, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _compare_maps(g, o, S):
    """Bit-identical maps: the same texels hit, with the same binary32 depth
    (the GPU walk tests every voxel the oracle's brute force can find)."""
    assert not np.isnan(g).any()
    assert np.array_equal(np.isinf(g), np.isinf(o))
    hit = ~np.isinf(o)
    assert hit.sum() > 0
    assert np.array_equal(g[hit], o[hit]), float(np.abs(g[hit] - o[hit]).max())


@pytest.mark.parametrize("d", LIGHTS)
def test_shadow_map_sphere(lib, orc, d):
    n, R = 48, 96
    mask, _ = I.sphere_mask(n, 9.0, 3)
    _compare_maps(_gpu_map(lib, mask, d, R), orc.shadow_map(mask, d, R), math.sqrt(3) * n)


def test_shadow_map_ragged_grid_and_slab(lib, orc):
    mask = np.zeros((20, 13, 27), np.uint8)
    mask[:, :4, :] = 1
    mask[5:9, 8:11, 3:20] = 1
    for d in LIGHTS:
        _compare_maps(_gpu_map(lib, mask, d, 64), orc.shadow_map(mask, d, 64), math.sqrt(20 ** 2 + 13 ** 2 + 27 ** 2))


def test_shadow_map_grazing_lattice(lib, orc):
    """Voxel columns on every other cell: texel lines run along the shared
    faces and edges of the columns, where the oracle's slab test reports
    touching voxels that a plain voxel walk steps past."""
    m = np.zeros((16, 16, 16), np.uint8)
    m[:, ::2, ::2] = 1
    for d in LIGHTS:
        _compare_maps(_gpu_map(lib, m, d, 64), orc.shadow_map(m, d, 64), math.sqrt(3) * 16)


def test_shadow_map_obstacle_128(lib, orc):
    pf = I.config_obstacle_128()
    d = pf.light.dir
    _compare_maps(_gpu_map(lib, pf.mask, d, 96), orc.shadow_map(pf.mask, d, 96), math.sqrt(3) * 128)


def _frame(lib):
    import torch
    pf = I.small_case(32, 48, 40, seed=21, kind=I.PERSP, step=2.0)
    mask = np.zeros_like(pf.density, dtype=np.uint8)
    n = pf.density.shape[0]
    mask[:, n // 2 + 4: n // 2 + 8, : n // 2] = 1      # a shelf over half the grid
    H, W = pf.camera.height, pf.camera.width
    ctx = PT.make_ctx(pf)
    g = torch.from_numpy(PT.gpu_guide(ctx, pf).astype(np.float32)).cuda()
    rng = np.random.default_rng(8)
    lm = torch.from_numpy(rng.uniform(0.0, 1.0, (8, H, W)).astype(np.float32)).cuda()
    lights = [I.Light((0.1, 1.0, 0.05), (1.0, 0.8, 0.6)), I.Light((-0.4, 0.6, 0.7), (0.5, 0.5, 0.9)),
              I.Light((0.9, -0.2, 0.1), (0.2, 0.4, 0.3))]
    return pf, mask, ctx, g, lm, lights


def _shade(lib, ctx, lm, g, pf, lights, maps, R, bias):
    import torch
    H, W = pf.camera.height, pf.camera.width
    rgba = torch.empty((4, H, W), device="cuda")
    lib.nsl_shade_shadowed(ctx.ctx, lm, g, W, H, pf.camera, lights, maps, R, bias, rgba)
    torch.cuda.synchronize()
    return rgba.cpu().numpy().astype(np.float64)


def test_shade_shadowed_same_maps(lib, orc):
    import torch
    pf, mask, ctx, g, lm, lights = _frame(lib)
    R = 80
    omaps = [orc.shadow_map(mask, L.dir, R) for L in lights[:2]] + [None]
    dmaps = [torch.from_numpy(m).cuda() if m is not None else None for m in omaps]
    got = _shade(lib, ctx, lm, g, pf, lights, dmaps, R, 1.0)
    ref = orc.shade_shadowed(lm.cpu().numpy(), g.cpu().numpy(), pf.camera, lights, pf.density.shape, omaps, 1.0)
    plain = orc.shade(lm.cpu().numpy().astype(np.float64), pf.camera, lights)
    assert np.mean(np.abs(ref[:3] - plain[:3]).max(axis=0) > 1e-6) > 0.05     # some pixels are in shadow
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * scale
    ctx.close()


def test_shade_shadowed_end_to_end(lib, orc):
    import torch
    pf, mask, ctx, g, lm, lights = _frame(lib)
    R = 80
    m_gpu = []
    for L in lights[:2]:
        t = torch.empty((R, R), device="cuda")
        lib.nsl_obstacle_shadow_map(torch.from_numpy(mask).cuda(), L.dir, R, t)
        m_gpu.append(t)
    got = _shade(lib, ctx, lm, g, pf, lights, m_gpu + [None], R, 1.0)
    omaps = [orc.shadow_map(mask, L.dir, R) for L in lights[:2]] + [None]
    ref = orc.shade_shadowed(lm.cpu().numpy(), g.cpu().numpy(), pf.camera, lights, pf.density.shape, omaps, 1.0)
    for mg, mo in zip(m_gpu, omaps[:2]):
        assert np.array_equal(mg.cpu().numpy(), mo)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    ctx.close()


def test_shadow_arguments_rejected(lib):
    import torch
    m = torch.zeros((8, 8, 8), dtype=torch.uint8, device="cuda")
    out = torch.empty((16, 16), device="cuda")
    with pytest.raises(lib.NslError):
        lib.nsl_obstacle_shadow_map(m, (0.0, 0.0, 0.0), 16, out)        # zero direction
    with pytest.raises(ValueError):
        lib.nsl_obstacle_shadow_map(m, (0.0, 1.0, 0.0), 8, out)         # out is not [R][R]
    with pytest.raises(ValueError):
        lib.nsl_obstacle_shadow_map(m.float(), (0.0, 1.0, 0.0), 16, out)  # mask must be uint8
