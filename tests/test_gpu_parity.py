"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle
on the same seeded inputs.  Marked gpu (needs a GB300 and the built libnsl)."""
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


# ----------------------------------------------------------------------------
# guide march
# ----------------------------------------------------------------------------

GUIDE_CASES = {
    "plume64_ortho128_h4": lambda: I.config_plain_64(),
    "small24_persp_mask_ragged": lambda: I.small_case(24, 32, 24, seed=11, kind=I.PERSP, step=2.0),
    "small20_ortho_h3": lambda: I.small_case(20, 40, 16, seed=12, kind=I.ORTHO, step=3.0),
}


@pytest.mark.parametrize("name", list(GUIDE_CASES))
def test_guide_parity(lib, orc, name):
    pf = GUIDE_CASES[name]()
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    o, s, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= PT.MAX_EXCUSED_FRAC * g[0].size
    ctx.close()


def test_guide_parity_obstacle_128_full_size(lib, orc):
    """The 128^3 perspective 512^2 workload with the sphere obstacle, every pixel."""
    pf = I.config_obstacle_128()
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    o, s, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= PT.MAX_EXCUSED_FRAC * g[0].size
    ctx.close()


@pytest.mark.parametrize("opts", [{}, dict(shadow_volume=1, t_min=0.0)])
def test_guide_quad_staging_large_f32_grid(lib, orc, opts):
    """A float32 grid whose octo cells would take more than 60% of the L2
    (144^3: 97.6 MB) is staged as quad cells in a single-plume context; its
    guide, through the host-buffer entry point too, matches the oracle."""
    import dataclasses
    from paper_2604_03748_gb300 import nsl
    n = 144
    vol = I.blob_fbm_volume(n, 31)
    mask, _ = I.sphere_mask(n, 20.0, 31, lo=30.0, hi=float(n - 30))
    pf = I.PlumeFrame(vol, mask, I.perspective_camera(n, 31, 48, 40), I.random_light(31), 2.0)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf, **opts)
    o, s, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step, **opts)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= PT.MAX_EXCUSED_FRAC * g[0].size
    if not opts:
        hg = np.zeros((3, 40, 48), np.float32)
        nsl.nsl_render_frame_host(ctx.ctx, pf.density, pf.mask, pf.camera, [pf.light], pf.step,
                                  nsl.NSL_PREC_F16, hg, None, None)
        assert np.array_equal(hg.astype(np.float64), g)
    ctx.close()


@pytest.mark.parametrize("opts", [dict(jitter=0, t_min=0.0), dict(segment_exact=1),
                                  dict(phase_g=0.5, surrogate_I=(1.0, 0.5, 2.0)),
                                  dict(seed=123, frame=77, tau_depth=0.2),
                                  dict(light_set=1), dict(light_set=2),
                                  dict(light_set=2, phase_g=0.4, surrogate_I=(1.0, 0.6, 1.7)),
                                  dict(shadow_volume=1, t_min=0.0), dict(shadow_volume=1, light_set=2, t_min=0.0)])
def test_guide_options(lib, orc, opts):
    pf = I.small_case(24, 24, 16, seed=13, kind=I.PERSP, step=2.0)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf, **opts)
    o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step, **opts)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= max(1, PT.MAX_EXCUSED_FRAC * g[0].size)
    ctx.close()


def test_guide_edge_cases(lib, orc):
    # empty grid, fully masked grid, rays that miss, a tiny 8x8 image, ragged grid
    vol = np.zeros((9, 7, 11), np.float32)
    cam = I.perspective_camera(11, 2, 8, 8)
    pf = I.PlumeFrame(vol, None, cam, I.random_light(1), 1.5)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    assert np.all(g[0] == 0) and np.all(g[1] == 1) and np.all(g[2] == 0)
    ctx.close()
    vol = I.blob_fbm_volume(16, 3)
    pf = I.PlumeFrame(vol, np.ones_like(vol, np.uint8), I.orbit_ortho_camera(16, 3, 16, 8),
                      I.random_light(1), 2.0)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    assert np.all(g[0] == 0) and np.all(g[1] == 1) and np.all(g[2] == 0)
    ctx.close()
    cam = I.Camera(I.ORTHO, (8.0, 8.0, 40.0), (8.0, 8.0, 80.0), (0.0, 1.0, 0.0), 40.0, 16.0, 16, 16)
    pf = I.PlumeFrame(vol, None, cam, I.random_light(1), 2.0)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    assert np.all(g[1] == 1)
    ctx.close()
    # ragged non-cubic grid
    rng = np.random.default_rng(5)
    vol = (rng.uniform(0, 0.3, size=(13, 21, 17))).astype(np.float32)
    mask = (rng.uniform(size=vol.shape) < 0.1).astype(np.uint8)
    cam = I.perspective_camera(21, 5, 24, 16)
    pf = I.PlumeFrame(vol, mask, cam, I.random_light(2), 1.25)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    o, _, f = orc.guide(vol, mask, cam, 1.25)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE and bad <= 1, errs
    ctx.close()


def test_guide_fp16_density(lib, orc):
    pf = I.small_case(32, 32, 32, seed=14, kind=I.PERSP, step=2.0)
    pf.density = pf.density.astype(np.float16)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE and bad <= 1, errs
    ctx.close()


@pytest.mark.parametrize("opts", [dict(), dict(jitter=0, t_min=0.0), dict(segment_exact=1), dict(light_set=1),
                                  dict(light_set=2), dict(shadow_volume=1, t_min=0.0),
                                  dict(shadow_volume=1, light_set=2)])
def test_guide_fp16_density_options(lib, orc, opts):
    # an FP16 grid is staged as FP16 (sigma_scale applied after the blend):
    # masked, a ragged 27^3 grid and 40x24 image, every light set and the
    # shadow volumes
    pf = I.small_case(27, 40, 24, seed=15, kind=I.PERSP, step=1.75)
    pf.density = pf.density.astype(np.float16)
    assert pf.mask is not None and pf.mask.any()
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf, **opts)
    o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step, **opts)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= max(1, PT.MAX_EXCUSED_FRAC * g[0].size)
    ctx.close()


def test_guide_deterministic(lib):
    pf = I.config_plain_64()
    ctx = PT.make_ctx(pf)
    a = PT.gpu_guide(ctx, pf)
    b = PT.gpu_guide(ctx, pf)
    assert np.array_equal(a, b)
    ctx.close()


def test_invalid_arguments_rejected(lib):
    import torch
    from paper_2604_03748_gb300 import nsl
    pf = I.config_plain_64()
    ctx = PT.make_ctx(pf)
    d = torch.from_numpy(pf.density).cuda()
    g = torch.empty((3, 128, 128), dtype=torch.float32, device="cuda")
    big = I.orbit_ortho_camera(64, 1, 256, 256)
    with pytest.raises(nsl.NslError) as ei:
        ctx.guiding_map(d, None, big, 4.0, g)
    assert ei.value.status == nsl.NSL_ERR_INVALID_ARG
    with pytest.raises(nsl.NslError):
        ctx.guiding_map(d, None, pf.camera, 0.0, g)
    odd = I.orbit_ortho_camera(64, 1, 100, 128)
    with pytest.raises(nsl.NslError):
        ctx.guiding_map(d, None, odd, 4.0, g)
    with pytest.raises(nsl.NslError) as ei:
        ctx.predict_lightmaps(g, 128, 128, 7, torch.empty((8, 128, 128), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):       # a float64 output buffer is refused by the binding
        ctx.guiding_map(d, None, pf.camera, 4.0, torch.empty((3, 128, 128), dtype=torch.float64, device="cuda"))
    assert ei.value.status in (nsl.NSL_ERR_UNSUPPORTED, nsl.NSL_ERR_INVALID_ARG)
    ctx.close()


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------

def _guide_input(H, W, seed):
    rng = np.random.default_rng(seed)
    g = np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 100, (H, W))])
    return g.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("H,W", [(8, 8), (16, 40), (128, 128), (64, 96)])
def test_net_f32_parity(lib, orc, H, W):
    from paper_2604_03748_gb300 import nsl
    vol = np.zeros((64, 64, 64), np.float32)
    pf = I.PlumeFrame(vol, None, I.orbit_ortho_camera(64, 1, W, H), I.random_light(1), 4.0)
    ctx = PT.make_ctx(pf)
    guide = _guide_input(H, W, H * 7 + W)
    got = PT.gpu_net(ctx, guide, nsl.NSL_PREC_F32)
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, 16, 1.0 / math.sqrt(3 * 64 * 64))
    assert np.abs(got - ref).max() <= PT.TOL_NET_F32_ABS, np.abs(got - ref).max()
    ctx.close()


def test_net_f32_parity_on_oracle_guide_512(lib, orc):
    """The 512^2 workload: FP32 network on the oracle's guide of the obstacle scene."""
    from paper_2604_03748_gb300 import nsl
    pf = I.config_obstacle_128()
    o, _, _ = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    guide = o.astype(np.float32).astype(np.float64)
    ctx = PT.make_ctx(pf)
    got = PT.gpu_net(ctx, guide, nsl.NSL_PREC_F32)
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, 16, 1.0 / math.sqrt(3 * 128 * 128))
    assert np.abs(got - ref).max() <= PT.TOL_NET_F32_ABS, np.abs(got - ref).max()
    ctx.close()


HALF_PRECISIONS = [("f16", 3, "TOL_NET_F16"), ("bf16", 1, "TOL_NET_BF16")]


@pytest.mark.parametrize("prec", HALF_PRECISIONS, ids=[p[0] for p in HALF_PRECISIONS])
@pytest.mark.parametrize("H,W", [(8, 8), (16, 40), (128, 128), (64, 96), (24, 136)])
def test_net_half_parity(lib, orc, H, W, prec):
    """Tensor-core network (16-bit operands, FP32 accumulation) vs the FP64 oracle,
    per plane relative to the oracle's range."""
    vol = np.zeros((64, 64, 64), np.float32)
    pf = I.PlumeFrame(vol, None, I.orbit_ortho_camera(64, 1, W, H), I.random_light(1), 4.0)
    ctx = PT.make_ctx(pf)
    guide = _guide_input(H, W, H * 5 + W)
    got = PT.gpu_net(ctx, guide, prec[1])
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, 16, 1.0 / math.sqrt(3 * 64 * 64))
    errs = PT.range_err(got, ref)
    assert max(errs) <= getattr(PT, prec[2]), errs
    ctx.close()


@pytest.mark.parametrize("prec", HALF_PRECISIONS, ids=[p[0] for p in HALF_PRECISIONS])
def test_net_half_parity_on_oracle_guide_512(lib, orc, prec):
    """The 512^2 workload: tensor-core network on the oracle's guide of the obstacle scene."""
    pf = I.config_obstacle_128()
    o, _, _ = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    guide = o.astype(np.float32).astype(np.float64)
    ctx = PT.make_ctx(pf)
    got = PT.gpu_net(ctx, guide, prec[1])
    again = PT.gpu_net(ctx, guide, prec[1])
    assert np.array_equal(got, again)          # deterministic
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref = orc.net_forward(guide, flat, 16, 1.0 / math.sqrt(3 * 128 * 128))
    errs = PT.range_err(got, ref)
    assert max(errs) <= getattr(PT, prec[2]), errs
    ctx.close()


# ----------------------------------------------------------------------------
# shading
# ----------------------------------------------------------------------------

def test_shade_parity(lib, orc):
    import torch
    rng = np.random.default_rng(3)
    H, W = 24, 40
    lm = rng.uniform(-0.2, 1.0, size=(8, H, W)).astype(np.float32)
    cam = I.perspective_camera(32, 4, W, H)
    lights = [I.random_light(s) for s in range(5)]
    pf = I.PlumeFrame(np.zeros((8, 8, 8), np.float32), None, cam, lights[0], 1.0)
    ctx = PT.make_ctx(pf)
    lm_dev = torch.from_numpy(lm).cuda()
    out = torch.full((4, H, W), float("nan"), dtype=torch.float32, device="cuda")
    ctx.shade(lm_dev, W, H, cam, lights, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = orc.shade(lm.astype(np.float64), cam, lights)
    errs = PT.range_err(got, ref)
    assert max(errs) <= PT.TOL_SHADE, errs
    # no lights: emissive and alpha only
    out.fill_(float("nan"))
    ctx.shade(lm_dev, W, H, cam, [], out)
    torch.cuda.synchronize()
    ref = orc.shade(lm.astype(np.float64), cam, [])
    assert max(PT.range_err(out.cpu().numpy().astype(np.float64), ref)) <= PT.TOL_SHADE
    ctx.close()


# ----------------------------------------------------------------------------
# whole frame through the host entry point
# ----------------------------------------------------------------------------

def test_render_frame_host_matches_device_calls(lib, orc):
    from paper_2604_03748_gb300 import nsl
    pf = I.config_plain_64()
    ctx = PT.make_ctx(pf)
    H, W = pf.camera.height, pf.camera.width
    guide = np.zeros((3, H, W), np.float32)
    lm = np.zeros((8, H, W), np.float32)
    rgba = np.zeros((4, H, W), np.float32)
    nsl.nsl_render_frame_host(ctx.ctx, pf.density, None, pf.camera, [pf.light], pf.step,
                              nsl.NSL_PREC_F32, guide, lm, rgba)
    o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    errs, bad = PT.compare_guide(guide.astype(np.float64), o, f)
    assert max(errs) <= PT.TOL_GUIDE
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref_lm = orc.net_forward(guide.astype(np.float64), flat, 16, 1.0 / math.sqrt(3 * 64 * 64))
    assert np.abs(lm - ref_lm).max() <= PT.TOL_NET_F32_ABS
    ref_rgba = orc.shade(lm.astype(np.float64), pf.camera, [pf.light])
    assert max(PT.range_err(rgba.astype(np.float64), ref_rgba)) <= PT.TOL_SHADE
    ctx.close()


@pytest.mark.parametrize("case", ["obstacle128_f32_mask", "ragged27_f16_mask", "thin3_f32"])
def test_render_frame_host_slab_upload_bitwise(lib, case):
    """The host entry point uploads the grid in slabs of z slices and stages
    each slab while the next one is copied; its guide, lightmaps and rgba equal
    the device-buffer calls (one staging of the whole grid) bit for bit: a
    masked 128^3 FP32 grid, a ragged masked FP16 grid, and a grid thinner
    (3 slices) than the number of slabs."""
    import dataclasses
    import torch
    from paper_2604_03748_gb300 import nsl
    if case == "obstacle128_f32_mask":
        pf = I.config_obstacle_128()
        pf = dataclasses.replace(pf, camera=dataclasses.replace(pf.camera, width=128, height=96))
    elif case == "ragged27_f16_mask":
        pf = I.small_case(27, 40, 24, seed=21, kind=I.PERSP, step=1.5)
        pf = dataclasses.replace(pf, density=pf.density.astype(np.float16))
    else:
        pf = I.small_case(20, 24, 16, seed=22, kind=I.ORTHO, step=2.0)
        pf = dataclasses.replace(pf, density=np.ascontiguousarray(pf.density[:3]),
                                 mask=np.ascontiguousarray(pf.mask[:3]))
    H, W = pf.camera.height, pf.camera.width
    dev = torch.device("cuda:0")
    ctx = PT.make_ctx(pf)
    d = torch.from_numpy(pf.density).to(dev)
    m = torch.from_numpy(pf.mask).to(dev)
    guide = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    lm = torch.empty((8, H, W), dtype=torch.float32, device=dev)
    rgba = torch.empty((4, H, W), dtype=torch.float32, device=dev)
    ctx.guiding_map(d, m, pf.camera, pf.step, guide)
    ctx.predict_lightmaps(guide, W, H, nsl.NSL_PREC_F16, lm)
    ctx.shade(lm, W, H, pf.camera, [pf.light], rgba)
    torch.cuda.synchronize()
    hg = np.zeros((3, H, W), np.float32)
    hl = np.zeros((8, H, W), np.float32)
    hr = np.zeros((4, H, W), np.float32)
    nsl.nsl_render_frame_host(ctx.ctx, pf.density, pf.mask, pf.camera, [pf.light], pf.step,
                              nsl.NSL_PREC_F16, hg, hl, hr)
    assert np.array_equal(hg, guide.cpu().numpy())
    assert np.array_equal(hl, lm.cpu().numpy())
    assert np.array_equal(hr, rgba.cpu().numpy())
    ctx.close()


def test_render_frame_host_async_two_contexts(lib):
    """Frames alternating between two contexts on two streams through the
    asynchronous host entry point equal the synchronous call, frame by frame
    (different cameras per frame, page-locked host buffers)."""
    import torch
    from paper_2604_03748_gb300 import nsl
    pf = I.config_plain_64()
    H, W = pf.camera.height, pf.camera.width
    cams = [I.orbit_ortho_camera(64, 40 + k, W, H) for k in range(6)]
    dens = torch.from_numpy(pf.density).pin_memory()
    ref = []
    ctx0 = PT.make_ctx(pf)
    for cam in cams:
        lm = np.zeros((8, H, W), np.float32)
        rgba = np.zeros((4, H, W), np.float32)
        nsl.nsl_render_frame_host(ctx0.ctx, pf.density, None, cam, [pf.light], pf.step, nsl.NSL_PREC_F16,
                                  None, lm, rgba)
        ref.append((lm, rgba))
    ctxs = [ctx0, PT.make_ctx(pf)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [(torch.zeros((8, H, W)).pin_memory(), torch.zeros((4, H, W)).pin_memory()) for _ in cams]
    for i, cam in enumerate(cams):
        if i >= 2:
            streams[i % 2].synchronize()
        nsl.nsl_render_frame_host_async(ctxs[i % 2].ctx, dens.numpy(), None, cam, [pf.light], pf.step,
                                        nsl.NSL_PREC_F16, None, outs[i][0].numpy(), outs[i][1].numpy(),
                                        stream=streams[i % 2])
    for s in streams:
        s.synchronize()
    for (lm, rgba), (glm, grgba) in zip(ref, outs):
        assert np.array_equal(glm.numpy(), lm)
        assert np.array_equal(grgba.numpy(), rgba)
    for c in ctxs:
        c.close()


def test_guide_parity_paper_step_10(lib, orc):
    """The paper's own sampling distance (h = 10 voxels) on the 512^2 obstacle
    workload, every pixel."""
    import dataclasses
    pf = dataclasses.replace(I.config_obstacle_128(), step=10.0)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf)
    o, s, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
    errs, bad = PT.compare_guide(g, o, f)
    assert max(errs) <= PT.TOL_GUIDE, errs
    assert bad <= PT.MAX_EXCUSED_FRAC * g[0].size
    ctx.close()


def test_guide_shadow_volume_with_early_termination(lib, orc):
    """Transmittance-volume mode with shadow rays stopped at t_min: a voxel
    ray whose stopping decision sits at the threshold moves that voxel's
    transmittance by at most about t_min, so the guide is held to 1e-4 of its
    range here (1e-5 with t_min = 0 above)."""
    pf = I.small_case(24, 32, 24, seed=11, kind=I.PERSP, step=2.0)
    ctx = PT.make_ctx(pf)
    g = PT.gpu_guide(ctx, pf, shadow_volume=1)
    o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step, shadow_volume=1)
    errs, bad = PT.compare_guide(g, o, f, tol=1e-4)
    assert max(errs) <= 1e-4, errs
    ctx.close()


def test_shadow_volume_rejected_where_unsupported(lib):
    """The option needs a context: the grouped and allocation-free paths refuse it."""
    import torch
    pf = I.small_case(16, 16, 16, seed=3, kind=I.ORTHO, step=2.0, with_mask=False)
    b = lib.Batch(I.pack_blob(I.make_params(16, 0), 16), 1)
    item = dict(density=torch.from_numpy(pf.density).cuda(), mask=None, camera=pf.camera, step=pf.step,
                light=pf.light, guide=torch.empty((3, 16, 16), device="cuda"),
                lightmaps=torch.empty((8, 16, 16), device="cuda"), rgba=torch.empty((4, 16, 16), device="cuda"))
    with pytest.raises(lib.NslError) as ei:
        b.render([item], lib.NSL_PREC_F16, opts=lib.march_opts(shadow_volume=1))
    assert ei.value.status == lib.NSL_ERR_UNSUPPORTED
    b.close()
