"""Batched frames through the C ABI: one call renders many plumes of different
grid and billboard sizes.  Each plume's guide, lightmaps and shading must equal
what the single-plume entry points give for it (same kernels per pixel, same
fixed summation orders), and a small plume is also checked against the FP64
oracle directly.  Graph capture, table updates between replays and the
autotuner are covered here as well."""
import math
import os

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I
import parity as PT

pytestmark = pytest.mark.gpu

C0 = 16


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


def _frames():
    """Six plumes: FP32 and FP16 grids, with and without obstacle masks,
    orthographic and perspective cameras, billboards from 16x8 to 256^2."""
    out = [
        I.small_case(24, 32, 24, seed=21, kind=I.PERSP, step=2.0),
        I.small_case(20, 40, 16, seed=22, kind=I.ORTHO, step=3.0, with_mask=False),
        I.small_case(32, 64, 64, seed=23, kind=I.PERSP, step=2.0),
    ]
    n = 48
    vol = I.blob_fbm_volume(n, 24).astype(np.float16)
    cam = I.perspective_camera(n, 24, 128, 96)
    out.append(I.PlumeFrame(vol, None, cam, I.random_light(24), 2.0, sigma_scale=0.7))
    n = 64
    vol = I.blob_fbm_volume(n, 25)
    mask, _ = I.sphere_mask(n, n / 6.0, 25)
    cam = I.orbit_ortho_camera(n, 25, 256, 256)
    out.append(I.PlumeFrame(vol, mask, cam, I.random_light(25), 4.0))
    vol = np.zeros((9, 7, 11), np.float32)
    out.append(I.PlumeFrame(vol, None, I.perspective_camera(11, 2, 16, 8), I.random_light(2), 1.5))
    return out


def _device_plumes(frames, with_rgba=True):
    import torch
    dev = torch.device("cuda:0")
    items = []
    for pf in frames:
        H, W = pf.camera.height, pf.camera.width
        items.append(dict(
            density=torch.from_numpy(np.ascontiguousarray(pf.density)).to(dev),
            mask=None if pf.mask is None else torch.from_numpy(np.ascontiguousarray(pf.mask)).to(dev),
            sigma_scale=pf.sigma_scale, camera=pf.camera, step=pf.step, light=pf.light,
            guide=torch.full((3, H, W), float("nan"), dtype=torch.float32, device=dev),
            lightmaps=torch.full((8, H, W), float("nan"), dtype=torch.float32, device=dev),
            rgba=torch.full((4, H, W), float("nan"), dtype=torch.float32, device=dev) if with_rgba else None))
    return items


def _single(lib, pf, precision, guide=None):
    """The single-plume entry points on one frame: guide, lightmaps, rgba (the
    network and shading on `guide` when given)."""
    import torch
    ctx = PT.make_ctx(pf, c0=C0)
    g = PT.gpu_guide(ctx, pf) if guide is None else guide
    dev = torch.device("cuda:0")
    H, W = pf.camera.height, pf.camera.width
    gd = torch.from_numpy(g.astype(np.float32)).to(dev)
    lm = torch.empty((8, H, W), dtype=torch.float32, device=dev)
    ctx.predict_lightmaps(gd, W, H, precision, lm)
    rgba = torch.empty((4, H, W), dtype=torch.float32, device=dev)
    ctx.shade(lm, W, H, pf.camera, [pf.light], rgba)
    torch.cuda.synchronize()
    out = (g, lm.cpu().numpy().astype(np.float64), rgba.cpu().numpy().astype(np.float64))
    ctx.close()
    return out


def _host(items, key):
    import torch
    torch.cuda.synchronize()
    return [it[key].cpu().numpy().astype(np.float64) for it in items]


@pytest.mark.parametrize("precision", [3, 1, 2, 4], ids=["f16", "bf16", "fp8", "bf16x3"])
def test_batch_equals_single_plume_path(lib, precision):
    frames = _frames()
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=8)
    items = _device_plumes(frames)
    b.render(items, precision)
    guides, lms, rgbas = _host(items, "guide"), _host(items, "lightmaps"), _host(items, "rgba")
    for k, pf in enumerate(frames):
        # the grouped march takes every shadow sample at its exact position,
        # the single-plume march the in-ray ones from p - 0.5 + k h u: the
        # guides agree to rounding
        g1, _, _ = _single(lib, pf, precision)
        for c in range(3):
            assert np.abs(guides[k][c] - g1[c]).max() <= 1e-6 * max(np.abs(g1[c]).max(), 1e-30), (k, c)
        # the same network and shading kernels: bitwise on the batch's guide
        _, lm1, rgba1 = _single(lib, pf, precision, guide=guides[k])
        assert np.array_equal(lms[k], lm1), k
        assert np.allclose(rgbas[k], rgba1, rtol=1e-6, atol=1e-7), k
    # a second render of the same batch is bitwise identical (deterministic)
    b.render(items, precision)
    assert all(np.array_equal(a, c) for a, c in zip(_host(items, "lightmaps"), lms))
    b.close()


def test_batch_against_oracle(lib, orc):
    """A three-plume batch checked plume by plume against the FP64 oracle:
    guide within the march tolerance, FP16 lightmaps within the FP16 bound on
    the oracle's own network evaluated on the batch's guide, shading of the
    batch's lightmaps within the shading tolerance."""
    frames = _frames()[:3]
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=3)
    items = _device_plumes(frames)
    b.render(items, 3)
    guides, lms, rgbas = _host(items, "guide"), _host(items, "lightmaps"), _host(items, "rgba")
    flat = I.flat_params(I.make_params(C0, 0)).astype(np.float64)
    for k, pf in enumerate(frames):
        o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step)
        errs, bad = PT.compare_guide(guides[k], o, f)
        assert max(errs) <= PT.TOL_GUIDE, (k, errs)
        assert bad <= max(1, PT.MAX_EXCUSED_FRAC * o[0].size)
        n = pf.density.shape[0]
        ref = orc.net_forward(guides[k].astype(np.float32).astype(np.float64), flat, C0,
                              1.0 / math.sqrt(3 * n * n))
        assert max(PT.range_err(lms[k], ref)) <= PT.TOL_NET_F16, k
        ref_rgba = orc.shade(lms[k].astype(np.float32).astype(np.float64), pf.camera, [pf.light])
        assert max(PT.range_err(rgbas[k], ref_rgba)) <= PT.TOL_SHADE, k
    b.close()


@pytest.mark.parametrize("opts", [dict(light_set=1), dict(light_set=2, phase_g=0.3),
                                  dict(segment_exact=1, jitter=0)])
def test_batch_march_options_against_oracle(lib, orc, opts):
    """The march options reach the grouped march: light sets of the Sec. 5
    ablation, HG phase, segment-exact A_n, no jitter."""
    frames = _frames()[:3]
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=3)
    items = _device_plumes(frames)
    b.render(items, 3, opts=lib.march_opts(**opts))
    guides = _host(items, "guide")
    for k, pf in enumerate(frames):
        o, _, f = orc.guide(pf.density, pf.mask, pf.camera, pf.step, **opts)
        errs, bad = PT.compare_guide(guides[k], o, f)
        assert max(errs) <= PT.TOL_GUIDE, (k, errs)
        assert bad <= max(1, PT.MAX_EXCUSED_FRAC * o[0].size)
    b.close()


def test_batch_graph_replay_and_update(lib):
    import torch
    frames = _frames()
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=8)
    items = _device_plumes(frames)
    s = torch.cuda.Stream()
    b.render(items, 3, stream=s)
    s.synchronize()
    want = [_host(items, k) for k in ("guide", "lightmaps", "rgba")]
    for it in items:
        for key in ("guide", "lightmaps", "rgba"):
            it[key].fill_(float("nan"))
    b.capture_graph(items, 3, s)
    for it in items:
        for key in ("guide", "lightmaps", "rgba"):
            it[key].fill_(float("nan"))
    torch.cuda.synchronize()
    for _ in range(2):
        b.launch_graph(s)
    s.synchronize()
    got = [_host(items, k) for k in ("guide", "lightmaps", "rgba")]
    for w, g in zip(want, got):
        assert all(np.array_equal(a, c) for a, c in zip(w, g))
    before = got[0]

    # new cameras and lights through the graph == a plain render with them
    moved = []
    for k, pf in enumerate(frames):
        n = pf.density.shape[0]
        W, H = pf.camera.width, pf.camera.height
        cam = (I.perspective_camera(n, 100 + k, W, H) if pf.camera.kind == I.PERSP
               else I.orbit_ortho_camera(n, 100 + k, W, H))
        moved.append(I.PlumeFrame(pf.density, pf.mask, cam, I.random_light(100 + k), pf.step,
                                  sigma_scale=pf.sigma_scale))
    items2 = [dict(it, camera=m.camera, light=m.light) for it, m in zip(items, moved)]
    b.update_graph(items2)
    b.launch_graph(s)
    s.synchronize()
    got = [_host(items2, k) for k in ("guide", "lightmaps", "rgba")]
    ref_items = _device_plumes(moved)
    b2 = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=8)
    b2.render(ref_items, 3)
    want = [_host(ref_items, k) for k in ("guide", "lightmaps", "rgba")]
    for w, g in zip(want, got):
        assert all(np.array_equal(a, c) for a, c in zip(w, g))
    assert not np.array_equal(got[0][4], before[4])        # the update took effect

    # a size change is refused
    bad = [dict(it) for it in items2]
    bad[0]["step"] = bad[0]["step"] * 2
    with pytest.raises(lib.NslError):
        b.update_graph(bad)
    b.close()
    b2.close()


def test_batch_autotune_and_cache(lib, tmp_path):
    import torch
    frames = _frames()[:4]
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=4)
    items = _device_plumes(frames)
    cache = str(tmp_path / "tune.jsonl")
    ms = b.autotune(items, 3, cache_path=cache)
    assert ms > 0
    seg_len, mb, cc = b.get_tuning()
    assert seg_len in (4, 6, 8) and mb in (0, 5, 6) and cc in (1, 2, 4)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    # the cached entry is applied without timing: plant a marker time and tuning
    import json
    rec = json.loads(lines[0])
    assert rec["march_tile_width"] in (4, 8) and rec["persistent_march"] in (0, 1)
    rec.update(seg_len=8, march_blocks_per_sm=4, conv_ctas_per_sm=1, march_tile_width=16, persistent_march=0,
               ms=123.5)
    with open(cache, "w") as f:
        f.write(json.dumps(rec) + "\n")
    ms2 = b.autotune(items, 3, cache_path=cache)
    assert abs(ms2 - 123.5) < 1e-3 and b.get_tuning() == (8, 4, 1) and b.get_march_tile() == 16
    assert b.get_march_form() == 0
    # every pixel marches the same whatever the warp's tile: bitwise equal guides
    b.render(items, 3)
    g16 = _host(items, "guide")
    b.set_march_tile(4)
    b.render(items, 3)
    for a, c in zip(g16, _host(items, "guide")):
        assert np.array_equal(a, c)
    with pytest.raises(lib.NslError):
        b.set_march_tile(6)
    b.set_march_tile(8)
    # another segment length groups the per-segment in-scattering partial sums
    # differently: the guide moves by rounding only, the lightmaps by what
    # the network makes of that; the same tuning again is bitwise identical
    b.render(items, 3)
    ref = _host(items, "guide"), _host(items, "lightmaps")
    b.set_tuning(4, 0, 2)
    b.render(items, 3)
    got = _host(items, "guide"), _host(items, "lightmaps")
    for a, c in zip(ref[0], got[0]):
        assert max(PT.range_err(c, a)) <= PT.TOL_GUIDE
    for a, c in zip(ref[1], got[1]):
        assert max(PT.range_err(c, a)) <= PT.TOL_NET_F16
    b.set_tuning(8, 4, 1)
    b.render(items, 3)
    again = _host(items, "guide"), _host(items, "lightmaps")
    for r, g in zip(ref, again):
        assert all(np.array_equal(a, c) for a, c in zip(r, g))
    b.close()


def test_batch_errors(lib):
    import torch
    frames = _frames()[:2]
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=2)
    items = _device_plumes(frames)
    with pytest.raises(lib.NslError):
        b.render(items, 0)                          # FP32 network is not batched
    with pytest.raises(lib.NslError):
        b.render(items * 2, 3)                      # more than max_plumes
    with pytest.raises(lib.NslError):
        b.launch_graph(None)                        # nothing captured
    bad = [dict(it) for it in items]
    H, W = frames[0].camera.height, frames[0].camera.width
    buf = torch.empty(3 * H * W + 1, dtype=torch.float32, device="cuda")
    bad[0]["guide"] = buf[1:].view(3, H, W)         # 4-byte offset: not 16-byte aligned
    with pytest.raises(lib.NslError):
        b.render(bad, 3)
    b.render(items, 3)                              # still usable
    torch.cuda.synchronize()
    b.close()


def test_persistent_march_equals_three_passes(lib):
    """The batched march as one cooperative launch with grid-wide barriers gives
    bitwise the guides (and so the lightmaps) of its three-launch form, with
    float16 and float32 grids, and inside a captured graph."""
    import torch
    frames = _frames()
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=len(frames))
    items = _device_plumes(frames)
    b.set_march_form(0)
    b.render(items, 3)
    ref = _host(items, "guide"), _host(items, "lightmaps")
    b.set_march_form(1)
    assert b.get_march_form() == 1
    for _ in range(2):                       # twice: the barrier words are reused
        b.render(items, 3)
        got = _host(items, "guide"), _host(items, "lightmaps")
        for r, g in zip(ref, got):
            assert all(np.array_equal(a, c) for a, c in zip(r, g))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.capture_graph(items, 3, stream)
        for it in items:
            it["guide"].zero_()
        b.launch_graph(stream)
    stream.synchronize()
    for a, c in zip(ref[0], _host(items, "guide")):
        assert np.array_equal(a, c)
    with pytest.raises(lib.NslError):
        b.set_march_form(2)
    b.close()
