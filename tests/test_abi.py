"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/nsl.h declares.  No compute calls (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "nsl.h")).read()
    return sorted(set(re.findall(r"NSL_API\s+[\w\s\*]*?\b(nsl_\w+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("nsl_create", "nsl_guiding_map", "nsl_predict_lightmaps", "nsl_shade", "nsl_destroy"):
        assert n in names


def test_library_builds_and_exports_all_symbols():
    from paper_2604_03748_gb300 import build, nsl
    path = build.build()
    assert os.path.exists(path)
    lib = nsl.load()
    for n in declared_symbols():
        assert hasattr(lib, n), n
    assert sorted(nsl.EXPORTS) == sorted(declared_symbols()) or set(declared_symbols()) <= set(nsl.EXPORTS)


def test_status_strings_without_gpu():
    from paper_2604_03748_gb300 import nsl
    lib = nsl.load()
    assert lib.nsl_status_str(0) == b"ok"
    assert lib.nsl_status_str(1) == b"invalid argument"


def test_create_rejects_bad_blob_without_touching_the_gpu():
    """Blob validation happens before any CUDA call."""
    from paper_2604_03748_gb300 import nsl
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_create(8, 8, 8, nsl.NSL_F32, 1.0, b"XXXX" + b"\0" * 40, 64, 64)
    assert ei.value.status == nsl.NSL_ERR_INVALID_ARG
    from paper_2604_03748_gb300 import inputs as I
    blob = bytearray(I.pack_blob(I.make_params(16), 16))
    blob[40] ^= 1  # corrupt one parameter byte: checksum must catch it
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_create(8, 8, 8, nsl.NSL_F32, 1.0, bytes(blob), 64, 64)
    assert "checksum" in str(ei.value)
    blob8 = I.pack_blob(I.make_params(8), 8)
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_create(8, 8, 8, nsl.NSL_F32, 1.0, blob8, 64, 64)
    assert ei.value.status == nsl.NSL_ERR_UNSUPPORTED


def test_create_rejects_grids_past_32_bit_cell_indices_without_touching_the_gpu():
    """Grid dimensions are checked before any CUDA call: each axis in
    [1, 4096] and (nx+1)(ny+1)(nz+2) staged cells below 2^32."""
    from paper_2604_03748_gb300 import inputs as I, nsl
    blob = I.pack_blob(I.make_params(16), 16)
    for dims in ((0, 8, 8), (8, 4097, 8), (2048, 2048, 1024), (4096, 4096, 300)):
        with pytest.raises(nsl.NslError) as ei:
            nsl.nsl_create(*dims, nsl.NSL_F32, 1.0, blob, 64, 64)
        assert ei.value.status == nsl.NSL_ERR_INVALID_ARG, dims


def test_default_options_without_gpu():
    """Documented defaults: t_min 1e-4 (early termination), tau_depth 0.01,
    jitter on, unit surrogate intensities, HG g = 0, front/top/bottom lights;
    the server's 40 GiB budget, 2 streams, batches of up to 64 requests and 1 Mi pixels
    with requests of up to 256^2 pixels first, FP16 network."""
    from paper_2604_03748_gb300 import nsl
    o = nsl.march_opts()
    assert o.t_min == pytest.approx(1e-4) and o.tau_depth == pytest.approx(0.01)
    assert o.jitter == 1 and o.seed == 0 and o.frame == 0 and o.phase_g == 0.0
    assert list(o.surrogate_I) == [1.0, 1.0, 1.0]
    assert o.segment_exact == 0 and o.light_set == nsl.NSL_LIGHTS_FTB and o.shadow_volume == 0
    s = nsl.server_opts()
    assert s.hbm_budget_bytes == 40 << 30 and s.streams == 2 and s.max_batch == 64
    assert s.max_batch_pixels == 1 << 20 and s.small_first_pixels == 256 * 256
    assert s.precision == nsl.NSL_PREC_F16 and s.scratch_bytes_per_stream == 0
    assert s.march.t_min == pytest.approx(1e-4) and s.march.jitter == 1


def test_precision_codes_and_trace_size_without_gpu():
    """The precision codes of include/nsl.h, and the trace size: 144 stored
    activation values per pixel (the 17 network tensors) at four bytes, enough
    for the binary32 trace of the split-BF16 form."""
    import re
    from paper_2604_03748_gb300 import nsl
    hdr = open(os.path.join(ROOT, "include", "nsl.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"(NSL_PREC_\w+) = (\d+)", hdr))
    assert codes == {"NSL_PREC_F32": nsl.NSL_PREC_F32, "NSL_PREC_BF16": nsl.NSL_PREC_BF16,
                     "NSL_PREC_FP8": nsl.NSL_PREC_FP8, "NSL_PREC_F16": nsl.NSL_PREC_F16,
                     "NSL_PREC_BF16X3": nsl.NSL_PREC_BF16X3}
    lib = nsl.load()
    assert lib.nsl_lightmap_trace_bytes(512, 256) == 512 * 256 * 144 * 4
    assert lib.nsl_lightmap_trace_bytes(0, 8) == 0


def test_null_handles_rejected_without_gpu():
    """Host-side argument checks return an error status and set the last-error
    message before any CUDA call."""
    import ctypes as C
    from paper_2604_03748_gb300 import nsl
    lib = nsl.load()
    st = lib.nsl_server_create(None, 0, None, None)
    assert st == nsl.NSL_ERR_INVALID_ARG and b"NULL" in lib.nsl_last_error()
    out = C.c_void_p()
    bad = nsl.server_opts(streams=0)
    st = lib.nsl_server_create(None, 0, C.byref(bad), C.byref(out))
    assert st == nsl.NSL_ERR_INVALID_ARG and not out.value


def test_binding_refuses_undersized_buffers_without_gpu():
    """The C ABI takes plain pointers; the binding checks each buffer's element
    count against the sizes of the call before anything reaches the library
    (CPU tensors here: the size check comes before the device check)."""
    import torch
    from paper_2604_03748_gb300 import inputs as I, nsl
    H, W = 16, 24
    small = torch.empty(3 * H * W - 1)
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_predict_lightmaps(None, small, W, H, nsl.NSL_PREC_F32, torch.empty(8 * H * W))
    assert ei.value.status == nsl.NSL_ERR_INVALID_ARG and "guide" in str(ei.value)
    with pytest.raises(nsl.NslError):
        nsl.nsl_predict_lightmaps(None, torch.empty(3 * H * W), W, H, nsl.NSL_PREC_F32, torch.empty(8 * H * W - 8))
    with pytest.raises(nsl.NslError):
        nsl.nsl_shade(None, torch.empty(8 * H * W), W, H, I.perspective_camera(16, 1, W, H), [],
                      torch.empty((3, H, W)))
    cam = I.perspective_camera(16, 1, W, H)
    with pytest.raises(nsl.NslError):
        nsl.nsl_guiding_map(None, torch.empty(16 ** 3), None, cam, 2.0, torch.empty((3, H, W - 8)))
    item = dict(density=torch.empty((16, 16, 16)), mask=None, camera=cam, step=2.0,
                light=I.random_light(1), guide=torch.empty((3, H, W)), lightmaps=torch.empty((8, H, W - 1)),
                rgba=None)
    with pytest.raises(nsl.NslError) as ei:
        nsl.plume_array([item])
    assert "lightmaps" in str(ei.value)
    # buffers of the right size get as far as the device check
    with pytest.raises(ValueError):
        nsl.nsl_predict_lightmaps(None, torch.empty(3 * H * W), W, H, nsl.NSL_PREC_F32, torch.empty(8 * H * W))


def test_binding_refuses_a_density_of_the_wrong_type_without_gpu():
    """A float16 density passed for a float32 grid would be read past its end by
    the staging kernel: the binding refuses it before the call, for the
    allocation-free entry point and for a context's grid (CPU tensors here)."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_2604_03748_gb300 import inputs as I, nsl
    cam = I.perspective_camera(16, 1, 16, 16)
    g = torch.empty((3, 16, 16))
    half = torch.empty((16, 16, 16), dtype=torch.float16)
    with pytest.raises(nsl.NslError) as ei:
        nsl.nsl_guiding_map_noalloc(half.shape, nsl.NSL_F32, 1.0, half, None, cam, 2.0, g)
    assert ei.value.status == nsl.NSL_ERR_INVALID_ARG and "float16" in str(ei.value)
    with pytest.raises(nsl.NslError):
        nsl.nsl_guiding_map_noalloc(half.shape, nsl.NSL_F16, 1.0, half.float(), None, cam, 2.0, g)
    fake = C.c_void_p(0x10000)   # a handle the binding knows, never passed to the library
    nsl._ctx_grid[fake.value] = (16 ** 3, nsl.NSL_F32)
    try:
        for fn in (lambda: nsl.nsl_stage_grid(fake, half, None),
                   lambda: nsl.nsl_guiding_map(fake, half, None, cam, 2.0, g),
                   lambda: nsl.nsl_render_frame_host(fake, half.numpy(), None, cam, [], 2.0, nsl.NSL_PREC_F32)):
            with pytest.raises(nsl.NslError) as ei:
                fn()
            assert "float16" in str(ei.value)
        with pytest.raises(nsl.NslError):   # right type, too few voxels
            nsl.nsl_stage_grid(fake, torch.empty(16 ** 3 - 1), None)
        with pytest.raises(nsl.NslError):   # a numpy host buffer, too few voxels
            nsl.nsl_render_frame_host(fake, np.empty(16 ** 3 - 1, np.float32), None, cam, [], 2.0,
                                      nsl.NSL_PREC_F32)
    finally:
        nsl._ctx_grid.pop(fake.value, None)


def test_noalloc_size_limit_without_gpu():
    """The allocation-free entry point's scratch holds a float32 136^3 grid and
    a float16 172^3 one; one voxel more per axis is refused by the size check,
    which runs before any CUDA call (the pointers below are never read)."""
    import ctypes as C
    from paper_2604_03748_gb300 import inputs as I, nsl
    lib = nsl.load()
    cam = nsl.camera(I.perspective_camera(16, 1, 16, 16))
    fake = C.c_void_p(0x10000)
    for n, dt in ((137, nsl.NSL_F32), (173, nsl.NSL_F16)):
        g = nsl.nsl_grid_desc(n, n, n, dt, 1.0)
        st = lib.nsl_guiding_map_noalloc(C.byref(g), fake, None, C.byref(cam), 2.0, None, fake, None)
        assert st == nsl.NSL_ERR_INVALID_ARG, n
        assert b"scratch" in lib.nsl_last_error()
    # the limits themselves: 16 or 8 bytes per cell of (n+1)^2 (n+2) cells
    lim = 40 << 20
    assert 137 * 137 * 138 * 16 <= lim < 138 * 138 * 139 * 16
    assert 173 * 173 * 174 * 8 <= lim < 174 * 174 * 175 * 8
