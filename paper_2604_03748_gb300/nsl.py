"""Thin ctypes binding of libnsl.so (the C ABI declared in include/nsl.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device
memory and streams).  The library must have been built (``build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnsl.so")

NSL_OK, NSL_ERR_INVALID_ARG, NSL_ERR_OOM, NSL_ERR_CUDA, NSL_ERR_UNSUPPORTED, NSL_ERR_TIMEOUT, NSL_ERR_BUDGET = range(7)
NSL_F32, NSL_F16 = 0, 1
NSL_PREC_F32, NSL_PREC_BF16, NSL_PREC_FP8, NSL_PREC_F16, NSL_PREC_BF16X3 = 0, 1, 2, 3, 4
NSL_CAM_ORTHO, NSL_CAM_PERSP = 0, 1
NSL_LIGHTS_FTB, NSL_LIGHTS_F, NSL_LIGHTS_FLR = 0, 1, 2
NSL_TEX_RGBA8, NSL_TEX_RGBA16F, NSL_TEX_RGBA32F = 0, 1, 2

# every symbol include/nsl.h declares
EXPORTS = ["nsl_default_march_opts", "nsl_create", "nsl_destroy", "nsl_stage_grid",
           "nsl_guiding_map", "nsl_guiding_map_noalloc", "nsl_guide_sample_count",
           "nsl_predict_lightmaps", "nsl_shade", "nsl_render_frame_host", "nsl_last_error",
           "nsl_status_str", "nsl_render_frame_host_async", "nsl_batch_create", "nsl_batch_destroy", "nsl_batch_render",
           "nsl_batch_capture_graph", "nsl_batch_update_graph", "nsl_batch_launch_graph",
           "nsl_batch_set_tuning", "nsl_batch_get_tuning", "nsl_batch_autotune",
           "nsl_default_server_opts", "nsl_server_create", "nsl_server_destroy",
           "nsl_server_add_plume", "nsl_server_remove_plume", "nsl_server_submit", "nsl_server_wait",
           "nsl_server_drain", "nsl_server_plume_state", "nsl_server_get_stats",
           "nsl_server_reset_stats", "nsl_pack_lightmaps", "nsl_obstacle_shadow_map",
           "nsl_shade_shadowed", "nsl_selftest_wait_timeout", "nsl_predict_lightmaps_trace",
           "nsl_lightmap_trace_bytes", "nsl_measure_peaks", "nsl_reference_lightmaps",
           "nsl_default_train_opts", "nsl_trainer_create", "nsl_trainer_step", "nsl_trainer_gradients",
           "nsl_trainer_get_blob", "nsl_trainer_destroy", "nsl_trainer_set_lr", "nsl_batch_set_march_tile",
           "nsl_batch_get_march_tile", "nsl_batch_set_march_form", "nsl_batch_get_march_form"]


class nsl_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dtype", C.c_int),
                ("sigma_scale", C.c_float)]


class nsl_camera(C.Structure):
    _fields_ = [("kind", C.c_int), ("eye", C.c_float * 3), ("target", C.c_float * 3),
                ("up", C.c_float * 3), ("fov_y_deg", C.c_float), ("ortho_height", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class nsl_light(C.Structure):
    _fields_ = [("dir", C.c_float * 3), ("intensity", C.c_float * 3)]


class nsl_march_opts(C.Structure):
    _fields_ = [("tau_depth", C.c_float), ("t_min", C.c_float), ("jitter", C.c_int),
                ("seed", C.c_uint32), ("frame", C.c_uint32), ("phase_g", C.c_float),
                ("surrogate_I", C.c_float * 3), ("segment_exact", C.c_int), ("light_set", C.c_int),
                ("shadow_volume", C.c_int)]


class nsl_plume(C.Structure):
    _fields_ = [("density_dev", C.c_void_p), ("mask_dev", C.c_void_p), ("grid", nsl_grid_desc),
                ("camera", nsl_camera), ("step_voxels", C.c_float), ("light", nsl_light),
                ("guide_dev", C.c_void_p), ("lightmaps_dev", C.c_void_p), ("rgba_dev", C.c_void_p)]


class nsl_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("scratch_bytes_per_stream", C.c_size_t),
                ("streams", C.c_int), ("max_batch", C.c_int), ("precision", C.c_int),
                ("march", nsl_march_opts), ("max_batch_pixels", C.c_size_t), ("small_first_pixels", C.c_size_t)]


class nsl_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("queued", C.c_uint64), ("running", C.c_uint64), ("batches", C.c_uint64),
                ("admissions", C.c_uint64), ("evictions", C.c_uint64), ("pixels_completed", C.c_double),
                ("resident_plumes", C.c_int), ("resident_bytes", C.c_size_t), ("used_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("mean_batch", C.c_double), ("busy_s", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class nsl_peaks(C.Structure):
    _fields_ = [("sms", C.c_int), ("fp32_tflops", C.c_double), ("l1_gbps", C.c_double),
                ("l2_gather_gbps", C.c_double)]


class nsl_train_opts(C.Structure):
    _fields_ = [("batch", C.c_int), ("width", C.c_int), ("height", C.c_int), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("plane_weight", C.c_float * 8)]


class NslError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libnsl.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is not built; run paper_2604_03748_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, f = C.c_void_p, C.c_int, C.c_float
    lib.nsl_default_march_opts.argtypes = [C.POINTER(nsl_march_opts)]
    lib.nsl_default_march_opts.restype = None
    lib.nsl_create.argtypes = [C.POINTER(nsl_grid_desc), vp, C.c_size_t, i, i, C.POINTER(vp)]
    lib.nsl_destroy.argtypes = [vp]
    lib.nsl_destroy.restype = None
    lib.nsl_guiding_map.argtypes = [vp, vp, vp, C.POINTER(nsl_camera), C.POINTER(nsl_light), f,
                                    C.POINTER(nsl_march_opts), vp, vp]
    lib.nsl_stage_grid.argtypes = [vp, vp, vp, vp]
    lib.nsl_guiding_map_noalloc.argtypes = [C.POINTER(nsl_grid_desc), vp, vp, C.POINTER(nsl_camera),
                                            f, C.POINTER(nsl_march_opts), vp, vp]
    lib.nsl_guide_sample_count.argtypes = [vp, C.POINTER(nsl_camera), f, C.POINTER(nsl_march_opts),
                                           C.POINTER(C.c_ulonglong), vp]
    lib.nsl_predict_lightmaps.argtypes = [vp, vp, i, i, i, vp, vp]
    lib.nsl_predict_lightmaps_trace.argtypes = [vp, vp, i, i, i, vp, vp, C.c_size_t, vp]
    lib.nsl_predict_lightmaps_trace.restype = C.c_int
    lib.nsl_reference_lightmaps.argtypes = [vp, vp, vp, C.POINTER(nsl_camera), f, f, vp, vp]
    lib.nsl_reference_lightmaps.restype = C.c_int
    lib.nsl_default_train_opts.argtypes = [C.POINTER(nsl_train_opts)]
    lib.nsl_default_train_opts.restype = None
    lib.nsl_trainer_create.argtypes = [vp, C.c_size_t, C.POINTER(nsl_train_opts), C.POINTER(vp)]
    lib.nsl_trainer_step.argtypes = [vp, vp, vp, f, i, C.POINTER(C.c_float), vp]
    lib.nsl_trainer_gradients.argtypes = [vp, vp, C.c_size_t, vp]
    lib.nsl_trainer_get_blob.argtypes = [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    lib.nsl_trainer_set_lr.argtypes = [vp, f]
    for name in ("nsl_trainer_create", "nsl_trainer_step", "nsl_trainer_gradients", "nsl_trainer_get_blob",
                 "nsl_trainer_set_lr"):
        getattr(lib, name).restype = C.c_int
    lib.nsl_trainer_destroy.argtypes = [vp]
    lib.nsl_trainer_destroy.restype = None
    lib.nsl_measure_peaks.argtypes = [C.POINTER(nsl_peaks), vp]
    lib.nsl_measure_peaks.restype = C.c_int
    lib.nsl_lightmap_trace_bytes.argtypes = [i, i]
    lib.nsl_lightmap_trace_bytes.restype = C.c_size_t
    lib.nsl_shade.argtypes = [vp, vp, i, i, C.POINTER(nsl_camera), C.POINTER(nsl_light), i, vp, vp]
    lib.nsl_pack_lightmaps.argtypes = [vp, i, i, i, vp, vp, vp]
    lib.nsl_pack_lightmaps.restype = C.c_int
    lib.nsl_selftest_wait_timeout.argtypes = [vp, vp]
    lib.nsl_selftest_wait_timeout.restype = C.c_int
    lib.nsl_obstacle_shadow_map.argtypes = [vp, i, i, i, C.POINTER(C.c_float * 3), i, vp, vp]
    lib.nsl_obstacle_shadow_map.restype = C.c_int
    lib.nsl_shade_shadowed.argtypes = [vp, vp, vp, i, i, C.POINTER(nsl_camera), C.POINTER(nsl_light), i,
                                       C.POINTER(vp), i, f, vp, vp]
    lib.nsl_shade_shadowed.restype = C.c_int
    lib.nsl_render_frame_host.argtypes = [vp, vp, vp, C.POINTER(nsl_camera), C.POINTER(nsl_light),
                                          i, f, C.POINTER(nsl_march_opts), i, vp, vp, vp, vp]
    lib.nsl_render_frame_host_async.argtypes = lib.nsl_render_frame_host.argtypes
    lib.nsl_render_frame_host_async.restype = C.c_int
    lib.nsl_batch_create.argtypes = [vp, C.c_size_t, i, C.POINTER(vp)]
    lib.nsl_batch_destroy.argtypes = [vp]
    lib.nsl_batch_destroy.restype = None
    lib.nsl_batch_render.argtypes = [vp, C.POINTER(nsl_plume), i, C.POINTER(nsl_march_opts), i, vp]
    lib.nsl_batch_capture_graph.argtypes = [vp, C.POINTER(nsl_plume), i, C.POINTER(nsl_march_opts), i, vp]
    lib.nsl_batch_update_graph.argtypes = [vp, C.POINTER(nsl_plume), i, C.POINTER(nsl_march_opts)]
    lib.nsl_batch_launch_graph.argtypes = [vp, vp]
    lib.nsl_batch_set_tuning.argtypes = [vp, i, i, i]
    lib.nsl_batch_get_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.nsl_batch_set_march_tile.argtypes = [vp, i]
    lib.nsl_batch_get_march_tile.argtypes = [vp, C.POINTER(C.c_int)]
    lib.nsl_batch_set_march_form.argtypes = [vp, i]
    lib.nsl_batch_get_march_form.argtypes = [vp, C.POINTER(C.c_int)]
    lib.nsl_batch_autotune.argtypes = [vp, C.POINTER(nsl_plume), i, C.POINTER(nsl_march_opts), i,
                                       C.c_char_p, vp, C.POINTER(C.c_float)]
    for name in ("nsl_batch_create", "nsl_batch_render", "nsl_batch_capture_graph",
                 "nsl_batch_update_graph", "nsl_batch_launch_graph", "nsl_batch_set_tuning",
                 "nsl_batch_get_tuning", "nsl_batch_autotune", "nsl_batch_set_march_tile",
                 "nsl_batch_get_march_tile", "nsl_batch_set_march_form", "nsl_batch_get_march_form"):
        getattr(lib, name).restype = C.c_int
    lib.nsl_default_server_opts.argtypes = [C.POINTER(nsl_server_opts)]
    lib.nsl_default_server_opts.restype = None
    lib.nsl_server_create.argtypes = [vp, C.c_size_t, C.POINTER(nsl_server_opts), C.POINTER(vp)]
    lib.nsl_server_destroy.argtypes = [vp]
    lib.nsl_server_destroy.restype = None
    lib.nsl_server_add_plume.argtypes = [vp, C.POINTER(nsl_grid_desc), vp, vp, C.c_float, i, i,
                                         C.POINTER(C.c_int)]
    lib.nsl_server_remove_plume.argtypes = [vp, i]
    lib.nsl_server_submit.argtypes = [vp, i, C.POINTER(nsl_camera), C.POINTER(nsl_light), vp, vp,
                                      C.POINTER(C.c_uint64)]
    lib.nsl_server_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(C.c_double)]
    lib.nsl_server_drain.argtypes = [vp, C.c_double]
    lib.nsl_server_plume_state.argtypes = [vp, i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                           C.POINTER(C.c_int)]
    lib.nsl_server_get_stats.argtypes = [vp, C.POINTER(nsl_server_stats)]
    lib.nsl_server_reset_stats.argtypes = [vp]
    for name in ("nsl_server_create", "nsl_server_add_plume", "nsl_server_remove_plume",
                 "nsl_server_submit", "nsl_server_wait", "nsl_server_drain", "nsl_server_plume_state",
                 "nsl_server_get_stats", "nsl_server_reset_stats"):
        getattr(lib, name).restype = C.c_int
    lib.nsl_last_error.argtypes = []
    lib.nsl_last_error.restype = C.c_char_p
    lib.nsl_status_str.argtypes = [i]
    lib.nsl_status_str.restype = C.c_char_p
    for name in ("nsl_create", "nsl_stage_grid", "nsl_guiding_map", "nsl_guiding_map_noalloc",
                 "nsl_guide_sample_count",
                 "nsl_predict_lightmaps", "nsl_shade", "nsl_render_frame_host"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(status: int, what: str = "nsl"):
    if status != NSL_OK:
        msg = load().nsl_last_error().decode(errors="replace")
        raise NslError(status, f"{what}: {msg}")


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def camera(cam) -> nsl_camera:
    c = nsl_camera()
    c.kind = int(cam.kind)
    c.eye[:] = [float(v) for v in cam.eye]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fov_y_deg = float(cam.fov_y_deg)
    c.ortho_height = float(cam.ortho_height)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def lights(ls):
    arr = (nsl_light * max(1, len(ls)))()
    for k, li in enumerate(ls):
        arr[k].dir[:] = [float(v) for v in li.dir]
        arr[k].intensity[:] = [float(v) for v in li.intensity]
    return arr


def march_opts(**kw) -> nsl_march_opts:
    o = nsl_march_opts()
    load().nsl_default_march_opts(C.byref(o))
    for k, v in kw.items():
        if k == "surrogate_I":
            o.surrogate_I[:] = [float(x) for x in v]
        elif k in ("seed", "frame"):
            setattr(o, k, int(v) & 0xFFFFFFFF)
        else:
            setattr(o, k, type(getattr(o, k))(v))
    return o


def _dptr(t, dtypes=None):
    """Device pointer of a contiguous CUDA tensor whose dtype is one of `dtypes`
    (names such as 'float32'); the C ABI takes plain pointers, so a wrong element
    type would otherwise be read or written silently."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtypes is not None and str(t.dtype).replace("torch.", "") not in dtypes:
        raise ValueError(f"expected a tensor of dtype {' or '.join(dtypes)}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _need(t, count, what):
    """The C ABI takes plain pointers and cannot see a buffer's size: refuse a
    tensor with fewer than `count` elements before the call (a kernel would
    read or write past its end)."""
    if t is None:
        return
    n = t.numel() if hasattr(t, "numel") else int(t.size)   # torch tensor or numpy array
    if n < count:
        raise NslError(NSL_ERR_INVALID_ARG, f"{what}: buffer holds {n} elements, needs {count}")


F32 = ("float32",)
GRID_TYPES = ("float32", "float16")
U8 = ("uint8",)
_GRID_DTYPE_NAME = {NSL_F32: "float32", NSL_F16: "float16"}
# grid (voxel count, dtype) of every live context, keyed by its handle: the C
# ABI's density pointer carries neither, and a float16 buffer read as float32
# would be read past its end
_ctx_grid: dict = {}


def _check_grid(t, dtype, voxels, what):
    """Refuse a density buffer (torch tensor or numpy array) whose element type
    is not the grid's `dtype` or that holds fewer than `voxels` elements."""
    if t is None:
        return
    want = _GRID_DTYPE_NAME.get(int(dtype))
    if want is None:
        raise NslError(NSL_ERR_INVALID_ARG, f"{what}: bad grid dtype {dtype}")
    got = str(t.dtype).replace("torch.", "")
    if got != want:
        raise NslError(NSL_ERR_INVALID_ARG, f"{what}: density is {got} but the grid is {want}")
    _need(t, voxels, what)


def _ctx_check_grid(ctx, density, mask, what):
    info = _ctx_grid.get(getattr(ctx, "value", ctx))
    if info is None:
        return
    voxels, dtype = info
    _check_grid(density, dtype, voxels, f"{what}: density")
    if mask is not None and str(mask.dtype).replace("torch.", "") != "uint8":
        raise NslError(NSL_ERR_INVALID_ARG, f"{what}: mask must be uint8, got {mask.dtype}")
    _need(mask, voxels, f"{what}: mask")


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------
# the C ABI, same names
# --------------------------------------------------------------------------

def nsl_create(nx, ny, nz, dtype, sigma_scale, blob: bytes, max_width, max_height):
    lib = load()
    g = nsl_grid_desc(nx, ny, nz, dtype, sigma_scale)
    out = C.c_void_p()
    buf = C.create_string_buffer(blob, len(blob))
    check(lib.nsl_create(C.byref(g), buf, len(blob), max_width, max_height, C.byref(out)), "nsl_create")
    _ctx_grid[out.value] = (int(nx) * int(ny) * int(nz), int(dtype))
    return out


def nsl_destroy(ctx):
    _ctx_grid.pop(getattr(ctx, "value", ctx), None)
    load().nsl_destroy(ctx)


def nsl_stage_grid(ctx, density, mask, stream=None):
    _ctx_check_grid(ctx, density, mask, "nsl_stage_grid")
    check(load().nsl_stage_grid(ctx, _dptr(density, GRID_TYPES), _dptr(mask, U8), _stream(stream)),
          "nsl_stage_grid")


def nsl_guide_sample_count(ctx, cam, step, opts=None, stream=None) -> int:
    out = C.c_ulonglong(0)
    check(load().nsl_guide_sample_count(ctx, C.byref(camera(cam)), float(step),
                                        C.byref(opts) if opts is not None else None, C.byref(out),
                                        _stream(stream)), "nsl_guide_sample_count")
    return int(out.value)


def nsl_guiding_map(ctx, density, mask, cam, step, guide, light=None, opts=None, stream=None):
    _need(guide, 3 * int(cam.width) * int(cam.height), "nsl_guiding_map: guide")
    _ctx_check_grid(ctx, density, mask, "nsl_guiding_map")
    lib = load()
    li = lights([light])[0] if light is not None else None
    check(lib.nsl_guiding_map(ctx, _dptr(density, GRID_TYPES), _dptr(mask, U8), C.byref(camera(cam)),
                              C.byref(li) if li is not None else None, float(step),
                              C.byref(opts) if opts is not None else None, _dptr(guide, F32),
                              _stream(stream)), "nsl_guiding_map")


def nsl_guiding_map_noalloc(grid_shape, dtype, sigma_scale, density, mask, cam, step, guide,
                            opts=None, stream=None):
    """Guide march whose scratch is the library's static device array (no allocation)."""
    nz, ny, nx = grid_shape
    _check_grid(density, dtype, nx * ny * nz, "nsl_guiding_map_noalloc: density")
    _need(mask, nx * ny * nz, "nsl_guiding_map_noalloc: mask")
    _need(guide, 3 * int(cam.width) * int(cam.height), "nsl_guiding_map_noalloc: guide")
    g = nsl_grid_desc(nx, ny, nz, dtype, sigma_scale)
    check(load().nsl_guiding_map_noalloc(C.byref(g), _dptr(density, GRID_TYPES), _dptr(mask, U8),
                                         C.byref(camera(cam)), float(step),
                                         C.byref(opts) if opts is not None else None,
                                         _dptr(guide, F32), _stream(stream)), "nsl_guiding_map_noalloc")


def nsl_reference_lightmaps(ctx, density, mask, cam, hf, out, phase_g=0.0, stream=None):
    """Fine-step six-light reference lightmaps [7][H][W] of the grid (see include/nsl.h)."""
    _need(out, 7 * int(cam.width) * int(cam.height), "nsl_reference_lightmaps: out")
    _ctx_check_grid(ctx, density, mask, "nsl_reference_lightmaps")
    check(load().nsl_reference_lightmaps(ctx, _dptr(density, GRID_TYPES), _dptr(mask, U8), C.byref(camera(cam)),
                                         float(hf), float(phase_g), _dptr(out, F32), _stream(stream)),
          "nsl_reference_lightmaps")


def nsl_predict_lightmaps(ctx, guide, width, height, precision, lightmaps, stream=None):
    _need(guide, 3 * int(width) * int(height), "nsl_predict_lightmaps: guide")
    _need(lightmaps, 8 * int(width) * int(height), "nsl_predict_lightmaps: lightmaps")
    check(load().nsl_predict_lightmaps(ctx, _dptr(guide, F32), int(width), int(height), int(precision),
                                       _dptr(lightmaps, F32), _stream(stream)), "nsl_predict_lightmaps")


# channels and level of the 17 stored tensors of the network, in order
TRACE_LAYERS = (("enc1a", 16, 0), ("enc1b", 16, 0), ("enc2a", 32, 1), ("enc2b", 32, 1), ("enc3a", 64, 2),
                ("enc3b", 64, 2), ("enc4a", 128, 3), ("enc4b", 128, 3), ("up3", 64, 2), ("dec3a", 64, 2),
                ("dec3b", 64, 2), ("up2", 32, 1), ("dec2a", 32, 1), ("dec2b", 32, 1), ("up1", 16, 0),
                ("dec1a", 16, 0), ("dec1b", 16, 0))


def nsl_predict_lightmaps_trace(ctx, guide, width, height, precision, lightmaps, trace, stream=None):
    """nsl_predict_lightmaps that also copies every layer's stored output into
    `trace`, a CUDA uint8 tensor of at least nsl_lightmap_trace_bytes bytes."""
    _need(guide, 3 * int(width) * int(height), "nsl_predict_lightmaps_trace: guide")
    _need(lightmaps, 8 * int(width) * int(height), "nsl_predict_lightmaps_trace: lightmaps")
    need = int(load().nsl_lightmap_trace_bytes(int(width), int(height)))
    _need(trace, need, "nsl_predict_lightmaps_trace: trace")
    check(load().nsl_predict_lightmaps_trace(ctx, _dptr(guide, F32), int(width), int(height), int(precision),
                                             _dptr(lightmaps, F32), _dptr(trace, U8), trace.numel(),
                                             _stream(stream)), "nsl_predict_lightmaps_trace")


def split_trace(trace_u8, width, height, dtype_name):
    """The 17 NHWC tensors of a trace (a flat uint8 tensor) as [C, H_l, W_l]
    float64 numpy arrays; dtype_name is 'bfloat16', 'float16' or 'float32'."""
    import numpy as np
    import torch
    tdt = getattr(torch, dtype_name)
    esz = torch.empty((), dtype=tdt).element_size()
    out, off = [], 0
    for _, ch, lv in TRACE_LAYERS:
        h, w = int(height) >> lv, int(width) >> lv
        n = h * w * ch * esz
        t = trace_u8[off:off + n].view(tdt).reshape(h, w, ch).permute(2, 0, 1)
        out.append(t.to(torch.float64).cpu().numpy())
        off += n
    return out


def nsl_measure_peaks(stream=None) -> dict:
    """Measured FP32 FMA rate, L1 data-path rate and L2 random-gather rate of
    the current device (see include/nsl.h)."""
    p = nsl_peaks()
    check(load().nsl_measure_peaks(C.byref(p), _stream(stream)), "nsl_measure_peaks")
    return {"sms": p.sms, "fp32_tflops": p.fp32_tflops, "l1_gbps": p.l1_gbps,
            "l2_gather_gbps": p.l2_gather_gbps}


def nsl_shade(ctx, lightmaps, width, height, cam, light_list, rgba, stream=None):
    _need(lightmaps, 8 * int(width) * int(height), "nsl_shade: lightmaps")
    _need(rgba, 4 * int(width) * int(height), "nsl_shade: rgba")
    check(load().nsl_shade(ctx, _dptr(lightmaps, F32), int(width), int(height), C.byref(camera(cam)),
                           lights(light_list), len(light_list), _dptr(rgba, F32), _stream(stream)),
          "nsl_shade")


_TEX_DTYPES = {NSL_TEX_RGBA8: ("uint8",), NSL_TEX_RGBA16F: ("float16",), NSL_TEX_RGBA32F: ("float32",)}


def nsl_pack_lightmaps(lightmaps, width, height, fmt, tex1, tex2, stream=None):
    """Two RGBA textures of the six-way layout; tex1/tex2 are [H][W][4] CUDA
    tensors of uint8, float16 or float32 for NSL_TEX_RGBA8 / 16F / 32F."""
    if fmt not in _TEX_DTYPES:
        raise ValueError(f"bad texture format {fmt}")
    for t in (tex1, tex2):
        if tuple(t.shape) != (int(height), int(width), 4):
            raise ValueError("textures must be [H][W][4]")
    _need(lightmaps, 8 * int(width) * int(height), "nsl_pack_lightmaps: lightmaps")
    check(load().nsl_pack_lightmaps(_dptr(lightmaps, F32), int(width), int(height), int(fmt),
                                    _dptr(tex1, _TEX_DTYPES[fmt]), _dptr(tex2, _TEX_DTYPES[fmt]),
                                    _stream(stream)), "nsl_pack_lightmaps")


def nsl_obstacle_shadow_map(mask, light_dir, resolution, out, stream=None):
    """Shadow map of a [nz][ny][nx] uint8 CUDA mask for a light toward light_dir
    into out, a [R][R] float32 CUDA tensor."""
    nz, ny, nx = mask.shape
    if tuple(out.shape) != (int(resolution), int(resolution)):
        raise ValueError("out must be [R][R]")
    d = (C.c_float * 3)(*[float(v) for v in light_dir])
    check(load().nsl_obstacle_shadow_map(_dptr(mask, ("uint8",)), nx, ny, nz, C.byref(d), int(resolution),
                                         _dptr(out, F32), _stream(stream)), "nsl_obstacle_shadow_map")


def nsl_shade_shadowed(ctx, lightmaps, guide, width, height, cam, light_list, maps, resolution, bias, rgba,
                       stream=None):
    """Six-way shading with obstacle shadows; maps: one [R][R] CUDA tensor (or
    None) per light."""
    if len(maps) != len(light_list):
        raise ValueError("one map (or None) per light")
    hw = int(width) * int(height)
    _need(lightmaps, 8 * hw, "nsl_shade_shadowed: lightmaps")
    _need(guide, 3 * hw, "nsl_shade_shadowed: guide")
    _need(rgba, 4 * hw, "nsl_shade_shadowed: rgba")
    for m in maps:
        _need(m, int(resolution) * int(resolution), "nsl_shade_shadowed: shadow map")
    ptrs = (C.c_void_p * max(1, len(maps)))(*[None if m is None else _dptr(m, F32).value for m in maps])
    check(load().nsl_shade_shadowed(ctx, _dptr(lightmaps, F32), _dptr(guide, F32), int(width), int(height),
                                    C.byref(camera(cam)), lights(light_list), len(light_list), ptrs,
                                    int(resolution), float(bias), _dptr(rgba, F32), _stream(stream)),
          "nsl_shade_shadowed")


def nsl_render_frame_host(ctx, density_np, mask_np, cam, light_list, step, precision,
                          guide_np=None, lightmaps_np=None, rgba_np=None, opts=None, stream=None):
    """Whole frame from host numpy buffers (copies in and out inside the call)."""
    _ctx_check_grid(ctx, density_np, mask_np, "nsl_render_frame_host")

    def hp(a):
        return None if a is None else C.c_void_p(a.ctypes.data)
    check(load().nsl_render_frame_host(ctx, hp(density_np), hp(mask_np), C.byref(camera(cam)),
                                       lights(light_list), len(light_list), float(step),
                                       C.byref(opts) if opts is not None else None, int(precision),
                                       hp(guide_np), hp(lightmaps_np), hp(rgba_np), _stream(stream)),
          "nsl_render_frame_host")


def nsl_render_frame_host_async(ctx, density_np, mask_np, cam, light_list, step, precision,
                                guide_np=None, lightmaps_np=None, rgba_np=None, opts=None, stream=None):
    """nsl_render_frame_host without the final synchronisation (page-locked
    host buffers make the copies asynchronous); synchronise `stream` before
    touching the buffers."""
    _ctx_check_grid(ctx, density_np, mask_np, "nsl_render_frame_host_async")

    def hp(a):
        return None if a is None else C.c_void_p(a.ctypes.data)
    check(load().nsl_render_frame_host_async(ctx, hp(density_np), hp(mask_np), C.byref(camera(cam)),
                                             lights(light_list), len(light_list), float(step),
                                             C.byref(opts) if opts is not None else None, int(precision),
                                             hp(guide_np), hp(lightmaps_np), hp(rgba_np), _stream(stream)),
          "nsl_render_frame_host_async")


class Context:
    """Owns an nsl_ctx; the methods forward to the C ABI."""

    def __init__(self, grid_shape, dtype, blob, max_width, max_height, sigma_scale=1.0):
        nz, ny, nx = grid_shape
        self.ctx = nsl_create(nx, ny, nz, dtype, sigma_scale, blob, max_width, max_height)
        self.voxels = nx * ny * nz

    def close(self):
        if self.ctx:
            nsl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stage_grid(self, density, mask, stream=None):
        _need(density, self.voxels, "nsl_stage_grid: density")
        _need(mask, self.voxels, "nsl_stage_grid: mask")
        nsl_stage_grid(self.ctx, density, mask, stream=stream)

    def guide_sample_count(self, cam, step, opts=None, stream=None):
        return nsl_guide_sample_count(self.ctx, cam, step, opts=opts, stream=stream)

    def guiding_map(self, density, mask, cam, step, guide, opts=None, stream=None):
        _need(density, self.voxels, "nsl_guiding_map: density")
        _need(mask, self.voxels, "nsl_guiding_map: mask")
        nsl_guiding_map(self.ctx, density, mask, cam, step, guide, opts=opts, stream=stream)

    def predict_lightmaps(self, guide, width, height, precision, lightmaps, stream=None):
        nsl_predict_lightmaps(self.ctx, guide, width, height, precision, lightmaps, stream=stream)

    def predict_lightmaps_trace(self, guide, width, height, precision, lightmaps, trace, stream=None):
        nsl_predict_lightmaps_trace(self.ctx, guide, width, height, precision, lightmaps, trace, stream=stream)

    def shade(self, lightmaps, width, height, cam, light_list, rgba, stream=None):
        nsl_shade(self.ctx, lightmaps, width, height, cam, light_list, rgba, stream=stream)


# --------------------------------------------------------------------------
# batched frames
# --------------------------------------------------------------------------

def plume_array(items):
    """items: sequence of dicts with density, mask, grid_dtype, sigma_scale,
    camera, step, light, guide, lightmaps, rgba (torch tensors / descriptions)."""
    arr = (nsl_plume * len(items))()
    for k, it in enumerate(items):
        p = arr[k]
        d = it["density"]
        nz, ny, nx = d.shape
        hw = int(it["camera"].width) * int(it["camera"].height)
        _need(it.get("mask"), nx * ny * nz, f"plume {k}: mask")
        _need(it["guide"], 3 * hw, f"plume {k}: guide")
        _need(it["lightmaps"], 8 * hw, f"plume {k}: lightmaps")
        _need(it.get("rgba"), 4 * hw, f"plume {k}: rgba")
        p.density_dev = _dptr(d, GRID_TYPES)
        p.mask_dev = _dptr(it.get("mask"), U8)
        p.grid = nsl_grid_desc(nx, ny, nz, NSL_F16 if str(d.dtype).endswith("float16") else NSL_F32,
                               float(it.get("sigma_scale", 1.0)))
        p.camera = camera(it["camera"])
        p.step_voxels = float(it["step"])
        p.light = lights([it["light"]])[0]
        p.guide_dev = _dptr(it["guide"], F32)
        p.lightmaps_dev = _dptr(it["lightmaps"], F32)
        p.rgba_dev = _dptr(it.get("rgba"), F32)
    return arr


class Batch:
    """Owns an nsl_batch; the methods forward to the C ABI."""

    def __init__(self, blob: bytes, max_plumes: int = 64):
        lib = load()
        out = C.c_void_p()
        buf = C.create_string_buffer(blob, len(blob))
        check(lib.nsl_batch_create(buf, len(blob), int(max_plumes), C.byref(out)), "nsl_batch_create")
        self.b = out

    def close(self):
        if self.b:
            load().nsl_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, plumes, precision, opts=None, stream=None):
        arr = plume_array(plumes)
        check(load().nsl_batch_render(self.b, arr, len(plumes), C.byref(opts) if opts else None,
                                      int(precision), _stream(stream)), "nsl_batch_render")

    def capture_graph(self, plumes, precision, stream, opts=None):
        arr = plume_array(plumes)
        check(load().nsl_batch_capture_graph(self.b, arr, len(plumes), C.byref(opts) if opts else None,
                                             int(precision), _stream(stream)), "nsl_batch_capture_graph")

    def update_graph(self, plumes, opts=None):
        arr = plume_array(plumes)
        check(load().nsl_batch_update_graph(self.b, arr, len(plumes), C.byref(opts) if opts else None),
              "nsl_batch_update_graph")

    def launch_graph(self, stream):
        check(load().nsl_batch_launch_graph(self.b, _stream(stream)), "nsl_batch_launch_graph")

    def set_tuning(self, seg_len, march_blocks_per_sm, conv_ctas_per_sm):
        check(load().nsl_batch_set_tuning(self.b, int(seg_len), int(march_blocks_per_sm),
                                          int(conv_ctas_per_sm)), "nsl_batch_set_tuning")

    def get_tuning(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        check(load().nsl_batch_get_tuning(self.b, C.byref(a), C.byref(b), C.byref(c)), "nsl_batch_get_tuning")
        return a.value, b.value, c.value

    def set_march_tile(self, width):
        check(load().nsl_batch_set_march_tile(self.b, int(width)), "nsl_batch_set_march_tile")

    def get_march_tile(self):
        w = C.c_int()
        check(load().nsl_batch_get_march_tile(self.b, C.byref(w)), "nsl_batch_get_march_tile")
        return int(w.value)

    def set_march_form(self, persistent):
        check(load().nsl_batch_set_march_form(self.b, int(persistent)), "nsl_batch_set_march_form")

    def get_march_form(self):
        v = C.c_int()
        check(load().nsl_batch_get_march_form(self.b, C.byref(v)), "nsl_batch_get_march_form")
        return int(v.value)

    def autotune(self, plumes, precision, cache_path=None, opts=None, stream=None):
        arr = plume_array(plumes)
        ms = C.c_float(0)
        check(load().nsl_batch_autotune(self.b, arr, len(plumes), C.byref(opts) if opts else None,
                                        int(precision), cache_path.encode() if cache_path else None,
                                        _stream(stream), C.byref(ms)), "nsl_batch_autotune")
        return ms.value


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

def server_opts(**kw) -> nsl_server_opts:
    o = nsl_server_opts()
    load().nsl_default_server_opts(C.byref(o))
    for k, v in kw.items():
        if k == "march":
            o.march = v
        else:
            setattr(o, k, v)
    return o


class Server:
    """Owns an nsl_server; the methods forward to the C ABI.  Host density
    arrays handed to add_plume are kept referenced here until removal."""

    def __init__(self, blob: bytes, opts: nsl_server_opts | None = None):
        lib = load()
        out = C.c_void_p()
        buf = C.create_string_buffer(blob, len(blob))
        check(lib.nsl_server_create(buf, len(blob), C.byref(opts) if opts else None, C.byref(out)),
              "nsl_server_create")
        self.s = out
        self._keep = {}

    def close(self):
        if self.s:
            load().nsl_server_destroy(self.s)
            self.s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_plume(self, density, mask, step, max_width, max_height, sigma_scale=1.0) -> int:
        import numpy as np
        density = np.ascontiguousarray(density)
        nz, ny, nx = density.shape
        dt = NSL_F16 if density.dtype == np.float16 else NSL_F32
        if density.dtype not in (np.float16, np.float32):
            raise ValueError("density must be float32 or float16")
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        g = nsl_grid_desc(nx, ny, nz, dt, float(sigma_scale))
        pid = C.c_int()
        check(load().nsl_server_add_plume(self.s, C.byref(g), C.c_void_p(density.ctypes.data),
                                          None if m is None else C.c_void_p(m.ctypes.data), float(step),
                                          int(max_width), int(max_height), C.byref(pid)),
              "nsl_server_add_plume")
        self._keep[pid.value] = (density, m)
        return pid.value

    def remove_plume(self, pid):
        check(load().nsl_server_remove_plume(self.s, int(pid)), "nsl_server_remove_plume")
        self._keep.pop(pid, None)

    def submit(self, pid, cam, light, lightmaps=None, rgba=None) -> int:
        hw = int(cam.width) * int(cam.height)
        _need(lightmaps, 8 * hw, "nsl_server_submit: lightmaps")
        _need(rgba, 4 * hw, "nsl_server_submit: rgba")
        rid = C.c_uint64()
        c = camera(cam)
        lt = lights([light])
        check(load().nsl_server_submit(self.s, int(pid), C.byref(c), lt, _dptr(lightmaps, F32), _dptr(rgba, F32),
                                       C.byref(rid)), "nsl_server_submit")
        return rid.value

    def wait(self, rid, timeout_ms=60000.0) -> float:
        lat = C.c_double()
        check(load().nsl_server_wait(self.s, C.c_uint64(rid), float(timeout_ms), C.byref(lat)), "nsl_server_wait")
        return lat.value

    def drain(self, timeout_ms=120000.0):
        check(load().nsl_server_drain(self.s, float(timeout_ms)), "nsl_server_drain")

    def plume_state(self, pid):
        g, lm, rgba, res = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int()
        check(load().nsl_server_plume_state(self.s, int(pid), C.byref(g), C.byref(lm), C.byref(rgba),
                                            C.byref(res)), "nsl_server_plume_state")
        return g.value, lm.value, rgba.value, bool(res.value)

    def stats(self) -> dict:
        st = nsl_server_stats()
        check(load().nsl_server_get_stats(self.s, C.byref(st)), "nsl_server_get_stats")
        return st.as_dict()

    def reset_stats(self):
        check(load().nsl_server_reset_stats(self.s), "nsl_server_reset_stats")


# --------------------------------------------------------------------------
# training slice
# --------------------------------------------------------------------------

def train_opts(**kw) -> nsl_train_opts:
    o = nsl_train_opts()
    load().nsl_default_train_opts(C.byref(o))
    for k, v in kw.items():
        if k == "plane_weight":
            o.plane_weight[:] = [float(x) for x in v]
        else:
            setattr(o, k, type(getattr(o, k))(v))
    return o


class Trainer:
    """Owns an nsl_trainer (Adam on the MSE of the eight output planes)."""

    def __init__(self, blob: bytes, opts: nsl_train_opts | None = None):
        self.o = opts if opts is not None else train_opts()
        out = C.c_void_p()
        buf = C.create_string_buffer(blob, len(blob))
        check(load().nsl_trainer_create(buf, len(blob), C.byref(self.o), C.byref(out)), "nsl_trainer_create")
        self.t = out
        self.n_params = (len(blob) - 20) // 4

    def close(self):
        if self.t:
            load().nsl_trainer_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, guides, targets, depth_scale, update=True, stream=None) -> float:
        """guides [B,3,H,W], targets [B,8,H,W]: float32 CUDA tensors."""
        B, H, W = int(self.o.batch), int(self.o.height), int(self.o.width)
        _need(guides, B * 3 * H * W, "nsl_trainer_step: guides")
        _need(targets, B * 8 * H * W, "nsl_trainer_step: targets")
        loss = C.c_float()
        check(load().nsl_trainer_step(self.t, _dptr(guides, F32), _dptr(targets, F32), float(depth_scale),
                                      1 if update else 0, C.byref(loss), _stream(stream)), "nsl_trainer_step")
        return float(loss.value)

    def set_lr(self, lr):
        check(load().nsl_trainer_set_lr(self.t, float(lr)), "nsl_trainer_set_lr")

    def gradients(self, out, stream=None):
        _need(out, self.n_params, "nsl_trainer_gradients: out")
        check(load().nsl_trainer_gradients(self.t, _dptr(out, F32), out.numel(), _stream(stream)),
              "nsl_trainer_gradients")

    def blob(self) -> bytes:
        need = C.c_size_t()
        check(load().nsl_trainer_get_blob(self.t, None, 0, C.byref(need)), "nsl_trainer_get_blob")
        buf = C.create_string_buffer(need.value)
        check(load().nsl_trainer_get_blob(self.t, buf, need.value, C.byref(need)), "nsl_trainer_get_blob")
        return buf.raw
