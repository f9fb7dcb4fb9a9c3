"""FP64 CPU oracle for the neural six-way lightmap hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares no
code with the CUDA path (``paper_2604_03748_gb300``) and imports nothing from
it; inputs arrive as plain numpy arrays and dataclass-like objects.

Parity status per function (pins live in tests/test_oracle_*.py):
  guide                 pinned (closed forms: empty, constant cube, linear field,
                        homogeneous sphere chords, perspective camera
                        chords, symmetry, mask, HG normalisation)
  reference_lightmaps   pinned (slab closed form, midpoint order)
  net_forward           pinned (PyTorch float64 conv/convT/pool/LayerNorm,
                        NAFBlock identity at beta=gamma=0)
  net_forward_q8        pinned (E4M3 and binary16 rounding against PyTorch's
                        float8_e4m3fn / float16 casts and brute force over all
                        E4M3 codes; the quantised network against a PyTorch
                        float64 assembly using those casts)
  shade                 pinned (axis lights select one plane; linearity)
  pack_lightmaps        pinned (Fig. 2 channel layout on exact binary fractions,
                        ties to even, clamping; binary16 against numpy's cast)
  guide light sets      pinned (constant-cube closed form for front only and
                        front/left/right)
  guide shadow volume   pinned (constant-cube closed form of the interpolated
                        voxel-centre transmittances)
  shadow_map            pinned (single voxel and slab closed forms, axis and
                        oblique lights)
  shade_shadowed        pinned (occluder slab: shadowed pixels keep only E,
                        lit ones equal shade(); no maps equals shade())
  paper-level quality   parity unpinned (no trained weights, no dataset)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library beside it (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(C.Structure):
    _fields_ = [("kind", C.c_int), ("eye", C.c_float * 3), ("target", C.c_float * 3),
                ("up", C.c_float * 3), ("fov_y_deg", C.c_float), ("ortho_height", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("tau_depth", C.c_float), ("t_min", C.c_float), ("jitter", C.c_int),
                ("seed", C.c_uint32), ("frame", C.c_uint32), ("phase_g", C.c_float),
                ("surrogate_I", C.c_float * 3), ("segment_exact", C.c_int), ("margin", C.c_float),
                ("light_set", C.c_int), ("shadow_volume", C.c_int)]


class _Light(C.Structure):
    _fields_ = [("dir", C.c_float * 3), ("intensity", C.c_float * 3)]


_P = np.ctypeslib.ndpointer


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    dptr = C.POINTER(C.c_double)
    lib.nslo_guide.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                               C.POINTER(_Camera), C.c_float, C.POINTER(_Opts), C.c_void_p,
                               C.c_void_p, C.c_void_p]
    lib.nslo_guide_rows.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                    C.POINTER(_Camera), C.c_float, C.POINTER(_Opts), C.c_int,
                                    C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.nslo_reference_lightmaps.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                             C.c_double, C.POINTER(_Camera), C.c_double,
                                             C.c_double, C.c_void_p]
    lib.nslo_reference_lightmaps_rows.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                                  C.c_double, C.POINTER(_Camera), C.c_double, C.c_double,
                                                  C.c_int, C.c_int, C.c_void_p]
    lib.nslo_net_forward.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                                     C.c_double, C.c_void_p]
    lib.nslo_net_forward_q8.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                                        C.c_double, C.c_void_p]
    lib.nslo_net_forward_prec.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                                          C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.nslo_net_trace_size.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    lib.nslo_net_trace_size.restype = C.c_int64
    lib.nslo_conv_layer_prec.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                         C.c_void_p, C.c_int, C.c_void_p]
    lib.nslo_store_as.argtypes = [C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
    lib.nslo_store_as.restype = None
    lib.nslo_net_adapters.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]
    lib.nslo_round_bf16.argtypes = [C.c_double]
    lib.nslo_round_bf16.restype = C.c_double
    lib.nslo_round_f16.argtypes = [C.c_double]
    lib.nslo_round_f16.restype = C.c_double
    lib.nslo_e4m3_rn.argtypes = [C.c_double]
    lib.nslo_e4m3_rn.restype = C.c_double
    lib.nslo_q8_tensor.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_float)]
    lib.nslo_q8_tensor.restype = None
    lib.nslo_q8_weights.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_void_p,
                                    C.c_void_p]
    lib.nslo_q8_weights.restype = None
    lib.nslo_shade.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(_Camera), C.POINTER(_Light),
                               C.c_int, C.c_void_p]
    lib.nslo_shadow_map.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float * 3),
                                    C.c_int, C.c_void_p]
    lib.nslo_shade_shadowed.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(_Camera),
                                        C.POINTER(_Light), C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.POINTER(C.c_void_p), C.c_int, C.c_float, C.c_void_p]
    lib.nslo_sample_sigma.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                      C.POINTER(C.c_float * 3)]
    lib.nslo_sample_sigma.restype = C.c_double
    lib.nslo_hg_phase.argtypes = [C.c_double, C.c_double]
    lib.nslo_hg_phase.restype = C.c_double
    lib.nslo_pcg_hash.argtypes = [C.c_uint32]
    lib.nslo_pcg_hash.restype = C.c_uint32
    lib.nslo_conv2d.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_int, C.c_int, C.c_void_p]
    lib.nslo_conv_transpose2x2.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                           C.c_void_p, C.c_int, C.c_void_p]
    lib.nslo_maxpool2.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]
    lib.nslo_layernorm.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_double, C.c_void_p]
    lib.nslo_dwconv3.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]
    lib.nslo_nafblock.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    lib.nslo_nafblock_params.argtypes = [C.c_int]
    lib.nslo_nafblock_params.restype = C.c_int64
    del dptr
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _cam(cam) -> _Camera:
    c = _Camera()
    c.kind = int(cam.kind)
    c.eye[:] = [float(v) for v in cam.eye]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fov_y_deg = float(cam.fov_y_deg)
    c.ortho_height = float(cam.ortho_height)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def _grid(density):
    d = np.ascontiguousarray(density)
    if d.dtype == np.float16:
        d = d.astype(np.float32)  # exact widening
    d = np.ascontiguousarray(d, dtype=np.float32)
    nz, ny, nx = d.shape
    return d, nx, ny, nz


def _mask(mask):
    return None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)


DEFAULT_OPTS = dict(tau_depth=0.01, t_min=1e-4, jitter=1, seed=0, frame=0, phase_g=0.0,
                    surrogate_I=(1.0, 1.0, 1.0), segment_exact=0, margin=1e-5, light_set=0,
                    shadow_volume=0)


def guide(density, mask, camera, step, sigma_scale=1.0, rows=None, **opts):
    """Alg. 1 guiding map.  Returns (guide[3,H,W] float64, samples[H,W] int64, flags[H,W] uint8).
    rows=(r0, r1) restricts the march to image rows [r0, r1) (others stay 0)."""
    lib = _load()
    o = dict(DEFAULT_OPTS)
    o.update(opts)
    d, nx, ny, nz = _grid(density)
    m = _mask(mask)
    H, W = camera.height, camera.width
    out = np.zeros((3, H, W), np.float64)
    samples = np.zeros((H, W), np.int64)
    flags = np.zeros((H, W), np.uint8)
    op = _Opts()
    op.tau_depth = o["tau_depth"]; op.t_min = o["t_min"]; op.jitter = int(o["jitter"])
    op.seed = int(o["seed"]) & 0xFFFFFFFF; op.frame = int(o["frame"]) & 0xFFFFFFFF
    op.phase_g = o["phase_g"]; op.surrogate_I[:] = list(o["surrogate_I"])
    op.segment_exact = int(o["segment_exact"]); op.margin = o["margin"]
    op.light_set = int(o["light_set"])
    op.shadow_volume = int(o["shadow_volume"])
    cam = _cam(camera)
    r0, r1 = (0, H) if rows is None else rows
    rc = lib.nslo_guide_rows(_ptr(d), _ptr(m), nx, ny, nz, float(sigma_scale), C.byref(cam),
                             float(step), C.byref(op), int(r0), int(r1), _ptr(out), _ptr(samples),
                             _ptr(flags))
    if rc != 0:
        raise ValueError(f"nslo_guide failed ({rc})")
    return out, samples, flags


def reference_lightmaps(density, mask, camera, hf=0.25, sigma_scale=1.0, phase_g=0.0, rows=None):
    """Fine-step six-light single-scattering reference: [7,H,W] = +X,-X,+Y,-Y,+Z,-Z,T.
    rows=(r0, r1) restricts it to image rows [r0, r1) (others stay 0)."""
    lib = _load()
    d, nx, ny, nz = _grid(density)
    m = _mask(mask)
    out = np.zeros((7, camera.height, camera.width), np.float64)
    cam = _cam(camera)
    r0, r1 = (0, camera.height) if rows is None else rows
    rc = lib.nslo_reference_lightmaps_rows(_ptr(d), _ptr(m), nx, ny, nz, float(sigma_scale),
                                           C.byref(cam), float(hf), float(phase_g), int(r0), int(r1),
                                           _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_reference_lightmaps failed ({rc})")
    return out


def net_forward_q8(guide_planes, params_flat, c0, depth_scale):
    """The network with FP8 E4M3 convolutions (see nslo_net_forward_q8)."""
    lib = _load()
    g = np.ascontiguousarray(guide_planes, dtype=np.float64)
    _, H, W = g.shape
    p = np.ascontiguousarray(params_flat, dtype=np.float64)
    out = np.zeros((8, H, W), np.float64)
    rc = lib.nslo_net_forward_q8(_ptr(g), H, W, _ptr(p), p.size, int(c0), float(depth_scale), _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_net_forward_q8 failed ({rc})")
    return out


PREC_F64, PREC_F16, PREC_BF16, PREC_FP8, PREC_BF16X3 = 0, 1, 2, 3, 4
# the network's 17 convolutions in order (nslo_net_forward_prec)
NET_LAYERS = ("enc1a", "enc1b", "enc2a", "enc2b", "enc3a", "enc3b", "enc4a", "enc4b", "up3", "dec3a",
              "dec3b", "up2", "dec2a", "dec2b", "up1", "dec1a", "dec1b")


def net_forward_prec(guide_planes, params_flat, c0, depth_scale, prec, trace=False):
    """The network with convolution l in precision form prec[l] (a sequence of
    17 codes, or one code for every layer); see nslo_net_forward_prec.
    Returns out [8,H,W], and with trace=True also the 17 stored layer outputs
    as a list of [C,H_l,W_l] arrays."""
    lib = _load()
    g = np.ascontiguousarray(guide_planes, np.float64)
    p = np.ascontiguousarray(params_flat, np.float64)
    H, W = g.shape[1:]
    codes = [int(prec)] * 17 if np.isscalar(prec) else [int(v) for v in prec]
    if len(codes) != 17:
        raise ValueError("prec needs 17 layer codes")
    pr = np.asarray(codes, np.int32)
    out = np.zeros((8, H, W), np.float64)
    sizes = [int(lib.nslo_net_trace_size(int(c0), H, W, l)) for l in range(17)]
    tr = np.zeros(sum(sizes), np.float64) if trace else None
    rc = lib.nslo_net_forward_prec(_ptr(g), H, W, _ptr(p), p.size, int(c0), float(depth_scale), _ptr(pr),
                                   _ptr(out), _ptr(tr) if trace else None)
    if rc != 0:
        raise ValueError(f"nslo_net_forward_prec failed ({rc})")
    if not trace:
        return out
    mult = (1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 4, 2, 2, 2, 1, 1, 1)
    lvl = (0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0)
    layers, off = [], 0
    for l in range(17):
        shp = (mult[l] * int(c0), H >> lvl[l], W >> lvl[l])
        layers.append(tr[off:off + sizes[l]].reshape(shp))
        off += sizes[l]
    return out, layers


def conv_layer_prec(prec, x, w, b, transposed=False):
    """One convolution of the network in precision form `prec` (see
    nslo_conv_layer_prec): x [cin,H,W]; w [cout,cin,3,3] (3x3 + ReLU) or, with
    transposed=True, [cin,cout,2,2] (2x2 stride 2)."""
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    cin, H, W = x.shape
    cout = w.shape[1] if transposed else w.shape[0]
    out = np.zeros((cout, 2 * H, 2 * W) if transposed else (cout, H, W), np.float64)
    rc = lib.nslo_conv_layer_prec(int(prec), 2 if transposed else 3, _ptr(x), cin, H, W, _ptr(w), _ptr(b),
                                  cout, _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_conv_layer_prec failed ({rc})")
    return out


def store_as(prec, x):
    """The values x are stored as after a layer of form `prec`."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(x)
    _load().nslo_store_as(int(prec), _ptr(x), x.size, _ptr(out))
    return out


def net_adapters(F, adapter_params, c0):
    """The four adapters and their heads on a feature map F [c0,H,W]: [8,H,W]."""
    lib = _load()
    F = np.ascontiguousarray(F, np.float64)
    p = np.ascontiguousarray(adapter_params, np.float64)
    _, H, W = F.shape
    out = np.zeros((8, H, W), np.float64)
    rc = lib.nslo_net_adapters(_ptr(F), int(c0), H, W, _ptr(p), p.size, _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_net_adapters failed ({rc})")
    return out


def round_bf16(x):
    lib = _load()
    return np.vectorize(lambda v: lib.nslo_round_bf16(float(v)), otypes=[np.float64])(x)


def round_f16(x):
    lib = _load()
    return np.vectorize(lambda v: lib.nslo_round_f16(float(v)), otypes=[np.float64])(x)


def e4m3_rn(x):
    lib = _load()
    return np.vectorize(lambda v: lib.nslo_e4m3_rn(float(v)), otypes=[np.float64])(x)


def q8_tensor(x):
    """(codes, dequantisation factor) of a tensor of binary16 values."""
    lib = _load()
    a = np.ascontiguousarray(x, dtype=np.float64)
    codes = np.zeros_like(a)
    deq = C.c_float()
    lib.nslo_q8_tensor(_ptr(a), a.size, _ptr(codes), C.byref(deq))
    return codes, deq.value


def q8_weights(w, cout, count, so, sj):
    lib = _load()
    a = np.ascontiguousarray(w, dtype=np.float64)
    codes = np.zeros_like(a)
    s = np.zeros(cout, np.float32)
    lib.nslo_q8_weights(_ptr(a), int(cout), int(count), int(so), int(sj), _ptr(codes), _ptr(s))
    return codes, s


def net_forward(guide_planes, params_flat, c0, depth_scale):
    """Lightmap network forward in FP64.  guide [3,H,W] -> [8,H,W]."""
    lib = _load()
    g = np.ascontiguousarray(guide_planes, dtype=np.float64)
    _, H, W = g.shape
    p = np.ascontiguousarray(params_flat, dtype=np.float64)
    out = np.zeros((8, H, W), np.float64)
    rc = lib.nslo_net_forward(_ptr(g), H, W, _ptr(p), p.size, int(c0), float(depth_scale), _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_net_forward failed ({rc})")
    return out


def shade(lightmaps, camera, lights):
    lib = _load()
    lm = np.ascontiguousarray(lightmaps, dtype=np.float64)
    _, H, W = lm.shape
    arr = (_Light * max(1, len(lights)))()
    for i, li in enumerate(lights):
        arr[i].dir[:] = [float(v) for v in li.dir]
        arr[i].intensity[:] = [float(v) for v in li.intensity]
    out = np.zeros((4, H, W), np.float64)
    cam = _cam(camera)
    rc = lib.nslo_shade(_ptr(lm), H, W, C.byref(cam), arr, len(lights), _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_shade failed ({rc})")
    return out


def shadow_map(mask, light_dir, R):
    """Obstacle shadow map (Sec. 4.5) of the uint8 mask [nz][ny][nx] for a light
    toward light_dir: float32 [R][R] of first-hit parameters (+inf = none)."""
    lib = _load()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = m.shape
    out = np.zeros((R, R), np.float32)
    d = (C.c_float * 3)(*[float(v) for v in light_dir])
    if lib.nslo_shadow_map(_ptr(m), nx, ny, nz, C.byref(d), int(R), _ptr(out)) != 0:
        raise ValueError("nslo_shadow_map failed")
    return out


def shade_shadowed(lightmaps, guide, camera, lights, grid_shape, maps, bias):
    """shade() with each light's term times the visibility of the pixel's smoke
    shell against that light's shadow map (maps[l] None = no obstacle shadow).
    guide: float32 [3][H][W]; grid_shape: (nz, ny, nx)."""
    lib = _load()
    lm = np.ascontiguousarray(lightmaps, dtype=np.float64)
    g = np.ascontiguousarray(guide, dtype=np.float32)
    _, H, W = lm.shape
    arr = (_Light * max(1, len(lights)))()
    for i, li in enumerate(lights):
        arr[i].dir[:] = [float(v) for v in li.dir]
        arr[i].intensity[:] = [float(v) for v in li.intensity]
    R = 1
    keep = [None if mp is None else np.ascontiguousarray(mp, dtype=np.float32) for mp in maps]
    for mp in keep:
        if mp is not None:
            R = mp.shape[0]
    ptrs = (C.c_void_p * max(1, len(keep)))(*[None if mp is None else mp.ctypes.data for mp in keep])
    nz, ny, nx = grid_shape
    out = np.zeros((4, H, W), np.float64)
    cam = _cam(camera)
    rc = lib.nslo_shade_shadowed(_ptr(lm), _ptr(g), H, W, C.byref(cam), arr, len(lights), nx, ny, nz,
                                 ptrs, int(R), float(bias), _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_shade_shadowed failed ({rc})")
    return out


TEX_RGBA8, TEX_RGBA16F, TEX_RGBA32F = 0, 1, 2


def pack_lightmaps(lightmaps, fmt):
    """The two RGBA textures of the six-way layout (Sec. 3, Fig. 2) from the
    eight planes [+X, -X, +Y, -Y, +Z, -Z, T, E] (camera frame: X right, Y up,
    Z away from the viewer).  Texture 1 = (right +X, top +Y, back +Z,
    transparency T); texture 2 = (left -X, bottom -Y, front -Z, emissive E);
    each [H][W][4].  RGBA8: the UNORM code of the value clamped to [0, 1] (NaN
    to 0), the float32 product v * 255 rounded to the nearest integer, ties to
    even.  RGBA16F: nearest binary16, ties to even.  RGBA32F: the values."""
    lm = np.asarray(lightmaps, np.float32)
    assert lm.ndim == 3 and lm.shape[0] == 8
    planes1 = (0, 2, 4, 6)
    planes2 = (1, 3, 5, 7)

    def one(idx):
        t = np.empty(lm.shape[1:] + (4,), np.float32)
        for c, q in enumerate(idx):
            t[..., c] = lm[q]
        if fmt == TEX_RGBA8:
            v = np.where(np.isnan(t), np.float32(0), t)
            v = np.minimum(np.maximum(v, np.float32(0)), np.float32(1))
            return np.rint(v * np.float32(255)).astype(np.uint8)
        if fmt == TEX_RGBA16F:
            return t.astype(np.float16)
        if fmt == TEX_RGBA32F:
            return t
        raise ValueError(fmt)
    return one(planes1), one(planes2)


def sample_sigma(density, mask, p, sigma_scale=1.0):
    lib = _load()
    d, nx, ny, nz = _grid(density)
    m = _mask(mask)
    pp = (C.c_float * 3)(*[float(v) for v in p])
    return lib.nslo_sample_sigma(_ptr(d), _ptr(m), nx, ny, nz, float(sigma_scale), C.byref(pp))


def hg_phase(g, cos_theta):
    return _load().nslo_hg_phase(float(g), float(cos_theta))


def pcg_hash(v):
    return int(_load().nslo_pcg_hash(int(v) & 0xFFFFFFFF))


def conv2d(x, w, b, k):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    cin, H, W = x.shape
    cout = w.shape[0]
    b = None if b is None else np.ascontiguousarray(b, np.float64)
    out = np.zeros((cout, H, W), np.float64)
    lib.nslo_conv2d(_ptr(x), cin, H, W, _ptr(w), _ptr(b), cout, int(k), _ptr(out))
    return out


def conv_transpose2x2(x, w, b):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    cin, H, W = x.shape
    cout = w.shape[1]
    b = None if b is None else np.ascontiguousarray(b, np.float64)
    out = np.zeros((cout, 2 * H, 2 * W), np.float64)
    lib.nslo_conv_transpose2x2(_ptr(x), cin, H, W, _ptr(w), _ptr(b), cout, _ptr(out))
    return out


def maxpool2(x):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    c, H, W = x.shape
    out = np.zeros((c, H // 2, W // 2), np.float64)
    lib.nslo_maxpool2(_ptr(x), c, H, W, _ptr(out))
    return out


def layernorm(x, g, b, eps=1e-6):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    c, H, W = x.shape
    out = np.zeros_like(x)
    lib.nslo_layernorm(_ptr(x), c, H, W, _ptr(np.ascontiguousarray(g, np.float64)),
                       _ptr(np.ascontiguousarray(b, np.float64)), float(eps), _ptr(out))
    return out


def dwconv3(x, w, b):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    c, H, W = x.shape
    out = np.zeros_like(x)
    lib.nslo_dwconv3(_ptr(x), c, H, W, _ptr(np.ascontiguousarray(w, np.float64)),
                     _ptr(np.ascontiguousarray(b, np.float64)), _ptr(out))
    return out


def nafblock(x, params_flat):
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    c, H, W = x.shape
    p = np.ascontiguousarray(params_flat, np.float64)
    if p.size != lib.nslo_nafblock_params(c):
        raise ValueError("wrong NAFBlock parameter count")
    out = np.zeros_like(x)
    rc = lib.nslo_nafblock(_ptr(x), c, H, W, _ptr(p), _ptr(out))
    if rc != 0:
        raise ValueError(f"nslo_nafblock failed ({rc})")
    return out


def nafblock_params(c):
    return int(_load().nslo_nafblock_params(int(c)))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
