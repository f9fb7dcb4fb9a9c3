"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module holds no arithmetic of the method itself (no ray marching, no
network layer, no shading).  It only draws inputs:

* smoke density grids: a sum of anisotropic Gaussian blobs multiplied by
  (0.5 + 0.5 * fBm) gradient noise, clamped to [0, 2].  They stand in for the
  lattice-Boltzmann smoke of the paper (Sec. 5, "Smoke Simulator" and
  "Performance": 400^3 density, inlet density 0.1), which is not available;
* voxelised obstacle masks (a signed-distance sphere);
* cameras (orthographic orbit, perspective) and directional lights;
* network parameters for the UNet + four NAFBlock adapters of Sec. 4.3,
  He-normal from a seed (no trained weights exist for this build), packed in
  the NSLW blob format that both sides parse.

Grids are stored [nz][ny][nx] with x fastest; voxel (i, j, k) has its centre at
(i + 0.5, j + 0.5, k + 0.5) in voxel units.
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# gradient noise / fBm
# ----------------------------------------------------------------------------


def _lattice_gradients(rng: np.random.Generator, period: int) -> np.ndarray:
    g = rng.normal(size=(period, period, period, 3)).astype(np.float64)
    g /= np.linalg.norm(g, axis=-1, keepdims=True) + 1e-12
    return g.astype(np.float32)


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def gradient_noise(px, py, pz, grads: np.ndarray) -> np.ndarray:
    """Periodic 3-D gradient noise at points (px, py, pz) in lattice units."""
    period = grads.shape[0]
    x0 = np.floor(px)
    y0 = np.floor(py)
    z0 = np.floor(pz)
    fx = (px - x0).astype(np.float32)
    fy = (py - y0).astype(np.float32)
    fz = (pz - z0).astype(np.float32)
    ix = x0.astype(np.int64) % period
    iy = y0.astype(np.int64) % period
    iz = z0.astype(np.int64) % period
    out = np.zeros(np.broadcast(px, py, pz).shape, np.float32)
    ux, uy, uz = _fade(fx), _fade(fy), _fade(fz)
    for dz in (0, 1):
        wz = uz if dz else 1.0 - uz
        for dy in (0, 1):
            wy = uy if dy else 1.0 - uy
            for dx in (0, 1):
                wx = ux if dx else 1.0 - ux
                g = grads[(iz + dz) % period, (iy + dy) % period, (ix + dx) % period]
                dot = g[..., 0] * (fx - dx) + g[..., 1] * (fy - dy) + g[..., 2] * (fz - dz)
                out += wx * wy * wz * dot
    return out


def fbm(n: int, seed: int, octaves: int = 4, base_period: float | None = None,
        lacunarity: float = 2.0, gain: float = 0.5, z_range=None) -> np.ndarray:
    """fBm of gradient noise on the voxel centres of an n^3 grid, in [-1, 1]."""
    rng = np.random.default_rng(seed)
    if base_period is None:
        base_period = n / 4.0
    z_lo, z_hi = (0, n) if z_range is None else z_range
    c = np.arange(n, dtype=np.float32) + 0.5
    zz = (np.arange(z_lo, z_hi, dtype=np.float32) + 0.5)[:, None, None]
    yy = c[None, :, None]
    xx = c[None, None, :]
    total = np.zeros((z_hi - z_lo, n, n), np.float32)
    amp, norm = 1.0, 0.0
    freq = 1.0 / base_period
    for o in range(octaves):
        grads = _lattice_gradients(rng, 64)
        off = rng.uniform(0, 64, size=3).astype(np.float32)
        total += amp * gradient_noise(xx * freq + off[0], yy * freq + off[1], zz * freq + off[2], grads)
        norm += amp
        amp *= gain
        freq *= lacunarity
    # gradient noise lies in about [-0.9, 0.9]; rescale and clip to [-1, 1]
    return np.clip(total / norm * 1.6, -1.0, 1.0)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def blob_fbm_volume(n: int, seed: int, n_blobs: int = 8, octaves: int = 4) -> np.ndarray:
    """Seeded smoke density: 8 anisotropic rotated Gaussian blobs x (0.5+0.5 fBm), clamp [0,2].

    Blob centres ~ U[0.25, 0.75] n, per-axis widths ~ U[0.05, 0.2] n, amplitude
    ~ U[0.5, 1.5]; fBm: 4 octaves, lacunarity 2, gain 0.5, base period n/4.
    Returns float32 [n][n][n] (z, y, x).
    """
    rng = np.random.default_rng(1_000_003 * seed + 17)
    blobs = []
    for _ in range(n_blobs):
        centre = rng.uniform(0.25, 0.75, size=3) * n
        widths = rng.uniform(0.05, 0.2, size=3) * n
        rot = _random_rotation(rng)
        amp = rng.uniform(0.5, 1.5)
        blobs.append((centre, widths, rot, amp))
    out = np.empty((n, n, n), np.float32)
    c = np.arange(n, dtype=np.float64) + 0.5
    chunk = max(1, (1 << 22) // (n * n))
    for z0 in range(0, n, chunk):
        z1 = min(n, z0 + chunk)
        zz, yy, xx = np.meshgrid(c[z0:z1], c, c, indexing="ij")
        pts = np.stack([xx, yy, zz], axis=-1)
        dens = np.zeros(zz.shape, np.float64)
        for centre, widths, rot, amp in blobs:
            local = (pts - centre) @ rot  # rotate into the blob frame
            dens += amp * np.exp(-0.5 * np.sum((local / widths) ** 2, axis=-1))
        noise = fbm(n, seed, octaves=octaves, z_range=(z0, z1))
        out[z0:z1] = np.clip(dens * (0.5 + 0.5 * noise), 0.0, 2.0)
    return out


def sphere_mask(n: int, radius: float, seed: int, lo: float = 30.0, hi: float = 98.0) -> tuple[np.ndarray, np.ndarray]:
    """Voxelised SDF sphere obstacle: mask=1 where |centre_of_voxel - c| <= radius.

    The centre is drawn ~ U[lo, hi]^3 (scaled by n/128 for other grid sizes).
    """
    rng = np.random.default_rng(7_000_001 * seed + 5)
    s = n / 128.0
    centre = rng.uniform(lo * s, hi * s, size=3)
    c = np.arange(n, dtype=np.float64) + 0.5
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    d2 = (xx - centre[0]) ** 2 + (yy - centre[1]) ** 2 + (zz - centre[2]) ** 2
    return (d2 <= radius * radius).astype(np.uint8), centre


# ----------------------------------------------------------------------------
# cameras and lights (plain descriptions; rays are computed by each side)
# ----------------------------------------------------------------------------

ORTHO = 0
PERSP = 1


@dataclass
class Camera:
    kind: int
    eye: tuple
    target: tuple
    up: tuple
    fov_y_deg: float
    ortho_height: float
    width: int
    height: int


@dataclass
class Light:
    dir: tuple          # unit vector toward the light, world space
    intensity: tuple    # RGB


def orbit_ortho_camera(n: int, seed: int, width: int, height: int) -> Camera:
    """Orthographic camera on an orbit around the grid centre (seeded angles).

    Azimuth ~ U[0, 2 pi), elevation ~ U[-30, 30] degrees, ortho height n sqrt(3).
    """
    rng = np.random.default_rng(3_000_017 * seed + 11)
    az = rng.uniform(0, 2 * math.pi)
    el = math.radians(rng.uniform(-30.0, 30.0))
    c = np.array([n / 2.0] * 3)
    dist = 2.5 * n
    off = np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)]) * dist
    eye = c + off
    return Camera(ORTHO, tuple(map(float, eye)), tuple(map(float, c)), (0.0, 1.0, 0.0),
                  40.0, float(n * math.sqrt(3.0)), width, height)


def perspective_camera(n: int, seed: int, width: int, height: int, fov_y_deg: float = 40.0,
                       dist_factor: float = 2.5) -> Camera:
    """Perspective camera 2.5 n from the grid centre at a seeded direction, fov_y 40 deg."""
    rng = np.random.default_rng(5_000_011 * seed + 13)
    az = rng.uniform(0, 2 * math.pi)
    el = math.radians(rng.uniform(-30.0, 30.0))
    c = np.array([n / 2.0] * 3)
    off = np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)]) * dist_factor * n
    eye = c + off
    return Camera(PERSP, tuple(map(float, eye)), tuple(map(float, c)), (0.0, 1.0, 0.0),
                  float(fov_y_deg), float(n), width, height)


def random_light(seed: int) -> Light:
    rng = np.random.default_rng(9_000_007 * seed + 3)
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    inten = rng.uniform(0.6, 1.4, size=3)
    return Light(tuple(map(float, v)), tuple(map(float, inten)))


# ----------------------------------------------------------------------------
# network parameters (layout of the UNet + adapters; values from a seed)
# ----------------------------------------------------------------------------

NSLW_MAGIC = b"NSLW"
NSLW_VERSION = 1
ADAPTERS = ("FB", "LR", "UD", "AE")   # order of Sec. 4.3 / Fig. 3


def param_spec(c0: int) -> list[tuple[str, tuple, str]]:
    """Ordered (name, shape, init) list of every network parameter.

    Conv weights are [Cout][Cin][kh][kw]; transposed-conv weights are
    [Cin][Cout][2][2]; 1x1 convs are [Cout][Cin].  init is one of
    'he:<fan_in>' (a ReLU follows: gain sqrt 2), 'lin:<fan_in>' (no ReLU
    follows: gain 1), 'bias', 'ln_w', 'ln_b', 'scale'.
    """
    c = [c0, 2 * c0, 4 * c0, 8 * c0]
    spec: list[tuple[str, tuple, str]] = []

    def conv3(name, cin, cout):
        spec.append((name + ".w", (cout, cin, 3, 3), f"he:{cin * 9}"))
        spec.append((name + ".b", (cout,), "bias"))

    def convt(name, cin, cout):
        spec.append((name + ".w", (cin, cout, 2, 2), f"lin:{cin}"))
        spec.append((name + ".b", (cout,), "bias"))

    def pw(name, cin, cout):
        spec.append((name + ".w", (cout, cin), f"lin:{cin}"))
        spec.append((name + ".b", (cout,), "bias"))

    conv3("enc1a", 3, c[0]); conv3("enc1b", c[0], c[0])
    conv3("enc2a", c[0], c[1]); conv3("enc2b", c[1], c[1])
    conv3("enc3a", c[1], c[2]); conv3("enc3b", c[2], c[2])
    conv3("enc4a", c[2], c[3]); conv3("enc4b", c[3], c[3])
    convt("up3", c[3], c[2]); conv3("dec3a", c[3], c[2]); conv3("dec3b", c[2], c[2])
    convt("up2", c[2], c[1]); conv3("dec2a", c[2], c[1]); conv3("dec2b", c[1], c[1])
    convt("up1", c[1], c[0]); conv3("dec1a", c[1], c[0]); conv3("dec1b", c[0], c[0])
    for a in ADAPTERS:
        p = "ad" + a
        spec.append((p + ".ln1.w", (c0,), "ln_w")); spec.append((p + ".ln1.b", (c0,), "ln_b"))
        pw(p + ".pw1", c0, 2 * c0)
        spec.append((p + ".dw.w", (2 * c0, 1, 3, 3), "lin:9")); spec.append((p + ".dw.b", (2 * c0,), "bias"))
        pw(p + ".sca", c0, c0)
        pw(p + ".pw2", c0, c0)
        spec.append((p + ".beta", (c0,), "scale"))
        spec.append((p + ".ln2.w", (c0,), "ln_w")); spec.append((p + ".ln2.b", (c0,), "ln_b"))
        pw(p + ".ffn1", c0, 2 * c0)
        pw(p + ".ffn2", c0, c0)
        spec.append((p + ".gamma", (c0,), "scale"))
        pw(p + ".head", c0, 2)
    return spec


def make_params(c0: int = 16, seed: int = 0, zero_residual_scales: bool = False) -> list[tuple[str, np.ndarray]]:
    """Kaiming-normal weights with the gain of the layer's nonlinearity: N(0, 2/fan_in)
    where a ReLU follows (the UNet 3x3 convs), N(0, 1/fan_in) where none does
    (transposed convs, adapter convs, heads); biases ~U(-0.1,0.1); NAFBlock beta,
    gamma ~U(0.5,1.5) (zero if zero_residual_scales); LayerNorm weight ~U(0.8,1.2),
    bias ~U(-0.1,0.1).  Values are float32."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape, init in param_spec(c0):
        if init.startswith("he:"):
            fan_in = int(init[3:])
            v = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=shape)
        elif init.startswith("lin:"):
            fan_in = int(init[4:])
            v = rng.normal(0.0, math.sqrt(1.0 / fan_in), size=shape)
        elif init == "bias":
            v = rng.uniform(-0.1, 0.1, size=shape)
        elif init == "ln_w":
            v = rng.uniform(0.8, 1.2, size=shape)
        elif init == "ln_b":
            v = rng.uniform(-0.1, 0.1, size=shape)
        elif init == "scale":
            v = np.zeros(shape) if zero_residual_scales else rng.uniform(0.5, 1.5, size=shape)
        else:
            raise ValueError(init)
        out.append((name, v.astype(np.float32)))
    return out


def flat_params(params) -> np.ndarray:
    return np.concatenate([p.reshape(-1) for _, p in params]).astype(np.float32)


def pack_blob(params, c0: int) -> bytes:
    """NSLW blob: 'NSLW', u32 version, u32 C0, u32 n_floats, then float32 values
    in param_spec order, then u32 checksum (sum of the float words as u32, mod 2^32)."""
    flat = flat_params(params)
    words = flat.view(np.uint32).astype(np.uint64)
    chk = int(words.sum() % (1 << 32))
    return (NSLW_MAGIC + struct.pack("<III", NSLW_VERSION, c0, flat.size) + flat.tobytes()
            + struct.pack("<I", chk))


def n_params(c0: int) -> int:
    return sum(int(np.prod(s)) for _, s, _ in param_spec(c0))


# ----------------------------------------------------------------------------
# workload descriptions
# ----------------------------------------------------------------------------


@dataclass
class PlumeFrame:
    density: np.ndarray          # float32 or float16 [nz][ny][nx]
    mask: np.ndarray | None      # uint8 or None
    camera: Camera
    light: Light
    step: float
    sigma_scale: float = 1.0
    meta: dict = field(default_factory=dict)


def config_plain_64(seed: int = 1) -> PlumeFrame:
    """64^3 FP32 blob x fBm, no obstacle, orthographic orbit, 128x128, step 4."""
    n = 64
    vol = blob_fbm_volume(n, seed)
    cam = orbit_ortho_camera(n, seed, 128, 128)
    return PlumeFrame(vol, None, cam, random_light(seed), 4.0, meta={"name": "plume64_ortho128_h4"})


def config_obstacle_128(seed: int = 2, width: int = 512, height: int = 512) -> PlumeFrame:
    """128^3 FP32 with a radius-20 voxelised sphere obstacle, perspective, 512^2, step 2."""
    n = 128
    vol = blob_fbm_volume(n, seed)
    mask, centre = sphere_mask(n, 20.0, seed)
    cam = perspective_camera(n, seed, width, height)
    return PlumeFrame(vol, mask, cam, random_light(seed), 2.0,
                      meta={"name": f"plume128_sphere20_persp{width}_h2", "sphere_centre": centre.tolist()})


def small_case(n: int = 24, width: int = 32, height: int = 24, seed: int = 11, kind: int = PERSP,
               step: float = 2.0, with_mask: bool = True) -> PlumeFrame:
    """A small ragged case (sizes not multiples of the kernels' tiles)."""
    vol = blob_fbm_volume(n, seed)
    mask = None
    if with_mask:
        mask, _ = sphere_mask(n, n / 6.0, seed)
    if kind == PERSP:
        cam = perspective_camera(n, seed, width, height)
    else:
        cam = orbit_ortho_camera(n, seed, width, height)
    return PlumeFrame(vol, mask, cam, random_light(seed), step, meta={"name": f"small{n}"})


def blob_fbm_volume_fast(n: int, seed: int, device=None):
    """blob_fbm_volume evaluated with torch (GPU when given): the same recipe and
    random draws, computed in float32 tensors; used for large batches."""
    import torch
    dev = torch.device(device or "cpu")
    rng = np.random.default_rng(1_000_003 * seed + 17)
    blobs = []
    for _ in range(8):
        centre = rng.uniform(0.25, 0.75, size=3) * n
        widths = rng.uniform(0.05, 0.2, size=3) * n
        rot = _random_rotation(rng)
        amp = rng.uniform(0.5, 1.5)
        blobs.append((centre, widths, rot, amp))
    c = torch.arange(n, dtype=torch.float32, device=dev) + 0.5
    zz, yy, xx = torch.meshgrid(c, c, c, indexing="ij")
    pts = torch.stack([xx, yy, zz], dim=-1)
    dens = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
    for centre, widths, rot, amp in blobs:
        local = (pts - torch.tensor(centre, dtype=torch.float32, device=dev)) @ torch.tensor(rot, dtype=torch.float32, device=dev)
        dens += float(amp) * torch.exp(-0.5 * ((local / torch.tensor(widths, dtype=torch.float32, device=dev)) ** 2).sum(-1))
    # fBm with the same lattice draws as fbm()
    rng2 = np.random.default_rng(seed)
    total = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
    amp, norm, freq = 1.0, 0.0, 1.0 / (n / 4.0)
    for _ in range(4):
        grads = torch.tensor(_lattice_gradients(rng2, 64), device=dev)
        off = rng2.uniform(0, 64, size=3).astype(np.float32)
        px, py, pz = xx * freq + float(off[0]), yy * freq + float(off[1]), zz * freq + float(off[2])
        x0, y0, z0 = torch.floor(px), torch.floor(py), torch.floor(pz)
        fx, fy, fz = px - x0, py - y0, pz - z0
        ix, iy, iz = x0.long() % 64, y0.long() % 64, z0.long() % 64
        fade = lambda t: t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
        ux, uy, uz = fade(fx), fade(fy), fade(fz)
        acc = torch.zeros_like(total)
        for dz in (0, 1):
            wz = uz if dz else 1.0 - uz
            for dy in (0, 1):
                wy = uy if dy else 1.0 - uy
                for dx in (0, 1):
                    wx = ux if dx else 1.0 - ux
                    g = grads[(iz + dz) % 64, (iy + dy) % 64, (ix + dx) % 64]
                    acc += wx * wy * wz * (g[..., 0] * (fx - dx) + g[..., 1] * (fy - dy) + g[..., 2] * (fz - dz))
        total += amp * acc
        norm += amp
        amp *= 0.5
        freq *= 2.0
    noise = torch.clamp(total / norm * 1.6, -1.0, 1.0)
    return torch.clamp(dens * (0.5 + 0.5 * noise), 0.0, 2.0)


@dataclass
class BatchPlume:
    n: int
    width: int
    height: int
    seed: int
    camera: Camera
    light: Light
    step: float


def batch_plumes_spec(count: int = 64, seed: int = 4, sizes=(32, 48, 64, 96, 128, 192),
                      billboards=(64, 128, 256, 512), step: float = 2.0) -> list:
    """The batched workload: `count` plumes with grid sizes drawn uniformly from
    `sizes` (cubic) and square billboards from `billboards`, each with its own
    seeded perspective camera and light."""
    rng = np.random.default_rng(11_000_003 * seed + 1)
    out = []
    for k in range(count):
        n = int(rng.choice(sizes))
        b = int(rng.choice(billboards))
        s = int(rng.integers(0, 1 << 30))
        out.append(BatchPlume(n, b, b, s, perspective_camera(n, s, b, b), random_light(s), step))
    return out


def serving_plumes_spec(count: int = 256, seed: int = 5, sizes=(32, 48, 64, 96, 128, 192, 256),
                        billboards=(64, 128, 256, 512, 1024), step: float = 2.0) -> list:
    """The serving workload's resident plumes: grid sizes drawn uniformly from
    `sizes` (cubic), square billboards from `billboards`, seeded per plume."""
    rng = np.random.default_rng(13_000_019 * seed + 7)
    out = []
    for k in range(count):
        n = int(rng.choice(sizes))
        b = int(rng.choice(billboards))
        s = int(rng.integers(0, 1 << 30))
        out.append(BatchPlume(n, b, b, s, perspective_camera(n, s, b, b), random_light(s), step))
    return out


def poisson_requests(count_plumes: int, rate_hz: float, duration_s: float, seed: int = 5):
    """Seeded Poisson arrivals: (arrival time in s, plume index, camera seed,
    light seed) with exponential inter-arrival times of mean 1/rate_hz and the
    plume drawn uniformly."""
    rng = np.random.default_rng(17_000_023 * seed + 9)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            return out
        out.append((t, int(rng.integers(0, count_plumes)), int(rng.integers(0, 1 << 30)),
                    int(rng.integers(0, 1 << 30))))


def fbm_torch(n: int, seed: int, device=None, octaves: int = 4, base_period: float | None = None):
    """fbm() evaluated with torch (float32, on `device`): same lattice draws,
    same recipe, values in [-1, 1]."""
    import torch
    dev = torch.device(device or "cpu")
    rng = np.random.default_rng(seed)
    if base_period is None:
        base_period = n / 4.0
    c = torch.arange(n, dtype=torch.float32, device=dev) + 0.5
    zz, yy, xx = torch.meshgrid(c, c, c, indexing="ij")
    total = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
    amp, norm, freq = 1.0, 0.0, 1.0 / base_period
    fade = lambda t: t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    for _ in range(octaves):
        grads = torch.tensor(_lattice_gradients(rng, 64), device=dev)
        off = rng.uniform(0, 64, size=3).astype(np.float32)
        px, py, pz = xx * freq + float(off[0]), yy * freq + float(off[1]), zz * freq + float(off[2])
        x0, y0, z0 = torch.floor(px), torch.floor(py), torch.floor(pz)
        fx, fy, fz = px - x0, py - y0, pz - z0
        ix, iy, iz = x0.long() % 64, y0.long() % 64, z0.long() % 64
        ux, uy, uz = fade(fx), fade(fy), fade(fz)
        acc = torch.zeros_like(total)
        for dz in (0, 1):
            wz = uz if dz else 1.0 - uz
            for dy in (0, 1):
                wy = uy if dy else 1.0 - uy
                for dx in (0, 1):
                    wx = ux if dx else 1.0 - ux
                    g = grads[(iz + dz) % 64, (iy + dy) % 64, (ix + dx) % 64]
                    acc += wx * wy * wz * (g[..., 0] * (fx - dx) + g[..., 1] * (fy - dy) + g[..., 2] * (fz - dz))
        total += amp * acc
        norm += amp
        amp *= 0.5
        freq *= 2.0
    return torch.clamp(total / norm * 1.6, -1.0, 1.0)


def _catmull_rom(p0, p1, p2, p3, t):
    t2, t3 = t * t, t * t * t
    return 0.5 * ((2.0 * p1) + (-p0 + p2) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t2
                  + (-p0 + 3.0 * p1 - 3.0 * p2 + p3) * t3)


@dataclass
class AnimatedSequence:
    n: int
    frames: dict           # frame index -> torch float16 tensor [n][n][n] on the device
    cameras: list          # Camera per frame
    lights: list           # Light per frame
    step: float


def animated_sequence(n: int = 256, count: int = 300, seed: int = 3, width: int = 1024,
                      height: int = 1024, step: float = 4.0, device=None, keep=None) -> AnimatedSequence:
    """The animated workload.  Frame 0 is the blob x fBm generator (seed); each
    later frame advects the previous one semi-Lagrangian (trilinear, zero
    outside the box) along a static divergence-free velocity, the curl of three
    seeded fBm potentials (2 octaves, base period n/2) scaled to a maximum speed
    of 1 voxel per frame, then re-injects 3% of frame 0 (rho <- 0.97 rho_adv +
    0.03 rho_0, clamped to [0, 2]); frames are stored as FP16.  The camera
    (perspective, fov 40) follows a closed Catmull-Rom spline through 8 seeded
    points 2.5 n from the centre (azimuth U[0, 2 pi), elevation U[-45, 45]
    degrees); the light starts at a seeded direction and turns 1 degree per frame
    about the world Y axis.  `keep` limits which frames are kept (all if None)."""
    import torch
    import torch.nn.functional as F
    dev = torch.device(device or "cuda")
    rho0 = blob_fbm_volume_fast(n, seed, device=dev)
    psi = [fbm_torch(n, 7_000_001 * seed + 101 + k, dev, octaves=2, base_period=n / 2.0) for k in range(3)]
    d = [torch.gradient(p) for p in psi]          # each: (d/dz, d/dy, d/dx)
    vx = d[2][1] - d[1][0]                        # d psi_z/dy - d psi_y/dz
    vy = d[0][0] - d[2][2]                        # d psi_x/dz - d psi_z/dx
    vz = d[1][2] - d[0][1]                        # d psi_y/dx - d psi_x/dy
    vmax = torch.sqrt(vx * vx + vy * vy + vz * vz).max()
    vx, vy, vz = vx / vmax, vy / vmax, vz / vmax
    del psi, d
    c = torch.arange(n, dtype=torch.float32, device=dev) + 0.5
    zz, yy, xx = torch.meshgrid(c, c, c, indexing="ij")
    # departure points x - v(x), as grid_sample coordinates (-1 at 0, +1 at n)
    grid = torch.stack([(xx - vx) / n * 2 - 1, (yy - vy) / n * 2 - 1, (zz - vz) / n * 2 - 1], dim=-1)[None]
    del zz, yy, xx, vx, vy, vz
    keep = set(range(count)) if keep is None else set(keep)
    frames = {}
    rho = rho0
    for t in range(count):
        if t in keep:
            frames[t] = rho.to(torch.float16)
        if t + 1 < count:
            adv = F.grid_sample(rho[None, None], grid, mode="bilinear", padding_mode="zeros",
                                align_corners=False)[0, 0]
            rho = torch.clamp(0.97 * adv + 0.03 * rho0, 0.0, 2.0)
    rng = np.random.default_rng(19_000_033 * seed + 5)
    ctr = np.array([n / 2.0] * 3)
    pts = []
    for _ in range(8):
        az = rng.uniform(0, 2 * math.pi)
        el = math.radians(rng.uniform(-45.0, 45.0))
        pts.append(ctr + 2.5 * n * np.array([math.cos(el) * math.cos(az), math.sin(el), math.cos(el) * math.sin(az)]))
    cams = []
    for t in range(count):
        s = 8.0 * t / count
        i = int(math.floor(s))
        u = s - i
        eye = _catmull_rom(pts[(i - 1) % 8], pts[i % 8], pts[(i + 1) % 8], pts[(i + 2) % 8], u)
        cams.append(Camera(PERSP, tuple(map(float, eye)), tuple(map(float, ctr)), (0.0, 1.0, 0.0), 40.0, 0.0,
                           width, height))
    l0 = random_light(seed)
    lights = []
    for t in range(count):
        a = math.radians(float(t))
        x, y, z = l0.dir
        lights.append(Light((math.cos(a) * x + math.sin(a) * z, y, -math.sin(a) * x + math.cos(a) * z),
                            l0.intensity))
    return AnimatedSequence(n, frames, cams, lights, step)
