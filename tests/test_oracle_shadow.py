"""Pins of the oracle's obstacle shadowing (Sec. 4.5): the shadow map of the
obstacle mask against closed forms, and the shadowed shading against the
plain six-way shading.  CPU only."""
import math

import numpy as np

from paper_2604_03748_gb300 import inputs as I


def frame(light_dir):
    """The light frame written out in float64 and rounded once (w, e1, e2)."""
    v = np.asarray(light_dir, np.float64)
    w = -v / np.linalg.norm(v)
    a = np.array([0.0, 0.0, 1.0]) if abs(w[1]) > 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(w, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(e1, w)
    return w.astype(np.float32), e1.astype(np.float32), e2.astype(np.float32)


def texel_origins(n, light_dir, R):
    w, e1, e2 = frame(light_dir)
    S = np.float32(math.sqrt(3.0 * n * n))
    c = np.full(3, np.float32(n / 2), np.float32)
    u = ((np.arange(R, dtype=np.float32) + np.float32(0.5)) / np.float32(R) - np.float32(0.5)) * S
    a = u[None, :]                      # column i
    b = u[:, None]                      # row j
    o = c[:, None, None] + a[None] * e1[:, None, None] + b[None] * e2[:, None, None]
    return o.astype(np.float64), w.astype(np.float64)


def test_single_voxel_under_a_vertical_light(orc):
    n, R = 8, 64
    mask = np.zeros((n, n, n), np.uint8)
    mask[5, 1, 2] = 1                    # voxel x in [2, 3], y in [1, 2], z in [5, 6]
    m = orc.shadow_map(mask, (0.0, 1.0, 0.0), R)
    o, w = texel_origins(n, (0.0, 1.0, 0.0), R)
    assert np.allclose(w, [0, -1, 0])
    x, z = o[0], o[2]                    # the light ray goes straight down from y = 4
    inside = (x > 2) & (x < 3) & (z > 5) & (z < 6)
    edge = (np.abs(x - 2) < 1e-4) | (np.abs(x - 3) < 1e-4) | (np.abs(z - 5) < 1e-4) | (np.abs(z - 6) < 1e-4)
    assert inside.sum() > 10
    assert np.all(m[inside] == 2.0)      # enters the top face y = 2 after 4 - 2 voxels
    assert np.all(np.isinf(m[~inside & ~edge]))


def test_slab_under_an_oblique_light(orc):
    n, R = 16, 48
    mask = np.zeros((n, n, n), np.uint8)
    mask[:, :4, :] = 1                   # every voxel with y < 4
    d = (0.3, 1.0, 0.2)
    m = orc.shadow_map(mask, d, R).astype(np.float64)
    o, w = texel_origins(n, d, R)
    t = (4.0 - o[1]) / w[1]              # the line meets the slab's top face y = 4
    xh, zh = o[0] + t * w[0], o[2] + t * w[2]
    top = (xh > 0.01) & (xh < n - 0.01) & (zh > 0.01) & (zh < n - 0.01)
    assert top.sum() > 100
    np.testing.assert_allclose(m[top], t[top], rtol=1e-5, atol=1e-4)
    # lines that never enter the box find nothing
    far = (np.abs(o[0] - n / 2) > n) | (np.abs(o[2] - n / 2) > n)
    assert np.all(np.isinf(m[far & ~top]))


def axis_camera(n, W, H, eye_z_off=18.0):
    return I.Camera(I.ORTHO, (n / 2, n / 2, n + eye_z_off), (n / 2, n / 2, 0.0), (0.0, 1.0, 0.0),
                    40.0, float(n), W, H)


def test_occluder_removes_one_lights_term(orc):
    """Camera down -z (pixel (i, j) at x = 2i + 1, y = 31 - 2j), the shell 5
    voxels behind the front face; an occluder slab over x < 16, y in [20, 24)
    under a light from +Y.  Its map holds t = -8 (top face y = 24, 8 voxels
    above the map plane y = 16) over x < 16; a shell point is shadowed when
    16 - y > -8 + bias, i.e. y < 23 at bias 1: those pixels keep only the
    second light's term."""
    n, W, H = 32, 16, 16
    cam = axis_camera(n, W, H)
    mask = np.zeros((n, n, n), np.uint8)
    mask[:, 20:24, :16] = 1
    L0 = I.Light((0.0, 1.0, 0.0), (1.0, 0.5, 0.25))
    L1 = I.Light((1.0, 0.2, 0.3), (0.3, 0.6, 0.9))
    m0 = orc.shadow_map(mask, L0.dir, 64)
    rng = np.random.default_rng(4)
    lm = rng.uniform(0.0, 1.0, (8, H, W))
    guide = np.zeros((3, H, W), np.float32)
    guide[2] = 5.0
    got = orc.shade_shadowed(lm, guide, cam, [L0, L1], (n, n, n), [m0, None], 1.0)
    both = orc.shade(lm, cam, [L0, L1])
    only1 = orc.shade(lm, cam, [L1])
    xs = 2 * np.arange(W)[None, :] + 1 + 0 * np.arange(H)[:, None]
    ys = 31 - 2 * np.arange(H)[:, None] + 0 * np.arange(W)[None, :]
    shadowed = (xs < 16) & (ys < 23)
    assert 0 < shadowed.sum() < W * H
    np.testing.assert_allclose(got[:3][:, shadowed], only1[:3][:, shadowed], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(got[:3][:, ~shadowed], both[:3][:, ~shadowed], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(got[3], both[3])
    # no shell (D = 0) means lit
    g0 = guide.copy()
    g0[2] = 0.0
    np.testing.assert_allclose(orc.shade_shadowed(lm, g0, cam, [L0, L1], (n, n, n), [m0, None], 1.0), both,
                               rtol=1e-12, atol=1e-15)


def test_without_maps_equals_plain_shading(orc):
    pf = I.small_case(16, 24, 16, seed=3)
    rng = np.random.default_rng(5)
    lm = rng.normal(size=(8, 16, 24))
    guide = rng.uniform(0, 10, (3, 16, 24)).astype(np.float32)
    lights = [I.random_light(1), I.random_light(2)]
    got = orc.shade_shadowed(lm, guide, pf.camera, lights, pf.density.shape, [None, None], 1.0)
    np.testing.assert_array_equal(got, orc.shade(lm, pf.camera, lights))
