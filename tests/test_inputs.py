"""The seeded synthetic input recipe (the stand-in for the paper's simulated
smoke): shapes, value ranges, distributions and determinism of every
generator the tests and the benchmark share.  CPU only."""
import math
import struct

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I


def test_blob_fbm_volume_range_and_determinism():
    a = I.blob_fbm_volume(32, 3)
    assert a.dtype == np.float32 and a.shape == (32, 32, 32)
    assert a.min() >= 0.0 and a.max() <= 2.0 and a.mean() > 0.01
    assert np.array_equal(a, I.blob_fbm_volume(32, 3))
    assert not np.array_equal(a, I.blob_fbm_volume(32, 4))
    # blob centres are drawn in the middle half of each axis: that eighth of the
    # box holds well over its volume share of the mass
    inner = a[8:24, 8:24, 8:24].sum()
    assert inner > 0.3 * a.sum()


def test_fbm_noise_range():
    f = I.fbm(32, 5)
    assert f.shape == (32, 32, 32) and np.isfinite(f).all()
    assert -1.0 <= f.min() and f.max() <= 1.0 and f.std() > 0.05


def test_blob_fbm_volume_fast_shape_and_range():
    t = I.blob_fbm_volume_fast(32, 3)
    a = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    assert a.shape == (32, 32, 32) and a.min() >= 0.0 and a.max() <= 2.0 and a.mean() > 0.01


def test_sphere_mask_radius_and_centre():
    m, c = I.sphere_mask(128, 20.0, 2)
    assert m.dtype == np.uint8 and m.shape == (128, 128, 128)
    assert np.all((c >= 30.0) & (c <= 98.0))
    vol = 4.0 / 3.0 * math.pi * 20.0 ** 3
    assert abs(int(m.sum()) - vol) < 0.02 * vol


def test_cameras_follow_the_recipe():
    n = 64
    for seed in range(8):
        o = I.orbit_ortho_camera(n, seed, 128, 96)
        p = I.perspective_camera(n, seed, 128, 96)
        for cam in (o, p):
            off = np.array(cam.eye) - np.array(cam.target)
            assert np.allclose(cam.target, (n / 2,) * 3)
            assert abs(np.linalg.norm(off) - 2.5 * n) < 1e-9
            el = math.degrees(math.asin(off[1] / np.linalg.norm(off)))
            assert -30.0 - 1e-9 <= el <= 30.0 + 1e-9
            assert cam.up == (0.0, 1.0, 0.0) and (cam.width, cam.height) == (128, 96)
        assert o.kind == I.ORTHO and o.ortho_height == pytest.approx(n * math.sqrt(3))
        assert p.kind == I.PERSP and p.fov_y_deg == 40.0


def test_random_light():
    for seed in range(16):
        li = I.random_light(seed)
        assert abs(np.linalg.norm(li.dir) - 1.0) < 1e-12
        assert all(0.6 <= v <= 1.4 for v in li.intensity)


def test_params_and_blob():
    c0 = 16
    params = I.make_params(c0, 0)
    flat = I.flat_params(params)
    assert flat.dtype == np.float32 and flat.size == I.n_params(c0)
    names = [name for name, _ in params]
    assert names == [name for name, _, _ in I.param_spec(c0)]
    blob = I.pack_blob(params, c0)
    magic, (ver, bc0, nf) = blob[:4], struct.unpack("<III", blob[4:16])
    assert magic == b"NSLW" and bc0 == c0 and nf == flat.size
    body = np.frombuffer(blob[16:16 + 4 * nf], np.float32)
    assert np.array_equal(body, flat)
    (chk,) = struct.unpack("<I", blob[16 + 4 * nf:])
    assert chk == int(body.view(np.uint32).astype(np.uint64).sum() % (1 << 32))
    assert len(blob) == 16 + 4 * nf + 4
    # Kaiming scale on the large UNet convolutions: N(0, 2 / fan_in) where a ReLU follows
    by_name = dict(params)
    big = [(k, v) for k, v in by_name.items() if v.ndim == 4 and v.shape[2:] == (3, 3) and v.size >= 20000]
    assert big
    for k, w in big:
        fan_in = w.shape[1] * 9
        assert abs(w.std() / math.sqrt(2.0 / fan_in) - 1.0) < 0.1, k
    assert np.array_equal(flat, I.flat_params(I.make_params(c0, 0)))


def test_batch_and_serving_specs():
    b = I.batch_plumes_spec(64, seed=4)
    assert len(b) == 64
    assert {p.n for p in b} <= {32, 48, 64, 96, 128, 192}
    assert {p.width for p in b} <= {64, 128, 256, 512} and all(p.width == p.height for p in b)
    assert len({p.n for p in b}) >= 4 and len({p.width for p in b}) >= 3
    s = I.serving_plumes_spec(256, seed=5)
    assert len(s) == 256
    assert {p.n for p in s} == {32, 48, 64, 96, 128, 192, 256}
    assert {p.width for p in s} == {64, 128, 256, 512, 1024}
    # billboard pixels: E = mean of b^2 over the five sizes
    e = np.mean([v * v for v in (64, 128, 256, 512, 1024)])
    px = np.array([p.width * p.height for p in s], np.float64)
    assert abs(px.mean() - e) < 4 * px.std() / math.sqrt(len(px))


def test_poisson_requests():
    rate, dur = 2000.0, 2.0
    r = I.poisson_requests(256, rate, dur, seed=5)
    n = len(r)
    assert abs(n - rate * dur) < 4 * math.sqrt(rate * dur)
    t = np.array([x[0] for x in r])
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < dur
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0 / rate) < 4 * (1.0 / rate) / math.sqrt(n)
    ids = np.array([x[1] for x in r])
    assert ids.min() >= 0 and ids.max() < 256
    counts = np.bincount(ids, minlength=256)
    # uniform plume choice: chi-square over 256 bins with 255 degrees of freedom
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    assert r == I.poisson_requests(256, rate, dur, seed=5)
