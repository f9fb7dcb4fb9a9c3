"""Pins of the FP64 oracle's lightmap network (Sec. 4.3) against PyTorch float64
library routines, brute force and identity special cases.  CPU only."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

from paper_2604_03748_gb300 import inputs as I



def T(a):
    return torch.from_numpy(np.asarray(a, np.float64))


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("cin,cout,H,W", [(3, 4, 8, 8), (5, 2, 6, 10), (16, 8, 8, 16)])
def test_conv2d_matches_torch(orc, k, cin, cout, H, W):
    rng = np.random.default_rng(cin * 100 + cout * 10 + k)
    x = rng.normal(size=(cin, H, W))
    w = rng.normal(size=(cout, cin, k, k))
    b = rng.normal(size=cout)
    ref = Fn.conv2d(T(x)[None], T(w), T(b), padding=(k - 1) // 2)[0].numpy()
    np.testing.assert_allclose(orc.conv2d(x, w, b, k), ref, rtol=1e-12, atol=1e-12)


def test_conv2d_brute_force_delta(orc):
    """A centred delta kernel is the identity; a shifted delta shifts with zero fill."""
    x = np.random.default_rng(1).normal(size=(2, 5, 7))
    w = np.zeros((2, 2, 3, 3))
    w[0, 0, 1, 1] = 1.0
    w[1, 1, 1, 1] = 1.0
    np.testing.assert_array_equal(orc.conv2d(x, w, None, 3), x)
    w2 = np.zeros((1, 1, 3, 3))
    w2[0, 0, 1, 2] = 1.0  # out(y, x) = in(y, x+1)
    out = orc.conv2d(x[:1], w2, None, 3)
    np.testing.assert_array_equal(out[0, :, :-1], x[0, :, 1:])
    assert np.all(out[0, :, -1] == 0)


def test_conv1x1_is_matmul(orc):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(6, 4, 5))
    w = rng.normal(size=(3, 6, 1, 1))
    ref = np.einsum("oc,chw->ohw", w[:, :, 0, 0], x)
    np.testing.assert_allclose(orc.conv2d(x, w, None, 1), ref, rtol=1e-12, atol=1e-12)


def test_conv_transpose_matches_torch(orc):
    rng = np.random.default_rng(3)
    x = rng.normal(size=(6, 4, 5))
    w = rng.normal(size=(6, 3, 2, 2))
    b = rng.normal(size=3)
    ref = Fn.conv_transpose2d(T(x)[None], T(w), T(b), stride=2)[0].numpy()
    np.testing.assert_allclose(orc.conv_transpose2x2(x, w, b), ref, rtol=1e-12, atol=1e-12)


def test_maxpool_matches_torch(orc):
    x = np.random.default_rng(4).normal(size=(3, 8, 6))
    np.testing.assert_array_equal(orc.maxpool2(x), Fn.max_pool2d(T(x)[None], 2)[0].numpy())


def test_layernorm_matches_torch(orc):
    rng = np.random.default_rng(5)
    x = rng.normal(size=(16, 4, 6)) * 3 + 1
    g = rng.uniform(0.5, 1.5, 16)
    b = rng.normal(size=16)
    ref = Fn.layer_norm(T(x).permute(1, 2, 0), (16,), T(g), T(b), eps=1e-6).permute(2, 0, 1).numpy()
    np.testing.assert_allclose(orc.layernorm(x, g, b), ref, rtol=1e-12, atol=1e-12)


def test_dwconv_matches_torch(orc):
    rng = np.random.default_rng(6)
    x = rng.normal(size=(8, 6, 7))
    w = rng.normal(size=(8, 1, 3, 3))
    b = rng.normal(size=8)
    ref = Fn.conv2d(T(x)[None], T(w), T(b), padding=1, groups=8)[0].numpy()
    np.testing.assert_allclose(orc.dwconv3(x, w, b), ref, rtol=1e-12, atol=1e-12)


def _nafblock_params(c, rng, zero_scales=False):
    parts = dict(
        ln1w=rng.uniform(0.8, 1.2, c), ln1b=rng.uniform(-0.1, 0.1, c),
        pw1w=rng.normal(size=(2 * c, c)) * 0.3, pw1b=rng.uniform(-0.1, 0.1, 2 * c),
        dww=rng.normal(size=(2 * c, 1, 3, 3)) * 0.3, dwb=rng.uniform(-0.1, 0.1, 2 * c),
        scaw=rng.normal(size=(c, c)) * 0.3, scab=rng.uniform(-0.1, 0.1, c),
        pw2w=rng.normal(size=(c, c)) * 0.3, pw2b=rng.uniform(-0.1, 0.1, c),
        beta=np.zeros(c) if zero_scales else rng.uniform(0.5, 1.5, c),
        ln2w=rng.uniform(0.8, 1.2, c), ln2b=rng.uniform(-0.1, 0.1, c),
        f1w=rng.normal(size=(2 * c, c)) * 0.3, f1b=rng.uniform(-0.1, 0.1, 2 * c),
        f2w=rng.normal(size=(c, c)) * 0.3, f2b=rng.uniform(-0.1, 0.1, c),
        gamma=np.zeros(c) if zero_scales else rng.uniform(0.5, 1.5, c),
    )
    flat = np.concatenate([np.asarray(v).reshape(-1) for v in parts.values()])
    return parts, flat


def _torch_nafblock(x, p, c):
    """NAFBlock written with PyTorch library ops (LayerNorm over channels, 1x1 and
    depthwise convs, adaptive average pooling)."""
    def ln(v, w, b):
        return Fn.layer_norm(v.permute(0, 2, 3, 1), (c,), T(w), T(b), eps=1e-6).permute(0, 3, 1, 2)

    def pw(v, w, b):
        return Fn.conv2d(v, T(w)[:, :, None, None], T(b))

    t = pw(ln(x, p["ln1w"], p["ln1b"]), p["pw1w"], p["pw1b"])
    t = Fn.conv2d(t, T(p["dww"]), T(p["dwb"]), padding=1, groups=2 * c)
    a, bb = t.chunk(2, dim=1)
    t = a * bb
    t = t * pw(Fn.adaptive_avg_pool2d(t, 1), p["scaw"], p["scab"])
    t = pw(t, p["pw2w"], p["pw2b"])
    y = x + t * T(p["beta"])[None, :, None, None]
    t = pw(ln(y, p["ln2w"], p["ln2b"]), p["f1w"], p["f1b"])
    a, bb = t.chunk(2, dim=1)
    t = pw(a * bb, p["f2w"], p["f2b"])
    return y + t * T(p["gamma"])[None, :, None, None]


def test_nafblock_identity_when_scales_zero(orc):
    rng = np.random.default_rng(7)
    _, flat = _nafblock_params(4, rng, zero_scales=True)
    x = rng.normal(size=(4, 6, 6))
    np.testing.assert_array_equal(orc.nafblock(x, flat), x)


def test_nafblock_matches_torch_composition(orc):
    rng = np.random.default_rng(8)
    c = 6
    parts, flat = _nafblock_params(c, rng)
    x = rng.normal(size=(c, 8, 10))
    assert flat.size == orc.nafblock_params(c)
    ref = _torch_nafblock(T(x)[None], parts, c)[0].numpy()
    np.testing.assert_allclose(orc.nafblock(x, flat), ref, rtol=1e-11, atol=1e-12)


def torch_unet_forward(guide, params, c0, depth_scale):
    """The Sec. 4.3 generator assembled from PyTorch float64 library ops, used to
    check the oracle's wiring (levels, skip order, adapter-to-plane mapping)."""
    P = {k: T(v) for k, v in params}
    x = T(guide).clone()[None]
    x[:, 2] *= depth_scale

    def c3(v, name):
        return torch.relu(Fn.conv2d(v, P[name + ".w"], P[name + ".b"], padding=1))

    s1 = c3(c3(x, "enc1a"), "enc1b")
    s2 = c3(c3(Fn.max_pool2d(s1, 2), "enc2a"), "enc2b")
    s3 = c3(c3(Fn.max_pool2d(s2, 2), "enc3a"), "enc3b")
    b = c3(c3(Fn.max_pool2d(s3, 2), "enc4a"), "enc4b")
    u = Fn.conv_transpose2d(b, P["up3.w"], P["up3.b"], stride=2)
    d = c3(c3(torch.cat([u, s3], 1), "dec3a"), "dec3b")
    u = Fn.conv_transpose2d(d, P["up2.w"], P["up2.b"], stride=2)
    d = c3(c3(torch.cat([u, s2], 1), "dec2a"), "dec2b")
    u = Fn.conv_transpose2d(d, P["up1.w"], P["up1.b"], stride=2)
    F = c3(c3(torch.cat([u, s1], 1), "dec1a"), "dec1b")
    out = torch.zeros(8, F.shape[2], F.shape[3], dtype=torch.float64)
    planes = {"FB": (4, 5), "LR": (0, 1), "UD": (2, 3), "AE": (6, 7)}
    for a in I.ADAPTERS:
        p = "ad" + a
        parts = dict(ln1w=P[p + ".ln1.w"], ln1b=P[p + ".ln1.b"], pw1w=P[p + ".pw1.w"], pw1b=P[p + ".pw1.b"],
                     dww=P[p + ".dw.w"], dwb=P[p + ".dw.b"], scaw=P[p + ".sca.w"], scab=P[p + ".sca.b"],
                     pw2w=P[p + ".pw2.w"], pw2b=P[p + ".pw2.b"], beta=P[p + ".beta"], ln2w=P[p + ".ln2.w"],
                     ln2b=P[p + ".ln2.b"], f1w=P[p + ".ffn1.w"], f1b=P[p + ".ffn1.b"], f2w=P[p + ".ffn2.w"],
                     f2b=P[p + ".ffn2.b"], gamma=P[p + ".gamma"])
        parts = {k: v.numpy() for k, v in parts.items()}
        z = _torch_nafblock(F, parts, c0)
        h = Fn.conv2d(z, P[p + ".head.w"][:, :, None, None], P[p + ".head.b"])[0]
        out[planes[a][0]] = h[0]
        out[planes[a][1]] = h[1]
    return out.numpy()


@pytest.mark.parametrize("c0,H,W", [(4, 16, 24), (8, 24, 16), (32, 16, 8)])
def test_net_forward_matches_torch_assembly(orc, c0, H, W):
    params = I.make_params(c0, seed=0)
    flat = I.flat_params(params).astype(np.float64)
    assert flat.size == I.n_params(c0)
    rng = np.random.default_rng(9)
    guide = np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 60, (H, W))])
    got = orc.net_forward(guide, flat, c0, 1 / 50.0)
    ref = torch_unet_forward(guide, params, c0, 1 / 50.0)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-11)


def test_net_forward_rejects_bad_sizes(orc):
    flat = I.flat_params(I.make_params(4)).astype(np.float64)
    with pytest.raises(ValueError):
        orc.net_forward(np.zeros((3, 12, 16)), flat, 4, 1.0)
    with pytest.raises(ValueError):
        orc.net_forward(np.zeros((3, 16, 16)), flat[:-1], 4, 1.0)


def test_blob_roundtrip():
    params = I.make_params(16, seed=0)
    blob = I.pack_blob(params, 16)
    assert blob[:4] == b"NSLW"
    n = I.n_params(16)
    assert len(blob) == 16 + 4 * n + 4
    # He-normal statistics of the largest conv weight
    w = dict(params)["enc4b.w"]
    assert abs(w.std() - np.sqrt(2.0 / (128 * 9))) < 0.01 * np.sqrt(2.0 / (128 * 9)) * 10
