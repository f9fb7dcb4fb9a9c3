"""Pins of the oracle's FP8 E4M3 network emulation (precision form).  The
rounding primitives are checked against PyTorch's float8_e4m3fn and float16
casts and against brute force over every E4M3 code decoded from the format's
definition; the quantised network against an assembly of PyTorch float64
library ops that uses those casts.  CPU only."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

from paper_2604_03748_gb300 import inputs as I
from test_oracle_net import T, _torch_nafblock


def e4m3_values():
    """Every finite E4M3 value from the bit layout: sign, 4 exponent bits
    (bias 7), 3 fraction bits; exponent field 0 is subnormal; S.1111.111 is NaN."""
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue
            mag = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
            vals.append((mag, m))
    return vals


def brute_e4m3(x):
    """Nearest finite E4M3 value, ties to the even fraction, saturating at 448."""
    a = abs(x)
    if a >= 448.0:
        return np.copysign(448.0, x)
    best = None
    for mag, m in e4m3_values():
        d = abs(mag - a)
        if best is None or d < best[0] or (d == best[0] and m % 2 == 0 and best[2] % 2 == 1):
            best = (d, mag, m)
    return np.copysign(best[1], x)


def test_e4m3_table_shape():
    vals = sorted(v for v, _ in e4m3_values())
    assert len(vals) == 127 and vals[0] == 0.0 and vals[1] == 2.0 ** -9 and vals[-1] == 448.0


def test_e4m3_matches_brute_force_and_torch(orc):
    rng = np.random.default_rng(3)
    mags = np.exp(rng.uniform(np.log(2.0 ** -12), np.log(440.0), 4000))
    x = mags * rng.choice([-1.0, 1.0], mags.size)
    # exact midpoints between neighbouring codes exercise ties-to-even
    vals = sorted(v for v, _ in e4m3_values())
    mids = np.array([(a + b) / 2 for a, b in zip(vals[:-1], vals[1:])])
    x = np.concatenate([x, mids, -mids[::7], np.array(vals), [0.0, 2.0 ** -10, 2.0 ** -10 * 3]])
    got = orc.e4m3_rn(x)
    ref_torch = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, ref_torch)
    sample = x[:: max(1, x.size // 600)]
    np.testing.assert_array_equal(orc.e4m3_rn(sample), np.array([brute_e4m3(v) for v in sample]))


def test_e4m3_saturates(orc):
    np.testing.assert_array_equal(orc.e4m3_rn(np.array([448.0, 460.0, 470.0, 1e6, -1e9])),
                                  [448.0, 448.0, 448.0, 448.0, -448.0])


def test_round_f16_matches_numpy(orc):
    rng = np.random.default_rng(4)
    x = np.exp(rng.uniform(np.log(1e-8), np.log(6e4), 3000)) * rng.choice([-1.0, 1.0], 3000)
    h = np.float16(1.0)
    ties = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 2.0 ** -24 * 1.5, 2.0 ** -24 * 2.5])
    x = np.concatenate([x, ties, -ties])
    np.testing.assert_array_equal(orc.round_f16(x), x.astype(np.float16).astype(np.float64))
    assert h == 1.0


def test_q8_tensor_scale_and_range(orc):
    rng = np.random.default_rng(5)
    x = np.float16(rng.normal(size=(4, 8, 8)) * 3).astype(np.float64)
    codes, deq = orc.q8_tensor(x)
    amax = np.abs(x).max()
    k = np.log2(deq)
    assert k == np.round(k)                               # a power of two ...
    assert 224.0 < amax / deq <= 448.0                    # ... the smallest with amax <= 448 s
    np.testing.assert_array_equal(codes, orc.e4m3_rn(x / deq))
    big = np.abs(x) > 2.0 ** -6 * deq * 8
    rel = np.abs(codes * deq - x)[big] / np.abs(x)[big]
    assert rel.max() <= 2.0 ** -4 * 1.0001
    zc, zd = orc.q8_tensor(np.zeros(5))
    assert np.all(zc == 0) and zd == 1.0


def test_q8_weights_per_channel(orc):
    rng = np.random.default_rng(6)
    w = rng.normal(size=(6, 5, 3, 3))
    w[2] = 0.0
    codes, s = orc.q8_weights(w.reshape(-1), 6, 45, 45, 1)
    codes = codes.reshape(w.shape)
    for co in range(6):
        if co == 2:
            assert s[co] == 1.0 and np.all(codes[co] == 0)
        else:
            assert np.abs(codes[co]).max() == 448.0
            assert s[co] == np.float32(np.float32(np.abs(w[co]).max()) / np.float32(448.0))


def _q8_torch(x):
    """Activation quantisation with PyTorch ops: power-of-two scale s (the
    smallest with amax <= 448 s, found by search), float8 cast of x / s."""
    a = float(x.abs().max())
    s = 1.0
    if a > 0:
        k = -200
        while a > 448.0 * 2.0 ** k:
            k += 1
        s = 2.0 ** k
    codes = (x / s).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64)
    return codes, torch.tensor(s, dtype=torch.float64)


def _w8_torch(w, dims):
    wf = w.to(torch.float32)
    amax = wf.abs().amax(dim=dims, keepdim=True)
    s = torch.where(amax > 0, amax / torch.tensor(448.0, dtype=torch.float32), torch.ones_like(amax))
    return (wf / s).to(torch.float8_e4m3fn).to(torch.float64), s.to(torch.float64)


def torch_q8_forward(guide, params, c0, depth_scale):
    P = {k: T(v) for k, v in params}
    x = T(guide).clone()[None]
    x[:, 2] *= depth_scale
    f16 = lambda v: v.to(torch.float16).to(torch.float64)

    def c3(v, name):
        xq, deq = _q8_torch(v)
        wq, s = _w8_torch(P[name + ".w"], (1, 2, 3))
        acc = Fn.conv2d(xq, wq, None, padding=1)
        return f16(torch.relu(acc * (deq * s.view(1, -1, 1, 1)) + P[name + ".b"].view(1, -1, 1, 1)))

    def up(v, name):
        xq, deq = _q8_torch(v)
        w = P[name + ".w"]                                  # [cin][cout][2][2]
        wq, s = _w8_torch(w, (0, 2, 3))
        acc = Fn.conv_transpose2d(xq, wq, None, stride=2)
        return f16(acc * (deq * s.view(1, -1, 1, 1)) + P[name + ".b"].view(1, -1, 1, 1))

    a0 = f16(torch.relu(Fn.conv2d(x, P["enc1a.w"], P["enc1a.b"], padding=1)))
    s1 = c3(a0, "enc1b")
    s2 = c3(c3(Fn.max_pool2d(s1, 2), "enc2a"), "enc2b")
    s3 = c3(c3(Fn.max_pool2d(s2, 2), "enc3a"), "enc3b")
    b = c3(c3(Fn.max_pool2d(s3, 2), "enc4a"), "enc4b")
    d = c3(c3(torch.cat([up(b, "up3"), s3], 1), "dec3a"), "dec3b")
    d = c3(c3(torch.cat([up(d, "up2"), s2], 1), "dec2a"), "dec2b")
    F = c3(c3(torch.cat([up(d, "up1"), s1], 1), "dec1a"), "dec1b")
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


@pytest.mark.parametrize("c0,H,W", [(8, 16, 24), (16, 24, 16)])
def test_net_forward_q8_matches_torch_assembly(orc, c0, H, W):
    params = I.make_params(c0, seed=0)
    flat = I.flat_params(params).astype(np.float64)
    rng = np.random.default_rng(10)
    guide = np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 60, (H, W))])
    got = orc.net_forward_q8(guide, flat, c0, 1 / 50.0)
    ref = torch_q8_forward(guide, params, c0, 1 / 50.0)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9)
    # the quantised network stays within the output range of the FP64 one
    full = orc.net_forward(guide, flat, c0, 1 / 50.0)
    assert np.abs(got - full).max() <= np.abs(full).max()
