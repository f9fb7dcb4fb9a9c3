"""Pins of the oracle's per-layer precision forms of the network
(nslo_net_forward_prec; the precision forms have no counterpart in the paper).
bfloat16 rounding is checked against PyTorch's bfloat16 casts (binary32 inputs,
one rounding) and against round-to-nearest-even on the binary64 bit pattern;
each form of the network against an assembly of PyTorch float64 library ops
that rounds with those independent helpers; the all-FP64 and all-FP8 forms
against the oracle's plain and FP8 forwards.  CPU only."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

from paper_2604_03748_gb300 import inputs as I
from test_oracle_net import T, _torch_nafblock


def bf16_bits(x):
    """Round binary64 values in the bfloat16 normal range to bfloat16 by
    round-to-nearest-even on the bit pattern: keep sign, 11 exponent bits and
    the top 7 of 52 fraction bits; the 45 dropped bits decide the rounding."""
    x = np.asarray(x, np.float64)
    u = x.view(np.uint64).copy()
    drop = np.uint64(45)
    low = u & np.uint64((1 << 45) - 1)
    half = np.uint64(1 << 44)
    keep = u >> drop
    up = (low > half) | ((low == half) & ((keep & np.uint64(1)) == np.uint64(1)))
    keep = keep + up.astype(np.uint64)
    return (keep << drop).view(np.float64)


def test_round_bf16_matches_torch_casts(orc):
    rng = np.random.default_rng(21)
    x = (np.exp(rng.uniform(np.log(1e-38), np.log(3e38), 4000)) * rng.choice([-1.0, 1.0], 4000))
    x = x.astype(np.float32).astype(np.float64)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0 + 2.0 ** -7, 2.0 ** -130 * 1.5, 2.0 ** -133 * 2.5,
                     2.0 ** -127, 2.0 ** -133, 2.0 ** -134 * 1.5])
    big = np.array([np.float32(3.3895e38), np.float32(3.39e38), float(np.finfo(np.float32).max)])
    x = np.concatenate([x, ties, -ties, big, [0.0, -0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(orc.round_bf16(x), ref)


def test_round_bf16_on_binary64_inputs(orc):
    """Binary64 inputs (no prior rounding to binary32), ties included."""
    rng = np.random.default_rng(22)
    x = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 4000)) * rng.choice([-1.0, 1.0], 4000)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -40, 1.0 + 3 * 2.0 ** -8 - 2.0 ** -45, 7.0 + 2.0 ** -6])
    x = np.concatenate([x, ties, -ties])
    np.testing.assert_array_equal(orc.round_bf16(x), bf16_bits(x))
    # relative error at most the unit roundoff 2^-8 of 8 significand bits
    r = orc.round_bf16(x)
    assert (np.abs(r - x) / np.abs(x)).max() <= 2.0 ** -8


def _rnd(kind, v):
    if kind == "bf16":
        return T(bf16_bits(v.numpy()))
    if kind == "f16":
        return T(v.numpy().astype(np.float16).astype(np.float64))
    if kind == "f32":
        return T(v.numpy().astype(np.float32).astype(np.float64))
    return v


def torch_prec_forward(guide, params, c0, depth_scale, kind):
    """The network with every convolution after the first in form `kind`
    (bf16, f16, or bf16x3: hi/lo bfloat16 splits, hi*hi + hi*lo + lo*hi, binary32
    storage), assembled from PyTorch float64 ops and the helpers above."""
    P = {k: T(v) for k, v in params}
    x = T(guide).clone()[None]
    x[:, 2] *= depth_scale
    store = {"bf16": "bf16", "f16": "f16", "bf16x3": "f32"}[kind]

    def mm(v, w, op):
        if kind == "bf16x3":
            vh = _rnd("bf16", v)
            vl = _rnd("bf16", v - vh)
            wh = _rnd("bf16", w)
            wl = _rnd("bf16", w - wh)
            return op(vh, wh) + op(vh, wl) + op(vl, wh)
        return op(_rnd(kind, v), _rnd(kind, w))

    def c3(v, name):
        acc = mm(v, P[name + ".w"], lambda a, b: Fn.conv2d(a, b, None, padding=1))
        return _rnd(store, torch.relu(acc + P[name + ".b"].view(1, -1, 1, 1)))

    def up(v, name):
        acc = mm(v, P[name + ".w"], lambda a, b: Fn.conv_transpose2d(a, b, None, stride=2))
        return _rnd(store, acc + P[name + ".b"].view(1, -1, 1, 1))

    a0 = _rnd(store, torch.relu(Fn.conv2d(x, P["enc1a.w"], P["enc1a.b"], padding=1)))
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
    return out.numpy(), F[0].numpy()


def _case(c0, H, W, seed):
    params = I.make_params(c0, seed=0)
    flat = I.flat_params(params).astype(np.float64)
    rng = np.random.default_rng(seed)
    guide = np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 60, (H, W))])
    return params, flat, guide


@pytest.mark.parametrize("kind,code", [("bf16", 2), ("f16", 1), ("bf16x3", 4)])
@pytest.mark.parametrize("c0,H,W", [(8, 16, 24), (16, 24, 16)])
def test_prec_forms_match_torch_assembly(orc, kind, code, c0, H, W):
    params, flat, guide = _case(c0, H, W, 30)
    got, layers = orc.net_forward_prec(guide, flat, c0, 1 / 50.0, code, trace=True)
    ref, F = torch_prec_forward(guide, params, c0, 1 / 50.0, kind)
    np.testing.assert_allclose(layers[16], F, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9)


def test_prec_f64_is_the_plain_forward(orc):
    params, flat, guide = _case(8, 24, 16, 31)
    got = orc.net_forward_prec(guide, flat, 8, 1 / 40.0, orc.PREC_F64)
    np.testing.assert_array_equal(got, orc.net_forward(guide, flat, 8, 1 / 40.0))


def test_prec_fp8_is_the_fp8_forward(orc):
    params, flat, guide = _case(8, 16, 16, 32)
    got = orc.net_forward_prec(guide, flat, 8, 1 / 40.0, orc.PREC_FP8)
    np.testing.assert_array_equal(got, orc.net_forward_q8(guide, flat, 8, 1 / 40.0))


def test_prec_trace_shapes_and_stored_types(orc):
    """The trace holds each layer's stored output: bfloat16 values for the BF16
    form, and the first stored tensor is the ReLU of the exact first convolution."""
    params, flat, guide = _case(8, 16, 24, 33)
    _, layers = orc.net_forward_prec(guide, flat, 8, 1 / 40.0, orc.PREC_BF16, trace=True)
    shapes = [l.shape for l in layers]
    assert shapes[0] == (8, 16, 24) and shapes[7] == (64, 2, 3) and shapes[8] == (32, 4, 6)
    assert shapes[14] == (8, 16, 24) and shapes[16] == (8, 16, 24)
    for l in layers:
        np.testing.assert_array_equal(l, bf16_bits(l))
    x = guide.copy()
    x[2] /= 40.0
    P = dict(params)
    a0 = orc.conv2d(x, P["enc1a.w"].astype(np.float64), P["enc1a.b"].astype(np.float64), 3)
    np.testing.assert_array_equal(layers[0], bf16_bits(np.maximum(a0, 0.0)))


def test_prec_mixed_layers_change_only_their_own_rounding(orc):
    """A form with only layer l in BF16 equals FP64 up to layer l - 1 and
    rounds layer l's output to bfloat16."""
    params, flat, guide = _case(8, 16, 16, 34)
    _, ref = orc.net_forward_prec(guide, flat, 8, 1 / 40.0, orc.PREC_F64, trace=True)
    for l in (3, 8, 16):
        codes = [orc.PREC_F64] * 17
        codes[l] = orc.PREC_BF16
        _, got = orc.net_forward_prec(guide, flat, 8, 1 / 40.0, codes, trace=True)
        for j in range(l):
            np.testing.assert_array_equal(got[j], ref[j])
        np.testing.assert_array_equal(got[l], bf16_bits(got[l]))
        assert np.abs(got[l] - ref[l]).max() <= 2.0 ** -8 * np.abs(ref[l]).max()


def test_layer_and_adapter_pieces_recompose_the_network(orc):
    """Running each convolution alone (nslo_conv_layer_prec) on the previous
    stored outputs, and the adapters alone on the stored feature map, gives the
    whole network's trace and output again."""
    c0, H, W = 8, 16, 24
    params, flat, guide = _case(c0, H, W, 35)
    P = {k: v.astype(np.float64) for k, v in params}
    ds = 1 / 40.0
    for code in (orc.PREC_BF16, orc.PREC_FP8, orc.PREC_F16):
        out, L = orc.net_forward_prec(guide, flat, c0, ds, code, trace=True)
        x0 = guide.copy()
        x0[2] *= ds
        a0 = orc.store_as(code, orc.conv_layer_prec(orc.PREC_F64, x0, P["enc1a.w"], P["enc1a.b"]))
        np.testing.assert_array_equal(a0, L[0])
        pool = orc.maxpool2
        ins = {1: L[0], 2: pool(L[1]), 3: L[2], 4: pool(L[3]), 5: L[4], 6: pool(L[5]), 7: L[6], 8: L[7],
               9: np.concatenate([L[8], L[5]]), 10: L[9], 11: L[10], 12: np.concatenate([L[11], L[3]]),
               13: L[12], 14: L[13], 15: np.concatenate([L[14], L[1]]), 16: L[15]}
        for l in range(1, 17):
            name = orc.NET_LAYERS[l]
            got = orc.conv_layer_prec(code, ins[l], P[name + ".w"], P[name + ".b"], transposed=name.startswith("up"))
            np.testing.assert_array_equal(got, L[l])
        n_ad = 4 * (orc.nafblock_params(c0) + 2 * c0 + 2)
        np.testing.assert_array_equal(orc.net_adapters(L[16], flat[-n_ad:], c0), out)
