"""Pins of the oracle's training-loss gradient (oracle/grad.py): its loss equals
the mean squared error of the C oracle's network (nslo_net_forward), and its
gradient equals central finite differences of that C oracle loss on
parameters of every kind (3x3 and transposed convolutions, LayerNorm affines,
1x1 and depthwise convolutions, the channel attention, the residual scales
beta and gamma, the heads).  CPU only."""
import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I


def _case(B=2, H=16, W=16, seed=40):
    params = I.make_params(16, seed=0)
    flat = I.flat_params(params).astype(np.float64)
    rng = np.random.default_rng(seed)
    guides = np.stack([np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 60, (H, W))])
                       for _ in range(B)])
    targets = rng.uniform(0, 0.1, (B, 8, H, W))
    return params, flat, guides, targets


def _c_loss(orc, flat, guides, targets, ds):
    outs = np.stack([orc.net_forward(g, flat, 16, ds) for g in guides])
    return float(((outs - targets) ** 2).mean())


def test_loss_equals_c_oracle(orc):
    from oracle import grad as OG
    _, flat, guides, targets = _case()
    loss, g, out = OG.mse_and_grad(flat, guides, targets, 16, 1 / 40.0)
    np.testing.assert_allclose(out, np.stack([orc.net_forward(x, flat, 16, 1 / 40.0) for x in guides]),
                               rtol=1e-10, atol=1e-12)
    assert loss == pytest.approx(_c_loss(orc, flat, guides, targets, 1 / 40.0), rel=1e-12)
    assert g.shape == flat.shape and np.abs(g).max() > 0


def _offsets():
    """(name, first flat index) of every parameter tensor, in blob order."""
    off, out = 0, []
    for name, shape, _ in I.param_spec(16):
        out.append((name, off, int(np.prod(shape))))
        off += int(np.prod(shape))
    return out


@pytest.mark.parametrize("names", [("enc1a.w", "enc2b.b", "enc4b.w", "up3.w", "up1.b", "dec1b.w"),
                                   ("adFB.ln1.w", "adLR.pw1.w", "adUD.dw.w", "adAE.sca.w", "adFB.pw2.b",
                                    "adLR.beta", "adUD.ln2.b", "adAE.ffn1.w", "adFB.ffn2.w", "adLR.gamma",
                                    "adUD.head.w", "adAE.head.b")])
def test_gradient_equals_central_differences(orc, names):
    from oracle import grad as OG
    _, flat, guides, targets = _case()
    ds = 1 / 40.0
    _, g, _ = OG.mse_and_grad(flat, guides, targets, 16, ds)
    table = {n: (o, k) for n, o, k in _offsets()}
    rng = np.random.default_rng(41)
    for name in names:
        o, k = table[name]
        idx = o + int(rng.integers(0, k))
        h = 1e-5 * max(1.0, abs(flat[idx]))
        fp, fm = flat.copy(), flat.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = (_c_loss(orc, fp, guides, targets, ds) - _c_loss(orc, fm, guides, targets, ds)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-5 * max(abs(g[idx]), 1e-4 * np.abs(g).max()), (name, fd, g[idx])


def test_plane_weights_scale_each_planes_term(orc):
    """With one plane weighted w and the others 0, the loss is w times that
    plane's share of the plain mean squared error."""
    from oracle import grad as OG
    _, flat, guides, targets = _case(B=1, H=16, W=16, seed=42)
    outs = np.stack([orc.net_forward(x, flat, 16, 1 / 40.0) for x in guides])
    for p in (0, 6):
        w = np.zeros(8)
        w[p] = 2.5
        loss, _, _ = OG.mse_and_grad(flat, guides, targets, 16, 1 / 40.0, plane_weight=w)
        share = float(((outs[:, p] - targets[:, p]) ** 2).sum() / outs.size)
        assert loss == pytest.approx(2.5 * share, rel=1e-10)
