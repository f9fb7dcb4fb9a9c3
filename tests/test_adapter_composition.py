"""The identity the tensor-core adapters' first pass is built on (Sec. 4.3,
Fig. 3: a NAFBlock's 1x1 convolution pw1 followed by its depthwise 3x3).

Both maps are linear and the depthwise convolution pads its input, pw1's output,
with zeros, so the pair equals one 3x3 convolution of the normalised input with
weights dw[o, tap] * W1[o, c] and zero padding, plus the per-pixel bias
dw_b[o] + b1[o] * (sum of dw[o, tap] over the taps that fall inside the image).
That bias depends only on which of a pixel's left, right, upper and lower
neighbours are missing: 16 cases.  Checked in binary64 against the oracle's own
pw1 and depthwise operators (the ones its NAFBlock uses), on images with
interior pixels, one-pixel-wide and one-pixel-tall images and a single pixel."""
import numpy as np
import pytest


def _edge_case(px, py, W, H):
    return (px < 1) | ((px + 1 >= W) << 1) | ((py < 1) << 2) | ((py + 1 >= H) << 3)


def _bias_table(dw, dwb, b1):
    tab = np.zeros((16, dw.shape[0]))
    for e in range(16):
        inside = np.ones((3, 3), bool)
        if e & 1:
            inside[:, 0] = False
        if e & 2:
            inside[:, 2] = False
        if e & 4:
            inside[0, :] = False
        if e & 8:
            inside[2, :] = False
        tab[e] = dwb + b1 * (dw * inside.reshape(1, 9)).sum(axis=1)
    return tab


@pytest.mark.parametrize("H,W", [(9, 14), (1, 6), (5, 1), (1, 1), (2, 2)])
def test_pw1_then_depthwise_equals_one_3x3_convolution(orc, H, W):
    rng = np.random.default_rng(H * 31 + W)
    cin, cout = 16, 32
    x = rng.standard_normal((cin, H, W))
    W1 = rng.standard_normal((cout, cin))
    b1 = rng.uniform(-1, 1, cout)
    dw = rng.standard_normal((cout, 9))
    dwb = rng.uniform(-1, 1, cout)
    ref = orc.dwconv3(orc.conv2d(x, W1.reshape(cout, cin, 1, 1), b1, 1), dw, dwb)

    comp = (dw[:, None, :] * W1[:, :, None]).reshape(cout, cin, 3, 3)   # [o][c][dy][dx]
    got = orc.conv2d(x, comp, None, 3)
    tab = _bias_table(dw, dwb, b1)
    for py in range(H):
        for px in range(W):
            got[:, py, px] += tab[_edge_case(px, py, W, H)]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-11)


def test_bias_table_interior_row_is_the_full_tap_sum():
    rng = np.random.default_rng(5)
    dw, dwb, b1 = rng.standard_normal((8, 9)), rng.standard_normal(8), rng.standard_normal(8)
    tab = _bias_table(dw, dwb, b1)
    np.testing.assert_allclose(tab[0], dwb + b1 * dw.sum(axis=1), rtol=0, atol=1e-14)
    # a pixel with no neighbour on any side keeps only the centre tap
    np.testing.assert_allclose(tab[15], dwb + b1 * dw[:, 4], rtol=0, atol=1e-14)
