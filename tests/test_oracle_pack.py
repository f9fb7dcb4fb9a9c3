"""Pins of the oracle's packed two-texture export (Sec. 3, Fig. 2).  CPU only."""
import numpy as np
import pytest

TEX_RGBA8, TEX_RGBA16F, TEX_RGBA32F = 0, 1, 2


def test_fig2_layout_on_exact_fractions(orc):
    """Plane q holds q/8 (exact in binary): texture 1 carries planes +X, +Y, +Z,
    T = (0, 2/8, 4/8, 6/8) and texture 2 planes -X, -Y, -Z, E = (1/8, 3/8,
    5/8, 7/8) (Fig. 2: right/top/back/transparency and left/bottom/front/
    emissive).  UNORM codes of q/8 * 255: 0, 31.875 -> 32, 63.75 -> 64,
    95.625 -> 96, 127.5 -> 128 (tie to even), 159.375 -> 159, 191.25 -> 191,
    223.125 -> 223."""
    lm = np.stack([np.full((2, 3), q / 8.0, np.float32) for q in range(8)])
    t1, t2 = orc.pack_lightmaps(lm, TEX_RGBA8)
    assert t1.shape == (2, 3, 4) and t1.dtype == np.uint8
    assert np.all(t1 == np.array([0, 64, 128, 191], np.uint8))
    assert np.all(t2 == np.array([32, 96, 159, 223], np.uint8))
    f1, f2 = orc.pack_lightmaps(lm, TEX_RGBA32F)
    assert np.all(f1 == np.array([0, 2, 4, 6], np.float32) / 8)
    assert np.all(f2 == np.array([1, 3, 5, 7], np.float32) / 8)


def test_unorm_ties_clamps_and_nan(orc):
    # clamps at both ends, NaN to 0, and exact products: 0.5 * 255 = 127.5 is a
    # tie (to even: 128), 0.25 * 255 = 63.75 rounds up
    vals = np.array([-0.5, -0.0, 0.0, 1.0, 1.7, np.inf, -np.inf, np.nan, 0.5, 0.25], np.float32)
    codes = [0, 0, 0, 255, 255, 255, 0, 0, 128, 64]   # 127.5 -> 128, 63.75 -> 64
    lm = np.zeros((8, 1, vals.size), np.float32)
    lm[0, 0] = vals
    t1, _ = orc.pack_lightmaps(lm, TEX_RGBA8)
    assert list(t1[0, :, 0]) == codes


@pytest.mark.parametrize("fmt", [TEX_RGBA16F, TEX_RGBA32F])
def test_float_formats(orc, fmt):
    rng = np.random.default_rng(2)
    lm = (rng.normal(size=(8, 5, 7)) * 3).astype(np.float32)
    t1, t2 = orc.pack_lightmaps(lm, fmt)
    dt = np.float16 if fmt == TEX_RGBA16F else np.float32
    for c, q in enumerate((0, 2, 4, 6)):
        np.testing.assert_array_equal(t1[..., c], lm[q].astype(dt))
    for c, q in enumerate((1, 3, 5, 7)):
        np.testing.assert_array_equal(t2[..., c], lm[q].astype(dt))
