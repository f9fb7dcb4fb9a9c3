"""Pins of the FP64 oracle's six-way shading (Sec. 3, directional interpolation)
and of the fine-step six-light reference renderer (Sec. 3, Eq. RE / Eq. scatter
in the single-scattering limit).  CPU only."""
import math

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I

FOUR_PI = 4 * math.pi


def _cam(W=8, H=6):
    return I.Camera(I.ORTHO, (4.0, 4.0, 30.0), (4.0, 4.0, 0.0), (0.0, 1.0, 0.0), 40.0, 8.0, W, H)


def _planes(H=6, W=8, seed=0):
    rng = np.random.default_rng(seed)
    lm = rng.uniform(0, 1, size=(8, H, W))
    return lm


@pytest.mark.parametrize("axis,sign,plane", [
    ((1, 0, 0), 1, 0), ((1, 0, 0), -1, 1),   # camera right is world +x here
    ((0, 1, 0), 1, 2), ((0, 1, 0), -1, 3),   # up
    ((0, 0, 1), -1, 4), ((0, 0, 1), 1, 5),   # camera looks along -z: behind the smoke is -z
])
def test_axis_light_selects_one_plane(orc, axis, sign, plane):
    lm = _planes()
    li = I.Light(tuple(sign * a for a in axis), (0.5, 1.0, 2.0))
    out = orc.shade(lm, _cam(), [li])
    for c, inten in enumerate(li.intensity):
        np.testing.assert_allclose(out[c], inten * lm[plane] + lm[7], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(out[3], np.clip(1 - lm[6], 0, 1))


def test_shade_linear_in_lights_and_planes(orc):
    lm1, lm2 = _planes(seed=1), _planes(seed=2)
    l1 = I.Light(tuple(np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])), (1.0, 0.7, 0.2))
    l2 = I.Light(tuple(np.array([-0.9, 0.1, 0.2]) / np.linalg.norm([-0.9, 0.1, 0.2])), (0.1, 0.4, 0.9))
    both = orc.shade(lm1, _cam(), [l1, l2])
    a = orc.shade(lm1, _cam(), [l1])
    b = orc.shade(lm1, _cam(), [l2])
    np.testing.assert_allclose(both[:3], a[:3] + b[:3] - lm1[7][None], rtol=1e-13, atol=1e-14)
    s12 = orc.shade(lm1 + lm2, _cam(), [l1])
    s1, s2 = orc.shade(lm1, _cam(), [l1]), orc.shade(lm2, _cam(), [l1])
    np.testing.assert_allclose(s12[:3], s1[:3] + s2[:3], rtol=1e-13, atol=1e-14)


def test_shade_diagonal_weights(orc):
    """|w_p| weights: a light along (1,1,1)/sqrt3 weighs +X, +Y and the plane of
    the z sign each by 1/sqrt3 (literal weights, no renormalisation)."""
    lm = _planes(seed=3)
    v = np.array([1.0, 1.0, 1.0]) / math.sqrt(3)
    out = orc.shade(lm, _cam(), [I.Light(tuple(v), (1.0, 1.0, 1.0))])
    exp = (lm[0] + lm[2] + lm[5]) / math.sqrt(3) + lm[7]
    np.testing.assert_allclose(out[0], exp, rtol=1e-13)


def test_alpha_clamped(orc):
    lm = np.zeros((8, 2, 2))
    lm[6] = [[-0.5, 0.3], [1.0, 2.0]]
    out = orc.shade(lm, _cam(2, 2), [])
    np.testing.assert_allclose(out[3], [[1.0, 0.7], [0.0, 0.0]])


def test_reference_slab_closed_form(orc):
    """Constant cube, orthographic camera along -z.  With the midpoint partition
    the front-lit plane (-Z) is exactly P sum_m e^{-s(m-1)h}(1-e^{-sh}) e^{-s(m-1/2)h},
    and tends to P(1 - e^{-2 s L})/2 with O(h^2) error; the back-lit plane (+Z)
    tends to P s L e^{-s L}."""
    n, sig = 16, 0.1
    vol = np.full((n, n, n), sig, np.float32)
    cam = I.Camera(I.ORTHO, (8.0, 8.0, 30.0), (8.0, 8.0, 0.0), (0.0, 1.0, 0.0), 40.0, 16.0, 4, 4)
    s = float(np.float32(sig))
    P = 1 / FOUR_PI
    errs = []
    for hf in (0.5, 0.25):
        ref = orc.reference_lightmaps(vol, None, cam, hf=hf)
        M = int(round(n / hf))
        disc = P * sum(math.exp(-s * (m - 1) * hf) * (1 - math.exp(-s * hf)) * math.exp(-s * (m - 0.5) * hf)
                       for m in range(1, M + 1))
        np.testing.assert_allclose(ref[5], disc, rtol=1e-9)
        np.testing.assert_allclose(ref[6], math.exp(-s * n), rtol=1e-9)
        errs.append(abs(ref[5].mean() - P * (1 - math.exp(-2 * s * n)) / 2))
        np.testing.assert_allclose(ref[4], P * s * n * math.exp(-s * n), rtol=5e-3)
    assert errs[1] < errs[0] / 3.5   # second order
    # side lights: by symmetry +X = -X and +Y = -Y on the centre pixels
    ref = orc.reference_lightmaps(vol, None, cam, hf=0.5)
    np.testing.assert_allclose(ref[0, 1:3, 1:3], ref[1, 1:3, 2:0:-1], rtol=1e-9)


def test_reference_guide_agree_on_transmittance(orc):
    """The guide's T channel (a first-order Riemann sum) converges to the
    reference's midpoint T as h -> 0."""
    vol = I.blob_fbm_volume(16, 9)
    cam = I.orbit_ortho_camera(16, 9, 8, 8)
    ref = orc.reference_lightmaps(vol, None, cam, hf=0.0625)
    errs = []
    for h in (0.5, 0.25, 0.125):
        g, _, _ = orc.guide(vol, None, cam, h, jitter=0, t_min=0.0)
        errs.append(np.abs(g[1] - ref[6]).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-3
