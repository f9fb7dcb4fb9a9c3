"""The stored expected values under tests/golden/ (written by
tests/golden/make_golden.py from the oracle alone) against the oracle as it
stands: a change of the oracle's arithmetic shows here and must come with
regenerated fixtures.  CPU only."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden as G  # noqa: E402


def _close(got, want):
    got = np.asarray(got, np.float64)
    scale = max(np.abs(want).max(), 1e-30)
    assert np.abs(got - want).max() <= 1e-12 * scale, np.abs(got - want).max() / scale


def test_golden_fixtures_match_the_oracle(orc):
    r = G.compute(orc)
    g = G.load("guide_small12_persp8.json")
    _close(r["guide"], g["array"])
    assert [int(v) for v in r["flags"].reshape(-1)] == g["flags"]
    assert int(r["samples"].sum()) == g["samples_total"]
    _close(r["lightmaps"], G.load("lightmaps_small12_persp8.json")["array"])
    _close(r["rgba"], G.load("shade_small12_persp8.json")["array"])


def test_golden_fixtures_are_cited_and_nontrivial():
    for name in ("guide_small12_persp8.json", "lightmaps_small12_persp8.json", "shade_small12_persp8.json"):
        obj = G.load(name)
        assert obj["cite"].startswith("Sec.")
        assert obj["array"].shape == tuple(obj["shape"]) and np.isfinite(obj["array"]).all()
    g = G.load("guide_small12_persp8.json")["array"]
    assert g[0].max() > 0 and 0 < g[1].min() < 1 and g[2].max() > 0   # scattering, T, depth all in play
