"""CPU checks of the seeded generators shared by the oracle side and the GPU path."""
import json
import os

import numpy as np

import lcsynth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_philox_known_answers():
    for v in json.load(open(GOLDEN))["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert list(lcsynth.philox4x32_10(ctr, key)) == out


def test_training_light_curve_recipe():
    sp = dict(lcsynth.TRAINING_SET, n_cadences=4096)
    for j in range(8):
        t, f, lab, P = lcsynth.training_light_curve(7, j, sp)
        assert t.shape == f.shape == (4096,)
        assert lab == float(j % 2 == 0)
        assert 0.2 <= P <= 1.0 + 1e-3
        z = (f - 1.0)
        assert np.all(np.abs(z) < 0.05)
    # noise-only light curve: the Box-Muller normals have unit variance
    t, f, lab, P = lcsynth.training_light_curve(7, 1, dict(lcsynth.TRAINING_SET, n_cadences=8192, sigma_min=1e-3,
                                                           sigma_max=1e-3))
    assert 0.95 < np.std(f) / 1e-3 < 1.05
