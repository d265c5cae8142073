"""GPU training-profile generator vs the same light curves regenerated on the CPU
(lcsynth, an independent Philox4x32-10) and folded by the FP64 oracle."""
import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def test_generated_profiles_match_oracle_fold():
    import paper_2312_02063_gb300 as g
    ctx = g.Context(0)
    seed = 12345
    sp = dict(lcsynth.TRAINING_SET, n_cadences=6000)  # ragged: not a multiple of the warp's 128
    js = list(range(8)) + [1001, 70000]
    for j in js:
        f, c, y, per, sd = g.gpfc_synth_profiles(ctx, seed, j, 1, 256, sp, want_period=True, want_std=True)
        ctx.sync()
        t, flux, lab, P = lcsynth.training_light_curve(seed, j, sp)
        assert float(per.item()) == P
        assert float(y.item()) == lab
        mean_o, cnt_o, _ = oracle.fold(t, flux.astype(np.float32), np.array([P]), 256, 0.0)
        np.testing.assert_array_equal(c.cpu().numpy()[0], cnt_o[0])
        fo = f.cpu().numpy()[0].astype(np.float64)
        nz = cnt_o[0] > 0
        assert np.max(np.abs(fo[nz] - mean_o[0][nz]) / mean_o[0][nz]) <= 1e-6
        assert abs(float(sd.item()) - np.std(flux)) <= 1e-5 * np.std(flux)
    ctx.close()


def test_paper_recipe_vectors_match_the_reference_generator(ctx):
    """gpfc_synth_vectors against lcsynth.paper_vector (the same Philox draws evaluated in
    FP64 on the CPU): values within FP32 rounding of the noise, labels, alpha and the
    per-bin noise exact to FP32."""
    import paper_2312_02063_gb300 as g
    seed, first, n = 4242, 1000, 64
    f, lab, al, sb = g.gpfc_synth_vectors(ctx, seed, first, n)
    ctx.sync()
    f, lab, al, sb = (x.cpu().numpy() for x in (f, lab, al, sb))
    for i in range(0, n, 3):
        v, l, a, s = lcsynth.paper_vector(seed, first + i)
        assert lab[i] == l
        assert abs(al[i] - a) <= 1e-6 * max(1.0, a)
        assert abs(sb[i] - s) <= 1e-6 * s
        np.testing.assert_allclose(f[i].astype(np.float64), v, rtol=0, atol=2e-7)
    # label balance and the negatives' split
    assert lab[0::2].min() == 1.0 and lab[1::2].max() == 0.0
    assert np.all(al[1::4] == 0.0) and np.all(al[3::4] < 5.0)
