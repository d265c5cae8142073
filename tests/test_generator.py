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


def test_paper_vector_recipe():
    """The paper-recipe vectors (Sec. 2.6-2.7): labels by index, alpha ranges, and the
    injected trapezoid: its depth satisfies Eq. 2 with the per-bin noise, its width at half
    depth is q of the phase (to one bin), and what is left after removing it is noise of
    the stated per-bin sigma."""
    nb, seed = 256, 7
    pv = lcsynth.PAPER_VECTORS
    for j in range(12):
        v, label, alpha, sb = lcsynth.paper_vector(99, j, nb)
        assert label == (1.0 if j % 2 == 0 else 0.0)
        if j % 2 == 0:
            assert pv["alpha_pos_min"] <= alpha <= pv["alpha_pos_max"]
        elif (j // 2) % 2 == 0:
            assert alpha == 0.0
        else:
            assert 0.0 <= alpha < pv["alpha_neg_max"]
    x = (np.arange(nb) + 0.5) / nb
    for j in (0, 2, 4, 6):
        v, _, alpha, sb = lcsynth.paper_vector(seed, j, nb)
        a = lcsynth.philox4x32_10((j, 0, 2, 0xFFFFFFFF), (seed, 0))
        b = lcsynth.philox4x32_10((j, 1, 2, 0xFFFFFFFF), (seed, 0))
        sigma = sb / np.sqrt(nb / pv["n_points"])
        q = pv["q_min"] + lcsynth._u64(a[2]) * (pv["q_max"] - pv["q_min"])
        r = lcsynth._u64(a[3])
        phi0 = lcsynth._u64(b[0])
        d = alpha * sigma / np.sqrt(pv["n_points"] * q)
        # Eq. 2 over the vector: alpha = d / sigma_bin * sqrt(nbins * q)
        assert abs(d / sb * np.sqrt(nb * q) - alpha) <= 1e-12 * alpha
        dphi = np.abs((x - phi0) - np.floor(x - phi0 + 0.5))
        t14 = 2 * q / (1 + r)
        t23 = r * t14
        shape = np.where(dphi <= t23 / 2, 1.0, np.where(dphi < t14 / 2, (t14 / 2 - dphi) / ((t14 - t23) / 2), 0.0))
        assert abs(np.sum(shape >= 0.5) / nb - q) <= 1.0 / nb + 1e-12
        noise = v - 1.0 + d * shape
        assert abs(np.std(noise) / sb - 1.0) < 0.2


def test_detection_stars_recipe():
    """Labelled stars: odd stars carry one box whose depth gives the target SNR of Eq. 2
    over the star's own samples; even stars are noise only; the set is reproducible."""
    import lcsynth
    d = lcsynth.detection_stars(40, seed=5, n_cad=2048, sigma=(2e-4, 2e-4), snr=(10.0, 10.0))
    assert list(d.label[:4]) == [0, 1, 0, 1] and d.lc_offsets[-1] == len(d.times) == len(d.flux)
    lens = np.diff(d.lc_offsets)
    assert lens.min() > 2048 - 2 * 5 / lcsynth.CADENCE_D - 1 and lens.max() <= 2048
    for s in range(40):
        t = d.times[d.lc_offsets[s]:d.lc_offsets[s + 1]]
        fl = d.flux[d.lc_offsets[s]:d.lc_offsets[s + 1]].astype(np.float64)
        assert np.all(np.diff(t) > 0)
        if d.label[s] == 0:
            assert np.isnan(d.period[s]) and abs(np.mean(fl) - 1) < 5 * 2e-4 / np.sqrt(len(fl)) + 1e-7
    d2 = lcsynth.detection_stars(40, seed=5, n_cad=2048, sigma=(2e-4, 2e-4), snr=(10.0, 10.0))
    assert np.array_equal(d.flux, d2.flux) and np.array_equal(d.times, d2.times)
    # in-transit samples sit lower by the Eq. 2 depth for SNR 10 (within 3 sigma of their mean)
    for s in range(1, 40, 2):
        t = d.times[d.lc_offsets[s]:d.lc_offsets[s + 1]]
        fl = d.flux[d.lc_offsets[s]:d.lc_offsets[s + 1]].astype(np.float64)
        P, e, w = d.period[s], d.epoch[s], d.duration[s]
        intr = np.abs(np.mod(t - e + P / 2, P) - P / 2) < w / 2
        n_in = intr.sum()
        assert abs(d.depth[s] - 10 * 2e-4 / np.sqrt(len(t) * w / P)) < 1e-15
        if n_in > 0:
            measured = 1.0 - fl[intr].mean()
            assert abs(measured - d.depth[s]) < 3 * 2e-4 / np.sqrt(n_in) + 1e-6, (s, measured, d.depth[s])
