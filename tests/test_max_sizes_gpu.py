"""GPU parity at the boundary's largest sizes: a light curve of 2^24 samples (the most a
star may have) and a search over 2^22 periods (4,194,304; scores only, so the outputs stay
at 16 MB). Checked against the FP64 oracle on sampled periods, with the fold's and the
box-SNR's tolerances (counts bit-exact, means 1e-6 relative, box-SNR 1e-5 relative plus
the fixed-point allowance of tolerances.py).
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle
from tolerances import box_atol, fixed_point_unit

pytestmark = pytest.mark.gpu

MEAN_RTOL = 1e-6
BOX_RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


def test_fold_and_search_of_2_pow_24_samples(ctx):
    import paper_2312_02063_gb300 as g
    n = 1 << 24
    rng = np.random.default_rng(24)
    # two-minute cadence over ~64 years with 3% of the cadences dropped, white noise 1e-3
    keep = rng.random(int(n * 1.04)) > 0.03
    times = (np.nonzero(keep)[0][:n] * (2.0 / 1440.0)).astype(np.float64)
    assert times.shape[0] == n
    flux = (1.0 + rng.normal(0.0, 1e-3, n)).astype(np.float32)
    periods = np.array([0.2137, 0.5, 0.99971, 3.3])
    t_d, f_d, p_d = _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods)
    fo, co = g.gpfc_fold(ctx, t_d, f_d, p_d, 256, 0.0)
    score, bi, _ = g.gpfc_search(ctx, t_d, f_d, p_d, 256, 0.0, g.SCORER_BOX, 1, 108, 1e-3)
    ctx.sync()
    mean_o, cnt_o, sum_o = oracle.fold(times, flux, periods, 256, 0.0)
    np.testing.assert_array_equal(co.cpu().numpy(), cnt_o)
    assert int(cnt_o.sum()) == n * len(periods)
    fo = fo.cpu().numpy().astype(np.float64)
    nz = cnt_o > 0
    assert np.all(np.abs(fo[nz] - mean_o[nz]) <= MEAN_RTOL * np.abs(mean_o[nz]))
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 108, 1e-3)
    sc = score.cpu().numpy().astype(np.float64)
    fin = np.isfinite(sc_o)
    np.testing.assert_array_equal(np.isfinite(sc), fin)
    tol = BOX_RTOL * np.maximum(np.abs(sc_o[fin]), 1.0) + box_atol(fixed_point_unit(flux), 1e-3)
    assert np.all(np.abs(sc[fin] - sc_o[fin]) <= tol)
    assert int(bi.item()) == oracle.argmax(score.cpu().numpy())


def test_search_over_4_million_periods(ctx):
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny(22)
    npd = 1 << 22
    periods = lcsynth.freq_grid(npd, 0.05, 2.0)
    score, bi, bs = g.gpfc_search(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), 256,
                                  lc.t0, g.SCORER_BOX, 1, 108, 2e-4)
    ctx.sync()
    sc = score.cpu().numpy()
    k = int(bi.item())
    assert k == oracle.argmax(sc) and float(bs.item()) == sc[k]
    idx = np.unique(np.concatenate([np.random.default_rng(22).choice(npd, 24, replace=False), [0, npd - 1, k]]))
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods[idx], 256, lc.t0)
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 108, 2e-4)
    fin = np.isfinite(sc_o)
    got = sc[idx].astype(np.float64)
    np.testing.assert_array_equal(np.isfinite(got), fin)
    assert np.all(np.abs(got[fin] - sc_o[fin]) <= BOX_RTOL * np.maximum(np.abs(sc_o[fin]), 1.0))
