"""GPU parity above 1024 bins, where the fold adds each sample with one exact fixed-point
shared-memory atomic per period (count << 40 plus the flux sum in quanta 2^-k) and the box
search runs on the fold's centred sums in the warp-per-profile kernel.

Tolerances as for the lane-private fold: counts bit-exact, means within 1e-6 relative,
box-SNR within 1e-5 relative (the score's own scale as floor when |score| < 1).
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle

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


def check_box(sc, sc_o):
    sc = sc.astype(np.float64)
    fin = np.isfinite(sc_o)
    np.testing.assert_array_equal(np.isfinite(sc), fin)
    err = np.abs(sc[fin] - sc_o[fin])
    assert np.all(err <= BOX_RTOL * np.maximum(np.abs(sc_o[fin]), 1.0)), float(np.max(err))


@pytest.mark.parametrize("n,npd,nbins", [(3001, 9, 2048), (20011, 7, 4096), (1, 3, 1025), (9000, 13, 1500),
                                         (65536, 5, 4096)])
def test_wide_fold_matches_the_oracle(ctx, n, npd, nbins):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(n + nbins)
    times = np.sort(rng.uniform(0.0, 400.0, n))
    flux = (1.0 + rng.normal(0, 3e-4, n)).astype(np.float32)
    periods = rng.uniform(0.05, 2.0, npd)
    t0 = float(rng.uniform(-2, 2))
    fo, co = g.gpfc_fold(ctx, _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods), nbins, t0)
    ctx.sync()
    fo, co = fo.cpu().numpy(), co.cpu().numpy()
    mean_o, cnt_o, _ = oracle.fold(times, flux, periods, nbins, t0)
    np.testing.assert_array_equal(co, cnt_o)
    nz = cnt_o > 0
    err = np.abs(fo[nz].astype(np.float64) - mean_o[nz])
    assert np.all(err <= MEAN_RTOL * np.abs(mean_o[nz])), float(np.max(err / np.abs(mean_o[nz])))
    assert np.all(np.isnan(fo[~nz]))


@pytest.mark.parametrize("nbins,w_min,w_max", [(2048, 1, 300), (4096, 5, 900), (1500, 2, 1500)])
def test_wide_box_search_matches_the_oracle(ctx, nbins, w_min, w_max):
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny(nbins)
    periods = lcsynth.freq_grid(1203)
    score, bi, bs = g.gpfc_search(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), nbins, lc.t0,
                                  g.SCORER_BOX, w_min, w_max, 2e-4)
    ctx.sync()
    sc = score.cpu().numpy()
    idx = np.unique(np.concatenate([np.random.default_rng(nbins).choice(len(periods), 10, replace=False),
                                    [0, len(periods) - 1, int(bi.item())]]))
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods[idx], nbins, lc.t0)
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, w_min, w_max, 2e-4)
    check_box(sc[idx], sc_o)
    k = int(bi.item())
    assert k == oracle.argmax(sc) and float(bs.item()) == sc[k]


def test_standalone_box_scoring_at_4096_bins(ctx):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(4096)
    n, nbins = 37, 4096
    counts = rng.integers(0, 6, (n, nbins)).astype(np.int32)
    prof = (1.0 + rng.normal(0, 1e-3, (n, nbins))).astype(np.float32)
    for k in range(n):
        st, w = rng.integers(0, nbins), rng.integers(1, 600)
        prof[k, (st + np.arange(w)) % nbins] -= 2e-3
    prof = np.where(counts > 0, prof, np.nan).astype(np.float32)
    sc, bs, bw = g.gpfc_score_box(ctx, _dev(ctx, prof), _dev(ctx, counts), 3, 700, 1e-3)
    ctx.sync()
    sc_o, _, _ = oracle.box_snr_from_means(prof, counts, 3, 700, 1e-3)
    check_box(sc.cpu().numpy(), sc_o)
    bs, bw = bs.cpu().numpy(), bw.cpu().numpy()
    sums = np.where(counts > 0, prof.astype(np.float64) * counts, 0.0)
    for k in range(0, n, 4):  # the reported box reaches the score
        assert 3 <= bw[k] <= 700 and 0 <= bs[k] < nbins
        v = oracle.box_snr_at(sums[k], counts[k], int(bs[k]), int(bw[k]), 1e-3)
        assert abs(v - sc_o[k]) <= BOX_RTOL * max(abs(sc_o[k]), 1.0)


def test_wide_limits(ctx):
    import paper_2312_02063_gb300 as g
    t = _dev(ctx, np.zeros(1 << 24))
    f = _dev(ctx, np.ones(1 << 24, np.float32))
    p = _dev(ctx, np.array([0.5]))
    with pytest.raises(g.GpfcError) as ei:  # the fixed-point fold takes fewer than 2^24 samples
        g.gpfc_fold(ctx, t, f, p, 2048, 0.0)
    assert ei.value.code == -1
    off = _dev(ctx, np.array([0, 100], np.int64))
    goff = _dev(ctx, np.array([0, 1], np.int64))
    with pytest.raises(g.GpfcError) as ei:  # the batched search stops at 1024 bins
        g.gpfc_search_batched(ctx, off, t[:100].contiguous(), f[:100].contiguous(), goff, p, 2048)
    assert ei.value.code == -6
