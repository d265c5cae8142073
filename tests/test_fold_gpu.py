"""GPU parity of the fold, box-SNR and best-period kernels against the FP64 oracle.

Tolerances: bin counts bit-exact; bin means within 1e-6 relative; box-SNR within 1e-5
relative (with the score's own scale as floor when |score| < 1).
"""
import math

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


def gpu_fold(ctx, times, flux, periods, nbins, t0):
    import paper_2312_02063_gb300 as g
    folded, counts = g.gpfc_fold(ctx, _dev(ctx, times), _dev(ctx, flux.astype(np.float32)),
                                 _dev(ctx, periods), nbins, t0)
    ctx.sync()
    return folded.cpu().numpy(), counts.cpu().numpy()


def check_fold(fo, co, mean_o, cnt_o):
    np.testing.assert_array_equal(co, cnt_o)
    nz = cnt_o > 0
    err = np.abs(fo[nz].astype(np.float64) - mean_o[nz])
    assert np.all(err <= MEAN_RTOL * np.abs(mean_o[nz])), float(np.max(err / np.abs(mean_o[nz])))
    assert np.all(np.isnan(fo[~nz]))


def check_box(sc, sc_o):
    sc = sc.astype(np.float64)
    fin = np.isfinite(sc_o)
    np.testing.assert_array_equal(np.isfinite(sc), fin)
    err = np.abs(sc[fin] - sc_o[fin])
    assert np.all(err <= BOX_RTOL * np.maximum(np.abs(sc_o[fin]), 1.0)), float(np.max(err))


def test_fold_tiny_config_matches_oracle(ctx):
    lc = lcsynth.light_curve_tiny()
    periods = lcsynth.freq_grid(2000)
    fo, co = gpu_fold(ctx, lc.times, lc.flux, periods, 64, lc.t0)
    mean_o, cnt_o, _ = oracle.fold(lc.times, lc.flux, periods, 64, lc.t0)
    check_fold(fo, co, mean_o, cnt_o)


@pytest.mark.parametrize("n,npd,nbins", [(1, 1, 2), (5, 3, 7), (1023, 37, 64), (1025, 33, 100),
                                         (3001, 65, 256), (4096 * 5 + 17, 129, 128), (2500, 40, 1024),
                                         (70001, 31, 256)])
def test_fold_ragged_sizes(ctx, n, npd, nbins):
    rng = np.random.default_rng(n + npd + nbins)
    times = np.sort(rng.uniform(0.0, 400.0, n))
    flux = (1.0 + rng.normal(0, 3e-4, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, npd)
    t0 = float(rng.uniform(-5, 5))
    fo, co = gpu_fold(ctx, times, flux, periods, nbins, t0)
    mean_o, cnt_o, _ = oracle.fold(times, flux, periods, nbins, t0)
    check_fold(fo, co, mean_o, cnt_o)


def test_fold_adversarial_edges_multiples_and_negative_tau(ctx):
    # t on a 2^-24 grid and power-of-two periods: many samples exactly on bin edges;
    # periods equal to multiples of the cadence leave most bins empty; t < t0.
    n = 5000
    dt = 2.0 ** -6
    times = np.arange(n) * dt - 20.0
    flux = (1.0 + 1e-4 * np.sin(np.arange(n))).astype(np.float32)
    periods = np.array([0.25, 0.5, 1.0, 2.0, 8 * dt, 13 * dt, 0.7, 1e-3, 123.0])
    for nbins in (64, 256, 100):
        fo, co = gpu_fold(ctx, times, flux, periods, nbins, 0.0)
        mean_o, cnt_o, _ = oracle.fold(times, flux, periods, nbins, 0.0)
        check_fold(fo, co, mean_o, cnt_o)


def test_fold_constant_flux_and_all_in_one_bin(ctx):
    n = 70000  # > 65535: one bin receives every sample (period far above the span)
    times = np.arange(n) * lcsynth.CADENCE_D
    flux = np.full(n, 0.99931, np.float32)
    periods = np.array([1e7, 0.5, 0.6123])
    fo, co = gpu_fold(ctx, times, flux, periods, 64, 0.0)
    mean_o, cnt_o, _ = oracle.fold(times, flux, periods, 64, 0.0)
    check_fold(fo, co, mean_o, cnt_o)
    assert co[0, 0] == n


def test_fold_is_deterministic(ctx):
    lc = lcsynth.light_curve_tiny(3)
    periods = lcsynth.freq_grid(777)
    a = gpu_fold(ctx, lc.times, lc.flux, periods, 64, lc.t0)
    b = gpu_fold(ctx, lc.times, lc.flux, periods, 64, lc.t0)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[1], b[1])


@pytest.fixture(scope="module")
def kepler():
    lc = lcsynth.light_curve_kepler()
    periods = lcsynth.freq_grid(250_000)
    return lc, periods


def test_fold_full_length_sampled_periods_and_invariants(ctx, kepler):
    lc, periods = kepler
    fo, co = gpu_fold(ctx, lc.times, lc.flux, periods, 256, lc.t0)
    n = lc.times.shape[0]
    assert np.all(co.sum(axis=1) == n)
    # sum of (mean * count) over bins equals the flux total for every period
    tot = float(np.sum(lc.flux.astype(np.float64)))
    s = np.where(co > 0, fo.astype(np.float64) * co, 0.0).sum(axis=1)
    assert np.max(np.abs(s - tot)) <= 1e-6 * tot
    idx = np.random.default_rng(0).choice(len(periods), 96, replace=False)
    idx = np.concatenate([idx, [0, len(periods) - 1]])
    mean_o, cnt_o, _ = oracle.fold(lc.times, lc.flux, periods[idx], 256, lc.t0)
    check_fold(fo[idx], co[idx], mean_o, cnt_o)


def test_search_box_tiny_config(ctx):
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny()
    periods = lcsynth.freq_grid(2000)
    sig = 1e-4
    score, bi, bs = g.gpfc_search(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), 64,
                                  lc.t0, g.SCORER_BOX, 1, 8, sig)
    ctx.sync()
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods, 64, lc.t0)
    sc_o, s_o, w_o = oracle.box_snr(sum_o, cnt_o, 1, 8, sig)
    sc = score.cpu().numpy()
    check_box(sc, sc_o)
    k = int(bi.item())
    assert k == oracle.argmax(sc)
    assert float(bs.item()) == sc[k]
    # the injected 0.7 d signal (or a harmonic) wins
    P = periods[k]
    assert min(abs(P - 0.7 * m) for m in (0.5, 1.0, 2.0)) < 2e-3


def test_search_box_full_length_sampled(ctx, kepler):
    import paper_2312_02063_gb300 as g
    lc, periods = kepler
    w_max = int(math.ceil(0.42 * 256))
    score, bi, bs = g.gpfc_search(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), 256,
                                  lc.t0, g.SCORER_BOX, 1, w_max, 0.0)
    ctx.sync()
    sc = score.cpu().numpy()
    sigma = float(np.std(lc.flux.astype(np.float64)))
    k = int(bi.item())
    idx = np.random.default_rng(1).choice(len(periods), 24, replace=False)
    idx = np.unique(np.concatenate([idx, [k]]))
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods[idx], 256, lc.t0)
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, w_max, sigma)
    # sigma: GPU uses its own FP64 population std, rounded to FP32
    check_box(sc[idx] * 1.0, sc_o * (sigma / np.float64(np.float32(sigma))))
    assert k == oracle.argmax(sc)


def test_score_box_standalone_matches_oracle(ctx):
    import paper_2312_02063_gb300 as g
    prof, _ = lcsynth.profiles_mixed(1500, seed=4)
    rng = np.random.default_rng(4)
    counts = rng.integers(0, 400, prof.shape).astype(np.int32)
    counts[:, ::17] = 0
    prof = np.where(counts > 0, prof, np.nan).astype(np.float32)
    sc, bs, bw = g.gpfc_score_box(ctx, _dev(ctx, prof), _dev(ctx, counts), 1, 32, 2e-4)
    ctx.sync()
    sc_o, _, _ = oracle.box_snr_from_means(prof, counts, 1, 32, 2e-4)
    check_box(sc.cpu().numpy(), sc_o)
    # the reported box must reach the score (several boxes may tie within rounding)
    bs, bw = bs.cpu().numpy(), bw.cpu().numpy()
    sums = np.where(counts > 0, prof.astype(np.float64) * counts, 0.0)
    for k in range(0, 1500, 97):
        v = oracle.box_snr_at(sums[k], counts[k], int(bs[k]), int(bw[k]), 2e-4)
        assert abs(v - sc_o[k]) <= BOX_RTOL * max(abs(sc_o[k]), 1.0)


@pytest.mark.parametrize("nbins,w_min,w_max", [(64, 1, 8), (100, 3, 17), (37, 2, 37), (256, 5, 108),
                                               (8, 1, 8), (13, 4, 4), (1024, 1, 40)])
def test_score_box_width_ranges_and_odd_bins(ctx, nbins, w_min, w_max):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(nbins * 1000 + w_min * 10 + w_max)
    n = 203
    counts = rng.integers(0, 30, (n, nbins)).astype(np.int32)
    counts[rng.random((n, nbins)) < 0.1] = 0
    prof = (1.0 + rng.normal(0, 1e-3, (n, nbins))).astype(np.float32)
    for k in range(0, n, 3):  # some boxes
        st, w = rng.integers(0, nbins), rng.integers(1, max(2, nbins // 3))
        prof[k, (st + np.arange(w)) % nbins] -= 3e-3
    prof = np.where(counts > 0, prof, np.nan).astype(np.float32)
    sc, bs, bw = g.gpfc_score_box(ctx, _dev(ctx, prof), _dev(ctx, counts), w_min, w_max, 1e-3)
    ctx.sync()
    sc_o, _, _ = oracle.box_snr_from_means(prof, counts, w_min, w_max, 1e-3)
    check_box(sc.cpu().numpy(), sc_o)
    bs, bw = bs.cpu().numpy(), bw.cpu().numpy()
    sums = np.where(counts > 0, prof.astype(np.float64) * counts, 0.0)
    for k in range(n):
        if np.isfinite(sc_o[k]):
            assert w_min <= bw[k] <= w_max and 0 <= bs[k] < nbins
            v = oracle.box_snr_at(sums[k], counts[k], int(bs[k]), int(bw[k]), 1e-3)
            assert abs(v - sc_o[k]) <= BOX_RTOL * max(abs(sc_o[k]), 1.0)


def test_search_box_odd_bins_and_width_range(ctx):
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny(5)
    periods = lcsynth.freq_grid(333)
    for nbins, w_min, w_max in ((100, 3, 17), (64, 2, 64), (7, 1, 6)):
        score, _, _ = g.gpfc_search(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), nbins,
                                    lc.t0, g.SCORER_BOX, w_min, w_max, 2e-4)
        ctx.sync()
        _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods, nbins, lc.t0)
        sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, w_min, w_max, 2e-4)
        check_box(score.cpu().numpy(), sc_o)


def test_score_box_degenerate_profiles(ctx):
    import paper_2312_02063_gb300 as g
    nb = 64
    prof = np.ones((3, nb), np.float32)
    counts = np.full((3, nb), 5, np.int32)
    counts[1] = 0
    counts[1, 9] = 70000  # one bin holds everything: no valid box, count > 65535
    prof[2] = 0.9995
    sc, bs, bw = g.gpfc_score_box(ctx, _dev(ctx, prof), _dev(ctx, counts), 3, 8, 1.0)
    ctx.sync()
    sc, bs, bw = sc.cpu().numpy(), bs.cpu().numpy(), bw.cpu().numpy()
    assert sc[0] == 0.0 and (bs[0], bw[0]) == (0, 3)
    assert sc[1] == -np.inf and (bs[1], bw[1]) == (-1, -1)
    assert sc[2] == 0.0


def test_best_period_ties_and_nan(ctx):
    import paper_2312_02063_gb300 as g
    s = np.full(100003, -1.0, np.float32)
    s[5] = 3.0
    s[77777] = 3.0
    s[9] = np.nan
    bi, bs = g.gpfc_best_period(ctx, _dev(ctx, s))
    ctx.sync()
    assert int(bi.item()) == 5 and float(bs.item()) == 3.0
    bi, bs = g.gpfc_best_period(ctx, _dev(ctx, np.full(7, np.nan, np.float32)))
    ctx.sync()
    assert int(bi.item()) == -1


def test_invalid_period_is_reported_at_sync(ctx):
    import paper_2312_02063_gb300 as g
    times = np.arange(100) * 0.02
    flux = np.ones(100, np.float32)
    periods = np.array([0.5, -1.0, 0.3])
    g.gpfc_fold(ctx, _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods), 64, 0.0)
    with pytest.raises(g.GpfcError) as ei:
        ctx.sync()
    assert ei.value.code == -4
    ctx.sync()  # cleared


def test_argument_errors_are_synchronous(ctx):
    import paper_2312_02063_gb300 as g
    times = _dev(ctx, np.arange(10) * 0.1)
    flux = _dev(ctx, np.ones(10, np.float32))
    per = _dev(ctx, np.array([0.5]))
    with pytest.raises(g.GpfcError) as ei:
        g.gpfc_fold(ctx, times, flux, per, 1, 0.0)
    assert ei.value.code == -1
    with pytest.raises(g.GpfcError) as ei:
        g.gpfc_fold(ctx, times, flux, per, 8192, 0.0)
    assert ei.value.code == -1


@pytest.mark.parametrize("layout,chunk", [(1, 1000), (2, 1000), (1, 0), (2, 0), (3, 1000), (3, 0)])
def test_fold_and_search_every_kernel_variant(ctx, layout, chunk):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(layout * 10 + chunk)
    n = 9001
    times = np.sort(rng.uniform(0.0, 300.0, n))
    times[100:107] = times[100]  # repeated timestamps: hazards inside a group
    flux = (1.0 + rng.normal(0, 2e-4, n)).astype(np.float32)
    periods = np.concatenate([rng.uniform(0.2, 1.0, 70), [1e6, 0.25]])
    try:
        for nbins in (256, 100):
            for warps in (1, ctx.fold_max_warps(nbins, layout)):
                ctx.set_fold_config(warps=warps, layout=layout, chunk=chunk)
                fo, co = gpu_fold(ctx, times, flux, periods, nbins, 0.0)
                mean_o, cnt_o, sum_o = oracle.fold(times, flux, periods, nbins, 0.0)
                check_fold(fo, co, mean_o, cnt_o)
                score, _, _ = g.gpfc_search(ctx, _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods), nbins,
                                            0.0, g.SCORER_BOX, 1, 20, 2e-4)
                ctx.sync()
                sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 20, 2e-4)
                check_box(score.cpu().numpy(), sc_o)
    finally:
        ctx.reset_fold_config()


def test_bounded_wait_gives_up_reports_timeout_and_context_recovers(ctx):
    """A wait that nothing completes (an mbarrier no copy or MMA arrives on) gives up after
    its cycle limit, latches the timeout bit and returns; the host reads GPFC_ETIMEOUT and
    the context keeps working."""
    import paper_2312_02063_gb300 as g
    ctx.check_wait_timeout(2_000_000)
    with pytest.raises(g.GpfcError) as ei:
        ctx.sync()
    assert ei.value.code == -5
    ctx.sync()  # the bit was cleared when it was reported
    lc = lcsynth.light_curve_tiny()
    periods = lcsynth.freq_grid(300)
    fo, co = gpu_fold(ctx, lc.times, lc.flux, periods, 64, lc.t0)
    mean_o, cnt_o, _ = oracle.fold(lc.times, lc.flux, periods, 64, lc.t0)
    check_fold(fo, co, mean_o, cnt_o)


def test_reduction_fold_is_identical_for_any_launch_shape(ctx):
    """Layout 3 sums integers exactly, so its outputs must not depend on how the work is
    spread: warps (period groups), sample streams per group, tile size and blocks per SM give
    bit-identical means, counts and box scores, on one chunk (the default) and on several
    (chunk 992: exact int64 flushes)."""
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(33)
    n = 20011
    times = np.sort(rng.uniform(0.0, 600.0, n))
    times[500:509] = times[500]
    flux = (1.0 + rng.normal(0, 5e-3, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, 700)
    t_d, f_d, p_d = _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods)
    try:
        for chunk in (0, 992):
            ref = None
            for warps, streams, tile in ((1, 1, 1024), (3, 4, 1024), (2, 6, 2048), (3, 2, 512), (1, 12, 1024)):
                ctx.set_fold_config(warps=warps, layout=3, chunk=chunk, tile=tile, streams=streams)
                fo, co = g.gpfc_fold(ctx, t_d, f_d, p_d, 256, 0.0)
                sc, _, _ = g.gpfc_search(ctx, t_d, f_d, p_d, 256, 0.0, g.SCORER_BOX, 1, 108, 5e-3)
                ctx.sync()
                got = (fo.cpu().numpy(), co.cpu().numpy(), sc.cpu().numpy())
                plan = ctx.last_fold_plan()
                assert plan["layout"] == 3 and plan["streams"] == streams
                if ref is None:
                    ref = got
                else:
                    np.testing.assert_array_equal(got[0], ref[0])
                    np.testing.assert_array_equal(got[1], ref[1])
                    np.testing.assert_array_equal(got[2], ref[2])
    finally:
        ctx.reset_fold_config()



@pytest.mark.parametrize("tail_per_sm", [40, 10])
def test_short_last_chunk_scores_equal_a_fixed_block_shape(ctx, tail_per_sm):
    """The searches fold a last chunk of periods too short to give every SM a block of three
    period groups with narrower blocks (two groups for 40 periods per SM, one for 10; layout
    3 only, whose sums are exact). Box and CNN scores must equal those of the same search with
    the block shape fixed at three groups, which folds every chunk alike."""
    import paper_2312_02063_gb300 as g
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rng = np.random.default_rng(41)
    n = 6000
    times = np.sort(rng.uniform(0.0, 400.0, n))
    flux = (1.0 + rng.normal(0, 2e-3, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, 96 * nsm + tail_per_sm * nsm)  # one full chunk and a short one
    w = lcsynth.cnn_init(5, bias_scale=0.05)
    w["fc2.w"] = lcsynth.round_to_bf16(w["fc2.w"] * 0.25)
    wd = {k: _dev(ctx, v.astype(np.float32)) for k, v in w.items()}
    t_d, f_d, p_d = _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods)

    def both():
        box = g.gpfc_search(ctx, t_d, f_d, p_d, 256, 0.0, g.SCORER_BOX, 1, 108, 2e-3)
        cnn = g.gpfc_search(ctx, t_d, f_d, p_d, 256, 0.0, g.SCORER_CNN, weights=wd)
        ctx.sync()
        assert ctx.last_fold_plan()["layout"] == 3
        return [[t.cpu().numpy() for t in r] for r in (box, cnn)]

    auto = both()
    try:
        ctx.set_fold_config(warps=3, layout=3)
        fixed = both()
    finally:
        ctx.reset_fold_config()
    for a, f in zip(auto, fixed):
        for x, y in zip(a, f):
            np.testing.assert_array_equal(x, y)
