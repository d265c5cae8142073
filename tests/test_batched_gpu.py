"""GPU parity of the batched search (many stars of uneven length, each with its own
period grid, in one launch sequence) and of the fold's launch-config variants.

The batched scores must equal, bit for bit, those of gpfc_search on each star alone
(same kernels, same per-sample order of additions); sampled (star, period) pairs are
also checked against the FP64 oracle with the single-star tolerances (box-SNR 1e-5
relative, CNN 2e-2 absolute).
"""
import math

import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

BOX_RTOL = 1e-5
SCORE_ATOL = 2e-2
MEAN_RTOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


def ragged_batch(seed=7):
    """Stars with edge-case sizes: 1 sample, less than a tile, tile +- 1, several chunks;
    grids of 1 period, one block +- 1, several blocks."""
    rng = np.random.default_rng(seed)
    sizes = [1, 15, 1023, 1025, 3 * 4096 + 5, 20011, 512, 2048]
    grids = [1, 129, 128, 33, 300, 700, 2, 257]
    lc_off, g_off = [0], [0]
    ts, fs, ps, t0s = [], [], [], []
    for n, npd in zip(sizes, grids):
        t = np.sort(rng.uniform(0.0, 1300.0, n)) if n > 4096 else np.arange(n) * (29.4 / 1440.0)
        f = (1.0 + rng.normal(0.0, 2e-4, n)).astype(np.float32)
        p = rng.uniform(0.2, 1.0, npd)
        ts.append(t)
        fs.append(f)
        ps.append(p)
        t0s.append(float(rng.uniform(-3.0, 3.0)))
        lc_off.append(lc_off[-1] + n)
        g_off.append(g_off[-1] + npd)
    return (np.array(lc_off, np.int64), np.concatenate(ts), np.concatenate(fs), np.array(g_off, np.int64),
            np.concatenate(ps), np.array(t0s))


def per_star(ctx, lc_off, times, flux, g_off, periods, t0s, nbins, scorer, **kw):
    import paper_2312_02063_gb300 as g
    out, bi, bs = [], [], []
    for s in range(len(lc_off) - 1):
        a, b = lc_off[s], lc_off[s + 1]
        c, d = g_off[s], g_off[s + 1]
        sc, i, v = g.gpfc_search(ctx, _dev(ctx, times[a:b]), _dev(ctx, flux[a:b]), _dev(ctx, periods[c:d]), nbins,
                                 float(t0s[s]), scorer, **kw)
        ctx.sync()
        out.append(sc.cpu().numpy())
        bi.append(int(i.item()))
        bs.append(float(v.item()))
    return np.concatenate(out), np.array(bi), np.array(bs, np.float32)


def batched(ctx, lc_off, times, flux, g_off, periods, t0s, nbins, scorer, **kw):
    import paper_2312_02063_gb300 as g
    sc, bi, bs = g.gpfc_search_batched(ctx, _dev(ctx, lc_off), _dev(ctx, times), _dev(ctx, flux), _dev(ctx, g_off),
                                       _dev(ctx, periods), nbins, None if t0s is None else _dev(ctx, t0s),
                                       scorer, **kw)
    ctx.sync()
    return sc.cpu().numpy(), bi.cpu().numpy(), bs.cpu().numpy()


def test_batched_box_equals_per_star_and_oracle(ctx):
    import paper_2312_02063_gb300 as g
    lc_off, times, flux, g_off, periods, t0s = ragged_batch()
    kw = dict(w_min=1, w_max=20, sigma=2e-4)
    sc, bi, bs = batched(ctx, lc_off, times, flux, g_off, periods, t0s, 256, g.SCORER_BOX, **kw)
    sc1, bi1, bs1 = per_star(ctx, lc_off, times, flux, g_off, periods, t0s, 256, g.SCORER_BOX, **kw)
    np.testing.assert_array_equal(sc, sc1)
    np.testing.assert_array_equal(bi, bi1)
    np.testing.assert_array_equal(bs, bs1)
    for s in range(len(lc_off) - 1):
        a, b, c, d = lc_off[s], lc_off[s + 1], g_off[s], g_off[s + 1]
        idx = np.arange(c, d)[:: max(1, (d - c) // 6)]
        _, cnt_o, sum_o = oracle.fold(times[a:b], flux[a:b], periods[idx], 256, t0s[s])
        sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 20, 2e-4)
        fin = np.isfinite(sc_o)
        got = sc[idx].astype(np.float64)
        np.testing.assert_array_equal(np.isfinite(got), fin)
        assert np.all(np.abs(got[fin] - sc_o[fin]) <= BOX_RTOL * np.maximum(np.abs(sc_o[fin]), 1.0))
        assert bi[s] == oracle.argmax(sc[c:d])


def test_batched_cnn_equals_per_star_and_oracle(ctx):
    import paper_2312_02063_gb300 as g
    lc_off, times, flux, g_off, periods, t0s = ragged_batch(11)
    w = lcsynth.cnn_init(5, bias_scale=0.05)
    w["fc2.w"] = lcsynth.round_to_bf16(w["fc2.w"] * 0.25)
    wd = {k: _dev(ctx, v.astype(np.float32)) for k, v in w.items()}
    sc, bi, bs = batched(ctx, lc_off, times, flux, g_off, periods, t0s, 256, g.SCORER_CNN, weights=wd)
    sc1, bi1, bs1 = per_star(ctx, lc_off, times, flux, g_off, periods, t0s, 256, g.SCORER_CNN, weights=wd)
    np.testing.assert_array_equal(sc, sc1)
    np.testing.assert_array_equal(bi, bi1)
    np.testing.assert_array_equal(bs, bs1)
    for s in (2, 4, 5):
        a, b, c, d = lc_off[s], lc_off[s + 1], g_off[s], g_off[s + 1]
        idx = np.arange(c, d)[:: max(1, (d - c) // 10)]
        mean_o, cnt_o, _ = oracle.fold(times[a:b], flux[a:b], periods[idx], 256, t0s[s])
        _, so = oracle.cnn_score(w, mean_o.astype(np.float32), cnt_o.astype(np.int32))
        assert np.max(np.abs(sc[idx] - so)) <= SCORE_ATOL


def test_batched_graph_replay_tracks_new_data(ctx):
    import paper_2312_02063_gb300 as g
    lc_off, times, flux, g_off, periods, t0s = ragged_batch(3)
    d = [_dev(ctx, x) for x in (lc_off, times, flux, g_off, periods, t0s)]
    score = torch.empty(len(periods), dtype=torch.float32, device=ctx.device)
    bi = torch.empty(len(lc_off) - 1, dtype=torch.int64, device=ctx.device)
    bs = torch.empty(len(lc_off) - 1, dtype=torch.float32, device=ctx.device)
    kw = dict(scorer=g.SCORER_BOX, w_min=2, w_max=30, sigma=0.0, score=score, best_index=bi, best_score=bs)
    ctx.set_graph(True)
    g.gpfc_search_batched(ctx, d[0], d[1], d[2], d[3], d[4], 128, d[5], **kw)
    ctx.sync()
    first = score.cpu().numpy().copy()
    g.gpfc_search_batched(ctx, d[0], d[1], d[2], d[3], d[4], 128, d[5], **kw)  # replay
    ctx.sync()
    np.testing.assert_array_equal(score.cpu().numpy(), first)
    # new flux in the same buffer: the replayed graph reads it
    d[2].copy_(_dev(ctx, (1.0 + np.random.default_rng(9).normal(0, 3e-4, len(flux))).astype(np.float32)))
    g.gpfc_search_batched(ctx, d[0], d[1], d[2], d[3], d[4], 128, d[5], **kw)
    ctx.sync()
    replayed = score.cpu().numpy().copy()
    replayed_bi = bi.cpu().numpy().copy()
    ctx.set_graph(False)
    try:
        g.gpfc_search_batched(ctx, d[0], d[1], d[2], d[3], d[4], 128, d[5], **kw)
        ctx.sync()
    finally:
        ctx.set_graph(True)
    np.testing.assert_array_equal(score.cpu().numpy(), replayed)
    np.testing.assert_array_equal(bi.cpu().numpy(), replayed_bi)
    assert not np.array_equal(replayed, first)


def test_batched_default_t0_is_each_stars_first_time(ctx):
    import paper_2312_02063_gb300 as g
    lc_off, times, flux, g_off, periods, _ = ragged_batch(5)
    first = times[lc_off[:-1]]
    sc_a, _, _ = batched(ctx, lc_off, times, flux, g_off, periods, None, 64, g.SCORER_BOX, w_max=8)
    sc_b, _, _ = batched(ctx, lc_off, times, flux, g_off, periods, first, 64, g.SCORER_BOX, w_max=8)
    np.testing.assert_array_equal(sc_a, sc_b)


def test_batched_invalid_offsets_are_reported(ctx):
    import paper_2312_02063_gb300 as g
    lc_off, times, flux, g_off, periods, t0s = ragged_batch(2)
    bad = lc_off.copy()
    bad[3], bad[4] = bad[4], bad[3]  # not monotone
    sc, _, _ = g.gpfc_search_batched(ctx, _dev(ctx, bad), _dev(ctx, times), _dev(ctx, flux), _dev(ctx, g_off),
                                     _dev(ctx, periods), 64, _dev(ctx, t0s), g.SCORER_BOX, w_max=8)
    with pytest.raises(g.GpfcError) as ei:
        ctx.sync()
    assert ei.value.code == -1
    bad_g = g_off.copy()
    bad_g[-1] += 5  # last offset past the periods
    g.gpfc_search_batched(ctx, _dev(ctx, lc_off), _dev(ctx, times), _dev(ctx, flux), _dev(ctx, bad_g),
                          _dev(ctx, periods), 64, _dev(ctx, t0s), g.SCORER_BOX, w_max=8)
    with pytest.raises(g.GpfcError):
        ctx.sync()
    # the context stays usable
    sc, _, _ = batched(ctx, lc_off, times, flux, g_off, periods, t0s, 64, g.SCORER_BOX, w_max=8)
    assert np.all(np.isfinite(sc) | (np.diff(lc_off).repeat(np.diff(g_off)) < 2))


def test_batched_argument_errors_are_synchronous(ctx):
    import paper_2312_02063_gb300 as g
    lc_off, times, flux, g_off, periods, t0s = ragged_batch(2)
    with pytest.raises(g.GpfcError):
        g.gpfc_search_batched(ctx, _dev(ctx, lc_off), _dev(ctx, times), _dev(ctx, flux), _dev(ctx, g_off),
                              _dev(ctx, periods), 100, None, g.SCORER_CNN,
                              weights={k: _dev(ctx, v) for k, v in lcsynth.cnn_init(1).items()})
    with pytest.raises(g.GpfcError):
        g.gpfc_search_batched(ctx, _dev(ctx, lc_off), _dev(ctx, times), _dev(ctx, flux), _dev(ctx, g_off),
                              _dev(ctx, periods), 64, None, g.SCORER_BOX, w_min=3, w_max=2)


@pytest.mark.parametrize("layout", [1, 2])
def test_fold_tile_and_occupancy_variants_are_bit_identical(ctx, layout):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(40 + layout)
    n = 3 * 2048 + 700
    times = np.arange(n) * (29.4 / 1440.0)
    times[1000:1500] += 0.3  # an irregular stretch: checked path between regular groups
    flux = (1.0 + rng.normal(0, 2e-4, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, 301)
    mean_o, cnt_o, sum_o = oracle.fold(times, flux, periods, 256, 0.0)
    ref = None
    try:
        for tile in (512, 1024, 2048):
            for warps in (1, 2, g.Context.fold_max_warps(ctx, 256, layout)):
                ctx.set_fold_config(warps=warps, layout=layout, tile=tile)
                fo, co = g.gpfc_fold(ctx, _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods), 256, 0.0)
                sc, _, _ = g.gpfc_search(ctx, _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods), 256, 0.0,
                                         g.SCORER_BOX, 1, 32, 2e-4)
                ctx.sync()
                plan = ctx.last_fold_plan()
                assert plan["tile"] == tile and plan["layout"] == layout
                fo, co, sc = fo.cpu().numpy(), co.cpu().numpy(), sc.cpu().numpy()
                np.testing.assert_array_equal(co, cnt_o)
                nz = cnt_o > 0
                assert np.all(np.abs(fo[nz] - mean_o[nz]) <= MEAN_RTOL * np.abs(mean_o[nz]))
                if ref is None:
                    ref = (fo, sc)
                else:
                    np.testing.assert_array_equal(fo, ref[0])
                    np.testing.assert_array_equal(sc, ref[1])
    finally:
        ctx.reset_fold_config()
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 32, 2e-4)
    assert np.all(np.abs(ref[1] - sc_o) <= BOX_RTOL * np.maximum(np.abs(sc_o), 1.0))


def test_autotune_picks_a_valid_config_with_identical_results(ctx):
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_kepler()
    periods = lcsynth.freq_grid(40000)
    t, f, p = _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods)
    ctx.set_autotune(0)
    ref, _, _ = g.gpfc_search(ctx, t, f, p, 256, lc.t0, g.SCORER_BOX, 1, 108, 0.0)
    ctx.sync()
    ctx.set_autotune(1)
    cfg = g.gpfc_autotune(ctx, t, f, p, 256, g.SCORER_BOX, 1, 108, 0.0)
    assert cfg["tile"] in (512, 1024, 2048) and cfg["layout"] in (1, 2, 3) and cfg["blocks_per_sm"] >= 1
    assert 1 <= cfg["warps"] <= ctx.fold_max_warps(256, cfg["layout"]) or cfg["tile"] != 1024
    sc, _, _ = g.gpfc_search(ctx, t, f, p, 256, lc.t0, g.SCORER_BOX, 1, 108, 0.0)
    ctx.sync()
    plan = ctx.last_fold_plan()
    assert (plan["warps"], plan["layout"], plan["tile"]) == (cfg["warps"], cfg["layout"], cfg["tile"])
    np.testing.assert_array_equal(sc.cpu().numpy(), ref.cpu().numpy())
    ctx.set_autotune(-1)
    ctx.set_autotune(1)


def test_batched_full_size_stars_sampled(ctx):
    """Stars of the batched workload's full sizes (8,192-70,000 samples with gaps,
    20,000-250,000 periods each), CNN and box scorers, in the launch configuration of the
    benchmark (autotuned, graph-captured): per-star equality on three stars and the
    oracle on sampled periods."""
    import paper_2312_02063_gb300 as g
    sb = lcsynth.star_batch(n_stars=12)
    w = lcsynth.cnn_init(3, bias_scale=0.05)
    wd = {k: _dev(ctx, v.astype(np.float32)) for k, v in w.items()}
    dargs = [_dev(ctx, x) for x in (sb.lc_offsets, sb.times, sb.flux, sb.grid_offsets, sb.periods, sb.t0s)]
    sc, bi, bs = g.gpfc_search_batched(ctx, *dargs[:5], 256, dargs[5], g.SCORER_CNN, weights=wd)
    sb_box, bib, _ = g.gpfc_search_batched(ctx, *dargs[:5], 256, dargs[5], g.SCORER_BOX, w_max=108)
    ctx.sync()
    sc, bi, bs, sb_box, bib = (x.cpu().numpy() for x in (sc, bi, bs, sb_box, bib))
    for s in (0, 5, 11):
        a, b, c, d = sb.lc_offsets[s], sb.lc_offsets[s + 1], sb.grid_offsets[s], sb.grid_offsets[s + 1]
        t, f, p = _dev(ctx, sb.times[a:b]), _dev(ctx, sb.flux[a:b]), _dev(ctx, sb.periods[c:d])
        one, i1, _ = g.gpfc_search(ctx, t, f, p, 256, float(sb.t0s[s]), g.SCORER_CNN, weights=wd)
        one_b, _, _ = g.gpfc_search(ctx, t, f, p, 256, float(sb.t0s[s]), g.SCORER_BOX, 1, 108, 0.0)
        ctx.sync()
        np.testing.assert_array_equal(sc[c:d], one.cpu().numpy())
        np.testing.assert_array_equal(sb_box[c:d], one_b.cpu().numpy())
        assert bi[s] == int(i1.item()) == oracle.argmax(sc[c:d])
        assert bib[s] == oracle.argmax(sb_box[c:d])
        idx = np.random.default_rng(s).choice(d - c, 6, replace=False)
        mean_o, cnt_o, sum_o = oracle.fold(sb.times[a:b], sb.flux[a:b], sb.periods[c:d][idx], 256, sb.t0s[s])
        _, so = oracle.cnn_score(w, mean_o.astype(np.float32), cnt_o.astype(np.int32))
        assert np.max(np.abs(sc[c:d][idx] - so)) <= SCORE_ATOL
        sigma = float(np.std(sb.flux[a:b].astype(np.float64)))
        sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 108, float(np.float32(sigma)))
        assert np.all(np.abs(sb_box[c:d][idx] - sc_o) <= BOX_RTOL * np.maximum(np.abs(sc_o), 1.0))
    assert math.isfinite(float(bs.max()))
