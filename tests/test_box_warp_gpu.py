"""GPU parity of the places the box-SNR search can run: the fold kernel's epilogue, the
separate warp-per-profile kernel fed by the fold's centred bin sums, and the one-kernel
search whose extra warp per fold block scores the block's previous task. All are checked
against the FP64 oracle (box-SNR within 1e-5 relative, the score's own scale as floor when
|score| < 1); the warp and one-kernel paths must agree bit for bit, and batched searches
must equal per-star ones bit for bit.
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

BOX_RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.set_box_path(g.BOX_AUTO)
    c.close()


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


def check_box(sc, sc_o):
    sc = sc.astype(np.float64)
    fin = np.isfinite(sc_o)
    np.testing.assert_array_equal(np.isfinite(sc), fin)
    err = np.abs(sc[fin] - sc_o[fin])
    assert np.all(err <= BOX_RTOL * np.maximum(np.abs(sc_o[fin]), 1.0)), float(np.max(err))


def search(ctx, path, times, flux, periods, nbins, t0, w_min, w_max, sigma):
    import paper_2312_02063_gb300 as g
    ctx.set_box_path(path)
    score, bi, bs = g.gpfc_search(ctx, _dev(ctx, times), _dev(ctx, flux), _dev(ctx, periods), nbins, t0,
                                  g.SCORER_BOX, w_min, w_max, sigma)
    ctx.sync()
    return score.cpu().numpy(), int(bi.item()), float(bs.item())


@pytest.mark.parametrize("nbins,w_min,w_max", [(256, 1, 108), (256, 5, 256), (100, 3, 17), (512, 2, 200),
                                               (300, 2, 120), (1024, 1, 40), (37, 2, 37), (2, 1, 2), (9, 1, 1)])
def test_both_box_paths_match_the_oracle(ctx, nbins, w_min, w_max):
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny(nbins)
    periods = lcsynth.freq_grid(517)
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods, nbins, lc.t0)
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, w_min, w_max, 2e-4)
    got = {}
    for path in (g.BOX_EPILOGUE, g.BOX_WARP, g.BOX_FUSED):
        sc, k, v = search(ctx, path, lc.times, lc.flux, periods, nbins, lc.t0, w_min, w_max, 2e-4)
        check_box(sc, sc_o)
        assert k == oracle.argmax(sc) and v == sc[k]
        got[path] = sc
    np.testing.assert_array_equal(got[g.BOX_WARP], got[g.BOX_FUSED])


@pytest.mark.parametrize("path_name", ["BOX_WARP", "BOX_FUSED"])
def test_box_warp_path_over_several_chunks(ctx, path_name):
    """More periods than one fold wave holds: the scorer runs on several chunks, and in the
    one-kernel search every block goes round its two-slot ring more than once."""
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny(3)
    periods = lcsynth.freq_grid(40000)
    sc, k, v = search(ctx, getattr(g, path_name), lc.times, lc.flux, periods, 256, lc.t0, 1, 108, 0.0)
    idx = np.unique(np.concatenate([np.random.default_rng(5).choice(len(periods), 40, replace=False),
                                    [0, len(periods) - 1, k]]))
    sigma = float(np.std(lc.flux.astype(np.float64)))
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods[idx], 256, lc.t0)
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 108, sigma)
    # the GPU's sigma is its own FP64 population std, rounded to FP32
    check_box(sc[idx], sc_o * (sigma / np.float64(np.float32(sigma))))
    assert k == oracle.argmax(sc) and v == sc[k]


def test_box_warp_degenerate_star(ctx):
    """One sample: every box has an empty side, so every score is -inf and no best exists."""
    import paper_2312_02063_gb300 as g
    args = (np.array([3.0]), np.array([1.0], np.float32), lcsynth.freq_grid(50), 256, 0.0, 1, 108, 1e-3)
    sc, k, v = search(ctx, g.BOX_WARP, *args)
    assert np.all(sc == -np.inf) and k == oracle.argmax(sc) and v == -np.inf
    assert search(ctx, g.BOX_EPILOGUE, *args)[1] == k
    sc2, k2, _ = search(ctx, g.BOX_FUSED, *args)
    assert np.all(sc2 == -np.inf) and k2 == k


def test_fused_search_equals_the_two_kernel_path_at_full_size(ctx):
    """The 250,000-period Kepler-like search: the one-kernel path gives the two-kernel
    path's scores bit for bit (same fold sums, same scorer), and its best period."""
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_kepler()
    periods = lcsynth.freq_grid(250000)
    a, ka, va = search(ctx, g.BOX_WARP, lc.times, lc.flux, periods, 256, lc.t0, 1, 108, 0.0)
    b, kb, vb = search(ctx, g.BOX_FUSED, lc.times, lc.flux, periods, 256, lc.t0, 1, 108, 0.0)
    np.testing.assert_array_equal(a, b)
    assert ka == kb and va == vb


@pytest.mark.parametrize("nbins", [128, 256])
def test_batched_equals_per_star_on_both_paths(ctx, nbins):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(nbins)
    sizes, grids = [1, 1023, 4096 * 3 + 5, 20011, 512], [1, 129, 300, 700, 257]
    lc_off, g_off, ts, fs, ps = [0], [0], [], [], []
    for n, npd in zip(sizes, grids):
        ts.append(np.sort(rng.uniform(0.0, 1300.0, n)))
        fs.append((1.0 + rng.normal(0.0, 2e-4, n)).astype(np.float32))
        ps.append(rng.uniform(0.2, 1.0, npd))
        lc_off.append(lc_off[-1] + n)
        g_off.append(g_off[-1] + npd)
    t0s = rng.uniform(-3.0, 3.0, len(sizes))
    lc_off, g_off = np.array(lc_off, np.int64), np.array(g_off, np.int64)
    times, flux, periods = np.concatenate(ts), np.concatenate(fs), np.concatenate(ps)
    for path in (g.BOX_EPILOGUE, g.BOX_WARP):
        ctx.set_box_path(path)
        sc, bi, bs = g.gpfc_search_batched(ctx, _dev(ctx, lc_off), _dev(ctx, times), _dev(ctx, flux),
                                           _dev(ctx, g_off), _dev(ctx, periods), nbins, _dev(ctx, t0s),
                                           g.SCORER_BOX, w_min=2, w_max=40, sigma=0.0)
        ctx.sync()
        sc, bi, bs = sc.cpu().numpy(), bi.cpu().numpy(), bs.cpu().numpy()
        for s in range(len(sizes)):
            a, b, c, d = lc_off[s], lc_off[s + 1], g_off[s], g_off[s + 1]
            one, k, v = search(ctx, path, times[a:b], flux[a:b], periods[c:d], nbins, float(t0s[s]), 2, 40, 0.0)
            np.testing.assert_array_equal(sc[c:d], one)
            assert bi[s] == k and bs[s] == v


def test_one_kernel_search_with_the_paired16_layout(ctx):
    """The one-kernel search with 6-byte bins (FP32 sums, paired 16-bit counts) and three
    fold warps, against the default 8-byte layout: the same fold sums, so the same scores."""
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_tiny(17)
    periods = lcsynth.freq_grid(3000)
    a, ka, _ = search(ctx, g.BOX_FUSED, lc.times, lc.flux, periods, 256, lc.t0, 1, 40, 2e-4)
    try:
        ctx.set_fold_config(warps=3, layout=g.LAYOUT_PAIRED16)
        b, kb, _ = search(ctx, g.BOX_FUSED, lc.times, lc.flux, periods, 256, lc.t0, 1, 40, 2e-4)
        assert ctx.last_fold_plan()["layout"] == g.LAYOUT_PAIRED16
    finally:
        ctx.reset_fold_config()
    _, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods, 256, lc.t0)
    sc_o, _, _ = oracle.box_snr(sum_o, cnt_o, 1, 40, 2e-4)
    check_box(b, sc_o)
    assert kb == oracle.argmax(b)
