"""GPU parity of the per-star decision (SDE of Eq. 3, the peak rule of Sec. 4.2, harmonic
flags) against the FP64 oracle: SDE, mean and sd within 1e-9 relative; peaks (index,
width, harmonic flag, height) and counts exact."""
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


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


def compare(sm, pk, ref, max_peaks):
    assert abs(sm["sde"] - ref["sde"]) <= 1e-9 * max(1.0, abs(ref["sde"]))
    assert abs(sm["mean"] - ref["mean"]) <= 1e-9 * max(1e-30, abs(ref["mean"])) + 1e-15
    assert abs(sm["sd"] - ref["sd"]) <= 1e-9 * max(1e-30, abs(ref["sd"]))
    assert sm["best_index"] == ref["best_index"]
    assert sm["n_peaks"] == ref["n_peaks"] and sm["truncated"] == 0
    n = len(ref["index"])
    assert sm["n_listed"] == n
    np.testing.assert_array_equal(pk["index"][:n], ref["index"])
    np.testing.assert_array_equal(pk["width"][:n], ref["width"])
    np.testing.assert_array_equal(pk["harmonic"][:n], ref["harmonic"])
    np.testing.assert_array_equal(pk["height"][:n], ref["height"])


def test_constructed_periodograms(ctx):
    import paper_2312_02063_gb300 as g
    N = 2000
    periods = np.linspace(0.1, 2.0, N)
    s = np.zeros(N, np.float32)
    for start, width, h in [(100, 3, 10.0), (300, 4, 9.0), (600, 6, 8.0), (1500, 5, 8.0), (1800, 9, 3.0)]:
        s[start:start + width] = h
    s[603] = 8.5
    s[1804] = np.nan
    sd_, pk_ = g.gpfc_peaks(ctx, _dev(ctx, s), _dev(ctx, periods), max_peaks=8)
    ctx.sync()
    sm, pk = g.peaks_to_numpy(sd_, pk_, 8)
    compare(sm[0], pk[0], oracle.peaks(s, periods, max_peaks=8), 8)


def test_batched_search_periodograms_box_and_cnn(ctx):
    import paper_2312_02063_gb300 as g
    sb = lcsynth.star_batch(n_stars=6, p_count_range=(20000, 60000))
    d = [_dev(ctx, x) for x in (sb.lc_offsets, sb.times, sb.flux, sb.grid_offsets, sb.periods, sb.t0s)]
    w = {k: _dev(ctx, v.astype(np.float32)) for k, v in lcsynth.cnn_init(3, bias_scale=0.05).items()}
    for scorer, kw in ((g.SCORER_BOX, {"w_max": 108}), (g.SCORER_CNN, {"weights": w})):
        score, _, _ = g.gpfc_search_batched(ctx, d[0], d[1], d[2], d[3], d[4], 256, d[5], scorer, **kw)
        sd_, pk_ = g.gpfc_peaks(ctx, score, d[4], d[3], max_peaks=6, harmonic_tol=2e-3)
        ctx.sync()
        sm, pk = g.peaks_to_numpy(sd_, pk_, 6)
        sc = score.cpu().numpy()
        for s in range(len(sb.lc_offsets) - 1):
            a, b = sb.grid_offsets[s], sb.grid_offsets[s + 1]
            ref = oracle.peaks(sc[a:b], sb.periods[a:b], max_peaks=6, harmonic_tol=2e-3)
            compare(sm[s], pk[s], ref, 6)


def test_peaks_without_list_and_argument_errors(ctx):
    import paper_2312_02063_gb300 as g
    s = np.zeros(100, np.float32)
    s[10:16] = 5.0
    sd_, _ = g.gpfc_peaks(ctx, _dev(ctx, s), _dev(ctx, np.linspace(0.2, 1, 100)), max_peaks=0)
    ctx.sync()
    sm, _ = g.peaks_to_numpy(sd_, torch.zeros(1, dtype=torch.uint8), 0)
    assert sm[0]["best_index"] == 10 and sm[0]["n_peaks"] == 1 and sm[0]["n_listed"] == 0
    with pytest.raises(g.GpfcError):
        g.gpfc_peaks(ctx, _dev(ctx, s), _dev(ctx, np.linspace(0.2, 1, 100)), min_width=0)
