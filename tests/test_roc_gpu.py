"""GPU ROC statistics (gpfc_roc, Sec. 3.2) against oracle.roc: exact equality of the
U statistic, thresholds and detection counts, on scores with many ties and NaNs, on large
random sets, and on star-level scores from a batched search of labelled stars."""
import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

FPRS = [0.0, 1e-3, 1e-2, 0.1, 0.5, 0.99]


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def check(ctx, pos, neg, fprs=FPRS):
    import paper_2312_02063_gb300 as g
    u2, thr, tp = g.gpfc_roc(ctx, torch.from_numpy(pos).to(ctx.device), torch.from_numpy(neg).to(ctx.device), fprs)
    ctx.sync()
    r = oracle.roc(pos, neg, fprs)
    assert int(u2.item()) == r["u2"]
    np.testing.assert_array_equal(thr.cpu().numpy().astype(np.float64), r["thr"])
    np.testing.assert_array_equal(tp.cpu().numpy(), r["tp"])
    return r


@pytest.mark.parametrize("seed", range(4))
def test_roc_ties_and_nan(ctx, seed):
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, 20, 3001).astype(np.float32)
    neg = rng.integers(0, 15, 2999).astype(np.float32)
    pos[rng.choice(3001, 50, replace=False)] = np.nan
    neg[rng.choice(2999, 70, replace=False)] = np.nan
    neg[:3] = [-np.inf, np.inf, -0.0]
    check(ctx, pos, neg)


def test_roc_large_and_ragged(ctx):
    rng = np.random.default_rng(9)
    pos = rng.normal(1.0, 1.0, 20011).astype(np.float32)
    neg = rng.normal(0.0, 1.0, 10007).astype(np.float32)   # several 2048-score tiles and a ragged tail
    r = check(ctx, pos, neg)
    assert 0.7 < r["auc"] < 0.8
    check(ctx, pos[:1], neg[:1], [0.0])


def test_star_level_pipeline(ctx):
    """Labelled stars through the batched box search; each star scored by its best period;
    the GPU ROC of those scores equals the oracle's, and the injections are detected."""
    import paper_2312_02063_gb300 as g
    ds = lcsynth.detection_stars(400, seed=77, n_cad=2048, snr=(8.0, 20.0))
    S, P = 400, 1500
    dev = ctx.device
    d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (ds.lc_offsets, ds.times, ds.flux)]
    grid = torch.from_numpy(lcsynth.freq_grid(P)).to(dev)
    periods = grid.repeat(S)
    goff = torch.arange(S + 1, dtype=torch.int64, device=dev) * P
    t0s = torch.zeros(S, dtype=torch.float64, device=dev)
    score = torch.empty(S * P, dtype=torch.float32, device=dev)
    bi = torch.empty(S, dtype=torch.int64, device=dev)
    bs = torch.empty(S, dtype=torch.float32, device=dev)
    g.gpfc_search_batched(ctx, d[0], d[1], d[2], goff, periods, 256, t0s, g.SCORER_BOX, score=score, best_index=bi,
                          best_score=bs, w_max=160)
    ctx.sync()
    best = bs.cpu().numpy()
    lab = ds.label == 1
    r = check(ctx, best[lab], best[~lab], [0.0, 0.01, 0.1])
    assert r["auc"] > 0.9, r["auc"]
