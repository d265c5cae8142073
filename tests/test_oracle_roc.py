"""Pins of oracle.roc (star-level detection statistics, Sec. 3.2): brute force over all
pairs on small sets with many ties and NaNs, closed forms, agreement with the existing
threshold rule (oracle.tpr_at_fpr) and, where scikit-learn is installed, its AUC."""
import numpy as np
import pytest

import oracle


def brute(pos, neg, fprs):
    pos = [(-np.inf if np.isnan(v) else float(v)) for v in pos]
    neg = [(-np.inf if np.isnan(v) else float(v)) for v in neg]
    u2 = sum(2 * (a > b) + (a == b) for a in pos for b in neg)
    out = []
    for f in fprs:
        k = int(np.floor(f * len(neg)))
        srt = sorted(neg, reverse=True)
        t = srt[k] if k < len(neg) else -np.inf
        out.append((t, sum(a > t for a in pos)))
    return u2, out


@pytest.mark.parametrize("seed", range(6))
def test_roc_matches_pairwise_brute_force_with_ties_and_nan(seed):
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, 12, 37).astype(np.float32)
    neg = rng.integers(0, 10, 41).astype(np.float32)
    pos[rng.choice(37, 3, replace=False)] = np.nan
    neg[rng.choice(41, 4, replace=False)] = np.nan
    fprs = [0.0, 0.01, 0.1, 0.25, 0.5, 0.9, 0.999]
    r = oracle.roc(pos, neg, fprs)
    u2, tt = brute(pos, neg, fprs)
    assert r["u2"] == u2
    assert r["auc"] == u2 / (2.0 * 37 * 41)
    for (t, tp), t2, tp2 in zip(tt, r["thr"], r["tp"]):
        assert t == t2 and tp == tp2


def test_roc_closed_forms():
    a = np.arange(10, dtype=np.float32)
    assert oracle.roc(a + 100, a)["auc"] == 1.0          # perfect separation
    assert oracle.roc(a, a + 100)["auc"] == 0.0          # reversed
    assert oracle.roc(np.ones(7), np.ones(5))["auc"] == 0.5   # all tied
    assert oracle.roc([np.nan], [np.nan])["auc"] == 0.5      # NaN ties NaN
    r = oracle.roc([5.0, 1.0], [2.0, 3.0, 4.0], [0.0, 1 / 3, 0.99])
    # thresholds: largest negative, 2nd largest, 3rd largest (k = 0, 1, 2)
    assert list(r["thr"]) == [4.0, 3.0, 2.0] and list(r["tp"]) == [1, 1, 1]
    r = oracle.roc([5.0], [2.0], [1.0])                  # k = n_neg: every score counts
    assert r["thr"][0] == -np.inf and r["tp"][0] == 1


def test_roc_threshold_rule_equals_tpr_at_fpr():
    rng = np.random.default_rng(3)
    pos, neg = rng.normal(1, 1, 500), rng.normal(0, 1, 2000)
    for f in (1e-3, 1e-2, 0.1):
        tpr, thr = oracle.tpr_at_fpr(pos, neg, f)
        r = oracle.roc(pos, neg, [f])
        assert r["thr"][0] == thr and r["tpr"][0] == tpr


def test_roc_auc_matches_scikit_learn():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(4)
    pos = np.round(rng.normal(0.6, 1, 300), 1)
    neg = np.round(rng.normal(0.0, 1, 400), 1)               # ties across and within classes
    y = np.r_[np.ones(300), np.zeros(400)]
    assert abs(oracle.roc(pos, neg)["auc"] - metrics.roc_auc_score(y, np.r_[pos, neg])) < 1e-12
