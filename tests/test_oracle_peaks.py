"""Pins of the oracle's per-star decision layer: SDE (Eq. 3) and the peak rule of Sec. 4.2
(runs above mean + 3 sd, wider than 3 periods), with harmonic flags (Fig. 14).

* SDE of N - 1 zeros and one spike h is sqrt(N - 1) exactly (population sd), whatever h.
* mean / sd equal numpy's mean / std (ddof 0) over the finite scores.
* Constructed periodograms with rectangular bumps of known widths and heights: which
  qualify, their order, the best index, ties, NaN/-inf handling, harmonic flags.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("N,h", [(10, 1.0), (1000, 7.5), (250000, 0.3)])
def test_sde_of_a_single_spike_is_sqrt_n_minus_1(N, h):
    s = np.zeros(N, np.float32)
    s[N // 3] = h
    r = oracle.peaks(s, np.linspace(0.2, 1.0, N))
    assert abs(r["sde"] - math.sqrt(N - 1)) <= 1e-9 * math.sqrt(N)


def test_statistics_match_numpy_over_finite_scores():
    rng = np.random.default_rng(1)
    s = rng.normal(0.3, 0.1, 5000).astype(np.float32)
    s[[5, 70, 900]] = [np.nan, -np.inf, np.inf]
    fin = s[np.isfinite(s)].astype(np.float64)
    r = oracle.peaks(s, np.linspace(0.2, 1.0, 5000))
    assert abs(r["mean"] - fin.mean()) <= 1e-12
    assert abs(r["sd"] - fin.std()) <= 1e-12
    assert abs(r["sde"] - (fin.max() - fin.mean()) / fin.std()) <= 1e-9


def bumps(N, spec):
    s = np.zeros(N, np.float32)
    for start, width, height in spec:
        s[start:start + width] = height
    return s


def test_peak_rule_width_more_than_three_and_order():
    s = bumps(1000, [(100, 3, 10.0), (300, 4, 9.0), (600, 6, 8.0)])
    s[603] = 8.5
    r = oracle.peaks(s, np.linspace(0.2, 1.0, 1000))
    assert r["n_peaks"] == 2
    assert r["best_index"] == 300
    assert list(r["index"]) == [300, 603]
    assert list(r["width"]) == [4, 6]
    np.testing.assert_array_equal(r["height"], np.float32([9.0, 8.5]))


def test_ties_go_to_the_smaller_index_and_no_peak_case():
    s = bumps(500, [(50, 5, 4.0), (200, 5, 4.0)])
    r = oracle.peaks(s, np.linspace(0.2, 1.0, 500))
    assert list(r["index"]) == [50, 200] and r["best_index"] == 50
    flat = np.full(500, 2.0, np.float32)
    r = oracle.peaks(flat, np.linspace(0.2, 1.0, 500))
    assert r["best_index"] == -1 and r["n_peaks"] == 0 and r["sde"] == 0.0


def test_non_finite_scores_break_runs():
    s = bumps(1000, [(100, 9, 6.0)])
    s[104] = np.nan  # splits the 9-wide run into 4 + 4
    r = oracle.peaks(s, np.linspace(0.2, 1.0, 1000))
    assert r["n_peaks"] == 2 and list(r["width"]) == [4, 4] and list(r["index"]) == [100, 105]
    s[104] = -np.inf
    r2 = oracle.peaks(s, np.linspace(0.2, 1.0, 1000))
    assert r2["n_peaks"] == 2


def test_harmonic_flags():
    N = 2000
    periods = np.linspace(0.1, 2.0, N)
    best = 500
    Pb = periods[best]

    def at(P):
        return int(np.argmin(np.abs(periods - P)))

    spec = [(best - 2, 5, 10.0), (at(2 * Pb) - 2, 5, 8.0), (at(Pb / 2) - 2, 5, 7.0), (at(3 * Pb) - 2, 5, 6.0),
            (at(2.5 * Pb) - 2, 5, 5.5)]
    s = bumps(N, spec)
    for start, width, height in spec:
        s[start + 2] = height + 0.25  # each peak's maximum at its centre
    r = oracle.peaks(s, periods, harmonic_tol=2e-3)
    assert r["best_index"] == best
    flags = dict(zip(r["index"].tolist(), r["harmonic"].tolist()))
    assert flags[best] == 1
    assert flags[at(2 * Pb)] == 2
    assert flags[at(Pb / 2)] == -2
    assert flags[at(3 * Pb)] == 3
    assert flags[at(2.5 * Pb)] == 0
