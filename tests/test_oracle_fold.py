"""Pins for the oracle's fold (phase, bins, counts, sums, means).

Each test checks the oracle against something other than its own formula: the
paper's phase definition frac((t - t0)/P) in exact rational arithmetic, closed-form
bin layouts, invariants, and the noise-free transit recovery of Sec. 2.1.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import lcsynth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def exact_bin(t, t0, P, nbins):
    """floor(frac((t - t0)/P) * nbins) on the exact values of the doubles t, t0, P."""
    q = (Fraction(t) - Fraction(t0)) / Fraction(P)
    frac = q - math.floor(q)
    return math.floor(frac * nbins), frac


def test_bins_match_exact_phase_when_quantisation_is_exact():
    # t - t0 on the 2^-24 grid and P a power of two make tau and F exact, so the
    # fixed-point bin must equal the paper's phase definition exactly, at every edge.
    rng = np.random.default_rng(1)
    t0 = 3.0
    tau = rng.integers(-2 ** 34, 2 ** 34, 400)
    times = t0 + tau.astype(np.float64) / 2 ** 24
    assert np.all((times - t0) * 2 ** 24 == tau)  # exactly representable
    periods = np.array([2.0 ** e for e in range(-6, 7)])
    for nbins in (2, 3, 7, 64, 100, 256, 4096):
        mean, cnt, _ = oracle.fold(times, np.ones_like(times, np.float32), periods, nbins, t0)
        b = oracle.bins(oracle.quantise_times(times, t0), oracle.quantise_periods(periods), nbins)
        for k, P in enumerate(periods):
            ref = np.array([exact_bin(t, t0, P, nbins)[0] for t in times])
            np.testing.assert_array_equal(b[k], ref)
            np.testing.assert_array_equal(cnt[k], np.bincount(ref, minlength=nbins))


def test_bins_match_exact_phase_up_to_quantisation_bound():
    # General doubles: the fixed-point phase differs from frac((t-t0)/P) by at most
    # eps = 2^-25/P + |t-t0| 2^-41 (+ FP64 rounding). Disagreements must sit within
    # eps of a bin edge, and be rare.
    rng = np.random.default_rng(2)
    times = np.sort(rng.uniform(0.0, 1500.0, 300))
    t0 = float(times[0]) - rng.uniform(0, 5)
    periods = rng.uniform(0.2, 1.0, 25)
    tau = oracle.quantise_times(times, t0)
    F = oracle.quantise_periods(periods)
    mism = 0
    for nbins in (64, 256, 100):
        b = oracle.bins(tau, F, nbins)
        for k, P in enumerate(periods):
            for i, t in enumerate(times):
                eb, frac = exact_bin(t, t0, P, nbins)
                if b[k, i] != eb:
                    mism += 1
                    eps = 2.0 ** -25 / P + abs(t - t0) * 2.0 ** -41 + 1e-15 * abs(t - t0) / P
                    x = frac * nbins
                    dist = min(abs(x - math.floor(x)), abs(math.ceil(x) - x)) / nbins
                    assert dist <= 2 * eps, (nbins, k, i, dist, eps)
                    assert (b[k, i] - eb) % nbins in (1, nbins - 1)
    assert mism <= 2


def test_negative_times_wrap_like_the_phase():
    # t < t0 gives negative tau; two's-complement wrap must still give frac((t-t0)/P).
    t0 = 10.0
    times = t0 - np.array([1, 3, 5, 1000, 2 ** 20 + 7], np.float64) / 2 ** 24 * 1000
    periods = np.array([0.5, 0.25, 1.0])
    b = oracle.bins(oracle.quantise_times(times, t0), oracle.quantise_periods(periods), 256)
    for k, P in enumerate(periods):
        np.testing.assert_array_equal(b[k], [exact_bin(t, t0, P, 256)[0] for t in times])


def test_golden_even_spread_gives_256_per_bin():
    g = json.load(open(GOLDEN))["bins_per_fold_example"]
    n, nb = g["n_samples"], g["nbins"]
    # P = 1 d and t_i = i/256 d put sample i at phase i/256 exactly: every bin gets n/nb.
    times = np.arange(n, dtype=np.float64) / 256.0
    flux = np.ones(n, np.float32)
    mean, cnt, s = oracle.fold(times, flux, np.array([1.0]), nb, 0.0)
    assert np.all(cnt == g["samples_per_bin"])
    np.testing.assert_array_equal(np.nonzero(cnt[0])[0], np.arange(nb))


def test_count_and_sum_invariants():
    lc = lcsynth.light_curve_tiny(7)
    periods = lcsynth.freq_grid(300)
    mean, cnt, s = oracle.fold(lc.times, lc.flux, periods, 64, lc.t0)
    n = lc.times.shape[0]
    assert np.all(cnt.sum(axis=1) == n)
    tot = float(np.sum(lc.flux.astype(np.float64)))
    np.testing.assert_allclose(s.sum(axis=1), tot, rtol=1e-13)
    nz = cnt > 0
    np.testing.assert_allclose(mean[nz] * cnt[nz], s[nz], rtol=1e-15)
    assert np.all(np.isnan(mean[~nz]))


def test_constant_flux_gives_the_constant():
    times = np.sort(np.random.default_rng(3).uniform(0, 90, 1000))
    flux = np.full(times.shape, 0.9993, np.float32)
    mean, cnt, _ = oracle.fold(times, flux, lcsynth.freq_grid(50), 256, 0.0)
    nz = cnt > 0
    assert np.all(mean[nz] == np.float64(np.float32(0.9993)))


def test_noise_free_box_recovered_at_true_period():
    # Sec. 2.1: at the true period the fold shows the transit. Bins whose phase interval
    # lies wholly inside the box hold exactly 1 - depth; bins wholly outside hold 1.
    n, dt = 4096, lcsynth.CADENCE_D
    times = np.arange(n) * dt
    P, depth, dur, epoch = 0.7, 3e-4, 1.0 / 24.0, 0.2345
    inbox = lcsynth.box_mask(times, P, epoch, dur)
    flux = np.where(inbox, np.float32(1.0 - depth), np.float32(1.0)).astype(np.float32)
    nb = 64
    mean, cnt, _ = oracle.fold(times, flux, np.array([P]), nb, 0.0)
    centre = (epoch / P) % 1.0
    half = 0.5 * dur / P
    lo, hi = centre - half, centre + half
    margin = 1e-6
    inside = outside = 0
    for b in range(nb):
        a0, a1 = b / nb, (b + 1) / nb
        # distance on the circle between the bin interval and the box interval
        fully_in = any(lo + s + margin <= a0 and a1 <= hi + s - margin for s in (-1, 0, 1))
        overlaps = any(a0 < hi + s + margin and lo + s - margin < a1 for s in (-1, 0, 1))
        if cnt[0, b] == 0:
            continue
        if fully_in:
            inside += 1
            assert mean[0, b] == np.float64(np.float32(1.0 - depth))
        elif not overlaps:
            outside += 1
            assert mean[0, b] == 1.0
    assert inside >= 2 and outside >= nb - 8
    bmin = int(np.nanargmin(mean[0]))
    a0, a1 = bmin / nb, (bmin + 1) / nb
    assert any(a0 < hi + s and lo + s < a1 for s in (-1, 0, 1))


def test_folding_noise_attenuation_matches_sec21():
    g = json.load(open(GOLDEN))["fold_noise_attenuation"]
    # The paper's 1/sqrt(N) with N = T/p folded cycles, at the two ends of the range.
    lo = 1.0 / math.sqrt(g["T_days"] / g["p_min"])
    hi = 1.0 / math.sqrt(g["T_days"] / g["p_max"])
    assert round(lo, 2) == g["lo"] and round(hi, 2) == g["hi"]
    # The oracle's fold of white noise (one sample per cycle per bin on average at
    # this cadence ratio) has per-bin mean scatter sigma/sqrt(count).
    rng = np.random.default_rng(5)
    n = 65536
    times = np.arange(n) * lcsynth.CADENCE_D
    sig = 1e-3
    flux = (1.0 + rng.normal(0, sig, n)).astype(np.float32)
    mean, cnt, _ = oracle.fold(times, flux, np.array([0.7123]), 256, 0.0)
    z = (mean[0] - 1.0) * np.sqrt(cnt[0]) / sig
    assert 0.85 < np.std(z) < 1.15


def test_grid_sizing_eq1_and_grid_endpoints():
    g = json.load(open(GOLDEN))["grid_sizing_eq1"]
    assert int(g["N_o"] * g["T_days"] / g["L_days"]) == g["N_sample"]
    p = lcsynth.freq_grid(2000)
    assert p[0] == 1.0 and abs(p[-1] - 0.2) < 1e-15
    f = 1.0 / p
    assert np.allclose(np.diff(f), 4.0 / 1999, rtol=1e-9)


def test_naive_fp64_phase_agrees_except_at_edges():
    # The FP64 evaluation of frac((t-t0)/P) and the fixed-point bins may disagree only
    # for samples whose exact phase lies on (or within ~1e-6 of) a bin edge. Regular
    # cadence and a rational frequency grid put some samples exactly on edges.
    lc = lcsynth.light_curve_tiny(11)
    periods = lcsynth.freq_grid(200)
    b_fixed = oracle.bins(oracle.quantise_times(lc.times, lc.t0), oracle.quantise_periods(periods), 64)
    b_naive = oracle.bins_naive_fp64(lc.times, periods, 64, lc.t0)
    ks, iis = np.nonzero(b_fixed != b_naive)
    assert len(ks) < 1e-3 * b_fixed.size
    for k, i in zip(ks, iis):
        _, frac = exact_bin(lc.times[i], lc.t0, periods[k], 64)
        x = frac * 64
        assert min(x - math.floor(x), math.ceil(x) - x) < 1e-6 * 64


def test_fixed_point_range_errors():
    with pytest.raises(ValueError):
        oracle.quantise_periods(np.array([0.0]))
    with pytest.raises(ValueError):
        oracle.quantise_periods(np.array([np.nan]))
    with pytest.raises(ValueError):
        oracle.quantise_times(np.array([3e11]), 0.0)
