"""Pins of the oracle's two-tier equal-count fold (Sec. 2.3, Fig. 4 (a)-(e)).

* The paper presents the two-tier fold as an emulation of the sort-based fold (sort the
  samples by phase, put n/nbins consecutive samples in each bin). With at most one sample
  per fine bin and n a multiple of nbins the two are the same computation: checked bit
  for bit against a sort of the samples.
* With several samples per fine bin and boundaries inside fine bins, each final bin is
  computed independently as an interval overlap in exact rationals (fractions.Fraction):
  fine bin f covers [C(f-1), C(f)) in cumulative samples, final bin j covers
  [j n/nbins, (j+1) n/nbins), and f gives j the share overlap/c_f of its flux sum.
* Conservation: the final sums add up to the total flux; the fine counts are the
  equal-width fold's counts.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def test_sort_based_fold_when_fine_bins_hold_single_samples():
    rng = np.random.default_rng(3)
    nfine, nbins, n = 4096, 16, 64
    fine = rng.choice(nfine, n, replace=False)
    cycles = rng.integers(0, 50, n)
    # period 1 d: the phase of (cycle + (f + 1/2) / nfine) d is exactly (f + 1/2) / nfine
    times = cycles + (fine + 0.5) / nfine
    flux = (1.0 + rng.normal(0, 1e-3, n)).astype(np.float32)
    mean, fc = oracle.fold_equal_count(times, flux, np.array([1.0]), nfine, nbins, 0.0)
    assert fc.max() == 1 and fc.sum() == n
    order = np.argsort(fine)
    per = n // nbins
    expect = np.empty(nbins)
    for j in range(nbins):
        acc = 0.0
        for i in order[j * per:(j + 1) * per]:
            acc += float(flux[i])
        expect[j] = acc / (n / nbins)
    np.testing.assert_array_equal(mean[0], expect)


def _exact_two_tier(times, flux, periods, nfine, nbins, t0):
    tau = oracle.quantise_times(times, t0)
    F = oracle.quantise_periods(periods)
    out = []
    for Fk in F:
        c = [0] * nfine
        s = [Fraction(0)] * nfine
        for ti, xi in zip(tau, flux):
            phase = Fraction((int(ti) * int(Fk)) % (1 << 64), 1 << 64)
            f = int(phase * nfine)  # floor
            c[f] += 1
            s[f] += Fraction(float(xi))
        n = len(times)
        width = Fraction(n, nbins)
        row = []
        for j in range(nbins):
            lo, hi = j * width, (j + 1) * width
            acc = Fraction(0)
            C = 0
            for f in range(nfine):
                a, b = C, C + c[f]
                C = b
                ov = min(b, hi) - max(a, lo)
                if c[f] and ov > 0:
                    acc += s[f] * ov / c[f]
            row.append(acc / width)
        out.append(row)
    return out


@pytest.mark.parametrize("n,nfine,nbins,seed", [(23, 16, 5, 1), (40, 32, 7, 2), (17, 8, 8, 3), (5, 64, 3, 4)])
def test_matches_exact_rational_interval_overlap(n, nfine, nbins, seed):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 30, n))
    flux = (1.0 + rng.normal(0, 1e-2, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, 3)
    mean, fc = oracle.fold_equal_count(times, flux, periods, nfine, nbins, 0.0)
    exact = _exact_two_tier(times, flux, periods, nfine, nbins, 0.0)
    for k in range(len(periods)):
        for j in range(nbins):
            e = float(exact[k][j])
            assert abs(mean[k, j] - e) <= 1e-12 * abs(e), (k, j, mean[k, j], e)


def test_conservation_and_fine_counts():
    rng = np.random.default_rng(9)
    n = 3001
    times = np.sort(rng.uniform(0, 200, n))
    flux = (1.0 + rng.normal(0, 5e-4, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, 20)
    mean, fc = oracle.fold_equal_count(times, flux, periods, 4096, 256, 0.0)
    total = float(np.sum(flux.astype(np.float64)))
    np.testing.assert_allclose(mean.sum(axis=1) * (n / 256), total, rtol=1e-12)
    _, cnt, _ = oracle.fold(times, flux, periods, 4096, 0.0)
    np.testing.assert_array_equal(fc, cnt)
    assert np.all(np.isfinite(mean))  # equal-count bins are never empty


def test_constant_flux_and_the_sec23_example():
    # Sec. 2.3: 65,536 samples over 256 bins put 65536/256 = 256 samples in each bin
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["two_tier_example"]
    n, nbins = g["n_samples"], g["nbins"]
    assert n // nbins == g["samples_per_bin"]
    rng = np.random.default_rng(5)
    times = np.arange(n) * (29.4 / 1440.0)
    flux = np.full(n, 1.25, np.float32)
    mean, fc = oracle.fold_equal_count(times, flux, np.array([0.7, rng.uniform(0.2, 1.0)]), 4096, nbins, 0.0)
    np.testing.assert_allclose(mean, 1.25, rtol=1e-14)
