"""Pins of the pre-processing oracle (Sec. 2.2, Fig. 3): the B-spline basis against
SciPy's, the unclipped fit against SciPy's least-squares spline, exact recovery of trends
the spline space contains, segmentation by brute force on constructed gaps and jumps,
clipping of outliers, masking of known transits and the edge clipping count."""
import numpy as np
import pytest

import oracle
from oracle import preprocess as dt

CAD = 0.020428


def test_basis_matches_scipy_and_partitions_unity():
    interp = pytest.importorskip("scipy.interpolate")
    t = np.sort(np.random.default_rng(1).uniform(2.0, 9.0, 500))
    t[0], t[-1] = 2.0, 9.0
    k = dt.knot_vector(2.0, 9.0, 1.3)
    B = dt.bspline_design(t, k)
    ref = interp.BSpline.design_matrix(t, k, 3).toarray()
    assert np.max(np.abs(B - ref)) < 1e-13
    assert np.max(np.abs(B.sum(axis=1) - 1.0)) < 1e-13


def test_unclipped_fit_equals_scipy_least_squares_spline():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(2)
    t = np.arange(1200) * CAD
    f = 1 + 0.01 * np.sin(t / 3.0) + rng.normal(0, 1e-3, t.size)
    k = dt.knot_vector(t[0], t[-1], 1.0)
    ref = interp.make_lsq_spline(t, f, k, 3)(t)
    _, trend, kept, p = dt.fit_segment(t, f, np.zeros(t.size, bool), 1.0, clip_sigma=np.inf, ridge=0.0)
    assert kept.all() and p == len(k) - 4
    assert np.max(np.abs(trend - ref)) < 1e-12
    # with the default penalty the fit moves by far less than the noise
    _, trend2, _, _ = dt.fit_segment(t, f, np.zeros(t.size, bool), 1.0, clip_sigma=np.inf)
    assert np.max(np.abs(trend2 - ref)) < 1e-8


def test_trend_in_the_spline_space_is_removed_exactly():
    t = np.arange(2500) * CAD
    trend = 1.0 + 1e-3 * (t / 10) - 2e-4 * (t / 10) ** 2 + 3e-5 * (t / 10) ** 3   # a cubic
    r = oracle.detrend(t, trend)
    assert len(r["starts"]) == 1
    assert np.max(np.abs(r["flux"] - 1.0)) < 1e-9
    # a B-spline on the knots of one candidate spacing, with noise of 1e-9: recovered to it
    k = dt.knot_vector(t[0], t[-1], 1.5)
    c = 1 + 0.01 * np.random.default_rng(8).normal(size=len(k) - 4)
    sp = dt.bspline_design(t, k) @ c
    r = oracle.detrend(t, sp * (1 + 1e-9 * np.random.default_rng(9).normal(size=t.size)), spacings=(1.5,))
    assert np.max(np.abs(r["flux"] - 1.0)) < 1e-8
    assert len(r["flux"]) == 2500 - 60 and np.array_equal(r["index"], np.arange(30, 2470))


def test_segmentation_brute_force():
    rng = np.random.default_rng(3)
    t = np.cumsum(np.where(rng.random(3000) < 0.003, 1.0, CAD))       # gaps of 1 d
    f = 1 + rng.normal(0, 1e-4, 3000)
    f[1700] += 0.05                      # a spike: two adjacent jumps far beyond 5 sigma
    s, e = dt.segments(t, f)
    sig = np.std(f)
    want = [0] + [i for i in range(1, 3000) if t[i] - t[i - 1] > 30 * CAD or abs(f[i] - f[i - 1]) > 5 * sig]
    assert list(s) == want and 1700 in want and 1701 in want and list(e) == want[1:] + [3000]
    assert sum(t[i] - t[i - 1] > 30 * CAD for i in range(1, 3000)) >= 3


def test_outliers_are_clipped_and_known_transits_masked():
    t = np.arange(3000) * CAD
    base = 1.0 + 2e-3 * np.sin(t / 9.0)
    f = base.copy()
    f[1500] += 3e-3                      # an outlier: 300 sigma of the residuals, below the flux gap
    m = np.zeros(3000, bool)
    m[800:830] = True
    f[800:830] *= 1 - 5e-3               # a known transit, masked
    rng = np.random.default_rng(4)
    f = f + rng.normal(0, 1e-5, 3000)
    r = oracle.detrend(t, f, m)
    out = np.full(3000, np.nan)
    out[r["index"]] = r["flux"]
    quiet = np.ones(3000, bool)
    quiet[[1500]] = False
    quiet[800:830] = False
    quiet[:30] = quiet[-30:] = False
    assert np.max(np.abs(out[quiet] - 1)) < 2e-4
    assert abs(out[1500] - (1 + 3e-3 / base[1500])) < 2e-4   # the outlier stays in the output
    assert len(r["starts"]) == 1
    assert np.max(np.abs(out[800:830] - (1 - 5e-3))) < 2e-4   # the transit depth survives


def test_short_segments_and_spacing_choice():
    t = np.r_[np.arange(50) * CAD, 10 + np.arange(4000) * CAD]   # a 50-point segment, dropped
    rng = np.random.default_rng(5)
    f = 1 + 0.02 * np.sin(t / 0.7) + rng.normal(0, 1e-4, t.size)  # fast variability
    r = oracle.detrend(t, f)
    assert np.isnan(r["spacing"][0]) and r["spacing"][1] == 0.5  # the finest knots win the BIC
    assert np.all(r["segment"] == 1) and len(r["flux"]) == 4000 - 60
    slow = 1 + 1e-3 * (t - 10) / 80 + rng.normal(0, 1e-4, t.size)
    r2 = oracle.detrend(t, slow)
    assert r2["spacing"][1] == 3.0                                # a straight line: fewest coefficients
