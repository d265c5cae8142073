"""GPU parity of the two-tier equal-count fold (Sec. 2.3) against the FP64 oracle.

Tolerance: bin means within 1e-6 relative (the fold's mean tolerance). The GPU sums in
exact fixed point (quantum 2^-k per light curve), the oracle in FP64.
"""
import math

import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

MEAN_RTOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


def gpu_eq(ctx, times, flux, periods, nfine, nbins, t0):
    import paper_2312_02063_gb300 as g
    out = g.gpfc_fold_equal_count(ctx, _dev(ctx, times), _dev(ctx, flux.astype(np.float32)), _dev(ctx, periods),
                                  nbins, nfine, t0)
    ctx.sync()
    return out.cpu().numpy().astype(np.float64)


def check(got, mean_o):
    assert np.all(np.isfinite(got))
    err = np.abs(got - mean_o)
    assert np.all(err <= MEAN_RTOL * np.abs(mean_o)), float(np.max(err / np.abs(mean_o)))


@pytest.mark.parametrize("n,npd,nfine,nbins", [(1, 3, 4096, 256), (100, 7, 4096, 256), (255, 9, 4096, 256),
                                               (4096 * 3 + 17, 13, 4096, 256), (3001, 20, 1000, 100),
                                               (7, 5, 16, 5), (20011, 31, 2048, 64), (65536, 4, 4096, 256)])
def test_two_tier_ragged_sizes(ctx, n, npd, nfine, nbins):
    rng = np.random.default_rng(n + npd + nfine + nbins)
    times = np.sort(rng.uniform(0.0, 1300.0, n))
    flux = (1.0 + rng.normal(0, 3e-4, n)).astype(np.float32)
    periods = rng.uniform(0.2, 1.0, npd)
    t0 = float(rng.uniform(-3, 3))
    got = gpu_eq(ctx, times, flux, periods, nfine, nbins, t0)
    mean_o, _ = oracle.fold_equal_count(times, flux, periods, nfine, nbins, t0)
    check(got, mean_o)


def test_two_tier_full_length_star_sampled_periods(ctx):
    lc = lcsynth.light_curve_kepler()
    periods = lcsynth.freq_grid(19456)
    got = gpu_eq(ctx, lc.times, lc.flux, periods, 4096, 256, lc.t0)
    idx = np.random.default_rng(2).choice(len(periods), 12, replace=False)
    mean_o, _ = oracle.fold_equal_count(lc.times, lc.flux, periods[idx], 4096, 256, lc.t0)
    check(got[idx], mean_o)
    # equal-count bins: every bin holds n/256 samples, so the bin means average to the flux mean
    np.testing.assert_allclose(got.mean(axis=1), np.mean(lc.flux.astype(np.float64)), rtol=1e-6)


def test_two_tier_sort_based_case_and_determinism(ctx):
    rng = np.random.default_rng(3)
    nfine, nbins, n = 4096, 16, 64
    fine = rng.choice(nfine, n, replace=False)
    times = rng.integers(0, 50, n) + (fine + 0.5) / nfine
    flux = (1.0 + rng.normal(0, 1e-3, n)).astype(np.float32)
    got = gpu_eq(ctx, times, flux, np.array([1.0, 0.5]), nfine, nbins, 0.0)
    mean_o, _ = oracle.fold_equal_count(times, flux, np.array([1.0, 0.5]), nfine, nbins, 0.0)
    check(got, mean_o)
    again = gpu_eq(ctx, times, flux, np.array([1.0, 0.5]), nfine, nbins, 0.0)
    np.testing.assert_array_equal(got, again)


def test_two_tier_argument_errors(ctx):
    import paper_2312_02063_gb300 as g
    t = _dev(ctx, np.arange(10.0))
    f = _dev(ctx, np.ones(10, np.float32))
    p = _dev(ctx, np.array([0.5]))
    for nbins, nfine in ((256, 128), (1, 16), (256, 8192)):
        with pytest.raises(g.GpfcError):
            g.gpfc_fold_equal_count(ctx, t, f, p, nbins, nfine, 0.0)
    bad = _dev(ctx, np.array([0.5, -1.0]))
    g.gpfc_fold_equal_count(ctx, t, f, bad, 8, 64, 0.0)
    with pytest.raises(g.GpfcError) as ei:
        ctx.sync()
    assert ei.value.code == -4
