"""CPU checks of the fixed-point error bounds in tolerances.py, by brute force: fold the
same light curve with exact FP64 flux and with flux rounded to multiples of the unit q
(oracle bin indices, Sec. 2.3), score both with the oracle's box-SNR (Sec. 2.4) and compare
the differences with the derived bounds.
"""
import math

import numpy as np

import lcsynth
import oracle
from tolerances import box_atol, fixed_point_unit


def _fold_both(times, flux, t0, periods, nbins, q):
    f32 = np.asarray(flux, np.float32)
    fref = float(np.mean(f32.astype(np.float64)))
    x = (f32.astype(np.float64) - fref).astype(np.float32).astype(np.float64)
    xq = np.rint(x / q) * q
    B = oracle.bins(oracle.quantise_times(times, t0), oracle.quantise_periods(periods), nbins)
    xe = f32.astype(np.float64) - fref
    S = np.stack([np.bincount(b, weights=xe, minlength=nbins) for b in B])
    Sq = np.stack([np.bincount(b, weights=xq, minlength=nbins) for b in B])
    C = np.stack([np.bincount(b, minlength=nbins) for b in B])
    return S, Sq, C


def test_unit_keeps_a_full_chunk_in_32_bits():
    rng = np.random.default_rng(3)
    for n, scale in ((5000, 1e-3), (70000, 3.0), (1000, 1e5)):
        flux = (scale * (1.0 + rng.normal(0.0, 0.01, n))).astype(np.float32)
        q = fixed_point_unit(flux)
        x = flux.astype(np.float64) - float(np.mean(flux.astype(np.float64)))
        lim = math.floor((2**31 - 1) / min(65520, n))
        assert np.max(np.abs(np.rint(x / q))) <= lim  # the worst bin of a chunk fits
        assert np.max(np.abs(x)) * 2.0 / q > lim       # and q is the smallest such power of two
        assert math.log2(q) == round(math.log2(q))


def test_box_snr_error_has_the_derived_spread_and_stays_in_bound():
    # a loud star: its fixed-point unit is coarser than the float32 flux grid
    lc = lcsynth.light_curve_tiny(4096)
    rng = np.random.default_rng(5)
    flux = (1.0 + rng.normal(0.0, 5e-2, lc.times.shape[0])).astype(np.float32)
    q = fixed_point_unit(flux)
    assert q > np.max(np.spacing(np.abs(flux)))
    periods = lcsynth.freq_grid(600)
    S, Sq, C = _fold_both(lc.times, flux, lc.t0, periods, 256, q)
    sigma = float(np.std(flux.astype(np.float64)))
    a, _, _ = oracle.box_snr(S, C, 1, 108, sigma)
    b, _, _ = oracle.box_snr(Sq, C, 1, 108, sigma)
    unit = q / (sigma * math.sqrt(12.0))
    d = (b - a) / unit
    assert 0.8 < float(np.std(d)) < 1.2  # one unit of spread, as derived
    assert np.all(np.abs(b - a) <= box_atol(q, sigma))
    # the means: off by at most q/2
    nz = C > 0
    assert np.all(np.abs(Sq[nz] - S[nz]) / C[nz] <= q / 2 + 1e-15)


def test_flux_on_a_grid_finer_than_the_unit_only_shifts_the_means():
    lc = lcsynth.light_curve_tiny(4096)
    flux = lc.flux.astype(np.float32)  # quiet star near 1: float32 spacing no finer than q
    q = fixed_point_unit(flux)
    assert np.min(np.spacing(np.abs(flux))) >= q
    periods = lcsynth.freq_grid(200)
    S, Sq, C = _fold_both(lc.times, flux, lc.t0, periods, 64, q)
    nz = C > 0
    shift = (Sq[nz] - S[nz]) / C[nz]
    assert np.ptp(shift) <= 1e-12 * q * 64  # one common offset ...
    assert np.all(np.abs(shift) <= q / 2)   # ... below half a unit
    sigma = float(np.std(flux.astype(np.float64)))
    a, _, _ = oracle.box_snr(S, C, 1, 26, sigma)
    b, _, _ = oracle.box_snr(Sq, C, 1, 26, sigma)
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(a))  # the box-SNR does not move
