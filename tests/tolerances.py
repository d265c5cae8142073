"""Error bounds of the GPU fold's fixed-point arithmetic (fold layout 3, the default from
256 bins), derived here so the parity tests can state them.

The fold sums x = float32(flux - mean(flux)) in units q = 2^-e, with e per star the largest
integer such that max|x| 2^e <= floor((2^31 - 1) / min(chunk, n)) (chunk = 65,520 samples
by default): every chunk's bin sum then fits in 32 bits and the integer sums are exact, so
the only error is each sample's rounding x -> q rint(x / q), at most q/2.

* A bin mean (sum / count) is therefore off by at most q/2.
* The box-SNR of a box (Sec. 2.4), (S n_in - S_in N) / (sigma sqrt(N n_in n_out)), changes
  by sum_i eps_i w_i / (sigma sqrt(N n_in n_out)), with eps_i the rounding errors and
  w_i = n_in - N [i in box]. Since sum_i w_i^2 = n_out n_in^2 + n_in n_out^2 = N n_in n_out,
  independent rounding errors (uniform on [-q/2, q/2], variance q^2/12) give the change a
  standard deviation of q / (sigma sqrt(12)) whatever the box. The tests allow eight of
  those on top of the FP32 tolerance of the box search.

Where the flux is a float32 whose spacing (ulp) is no finer than q, every flux value is a
multiple of q, so x / q has the same fraction for every sample: the rounding errors are all
equal, the box-SNR does not change at all and the means move by one common offset below
q/2 (the usual case of photometry normalised to 1 with a quiet star).
"""
import math

import numpy as np

DEFAULT_CHUNK = 65520


def fixed_point_unit(flux, chunk=DEFAULT_CHUNK):
    """q = 2^-e of a star's fixed-point flux, as defined above."""
    f32 = np.asarray(flux, np.float32)
    x = (f32.astype(np.float64) - float(np.mean(f32.astype(np.float64)))).astype(np.float32).astype(np.float64)
    xm = float(np.max(np.abs(x)))
    if xm == 0.0:
        return 1.0
    lim = math.floor((2**31 - 1) / min(chunk, x.shape[0]))
    e = math.floor(math.log2(lim / xm))
    while xm * 2.0 ** (e + 1) <= lim:
        e += 1
    while xm * 2.0 ** e > lim:
        e -= 1
    return 2.0 ** -e


def box_atol(q, sigma, k=8.0):
    """Absolute box-SNR allowance for flux rounded to multiples of q: k standard deviations."""
    return k * q / (sigma * math.sqrt(12.0))
