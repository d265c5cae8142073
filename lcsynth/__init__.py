"""Seeded synthetic inputs for the GPFC fold + score path.

This module only draws random inputs with the shapes of Kepler long-cadence light
curves (paper Sec. 2.2 and Sec. 3: 29.4-min cadence, 30k-70k epochs; Table 2
ranges). It holds none of the method's arithmetic (no phase, no binning, no
scoring): both the FP64 oracle and the CUDA path receive the arrays it returns.

Every generator takes an explicit integer seed and uses NumPy's PCG64, so the
same call gives the same arrays on every machine.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Kepler long cadence, 29.4 minutes, in days (the workload's stated cadence).
CADENCE_D = 29.4 / 1440.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def freq_grid(n_periods: int, p_min: float = 0.2, p_max: float = 1.0) -> np.ndarray:
    """Trial periods uniform in frequency over [1/p_max, 1/p_min], endpoints included.

    Returns float64 periods P_k = 1/f_k with f_k = f_lo + k (f_hi - f_lo)/(n-1).
    """
    f_lo, f_hi = 1.0 / p_max, 1.0 / p_min
    if n_periods == 1:
        return np.array([1.0 / f_lo])
    k = np.arange(n_periods, dtype=np.float64)
    f = f_lo + k * (f_hi - f_lo) / (n_periods - 1)
    return 1.0 / f


def period_grid(n_periods: int, p_min: float = 0.2, p_max: float = 1.0) -> np.ndarray:
    """Trial periods uniform in period (the paper's own grid form, Sec. 2.1)."""
    return np.linspace(p_min, p_max, n_periods, dtype=np.float64)


def box_mask(t: np.ndarray, period: float, epoch: float, duration: float) -> np.ndarray:
    """True where t lies within duration/2 of a mid-transit time epoch + j*period."""
    d = np.mod(t - epoch + 0.5 * period, period) - 0.5 * period
    return np.abs(d) < 0.5 * duration


@dataclasses.dataclass
class LightCurve:
    times: np.ndarray      # float64 [N], days
    flux: np.ndarray       # float32 [N], relative flux
    t0: float              # phase origin used by the workload
    truth: dict            # injected parameters (empty dict if none)


def _gaps(rng: np.random.Generator, n_cad: int, frac: float, lo_d: float, hi_d: float) -> np.ndarray:
    """Keep-mask after dropping seeded gaps of U[lo_d, hi_d] days until >= frac removed."""
    keep = np.ones(n_cad, dtype=bool)
    span = n_cad * CADENCE_D
    while (~keep).mean() < frac:
        start = rng.uniform(0.0, span)
        length = rng.uniform(lo_d, hi_d)
        a = int(start / CADENCE_D)
        b = min(n_cad, int((start + length) / CADENCE_D) + 1)
        keep[a:b] = False
    return keep


def light_curve_tiny(seed: int = 20231204) -> LightCurve:
    """4,096 cadences from t0 = 0, no gaps, white noise 1e-4, one box at P = 0.7 d.

    Box: depth 3e-4, duration 1 h, epoch uniform in [0, P).
    """
    rng = _rng(seed)
    n = 4096
    t = np.arange(n, dtype=np.float64) * CADENCE_D
    period, depth, dur = 0.7, 3e-4, 1.0 / 24.0
    epoch = rng.uniform(0.0, period)
    flux = 1.0 + rng.normal(0.0, 1e-4, n)
    flux = flux * np.where(box_mask(t, period, epoch, dur), 1.0 - depth, 1.0)
    return LightCurve(t, flux.astype(np.float32), 0.0,
                      dict(period=period, depth=depth, duration=dur, epoch=epoch))


def light_curve_kepler(seed: int = 20232204, n_cad: int = 65536, sigma_white: float = 2e-4,
                       ar_phi: float = 0.9, ar_sigma: float = 5e-5, gap_frac: float = 0.04,
                       inject: bool = True, depth_ppm=(50.0, 500.0), dur_h=(0.5, 2.0),
                       p_range=(0.2, 1.0)) -> LightCurve:
    """Full-length Kepler-like light curve.

    n_cad cadences at 29.4 min (65,536 -> ~1,338 d); ~gap_frac of cadences dropped in
    seeded 1-5 d gaps; white noise plus AR(1) red noise (ar_sigma is the marginal std,
    so the innovation std is ar_sigma*sqrt(1-phi^2)); one box transit with depth
    log-uniform in depth_ppm, duration uniform in dur_h hours, period uniform in
    p_range days, epoch uniform in [0, P). t0 = times[0] = 0.
    """
    rng = _rng(seed)
    t_all = np.arange(n_cad, dtype=np.float64) * CADENCE_D
    keep = _gaps(rng, n_cad, gap_frac, 1.0, 5.0)
    white = rng.normal(0.0, sigma_white, n_cad)
    innov = rng.normal(0.0, ar_sigma * np.sqrt(1.0 - ar_phi ** 2), n_cad)
    red = np.empty(n_cad)
    red[0] = rng.normal(0.0, ar_sigma)
    for i in range(1, n_cad):
        red[i] = ar_phi * red[i - 1] + innov[i]
    flux = 1.0 + white + red
    truth = {}
    if inject:
        depth = 1e-6 * np.exp(rng.uniform(np.log(depth_ppm[0]), np.log(depth_ppm[1])))
        dur = rng.uniform(dur_h[0], dur_h[1]) / 24.0
        period = rng.uniform(p_range[0], p_range[1])
        epoch = rng.uniform(0.0, period)
        flux = flux * np.where(box_mask(t_all, period, epoch, dur), 1.0 - depth, 1.0)
        truth = dict(period=period, depth=depth, duration=dur, epoch=epoch)
    return LightCurve(t_all[keep].copy(), flux[keep].astype(np.float32), 0.0, truth)


@dataclasses.dataclass
class DetectionSet:
    """Labelled stars (CSR) for the star-level detection comparison."""
    lc_offsets: np.ndarray    # int64 [S+1]
    times: np.ndarray         # float64 [sum N]
    flux: np.ndarray          # float32 [sum N]
    label: np.ndarray         # int8 [S]: 1 = one injected transit
    sigma: np.ndarray         # float64 [S]: white-noise standard deviation
    period: np.ndarray        # float64 [S]: injected period (NaN for label 0)
    snr: np.ndarray           # float64 [S]: target SNR of the injection (Eq. 2; NaN for label 0)
    epoch: np.ndarray         # float64 [S]: mid-transit epoch in [0, P) (NaN for label 0)
    duration: np.ndarray      # float64 [S]: transit duration in days (NaN for label 0)
    depth: np.ndarray         # float64 [S]: fractional depth (NaN for label 0)


def detection_stars(n_stars: int = 20000, seed: int = 20235404, n_cad: int = 4096, sigma=(1e-4, 1e-3),
                    snr=(4.0, 16.0), dur_h=(0.5, 3.0), p_range=(0.2, 1.0), gap_d=(1.0, 5.0),
                    chunk: int = 1024) -> DetectionSet:
    """Seeded labelled stars for star-level ROC curves (Sec. 3.2, Figs. 10-13): star s
    carries one box transit when s is odd, none when s is even (noise only).

    n_cad cadences at 29.4 min (t0 = 0) with two gaps of U[gap_d] days starting at uniform
    times (samples inside either are dropped); flux = 1 + white noise of sigma log-uniform in
    `sigma`; an injected box has period U[p_range] d, duration U[dur_h] h, epoch U[0, P) and
    depth d = snr sigma / sqrt(n q) with snr ~ U[snr], n the star's sample count and q the
    duty cycle dur / P (the SNR of Eq. 2); the flux is multiplied by (1 - d) in transit.
    Per-star parameters are drawn first for all stars (PCG64, `seed`); the noise comes
    from one generator per block of `chunk` stars (seed + 1 + block), so the set does not
    depend on how it is consumed.
    """
    rng = _rng(seed)
    S = int(n_stars)
    T = n_cad * CADENCE_D
    sig = np.exp(rng.uniform(np.log(sigma[0]), np.log(sigma[1]), S))
    g0 = rng.uniform(0.0, T, (S, 2))
    gl = rng.uniform(gap_d[0], gap_d[1], (S, 2))
    per = rng.uniform(p_range[0], p_range[1], S)
    dur = rng.uniform(dur_h[0], dur_h[1], S) / 24.0
    epo = rng.uniform(0.0, 1.0, S) * per
    tsnr = rng.uniform(snr[0], snr[1], S)
    label = (np.arange(S) % 2).astype(np.int8)
    t = np.arange(n_cad, dtype=np.float64) * CADENCE_D
    times, flux, lens = [], [], []
    for c0 in range(0, S, chunk):
        c1 = min(S, c0 + chunk)
        crng = _rng(seed + 1 + c0 // chunk)
        keep = np.ones((c1 - c0, n_cad), bool)
        for k in range(2):
            keep &= ~((t[None, :] >= g0[c0:c1, k, None]) & (t[None, :] < g0[c0:c1, k, None] + gl[c0:c1, k, None]))
        f = 1.0 + crng.normal(0.0, 1.0, (c1 - c0, n_cad)) * sig[c0:c1, None]
        n = keep.sum(axis=1)
        depth = tsnr[c0:c1] * sig[c0:c1] / np.sqrt(n * dur[c0:c1] / per[c0:c1])
        P = per[c0:c1, None]
        intr = np.abs(np.mod(t[None, :] - epo[c0:c1, None] + P / 2, P) - P / 2) < dur[c0:c1, None] / 2
        f = np.where(intr & (label[c0:c1, None] == 1), f * (1.0 - depth[:, None]), f)
        for r in range(c1 - c0):
            times.append(t[keep[r]])
            flux.append(f[r, keep[r]].astype(np.float32))
        lens.append(n)
    lens = np.concatenate(lens)
    off = np.zeros(S + 1, np.int64)
    off[1:] = np.cumsum(lens)
    inj = label == 1
    depth_all = tsnr * sig / np.sqrt(lens * dur / per)
    nan = np.nan
    return DetectionSet(off, np.concatenate(times), np.concatenate(flux), label, sig,
                        np.where(inj, per, nan), np.where(inj, tsnr, nan), np.where(inj, epo, nan),
                        np.where(inj, dur, nan), np.where(inj, depth_all, nan))


@dataclasses.dataclass
class StarBatch:
    """Many stars of uneven length, concatenated (CSR offsets)."""
    lc_offsets: np.ndarray    # int64 [S+1]
    times: np.ndarray         # float64 [sum N]
    flux: np.ndarray          # float32 [sum N]
    grid_offsets: np.ndarray  # int64 [S+1]
    periods: np.ndarray       # float64 [sum P]
    t0s: np.ndarray           # float64 [S]
    truths: list


def star_batch(n_stars: int = 1024, seed: int = 20235204, n_range=(8192, 70000),
               p_count_range=(20000, 250000), transit_frac: float = 0.3,
               sigma_range=(1e-4, 1e-3)) -> StarBatch:
    """Batch of stars with uneven lengths and grids (one frequency grid per star)."""
    rng = _rng(seed)
    lc_off = [0]
    g_off = [0]
    ts, fs, ps, t0s, truths = [], [], [], [], []
    for s in range(n_stars):
        n_cad = int(rng.integers(n_range[0], n_range[1] + 1))
        keep = _gaps(rng, n_cad, 0.04, 1.0, 5.0)
        t = np.arange(n_cad, dtype=np.float64) * CADENCE_D
        sig = np.exp(rng.uniform(np.log(sigma_range[0]), np.log(sigma_range[1])))
        flux = 1.0 + rng.normal(0.0, sig, n_cad)
        truth = dict(sigma=sig)
        if rng.uniform() < transit_frac:
            depth = 1e-6 * np.exp(rng.uniform(np.log(30.0), np.log(2000.0)))
            dur = rng.uniform(0.5, 3.0) / 24.0
            period = rng.uniform(0.2, 1.0)
            epoch = rng.uniform(0.0, period)
            flux = flux * np.where(box_mask(t, period, epoch, dur), 1.0 - depth, 1.0)
            truth.update(period=period, depth=depth, duration=dur, epoch=epoch)
        t, flux = t[keep], flux[keep]
        n_p = int(rng.integers(p_count_range[0], p_count_range[1] + 1))
        ts.append(t)
        fs.append(flux.astype(np.float32))
        ps.append(freq_grid(n_p))
        t0s.append(0.0)
        truths.append(truth)
        lc_off.append(lc_off[-1] + len(t))
        g_off.append(g_off[-1] + n_p)
    return StarBatch(np.array(lc_off, np.int64), np.concatenate(ts), np.concatenate(fs),
                     np.array(g_off, np.int64), np.concatenate(ps), np.array(t0s), truths)


def profiles_mixed(n: int, nbins: int = 256, seed: int = 20233204):
    """Folded-profile-like vectors: half boxes, half noise-only or sinusoids.

    Boxes: depth log-uniform 30-2,000 ppm, target SNR uniform 3-30 (Eq. 2 form,
    alpha = d*sqrt(w)/sigma_bin over the w in-box bins), width w = round(q*nbins) bins
    with q = duration/period, duration U[0.5, 3] h, period U[0.2, 1] d; the per-bin
    noise sigma_bin is set by the SNR target. Negatives: noise-only (sigma_bin
    log-uniform 1e-5..1e-3) or a sinusoid (amplitude 1e-4..1e-3, 1-5 cycles per
    profile, random phase) plus noise. Returns (profiles float32 [n][nbins], labels
    uint8 [n]).
    """
    rng = _rng(seed)
    out = np.empty((n, nbins), dtype=np.float32)
    lab = np.zeros(n, dtype=np.uint8)
    x = np.arange(nbins, dtype=np.float64)
    for j in range(n):
        if j % 2 == 0:
            depth = 1e-6 * np.exp(rng.uniform(np.log(30.0), np.log(2000.0)))
            snr = rng.uniform(3.0, 30.0)
            q = (rng.uniform(0.5, 3.0) / 24.0) / rng.uniform(0.2, 1.0)
            w = int(min(max(1, round(q * nbins)), nbins // 2))
            sig = depth * np.sqrt(w) / snr
            start = int(rng.integers(0, nbins))
            prof = 1.0 + rng.normal(0.0, sig, nbins)
            idx = (start + np.arange(w)) % nbins
            prof[idx] -= depth
            lab[j] = 1
        elif rng.uniform() < 0.5:
            sig = np.exp(rng.uniform(np.log(1e-5), np.log(1e-3)))
            prof = 1.0 + rng.normal(0.0, sig, nbins)
        else:
            amp = rng.uniform(1e-4, 1e-3)
            cyc = rng.uniform(1.0, 5.0)
            ph = rng.uniform(0.0, 2 * np.pi)
            sig = np.exp(rng.uniform(np.log(1e-5), np.log(1e-4)))
            prof = 1.0 + amp * np.sin(2 * np.pi * cyc * x / nbins + ph) + rng.normal(0.0, sig, nbins)
        out[j] = prof
    return out, lab


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


# Layer shapes of the scorer CNN, PyTorch layout: (name, shape, fan_in)
CNN_SHAPES = [
    ("conv1.w", (16, 1, 5), 5), ("conv1.b", (16,), None),
    ("conv2.w", (32, 16, 5), 80), ("conv2.b", (32,), None),
    ("conv3.w", (64, 32, 5), 160), ("conv3.b", (64,), None),
    ("fc1.w", (256, 2048), 2048), ("fc1.b", (256,), None),
    ("fc2.w", (1, 256), 256), ("fc2.b", (1,), None),
]


def cnn_init(seed: int = 20232304, bias_scale: float = 0.0) -> dict:
    """He-uniform weights U(+-sqrt(6/fan_in)), biases zero (or U(+-bias_scale)).

    Values are rounded to bfloat16-representable float32 so that every consumer sees
    the same numbers whatever precision it computes in.
    """
    rng = _rng(seed)
    out = {}
    for name, shape, fan_in in CNN_SHAPES:
        if fan_in is None:
            v = rng.uniform(-bias_scale, bias_scale, shape) if bias_scale > 0 else np.zeros(shape)
        else:
            lim = np.sqrt(6.0 / fan_in)
            v = rng.uniform(-lim, lim, shape)
        out[name] = round_to_bf16(v.astype(np.float32))
    return out


# ---------------------------------------------------------------- counter-based generator

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11): 4 x 32-bit counter,
    2 x 32-bit key -> 4 x 32-bit output. Each round multiplies words 0 and 2 by M0 and M1,
    mixes the high halves with words 1/3 and the key, and the key is bumped by (W0, W1)
    between rounds."""
    c0, c1, c2, c3 = (int(v) & _M32 for v in ctr)
    k0, k1 = (int(v) & _M32 for v in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _PHILOX_W0) & _M32
            k1 = (k1 + _PHILOX_W1) & _M32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & _M32, p1 & _M32, ((p0 >> 32) ^ c3 ^ k1) & _M32, p0 & _M32
    return (c0, c1, c2, c3)


def _u64(x):
    return (x >> 8) * (1.0 / 16777216.0)


TRAINING_SET = dict(n_cadences=65536, cadence=29.4 / 1440.0, sigma_min=1e-4, sigma_max=1e-3,
                    depth_min=30e-6, depth_max=2000e-6, dur_min_h=0.5, dur_max_h=3.0, p_min=0.2, p_max=1.0,
                    drift_bins=0.5)


def training_light_curve(seed: int, j: int, sp: dict = TRAINING_SET):
    """Light curve j of the seeded training set (the recipe of gpfc_synth_profiles).

    Returns (times f64, flux f64, label, fold_period). Parameters from Philox counters
    (j, 0, 0, 2^32-1) and (j, 1, 0, 2^32-1); normals of samples 4m..4m+3 from counter
    (j, m, 1, 0) by Box-Muller on u = (x >> 8) 2^-24.
    """
    key = (seed & _M32, (seed >> 32) & _M32)
    a = philox4x32_10((j, 0, 0, _M32), key)
    b = philox4x32_10((j, 1, 0, _M32), key)
    kind = 0 if j % 2 == 0 else 1 + (j // 2) % 3
    sigma = np.exp(np.log(sp["sigma_min"]) + _u64(a[0]) * np.log(sp["sigma_max"] / sp["sigma_min"]))
    period = sp["p_min"] + _u64(a[1]) * (sp["p_max"] - sp["p_min"])
    epoch = _u64(a[2]) * period
    dur = (sp["dur_min_h"] + _u64(a[3]) * (sp["dur_max_h"] - sp["dur_min_h"])) / 24.0
    depth = np.exp(np.log(sp["depth_min"]) + _u64(b[0]) * np.log(sp["depth_max"] / sp["depth_min"]))
    depth2 = depth * (0.2 + 0.8 * _u64(b[1]))
    amp = np.exp(np.log(sp["depth_min"]) + _u64(b[2]) * np.log(sp["depth_max"] / sp["depth_min"]))
    T = sp["n_cadences"] * sp["cadence"]
    df = (2.0 * _u64(b[3]) - 1.0) * sp["drift_bins"] / (256.0 * T)
    fold_period = 1.0 / (1.0 / period + df)
    n = sp["n_cadences"]
    t = np.arange(n, dtype=np.float64) * sp["cadence"]
    z = np.empty(n)
    for m in range((n + 3) // 4):
        r = philox4x32_10((j, m, 1, 0), key)
        for h in range(2):
            u1 = 1.0 - _u64(r[2 * h])
            u2 = _u64(r[2 * h + 1])
            rad = np.sqrt(-2.0 * np.log(u1))
            for q, v in ((2 * h, rad * np.cos(2 * np.pi * u2)), (2 * h + 1, rad * np.sin(2 * np.pi * u2))):
                if 4 * m + q < n:
                    z[4 * m + q] = v
    x = sigma * z

    def inbox(centre):
        d = np.mod(t - centre + 0.5 * period, period) - 0.5 * period
        return np.abs(d) < 0.5 * dur

    if kind == 0:
        x = x - depth * inbox(epoch)
    elif kind == 2:
        x = x + amp * np.sin(2 * np.pi * (t - epoch) / period)
    elif kind == 3:
        x = x - depth * inbox(epoch) - depth2 * inbox(epoch + 0.5 * period)
    return t, 1.0 + x, float(kind == 0), fold_period


# The paper's own training-set recipe (Sec. 2.6, Sec. 2.7): length-nbins vectors standing
# for folded light curves, Gaussian noise plus a trapezoid transit whose depth gives a
# target SNR alpha by Eq. 2. Positives: alpha in [6, 10]; negatives: noise only, or a
# transit injected with alpha below 5.
PAPER_VECTORS = dict(alpha_pos_min=6.0, alpha_pos_max=10.0, alpha_neg_max=5.0, q_min=0.04, q_max=0.12,
                     sigma_min=1e-4, sigma_max=5e-4, n_points=65536)


def paper_vector(seed: int, j: int, nbins: int = 256, pv: dict = PAPER_VECTORS):
    """Vector j of the seeded paper-recipe set (the recipe of gpfc_synth_vectors).

    Even j: positive (alpha ~ U[alpha_pos_min, alpha_pos_max]). Odd j: negative, noise only
    when (j // 2) is even, else a transit with alpha ~ U(0, alpha_neg_max). Per-point noise
    sigma log-uniform in [sigma_min, sigma_max]; a vector bin averages n_points / nbins points,
    so its noise is sigma sqrt(nbins / n_points). Trapezoid: duration at half depth
    q = L/p ~ U[q_min, q_max] (phase units), short-to-long base ratio r ~ U(0, 1), centre
    phi0 ~ U[0, 1), evaluated at the bin centres (b + 1/2) / nbins. Depth d = alpha sigma /
    sqrt(n_points q) (Eq. 2). Random numbers: Philox counters (j, 0, 2, 2^32-1) and
    (j, 1, 2, 2^32-1) for the parameters, (j, m, 3, 0) for the normals of bins 4m..4m+3.
    Returns (values f64 [nbins], label, alpha, sigma_bin).
    """
    key = (seed & _M32, (seed >> 32) & _M32)
    a = philox4x32_10((j, 0, 2, _M32), key)
    b = philox4x32_10((j, 1, 2, _M32), key)
    positive = j % 2 == 0
    inject = positive or (j // 2) % 2 == 1
    sigma = np.exp(np.log(pv["sigma_min"]) + _u64(a[0]) * np.log(pv["sigma_max"] / pv["sigma_min"]))
    if positive:
        alpha = pv["alpha_pos_min"] + _u64(a[1]) * (pv["alpha_pos_max"] - pv["alpha_pos_min"])
    else:
        alpha = _u64(a[1]) * pv["alpha_neg_max"] if inject else 0.0
    q = pv["q_min"] + _u64(a[2]) * (pv["q_max"] - pv["q_min"])
    r = _u64(a[3])
    phi0 = _u64(b[0])
    n = pv["n_points"]
    depth = alpha * sigma / np.sqrt(n * q)
    sigma_bin = sigma * np.sqrt(nbins / n)
    z = np.empty(nbins)
    for m in range((nbins + 3) // 4):
        rr = philox4x32_10((j, m, 3, 0), key)
        for h in range(2):
            u1 = 1.0 - _u64(rr[2 * h])
            u2 = _u64(rr[2 * h + 1])
            rad = np.sqrt(-2.0 * np.log(u1))
            for qq, v in ((2 * h, rad * np.cos(2 * np.pi * u2)), (2 * h + 1, rad * np.sin(2 * np.pi * u2))):
                if 4 * m + qq < nbins:
                    z[4 * m + qq] = v
    x = (np.arange(nbins) + 0.5) / nbins
    dphi = x - phi0
    dphi = np.abs(dphi - np.floor(dphi + 0.5))
    t14 = 2.0 * q / (1.0 + r)
    t23 = r * t14
    shape = np.where(dphi <= 0.5 * t23, 1.0,
                     np.where(dphi < 0.5 * t14, (0.5 * t14 - dphi) / (0.5 * (t14 - t23)), 0.0))
    values = 1.0 + sigma_bin * z - depth * shape
    return values, float(positive), float(alpha), float(sigma_bin)
