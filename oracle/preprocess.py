"""Oracle of the pre-processing of Sec. 2.2 (Fig. 3): segmentation at time and flux gaps,
an iteratively clipped spline fit per segment with the smoothing chosen by the Bayesian
Information Criterion, division by the fit, and clipping of each segment's edges.

Test infrastructure: written from the paper's description in plain NumPy, with one
library primitive (numpy.linalg.solve for the spline's normal equations). It shares no
code with the CUDA path.

Readings of the paper (it names the steps, not the spline or the criterion's form):
 * segments: a new segment starts at sample i when t_i - t_{i-1} > time_gap (30 cadences
   of 0.020428 d) or |f_i - f_{i-1}| > flux_gap_sigma (5) times the population standard
   deviation of the whole light curve's flux;
 * the spline: cubic, least squares, clamped end knots at the segment's first and last
   times, interior knots spaced `spacing` days apart from the first time (every knot
   strictly inside); its smoothing is the knot spacing, chosen per segment from
   `spacings` by the smallest BIC = n ln(RSS / n) + p ln n over the n points kept in the
   final fit, p = number of coefficients (ties: the earlier candidate); a candidate with
   fewer kept points than coefficients is skipped;
 * normal equations (B^T B + lambda D^T D) c = B^T y, D the (p - 2) x p second-difference
   operator on the coefficients and lambda = ridge * trace(B^T B) / p (ridge 1e-9): a knot
   interval left without points (clipping, masks) takes coefficients continued linearly
   from its neighbours, and smooth trends are left nearly unbiased;
 * clipping: residuals r = f - spline over all the segment's points; sigma_r = the RMS
   of r over the points used in the fit; the next fit uses the unmasked points with
   |r| <= max(clip_sigma sigma_r, 1e-9 RMS(f)) (points can return; residuals below 1e-9 of
   the flux are never clipped); iterate until the kept set repeats or max_iter
   fits have been made; known transits (mask true) are never used in a fit;
 * output: f / spline for every point of the segment, the first and last `edge` points
   of each segment dropped (a segment of 2 edge points or fewer is dropped whole);
   segments stitched in time order.
"""
from __future__ import annotations

import numpy as np

TIME_GAP = 30 * 0.020428
SPACINGS = (0.5, 1.0, 1.5, 2.0, 3.0)


def segments(times, flux, time_gap=TIME_GAP, flux_gap_sigma=5.0):
    """Start indices of the segments (the first is 0) and their ends (exclusive)."""
    t = np.asarray(times, np.float64)
    f = np.asarray(flux, np.float64)
    sig = np.std(f)
    starts = [0]
    for i in range(1, len(t)):
        if t[i] - t[i - 1] > time_gap or abs(f[i] - f[i - 1]) > flux_gap_sigma * sig:
            starts.append(i)
    ends = starts[1:] + [len(t)]
    return np.asarray(starts, np.int64), np.asarray(ends, np.int64)


def knot_vector(t0, t1, spacing):
    """Clamped cubic knots: t0 four times, t0 + spacing j strictly inside (t0, t1), t1 four times."""
    inner = []
    j = 1
    while t0 + spacing * j < t1:
        inner.append(t0 + spacing * j)
        j += 1
    return np.asarray([t0] * 4 + inner + [t1] * 4, np.float64)


def bspline_design(t, knots, degree=3):
    """B[i, j] = B_j(t_i) by the Cox-de Boor recursion; the right end t = knots[-1] belongs
    to the last interval."""
    t = np.asarray(t, np.float64)
    k = np.asarray(knots, np.float64)
    nb = len(k) - 1
    B = np.zeros((len(t), nb))
    last = np.max(np.nonzero(k[:-1] < k[1:])[0])          # last non-empty interval
    for j in range(nb):
        inside = (k[j] <= t) & (t < k[j + 1])
        if j == last:
            inside |= t == k[j + 1]
        B[:, j] = inside
    for d in range(1, degree + 1):
        Bn = np.zeros((len(t), nb - d))
        for j in range(nb - d):
            left = (t - k[j]) / (k[j + d] - k[j]) * B[:, j] if k[j + d] > k[j] else 0.0
            right = (k[j + d + 1] - t) / (k[j + d + 1] - k[j + 1]) * B[:, j + 1] if k[j + d + 1] > k[j + 1] else 0.0
            Bn[:, j] = left + right
        B = Bn
    return B


def fit_segment(t, f, mask, spacing, clip_sigma=3.0, max_iter=10, ridge=1e-9):
    """Clipped least-squares spline of one segment for one knot spacing.
    Returns (bic, trend [n], kept [n] bool, n_coefficients) or None when skipped."""
    knots = knot_vector(t[0], t[-1], spacing)
    B = bspline_design(t, knots)
    p = B.shape[1]
    free = ~mask
    used = free.copy()
    for it in range(max_iter):
        if used.sum() < p:
            return None
        Bu = B[used]
        G = Bu.T @ Bu
        D = np.zeros((p - 2, p))
        for i in range(p - 2):
            D[i, i:i + 3] = (1.0, -2.0, 1.0)
        G = G + ridge * np.trace(G) / p * (D.T @ D)
        c = np.linalg.solve(G, Bu.T @ f[used])
        trend = B @ c
        r = f - trend
        sr = np.sqrt(np.mean(r[used] ** 2))
        floor = 1e-9 * np.sqrt(np.mean(f[used] ** 2))  # residuals below 1e-9 of the flux stay
        nxt = free & (np.abs(r) <= max(clip_sigma * sr, floor))
        if np.array_equal(nxt, used) or it == max_iter - 1:
            break  # `used` is the point set of the last fit
        used = nxt
    r = f - trend
    n = int(used.sum())
    rss = float(np.sum(r[used] ** 2))
    bic = n * np.log(rss / n) + p * np.log(n) if rss > 0 else -np.inf
    return bic, trend, used, p


def detrend(times, flux, mask=None, time_gap=TIME_GAP, flux_gap_sigma=5.0, clip_sigma=3.0, edge=30,
            max_iter=10, spacings=SPACINGS, ridge=1e-9):
    """The pre-processing of Sec. 2.2. Returns dict(times, flux (f / spline), segment,
    index (into the input), spacing [per segment, NaN if dropped], starts, ends)."""
    t = np.asarray(times, np.float64)
    f = np.asarray(flux, np.float64)
    m = np.zeros(len(t), bool) if mask is None else np.asarray(mask, bool)
    starts, ends = segments(t, f, time_gap, flux_gap_sigma)
    out_t, out_f, out_s, out_i = [], [], [], []
    chosen = np.full(len(starts), np.nan)
    for s, (a, b) in enumerate(zip(starts, ends)):
        if b - a <= 2 * edge:
            continue
        best = None
        for sp in spacings:
            r = fit_segment(t[a:b], f[a:b], m[a:b], sp, clip_sigma, max_iter, ridge)
            if r is not None and (best is None or r[0] < best[0]):
                best = (r[0], r[1], sp)
        if best is None:
            continue
        chosen[s] = best[2]
        det = f[a:b] / best[1]
        idx = np.arange(a + edge, b - edge)
        out_t.append(t[idx])
        out_f.append(det[edge:b - a - edge])
        out_s.append(np.full(len(idx), s, np.int64))
        out_i.append(idx)
    cat = lambda xs, dt: np.concatenate(xs) if xs else np.zeros(0, dt)
    return {"times": cat(out_t, np.float64), "flux": cat(out_f, np.float64), "segment": cat(out_s, np.int64),
            "index": cat(out_i, np.int64), "spacing": chosen, "starts": starts, "ends": ends}
