"""FP64 CPU oracle for the GPFC fold + score path.

TEST INFRASTRUCTURE: only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg
of `bench.py` may import this package. The product library never calls it and shares
no code with it (no headers, kernels, helpers or constants).

The arithmetic lives in `gpfc_oracle.c` (plain C loops in FP64, index order); this
module compiles it with gcc on first use and wraps it with ctypes. `adam_step` is the
one routine written here in NumPy.

Parity status: every function is pinned by the `-m "not gpu"` tests (exact-rational
brute force, invariants, closed forms, library special cases, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpfc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile gpfc_oracle.c into _build/liboracle.so (gcc -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CnnParams(ctypes.Structure):
    _fields_ = [(n, _dp) for n in ("w1", "b1", "w2", "b2", "w3", "b3", "wf1", "bf1", "wf2", "bf2")]


_CnnGrads = type("_CnnGrads", (ctypes.Structure,), {"_fields_": _CnnParams._fields_})


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_quantise_times.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _i64p]
            L.or_quantise_periods.argtypes = [_dp, ctypes.c_int64, _u64p]
            L.or_bins.argtypes = [_i64p, ctypes.c_int64, _u64p, ctypes.c_int64, ctypes.c_int32, _i32p]
            L.or_fold.argtypes = [_dp, _fp, ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_double, _dp, _i64p, _dp]
            L.or_fold_equal_count.argtypes = [_dp, _fp, ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_double, _dp, _i64p]
            L.or_peaks.argtypes = [_fp, _dp, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_int32, _dp, _i64p, _i64p, _fp, _i32p, _i32p]
            L.or_peaks.restype = ctypes.c_int32
            L.or_bins_naive_fp64.argtypes = [_dp, ctypes.c_int64, _dp, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_double, _i32p]
            L.or_box_snr.argtypes = [_dp, _i64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_double, _dp, _i32p, _i32p]
            L.or_box_snr_at.argtypes = [_dp, _i64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double]
            L.or_box_snr_at.restype = ctypes.c_double
            L.or_argmax.argtypes = [_fp, ctypes.c_int64]
            L.or_argmax.restype = ctypes.c_int64
            L.or_cnn_normalise.argtypes = [_fp, _i32p, _dp]
            L.or_cnn_score.argtypes = [ctypes.POINTER(_CnnParams), _fp, _i32p, ctypes.c_int64, _dp, _dp]
            L.or_cnn_forward.argtypes = [ctypes.POINTER(_CnnParams), _dp, ctypes.c_int64, _dp]
            L.or_cnn_loss_backward.argtypes = [ctypes.POINTER(_CnnParams), _dp, _fp, ctypes.c_int64,
                                               ctypes.POINTER(_CnnGrads), _dp]
            L.or_cnn_loss_backward.restype = ctypes.c_double
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------- fold


def quantise_times(times, t0):
    """tau = rint((t - t0) * 2^24) as int64. Raises ValueError on fixed-point overflow."""
    times = _c(times, np.float64)
    tau = np.empty(times.shape[0], np.int64)
    rc = lib().or_quantise_times(_p(times, _dp), times.shape[0], float(t0), _p(tau, _i64p))
    if rc != 0:
        raise ValueError("time outside the 64-bit fixed-point range")
    return tau


def quantise_periods(periods):
    """F = rint(2^40 / P) as uint64. Raises ValueError on invalid periods."""
    periods = _c(periods, np.float64)
    F = np.empty(periods.shape[0], np.uint64)
    rc = lib().or_quantise_periods(_p(periods, _dp), periods.shape[0], _p(F, _u64p))
    if rc != 0:
        raise ValueError("period not finite/positive or outside the fixed-point range")
    return F


def bins(tau, F, nbins):
    """bins[k][i] = floor(((tau_i * F_k) mod 2^64) * nbins / 2^64)."""
    tau = _c(tau, np.int64)
    F = _c(F, np.uint64)
    out = np.empty((F.shape[0], tau.shape[0]), np.int32)
    lib().or_bins(_p(tau, _i64p), tau.shape[0], _p(F, _u64p), F.shape[0], int(nbins), _p(out, _i32p))
    return out


def fold(times, flux, periods, nbins, t0=None):
    """FP64 fold. Returns (mean [P][nbins] f64 with NaN for empty, count i64, sum f64)."""
    times = _c(times, np.float64)
    flux = _c(flux, np.float32)
    periods = _c(periods, np.float64)
    if t0 is None or (isinstance(t0, float) and np.isnan(t0)):
        t0 = float(times[0])
    n, npd = times.shape[0], periods.shape[0]
    mean = np.empty((npd, nbins), np.float64)
    cnt = np.empty((npd, nbins), np.int64)
    s = np.empty((npd, nbins), np.float64)
    rc = lib().or_fold(_p(times, _dp), _p(flux, _fp), n, _p(periods, _dp), npd, int(nbins),
                       float(t0), _p(mean, _dp), _p(cnt, _i64p), _p(s, _dp))
    if rc != 0:
        raise ValueError("time or period outside the 64-bit fixed-point range")
    return mean, cnt, s


def fold_equal_count(times, flux, periods, nfine, nbins, t0=None):
    """Two-tier equal-count fold (Sec. 2.3): nfine equal-width fine bins merged left to
    right into nbins bins of n/nbins samples each. Returns (mean [P][nbins] f64,
    fine_count [P][nfine] i64)."""
    times = _c(times, np.float64)
    flux = _c(flux, np.float32)
    periods = _c(periods, np.float64)
    if t0 is None or (isinstance(t0, float) and np.isnan(t0)):
        t0 = float(times[0])
    n, npd = times.shape[0], periods.shape[0]
    mean = np.empty((npd, nbins), np.float64)
    fc = np.empty((npd, nfine), np.int64)
    rc = lib().or_fold_equal_count(_p(times, _dp), _p(flux, _fp), n, _p(periods, _dp), npd, int(nfine),
                                   int(nbins), float(t0), _p(mean, _dp), _p(fc, _i64p))
    if rc != 0:
        raise ValueError("time or period outside the 64-bit fixed-point range")
    return mean, fc


def bins_naive_fp64(times, periods, nbins, t0):
    """floor(frac((t - t0)/P) * nbins) evaluated directly in FP64 (for reporting)."""
    times = _c(times, np.float64)
    periods = _c(periods, np.float64)
    out = np.empty((periods.shape[0], times.shape[0]), np.int32)
    lib().or_bins_naive_fp64(_p(times, _dp), times.shape[0], _p(periods, _dp), periods.shape[0],
                             int(nbins), float(t0), _p(out, _i32p))
    return out


# ---------------------------------------------------------------- box-SNR


def box_snr(sums, counts, w_min, w_max, sigma=1.0):
    """Box-SNR per profile from per-bin flux sums and counts ([P][nbins]).

    Returns (score f64 [P], best_s i32 [P], best_w i32 [P]).
    """
    sums = _c(np.atleast_2d(sums), np.float64)
    counts = _c(np.atleast_2d(counts), np.int64)
    npd, nb = sums.shape
    score = np.empty(npd, np.float64)
    bs = np.empty(npd, np.int32)
    bw = np.empty(npd, np.int32)
    lib().or_box_snr(_p(sums, _dp), _p(counts, _i64p), npd, nb, int(w_min), int(w_max),
                     float(sigma), _p(score, _dp), _p(bs, _i32p), _p(bw, _i32p))
    return score, bs, bw


def box_snr_from_means(means, counts, w_min, w_max, sigma=1.0):
    """Box-SNR of profiles given as per-bin means + counts (sum = mean * count in FP64)."""
    means = np.atleast_2d(np.asarray(means, np.float64))
    counts = np.atleast_2d(np.asarray(counts, np.int64))
    sums = np.where(counts > 0, means * counts, 0.0)
    return box_snr(sums, counts, w_min, w_max, sigma)


def box_snr_at(sums, counts, s, w, sigma=1.0):
    sums = _c(sums, np.float64)
    counts = _c(counts, np.int64)
    return lib().or_box_snr_at(_p(sums, _dp), _p(counts, _i64p), sums.shape[0], int(s), int(w),
                               float(sigma))


def argmax(score):
    score = _c(score, np.float32)
    return int(lib().or_argmax(_p(score, _fp), score.shape[0]))


# ---------------------------------------------------------------- CNN

CNN_NAMES = ["conv1.w", "conv1.b", "conv2.w", "conv2.b", "conv3.w", "conv3.b",
             "fc1.w", "fc1.b", "fc2.w", "fc2.b"]
_FIELDS = ["w1", "b1", "w2", "b2", "w3", "b3", "wf1", "bf1", "wf2", "bf2"]


def _params(weights):
    keep = [_c(weights[n], np.float64).ravel() for n in CNN_NAMES]
    p = _CnnParams(*[_p(a, _dp) for a in keep])
    return p, keep


def cnn_normalise(folded, counts=None):
    folded = _c(np.atleast_2d(folded), np.float32)
    out = np.empty(folded.shape, np.float64)
    for k in range(folded.shape[0]):
        c = None if counts is None else _c(np.atleast_2d(counts)[k], np.int32)
        lib().or_cnn_normalise(_p(folded[k], _fp), _p(c, _i32p) if c is not None else None,
                               _p(out[k], _dp))
    return out


def cnn_score(weights, folded, counts=None):
    """normalise + CNN forward. Returns (logits f64 [P], scores f64 [P])."""
    folded = _c(np.atleast_2d(folded), np.float32)
    cts = None if counts is None else _c(np.atleast_2d(counts), np.int32)
    npd = folded.shape[0]
    p, keep = _params(weights)
    z = np.empty(npd, np.float64)
    s = np.empty(npd, np.float64)
    lib().or_cnn_score(ctypes.byref(p), _p(folded, _fp), _p(cts, _i32p) if cts is not None else None,
                       npd, _p(z, _dp), _p(s, _dp))
    return z, s


def cnn_forward(weights, x):
    """CNN forward on already-normalised inputs x [P][256]; returns logits f64 [P]."""
    x = _c(np.atleast_2d(x), np.float64)
    p, keep = _params(weights)
    z = np.empty(x.shape[0], np.float64)
    lib().or_cnn_forward(ctypes.byref(p), _p(x, _dp), x.shape[0], _p(z, _dp))
    return z


def cnn_loss_backward(weights, x, labels, want_dx=False):
    """Mean BCE-with-logits loss and its FP64 gradients.

    Returns (loss, grads dict with the same names/shapes as weights, dx or None).
    """
    x = _c(np.atleast_2d(x), np.float64)
    labels = _c(labels, np.float32)
    p, keep = _params(weights)
    grads = {n: np.zeros(np.shape(weights[n]), np.float64) for n in CNN_NAMES}
    g = _CnnGrads(*[_p(grads[n].reshape(-1), _dp) for n in CNN_NAMES])
    dx = np.zeros(x.shape, np.float64) if want_dx else None
    loss = lib().or_cnn_loss_backward(ctypes.byref(p), _p(x, _dp), _p(labels, _fp), x.shape[0],
                                      ctypes.byref(g), _p(dx, _dp) if dx is not None else None)
    return loss, grads, dx


def adam_step(param, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), FP64, in place on copies.

    m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;  mhat = m/(1-b1^t);
    vhat = v/(1-b2^t);  param <- param - lr * mhat / (sqrt(vhat) + eps).
    Returns (param, m, v) as new arrays.
    """
    param = np.asarray(param, np.float64)
    grad = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


def peaks(score, periods, k_sigma=3.0, min_width=4, harmonic_tol=1e-3, max_peaks=8):
    """Per-star decision over a periodogram: SDE (Eq. 3) and the peak rule of Sec. 4.2.

    Returns a dict with mean, sd, sde, best_index (-1 if no qualifying peak), n_peaks and
    the listed peaks (index, height, width, harmonic), highest first.
    """
    score = _c(score, np.float32)
    periods = _c(periods, np.float64)
    npd = score.shape[0]
    st = np.empty(3, np.float64)
    best = np.empty(2, np.int64)
    idx = np.empty(max(1, max_peaks), np.int64)
    h = np.empty(max(1, max_peaks), np.float32)
    w = np.empty(max(1, max_peaks), np.int32)
    hm = np.empty(max(1, max_peaks), np.int32)
    n = lib().or_peaks(_p(score, _fp), _p(periods, _dp), npd, float(k_sigma), int(min_width), float(harmonic_tol),
                       int(max_peaks), _p(st, _dp), _p(best, _i64p), _p(idx, _i64p), _p(h, _fp), _p(w, _i32p),
                       _p(hm, _i32p))
    return {"mean": st[0], "sd": st[1], "sde": st[2], "best_index": int(best[0]), "n_peaks": int(best[1]),
            "index": idx[:n].copy(), "height": h[:n].copy(), "width": w[:n].copy(), "harmonic": hm[:n].copy()}


def sigmoid(z):
    z = np.asarray(z, np.float64)
    return 1.0 / (1.0 + np.exp(-z))


def tpr_at_fpr(scores_pos, scores_neg, fpr):
    """True-positive rate at a false-positive rate.

    k = floor(fpr * n_neg) negatives may be false alarms; the threshold is the
    (k+1)-th largest negative score and a profile counts as detected when its score
    is strictly above it. Returns (tpr, threshold).
    """
    neg = np.sort(np.asarray(scores_neg, np.float64))[::-1]
    k = int(np.floor(fpr * len(neg)))
    thr = neg[k] if k < len(neg) else -np.inf
    return float(np.mean(np.asarray(scores_pos, np.float64) > thr)), float(thr)


def roc(scores_pos, scores_neg, fprs=()):
    """Detection statistics of one detector on a labelled set (Sec. 3.2: ROC curves of
    stars scored by their best trial period, Figs. 10-13). A NaN score ranks below every
    number (it is never a detection).

    u2  = sum over (i, j) of 2 [pos_i > neg_j] + [pos_i == neg_j]   (an exact integer:
          twice the Mann-Whitney U statistic, ties counted one half)
    auc = u2 / (2 n_pos n_neg)
    for each fpr: k = floor(fpr n_neg); thr = the (k+1)-th largest negative score (-inf when
          k >= n_neg); tp = #{pos_i > thr}, tpr = tp / n_pos
    Returns dict(u2, auc, thr [n_fpr] f64, tp [n_fpr] int64, tpr [n_fpr] f64).
    """
    p = np.asarray(scores_pos, np.float64).ravel()
    n = np.asarray(scores_neg, np.float64).ravel()
    p = np.where(np.isnan(p), -np.inf, p)
    n = np.where(np.isnan(n), -np.inf, n)
    ns = np.sort(n)
    below = np.searchsorted(ns, p, side="left")      # negatives < p_i
    upto = np.searchsorted(ns, p, side="right")      # negatives <= p_i
    u2 = int(2 * np.sum(below, dtype=np.int64) + np.sum(upto - below, dtype=np.int64))
    thr, tp = [], []
    for f in fprs:
        k = int(np.floor(float(f) * len(n)))
        t = ns[len(n) - 1 - k] if k < len(n) else -np.inf
        thr.append(t)
        tp.append(int(np.sum(p > t)))
    tp = np.asarray(tp, np.int64)
    return {"u2": u2, "auc": u2 / (2.0 * len(p) * len(n)), "thr": np.asarray(thr, np.float64), "tp": tp,
            "tpr": tp / float(len(p))}


from .preprocess import bspline_design, detrend, knot_vector, segments  # noqa: E402  (pre-processing, Sec. 2.2)
