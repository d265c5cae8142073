"""Pins for the oracle's box-SNR statistic.

The oracle forms (out-of-box mean - in-box mean) * sqrt(n_in n_out / N) / sigma. It is
checked here against Kovacs et al.'s BLS signal residue SR = s^2 / (r (1 - r)), written
independently with prefix sums on a doubled profile, against the noise-free closed
form, and against the paper's Eq. 2 SNR.
"""
import numpy as np
import pytest

import oracle


def bls_sr_reference(sums, counts, w_min, w_max, sigma):
    """Signed sqrt(N*SR)/sigma from Kovacs' SR, by prefix sums over a doubled profile.

    With x the fluxes, xbar the profile mean, r = n_in/N and s = sum_in (x - xbar)/N,
    SR = s^2/(r(1-r)). A dip has s < 0, and we sign the result by -s.
    """
    nb = len(sums)
    N = counts.sum()
    S = sums[counts > 0].sum()
    xbar = S / N
    s2 = np.concatenate([np.where(counts > 0, sums, 0.0)] * 2)
    c2 = np.concatenate([counts] * 2)
    ps = np.concatenate([[0.0], np.cumsum(s2)])
    pc = np.concatenate([[0], np.cumsum(c2)])
    best = (-np.inf, -1, -1)
    for w in range(w_min, w_max + 1):
        for st in range(nb):
            nin = pc[st + w] - pc[st]
            if nin < 1 or N - nin < 1:
                continue
            sin_ = ps[st + w] - ps[st]
            r = nin / N
            s = (sin_ - nin * xbar) / N
            sr = s * s / (r * (1 - r))
            val = -np.sign(s) * np.sqrt(N * sr) / sigma
            if best[1] < 0 or val > best[0] + 1e-12 * max(1.0, abs(best[0])):
                best = (val, st, w)
    return best


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_matches_bls_signal_residue(seed):
    rng = np.random.default_rng(seed)
    nb = [16, 64, 37, 100][seed]
    counts = rng.integers(0, 20, nb)
    counts[rng.integers(0, nb)] = 0
    means = 1.0 + rng.normal(0, 1e-3, nb)
    sums = np.where(counts > 0, means * counts, 0.0)
    w_min, w_max = 1, max(2, nb // 4)
    sigma = 2e-4
    score, bs, bw = oracle.box_snr(sums[None], counts[None], w_min, w_max, sigma)
    ref, rs, rw = bls_sr_reference(sums, counts, w_min, w_max, sigma)
    assert score[0] == pytest.approx(ref, rel=1e-9)
    # the oracle's own box must reach the same value
    assert oracle.box_snr_at(sums, counts, bs[0], bw[0], sigma) == pytest.approx(ref, rel=1e-9)


def test_noise_free_box_closed_form_and_eq2():
    # w* whole bins of depth d, c samples per bin: delta = d exactly and
    # SNR = d sqrt(n_in n_out / N) / sigma = (d/sigma) sqrt(N q (1-q)) with q = w*/nb.
    # The paper's Eq. 2 (alpha = (d/sigma) sqrt(n L/p), n L/p = N q in-transit points)
    # is the same expression without the (1 - q) factor.
    nb, c, wstar, d, start, sigma = 256, 37, 9, 4e-4, 250, 1.5e-4
    counts = np.full(nb, c)
    means = np.ones(nb)
    idx = (start + np.arange(wstar)) % nb
    means[idx] = 1.0 - d
    sums = means * counts
    score, bs, bw = oracle.box_snr(sums[None], counts[None], 1, 40, sigma)
    N, q = nb * c, wstar / nb
    closed = d * np.sqrt(wstar * c * (N - wstar * c) / N) / sigma
    eq2 = (d / sigma) * np.sqrt(N * q)
    # FP64 on raw fluxes near 1 loses ~1e-16/d relative to the cancellation in delta
    assert score[0] == pytest.approx(closed, rel=1e-10)
    assert score[0] == pytest.approx(eq2 * np.sqrt(1 - q), rel=1e-10)
    assert (bs[0], bw[0]) == (start, wstar)


def test_direct_triple_loop():
    rng = np.random.default_rng(9)
    nb = 24
    counts = rng.integers(1, 9, nb)
    sums = counts * (1 + rng.normal(0, 1e-3, nb))
    sigma = 1.0
    N, S = counts.sum(), sums.sum()
    best = (-np.inf, -1, -1)
    for w in range(2, 7):
        for s in range(nb):
            idx = [(s + j) % nb for j in range(w)]
            nin = counts[idx].sum()
            sin_ = sums[idx].sum()
            nout = N - nin
            snr = ((S - sin_) / nout - sin_ / nin) * np.sqrt(nin * nout / N) / sigma
            if snr > best[0]:
                best = (snr, s, w)
    score, bs, bw = oracle.box_snr(sums[None], counts[None], 2, 6, sigma)
    assert score[0] == pytest.approx(best[0], rel=1e-12)
    assert (bs[0], bw[0]) == best[1:]


def test_ties_and_degenerate_profiles():
    # constant profile: every box gives 0; ties keep the smallest w, then smallest s
    counts = np.full(32, 5)
    sums = counts * 1.0
    score, bs, bw = oracle.box_snr(sums[None], counts[None], 3, 8, 1.0)
    assert score[0] == 0.0 and (bs[0], bw[0]) == (0, 3)
    # all samples in one bin: no box has both an inside and an outside sample
    counts = np.zeros(32, np.int64)
    counts[7] = 100
    sums = counts * 1.0
    score, bs, bw = oracle.box_snr(sums[None], counts[None], 1, 8, 1.0)
    assert score[0] == -np.inf and (bs[0], bw[0]) == (-1, -1)


def test_argmax_ties_and_nan():
    s = np.array([0.1, 0.5, np.nan, 0.5, 0.2], np.float32)
    assert oracle.argmax(s) == 1
    assert oracle.argmax(np.array([np.nan, np.nan], np.float32)) == -1


def test_tpr_at_fpr_small_example():
    neg = np.arange(1000) / 1000.0          # 0.000 .. 0.999
    pos = np.array([0.9985, 0.9995, 0.5, 1.5])
    tpr, thr = oracle.tpr_at_fpr(pos, neg, 1e-3)
    # one false alarm allowed: threshold is the 2nd largest negative, 0.998
    assert thr == pytest.approx(0.998)
    assert tpr == pytest.approx(0.75)
