/*
 * gpfc_oracle.c -- plain, slow FP64 reference for the GPFC fold + score path.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use this file. The product path never calls it and shares no code
 * with it.
 *
 * Every function is the definition written out with plain loops in index order, no
 * blocking or reordering:
 *   - phase fold (paper Sec. 2.3: modular residual of each timestamp by the trial
 *     period, map to a bin, per-bin count and flux sum, mean = sum / count), with the
 *     phase taken exactly in 64-bit fixed point: tau = rint((t - t0) * 2^24),
 *     F = rint(2^40 / P), phase = ((tau * F) mod 2^64) / 2^64, bin = floor(phase*nbins);
 *   - box-SNR statistic per folded profile (the box-fitting idea of Sec. 3.1: a box of
 *     w consecutive bins, circular, against the rest of the profile);
 *   - noise normalisation of a folded profile (Sec. 2.1: std scaled to 1 while the
 *     mean is kept);
 *   - forward and backward of the scorer CNN conv(k5,16)-pool2-conv(k5,32)-pool2-
 *     conv(k5,64)-pool2-FC(2048->256)-FC(256->1)-sigmoid with circular padding
 *     (Sec. 2.5 uses circular convolutions), ReLU after each conv and after FC1,
 *     max-pool k2 s2, channel-major flatten, binary cross-entropy with logits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TWO24 16777216.0
#define OR_TWO40 1099511627776.0

/* ---------------------------------------------------------------- quantisation */

/* tau_i = rint((t_i - t0) * 2^24), round to nearest even (default FP environment). */
int or_quantise_times(const double *times, int64_t n, double t0, int64_t *tau)
{
    int bad = 0;
    for (int64_t i = 0; i < n; i++) {
        double v = (times[i] - t0) * OR_TWO24;
        if (!(fabs(v) < 4611686018427387904.0)) { /* |tau| must stay below 2^62 */
            tau[i] = 0;
            bad = 1;
            continue;
        }
        tau[i] = llrint(v);
    }
    return bad ? -4 : 0;
}

/* F_k = rint(2^40 / P_k) as an unsigned 64-bit integer; P_k must be finite, > 0. */
int or_quantise_periods(const double *periods, int64_t np, uint64_t *F)
{
    int bad = 0;
    for (int64_t k = 0; k < np; k++) {
        double p = periods[k];
        if (!(p > 0.0) || !isfinite(p)) { F[k] = 0; bad = 1; continue; }
        double q = OR_TWO40 / p;
        if (!(q < 9223372036854775808.0)) { F[k] = 0; bad = 1; continue; }
        F[k] = (uint64_t)llrint(q);
    }
    return bad ? -4 : 0;
}

/* bin = floor(((tau * F) mod 2^64) * nbins / 2^64), exact integer arithmetic. */
static uint32_t or_bin(int64_t tau, uint64_t F, int32_t nbins)
{
    uint64_t phi = (uint64_t)tau * F; /* unsigned wrap = mod 2^64 */
    unsigned __int128 p = (unsigned __int128)phi * (uint64_t)(uint32_t)nbins;
    return (uint32_t)(p >> 64);
}

void or_bins(const int64_t *tau, int64_t n, const uint64_t *F, int64_t np, int32_t nbins,
             int32_t *bins /* [np][n] */)
{
    for (int64_t k = 0; k < np; k++)
        for (int64_t i = 0; i < n; i++)
            bins[k * n + i] = (int32_t)or_bin(tau[i], F[k], nbins);
}

/* ---------------------------------------------------------------- fold */

/*
 * Fold one light curve at every trial period.
 *   count[k][b] = #{i : bin_ik = b}
 *   sum[k][b]   = sum of flux_i over those i, in FP64, in index order
 *   mean[k][b]  = sum / count, NaN when count = 0
 * Any output pointer may be NULL. Returns 0, or -4 if a time or period does not
 * fit the fixed-point representation.
 */
int or_fold(const double *times, const float *flux, int64_t n, const double *periods,
            int64_t np, int32_t nbins, double t0, double *mean, int64_t *count, double *sum)
{
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t *F = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(np > 0 ? np : 1));
    double *s = (double *)malloc(sizeof(double) * (size_t)nbins);
    int64_t *c = (int64_t *)malloc(sizeof(int64_t) * (size_t)nbins);
    int rc = or_quantise_times(times, n, t0, tau);
    int rc2 = or_quantise_periods(periods, np, F);
    if (rc == 0) rc = rc2;
    for (int64_t k = 0; k < np; k++) {
        for (int32_t b = 0; b < nbins; b++) { s[b] = 0.0; c[b] = 0; }
        for (int64_t i = 0; i < n; i++) {
            uint32_t b = or_bin(tau[i], F[k], nbins);
            c[b] += 1;
            s[b] += (double)flux[i];
        }
        for (int32_t b = 0; b < nbins; b++) {
            if (count) count[k * nbins + b] = c[b];
            if (sum) sum[k * nbins + b] = s[b];
            if (mean) mean[k * nbins + b] = c[b] > 0 ? s[b] / (double)c[b] : NAN;
        }
    }
    free(tau); free(F); free(s); free(c);
    return rc;
}

/* Two-tier equal-count fold (Sec. 2.3, Fig. 4 (a)-(e)): the samples go to nfine
 * equal-width bins by their fixed-point phase, each fine bin keeping its count and flux
 * sum (steps 1-3); a left-to-right scan over the fine bins then fills the nbins final
 * bins one after the other with exactly n / nbins samples each, merging adjacent fine
 * bins and splitting the fine bin that straddles a boundary (step 4); each final mean is
 * its flux sum over n / nbins (step 5).
 * Reading of the split (the paper leaves it open): a fine bin that gives k of its c
 * samples to a final bin gives it k / c of its flux sum. The scan counts in units of
 * 1 / nbins sample, so every boundary (a multiple of n units) is exact in integers.
 * mean is [np][nbins]; fine_count (may be NULL) [np][nfine]. Returns 0 or -4. */
int or_fold_equal_count(const double *times, const float *flux, int64_t n, const double *periods,
                        int64_t np, int32_t nfine, int32_t nbins, double t0, double *mean,
                        int64_t *fine_count)
{
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t *F = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(np > 0 ? np : 1));
    double *s = (double *)malloc(sizeof(double) * (size_t)nfine);
    int64_t *c = (int64_t *)malloc(sizeof(int64_t) * (size_t)nfine);
    int rc = or_quantise_times(times, n, t0, tau);
    int rc2 = or_quantise_periods(periods, np, F);
    if (rc == 0) rc = rc2;
    const int64_t cap = n; /* units per final bin */
    for (int64_t k = 0; k < np; k++) {
        for (int32_t f = 0; f < nfine; f++) { s[f] = 0.0; c[f] = 0; }
        for (int64_t i = 0; i < n; i++) {
            uint32_t f = or_bin(tau[i], F[k], nfine);
            c[f] += 1;
            s[f] += (double)flux[i];
        }
        if (fine_count)
            for (int32_t f = 0; f < nfine; f++) fine_count[k * nfine + f] = c[f];
        int32_t j = 0;      /* final bin being filled */
        int64_t fill = 0;   /* units already in it */
        double acc = 0.0;   /* its flux sum */
        for (int32_t f = 0; f < nfine && j < nbins; f++) {
            int64_t left = c[f] * (int64_t)nbins; /* units of fine bin f not yet placed */
            const int64_t whole = left;
            while (left > 0 && j < nbins) {
                const int64_t room = cap - fill;
                const int64_t take = left < room ? left : room;
                acc += s[f] * ((double)take / (double)whole);
                fill += take;
                left -= take;
                if (fill == cap) {
                    mean[k * nbins + j] = acc / ((double)n / (double)nbins);
                    j++;
                    fill = 0;
                    acc = 0.0;
                }
            }
        }
        for (; j < nbins; j++) mean[k * nbins + j] = NAN; /* only when n == 0 */
    }
    free(tau); free(F); free(s); free(c);
    return rc;
}

/* The phase the paper states, frac((t - t0) / P), taken directly in FP64. Returns
 * floor(frac * nbins) per (k, i); used only to report how often the fixed-point bins
 * differ from it (at bin edges). */
void or_bins_naive_fp64(const double *times, int64_t n, const double *periods, int64_t np,
                        int32_t nbins, double t0, int32_t *bins /* [np][n] */)
{
    for (int64_t k = 0; k < np; k++)
        for (int64_t i = 0; i < n; i++) {
            double q = (times[i] - t0) / periods[k];
            double ph = q - floor(q);
            int32_t b = (int32_t)floor(ph * nbins);
            if (b >= nbins) b = nbins - 1;
            bins[k * n + i] = b;
        }
}

/* ---------------------------------------------------------------- box-SNR */

/*
 * Box-SNR of one folded profile from its per-bin flux sums and counts.
 * For every width w in [w_min, w_max] and start s in [0, nbins), the box holds bins
 * s, s+1, ..., s+w-1 (mod nbins). With n_in, S_in the count and flux sum inside,
 * N, S the profile totals and n_out = N - n_in, a box is valid when n_in >= 1 and
 * n_out >= 1, and
 *     delta = (S - S_in)/n_out - S_in/n_in          (out-of-box mean minus in-box mean)
 *     snr   = delta * sqrt(n_in * n_out / N) / sigma
 * The score is the largest snr; ties keep the smaller w, then the smaller s. With no
 * valid box the score is -inf and s = w = -1. The in-box sums are formed directly
 * from the bins for each (s, w).
 */
void or_box_snr_one(const double *sum, const int64_t *count, int32_t nbins, int32_t w_min,
                    int32_t w_max, double sigma, double *score, int32_t *best_s, int32_t *best_w)
{
    int64_t N = 0;
    double S = 0.0;
    for (int32_t b = 0; b < nbins; b++) { N += count[b]; S += count[b] > 0 ? sum[b] : 0.0; }
    double best = -INFINITY;
    int32_t bs = -1, bw = -1;
    for (int32_t w = w_min; w <= w_max; w++) {
        for (int32_t s = 0; s < nbins; s++) {
            int64_t nin = 0;
            double sin_ = 0.0;
            for (int32_t j = 0; j < w; j++) {
                int32_t b = (s + j) % nbins;
                nin += count[b];
                if (count[b] > 0) sin_ += sum[b];
            }
            int64_t nout = N - nin;
            if (nin < 1 || nout < 1) continue;
            double delta = (S - sin_) / (double)nout - sin_ / (double)nin;
            double snr = delta * sqrt((double)nin * (double)nout / (double)N) / sigma;
            if (snr > best) { best = snr; bs = s; bw = w; }
        }
    }
    *score = best;
    if (best_s) *best_s = bs;
    if (best_w) *best_w = bw;
}

/* Box-SNR over np profiles given as per-bin sums + counts (row-major [np][nbins]). */
void or_box_snr(const double *sum, const int64_t *count, int64_t np, int32_t nbins,
                int32_t w_min, int32_t w_max, double sigma, double *score, int32_t *best_s,
                int32_t *best_w)
{
    for (int64_t k = 0; k < np; k++)
        or_box_snr_one(sum + k * nbins, count + k * nbins, nbins, w_min, w_max, sigma,
                       score + k, best_s ? best_s + k : NULL, best_w ? best_w + k : NULL);
}

/* Box-SNR of one box (s, w) only; NAN if the box is not valid. */
double or_box_snr_at(const double *sum, const int64_t *count, int32_t nbins, int32_t s,
                     int32_t w, double sigma)
{
    int64_t N = 0, nin = 0;
    double S = 0.0, sin_ = 0.0;
    for (int32_t b = 0; b < nbins; b++) { N += count[b]; if (count[b] > 0) S += sum[b]; }
    for (int32_t j = 0; j < w; j++) {
        int32_t b = (s + j) % nbins;
        nin += count[b];
        if (count[b] > 0) sin_ += sum[b];
    }
    int64_t nout = N - nin;
    if (nin < 1 || nout < 1) return NAN;
    double delta = (S - sin_) / (double)nout - sin_ / (double)nin;
    return delta * sqrt((double)nin * (double)nout / (double)N) / sigma;
}

/* argmax of a score vector; ties go to the smallest index; NaN never wins. */
int64_t or_argmax(const float *score, int64_t np)
{
    int64_t best = -1;
    for (int64_t k = 0; k < np; k++)
        if (!isnan(score[k]) && (best < 0 || score[k] > score[best])) best = k;
    return best;
}

/* ---------------------------------------------------------------- per-star decision */

/* Decision over one star's periodogram score[0..np-1] (non-finite entries are left out
 * of the statistics and never belong to a peak):
 *  - mean and population standard deviation of the finite scores;
 *  - SDE = (max - mean) / sd (Eq. 3; 0 when sd is 0);
 *  - peaks (Sec. 4.2): maximal runs of consecutive periods scoring above
 *    mean + k_sigma * sd; a run qualifies when it is at least min_width periods wide
 *    ("more than 3" is min_width = 4). Its height is its largest score, at its first
 *    occurrence. The best peak is the highest (ties: smaller index);
 *  - the qualifying peaks by decreasing height (ties: smaller index), at most max_peaks,
 *    each with a harmonic flag against the best peak's period Pb (Fig. 14 notes peaks
 *    at harmonics): 1 for the best, +m if P = m Pb, -m if P = Pb / m (m = 2..4, within
 *    relative tolerance harmonic_tol), else 0.
 * out_stats: mean, sd, sde. out_best: best index (-1 if none), n_peaks.
 * peaks_*: [max_peaks]. Returns the number of peaks listed. */
int32_t or_peaks(const float *score, const double *periods, int64_t np, double k_sigma, int32_t min_width,
                 double harmonic_tol, int32_t max_peaks, double *out_stats, int64_t *out_best,
                 int64_t *peak_index, float *peak_height, int32_t *peak_width, int32_t *peak_harm)
{
    double sum = 0.0, cnt = 0.0, mx = -INFINITY;
    for (int64_t k = 0; k < np; k++)
        if (isfinite(score[k])) { sum += (double)score[k]; cnt += 1.0; if ((double)score[k] > mx) mx = score[k]; }
    const double mean = cnt > 0 ? sum / cnt : NAN;
    double ss = 0.0;
    for (int64_t k = 0; k < np; k++)
        if (isfinite(score[k])) { const double d = (double)score[k] - mean; ss += d * d; }
    const double sd = cnt > 0 ? sqrt(ss / cnt) : NAN;
    out_stats[0] = mean;
    out_stats[1] = sd;
    out_stats[2] = cnt > 0 ? (sd > 0 ? (mx - mean) / sd : 0.0) : NAN;
    const double thr = mean + k_sigma * sd;
    /* qualifying runs */
    int64_t nq = 0, cap = np > 0 ? np : 1;
    int64_t *ri = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    float *rh = (float *)malloc(sizeof(float) * (size_t)cap);
    int32_t *rw = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int64_t k = 0;
    while (k < np) {
        if (!(isfinite(score[k]) && (double)score[k] > thr)) { k++; continue; }
        int64_t e = k, arg = k;
        while (e < np && isfinite(score[e]) && (double)score[e] > thr) {
            if (score[e] > score[arg]) arg = e;
            e++;
        }
        if (e - k >= min_width) { ri[nq] = arg; rh[nq] = score[arg]; rw[nq] = (int32_t)(e - k); nq++; }
        k = e;
    }
    out_best[1] = nq;
    /* order by height, then index (selection of the top max_peaks) */
    int32_t listed = 0;
    char *taken = (char *)calloc((size_t)(nq > 0 ? nq : 1), 1);
    for (; listed < max_peaks && listed < nq; listed++) {
        int64_t b = -1;
        for (int64_t q = 0; q < nq; q++)
            if (!taken[q] && (b < 0 || rh[q] > rh[b] || (rh[q] == rh[b] && ri[q] < ri[b]))) b = q;
        taken[b] = 1;
        peak_index[listed] = ri[b];
        peak_height[listed] = rh[b];
        peak_width[listed] = rw[b];
    }
    out_best[0] = listed > 0 ? peak_index[0] : -1;
    for (int32_t q = 0; q < listed; q++) {
        int32_t h = 0;
        if (q == 0) h = 1;
        else {
            const double r = periods[peak_index[q]] / periods[peak_index[0]];
            for (int32_t m = 2; m <= 4 && h == 0; m++) {
                if (fabs(r - m) <= harmonic_tol * m) h = m;
                else if (fabs(1.0 / r - m) <= harmonic_tol * m) h = -m;
            }
        }
        peak_harm[q] = h;
    }
    free(ri); free(rh); free(rw); free(taken);
    return listed;
}

/* ---------------------------------------------------------------- CNN */

#define L0 256
#define C1 16
#define C2 32
#define C3 64
#define KW 5
#define NF 2048
#define NH 256

typedef struct {
    const double *w1, *b1, *w2, *b2, *w3, *b3, *wf1, *bf1, *wf2, *bf2;
} or_cnn_params;

typedef struct {
    double *w1, *b1, *w2, *b2, *w3, *b3, *wf1, *bf1, *wf2, *bf2;
} or_cnn_grads;

/*
 * Noise normalisation of one folded profile (Sec. 2.1): m = mean of the non-empty
 * bins, s = their population standard deviation, x_b = m + (v_b - m) / s; an empty
 * bin takes the value m; if s = 0 every bin takes m. A bin is empty when its count is
 * 0 (count != NULL) or its value is NaN (count == NULL).
 */
void or_cnn_normalise(const float *v, const int32_t *count, double *x)
{
    double m = 0.0, n = 0.0;
    for (int b = 0; b < L0; b++) {
        int empty = count ? (count[b] == 0) : isnan(v[b]);
        if (!empty) { m += v[b]; n += 1.0; }
    }
    if (n == 0.0) { for (int b = 0; b < L0; b++) x[b] = 0.0; return; }
    m /= n;
    double var = 0.0;
    for (int b = 0; b < L0; b++) {
        int empty = count ? (count[b] == 0) : isnan(v[b]);
        if (!empty) var += ((double)v[b] - m) * ((double)v[b] - m);
    }
    double s = sqrt(var / n);
    for (int b = 0; b < L0; b++) {
        int empty = count ? (count[b] == 0) : isnan(v[b]);
        x[b] = (empty || s == 0.0) ? m : m + ((double)v[b] - m) / s;
    }
}

/* Circular 1-D cross-correlation, padding 2: out[co][l] = b[co] +
 * sum_ci sum_k w[co][ci][k] * in[ci][(l + k - 2) mod L]. */
static void conv_circ(const double *in, int cin, int L, const double *w, const double *b,
                      int cout, double *out)
{
    for (int co = 0; co < cout; co++)
        for (int l = 0; l < L; l++) {
            double acc = b[co];
            for (int ci = 0; ci < cin; ci++)
                for (int k = 0; k < KW; k++) {
                    int src = ((l + k - 2) % L + L) % L;
                    acc += w[(co * cin + ci) * KW + k] * in[ci * L + src];
                }
            out[co * L + l] = acc;
        }
}

/* ReLU then max-pool (k2 s2): out[c][j] = max(relu(a[c][2j]), relu(a[c][2j+1])).
 * arg[c][j] records which input (2j or 2j+1) is the first maximum. */
static void relu_pool(const double *a, int C, int L, double *out, int *arg)
{
    for (int c = 0; c < C; c++)
        for (int j = 0; j < L / 2; j++) {
            double u = a[c * L + 2 * j], v = a[c * L + 2 * j + 1];
            u = u > 0.0 ? u : 0.0;
            v = v > 0.0 ? v : 0.0;
            int which = (v > u) ? 1 : 0;
            out[c * (L / 2) + j] = which ? v : u;
            if (arg) arg[c * (L / 2) + j] = 2 * j + which;
        }
}

/* Saved activations of one forward pass (per profile). */
typedef struct {
    double x[L0];
    double a1[C1 * 256], h1[C1 * 128];
    double a2[C2 * 128], h2[C2 * 64];
    double a3[C3 * 64], h3[C3 * 32];
    double z1[NH], r1[NH];
    double z;
    int p1[C1 * 128], p2[C2 * 64], p3[C3 * 32];
} or_cnn_acts;

size_t or_cnn_acts_size(void) { return sizeof(or_cnn_acts); }

/* Forward of one normalised profile x[256]; returns the logit z (sigmoid(z) is the
 * score). If acts != NULL the intermediate values are saved for the backward. */
double or_cnn_forward_one(const or_cnn_params *p, const double *x, or_cnn_acts *acts)
{
    or_cnn_acts local;
    or_cnn_acts *A = acts ? acts : &local;
    memcpy(A->x, x, sizeof(double) * L0);
    conv_circ(A->x, 1, 256, p->w1, p->b1, C1, A->a1);
    relu_pool(A->a1, C1, 256, A->h1, A->p1);
    conv_circ(A->h1, C1, 128, p->w2, p->b2, C2, A->a2);
    relu_pool(A->a2, C2, 128, A->h2, A->p2);
    conv_circ(A->h2, C2, 64, p->w3, p->b3, C3, A->a3);
    relu_pool(A->a3, C3, 64, A->h3, A->p3);
    /* flatten channel-major: feature f = c*32 + l, which is the h3 memory order */
    for (int j = 0; j < NH; j++) {
        double acc = p->bf1[j];
        for (int f = 0; f < NF; f++) acc += p->wf1[j * NF + f] * A->h3[f];
        A->z1[j] = acc;
        A->r1[j] = acc > 0.0 ? acc : 0.0;
    }
    double z = p->bf2[0];
    for (int j = 0; j < NH; j++) z += p->wf2[j] * A->r1[j];
    A->z = z;
    return z;
}

/* Scores of np profiles (means [np][256], optional counts) through normalise + CNN. */
void or_cnn_score(const or_cnn_params *p, const float *folded, const int32_t *counts,
                  int64_t np, double *logit, double *score)
{
    double x[L0];
    for (int64_t k = 0; k < np; k++) {
        or_cnn_normalise(folded + k * L0, counts ? counts + k * L0 : NULL, x);
        double z = or_cnn_forward_one(p, x, NULL);
        if (logit) logit[k] = z;
        if (score) score[k] = 1.0 / (1.0 + exp(-z));
    }
}

/* Forward on already-normalised inputs x[np][256] (no normalisation step). */
void or_cnn_forward(const or_cnn_params *p, const double *x, int64_t np, double *logit)
{
    for (int64_t k = 0; k < np; k++) logit[k] = or_cnn_forward_one(p, x + k * L0, NULL);
}

/* Gradient of a circular conv: given dout[co][l], accumulate dw, db and din. */
static void conv_circ_back(const double *in, int cin, int L, const double *w, int cout,
                           const double *dout, double *dw, double *db, double *din)
{
    if (din) for (int i = 0; i < cin * L; i++) din[i] = 0.0;
    for (int co = 0; co < cout; co++)
        for (int l = 0; l < L; l++) {
            double g = dout[co * L + l];
            db[co] += g;
            for (int ci = 0; ci < cin; ci++)
                for (int k = 0; k < KW; k++) {
                    int src = ((l + k - 2) % L + L) % L;
                    dw[(co * cin + ci) * KW + k] += g * in[ci * L + src];
                    if (din) din[ci * L + src] += g * w[(co * cin + ci) * KW + k];
                }
        }
}

/* Gradient through relu+maxpool: route dh[c][j] to the recorded argmax position if
 * the pre-activation there was positive (ReLU'(0) = 0). */
static void relu_pool_back(const double *a, int C, int L, const int *arg, const double *dh,
                           double *da)
{
    for (int i = 0; i < C * L; i++) da[i] = 0.0;
    for (int c = 0; c < C; c++)
        for (int j = 0; j < L / 2; j++) {
            int src = arg[c * (L / 2) + j];
            if (a[c * L + src] > 0.0) da[c * L + src] += dh[c * (L / 2) + j];
        }
}

/*
 * Binary cross-entropy with logits, mean over the batch, and its gradient w.r.t. every
 * parameter (accumulated into g, which the caller zeroes) and optionally w.r.t. the
 * inputs (dx[np][256]). loss = mean_k [max(z,0) - z*y + log1p(exp(-|z|))],
 * dloss/dz_k = (sigmoid(z_k) - y_k) / np. Returns the loss.
 */
double or_cnn_loss_backward(const or_cnn_params *p, const double *x, const float *labels,
                            int64_t np, or_cnn_grads *g, double *dx)
{
    or_cnn_acts *A = (or_cnn_acts *)malloc(sizeof(or_cnn_acts));
    double *d_r1 = (double *)malloc(sizeof(double) * NH);
    double *d_h3 = (double *)malloc(sizeof(double) * NF);
    double *d_a3 = (double *)malloc(sizeof(double) * C3 * 64);
    double *d_h2 = (double *)malloc(sizeof(double) * C2 * 64);
    double *d_a2 = (double *)malloc(sizeof(double) * C2 * 128);
    double *d_h1 = (double *)malloc(sizeof(double) * C1 * 128);
    double *d_a1 = (double *)malloc(sizeof(double) * C1 * 256);
    double loss = 0.0;
    for (int64_t k = 0; k < np; k++) {
        double z = or_cnn_forward_one(p, x + k * L0, A);
        double y = (double)labels[k];
        loss += (z > 0.0 ? z : 0.0) - z * y + log1p(exp(-fabs(z)));
        double dz = (1.0 / (1.0 + exp(-z)) - y) / (double)np;
        g->bf2[0] += dz;
        for (int j = 0; j < NH; j++) {
            g->wf2[j] += dz * A->r1[j];
            d_r1[j] = A->z1[j] > 0.0 ? dz * p->wf2[j] : 0.0;
        }
        for (int f = 0; f < NF; f++) d_h3[f] = 0.0;
        for (int j = 0; j < NH; j++) {
            g->bf1[j] += d_r1[j];
            for (int f = 0; f < NF; f++) {
                g->wf1[j * NF + f] += d_r1[j] * A->h3[f];
                d_h3[f] += d_r1[j] * p->wf1[j * NF + f];
            }
        }
        relu_pool_back(A->a3, C3, 64, A->p3, d_h3, d_a3);
        conv_circ_back(A->h2, C2, 64, p->w3, C3, d_a3, g->w3, g->b3, d_h2);
        relu_pool_back(A->a2, C2, 128, A->p2, d_h2, d_a2);
        conv_circ_back(A->h1, C1, 128, p->w2, C2, d_a2, g->w2, g->b2, d_h1);
        relu_pool_back(A->a1, C1, 256, A->p1, d_h1, d_a1);
        conv_circ_back(A->x, 1, 256, p->w1, C1, d_a1, g->w1, g->b1, dx ? dx + k * L0 : NULL);
    }
    free(A); free(d_r1); free(d_h3); free(d_a3); free(d_h2); free(d_a2); free(d_h1); free(d_a1);
    return loss / (double)np;
}
