/*
 * gpfc.h -- C ABI of the GPFC fold + score library (libgpfc.so, sm_103a).
 *
 * The library folds a detrended light curve at every trial period of a grid into
 * phase-binned profiles and scores each profile (paper Sec. 2.1, Fig. 1: fold, noise
 * normalisation, CNN score per trial period; Sec. 3.1: box-fitting statistic as the
 * plain detector).
 *
 * Conventions for every call:
 *  - Array arguments are DEVICE pointers owned by the caller (unless a comment says
 *    "host"). The library never frees them and never keeps them after the call.
 *  - Work is enqueued on the context's CUDA stream and runs asynchronously. A call
 *    returns GPFC_OK once its work is enqueued; argument errors found on the host are
 *    returned at once. Errors found on the device (an invalid period, a time outside
 *    the fixed-point range, a wait that timed out) are latched in the context and
 *    returned by gpfc_sync() and by the next call on the context.
 *  - Status codes are the negative gpfc_status values; GPFC_OK is 0. No call throws.
 *  - A context is used by one host thread at a time.
 */
#ifndef GPFC_H
#define GPFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPFC_OK = 0,
    GPFC_EINVAL = -1,   /* bad argument: NULL pointer, size out of range */
    GPFC_ENOMEM = -2,   /* device workspace allocation failed */
    GPFC_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    GPFC_ERANGE = -4,   /* a period is not finite and > 0, or |tau| / F overflow */
    GPFC_ETIMEOUT = -5, /* a bounded device-side wait gave up */
    GPFC_ENOTSUP = -6   /* valid but unsupported configuration (e.g. CNN with nbins != 256) */
} gpfc_status;

typedef struct gpfc_ctx gpfc_ctx;

/* Library version, major*10000 + minor*100 + patch. */
int gpfc_version(void);

/* Static message for a status code. */
const char *gpfc_strerror(int status);

/* Create a context on CUDA device `device`, enqueuing on `stream` (a cudaStream_t;
 * NULL = the legacy default stream). The stream is borrowed, not owned. The context
 * owns a device workspace that grows on demand; *out is set to NULL on failure. */
int gpfc_create(gpfc_ctx **out, int device, void *stream);

/* Release the context and its workspace (synchronises its stream first). */
void gpfc_destroy(gpfc_ctx *ctx);

/* Change the stream later calls enqueue on (synchronises the old stream first). */
int gpfc_set_stream(gpfc_ctx *ctx, void *stream);

/* Detail text for the last failing call on this context (empty if none). With
 * ctx == NULL: the detail of the calling thread's last failed gpfc_create. */
const char *gpfc_last_error(const gpfc_ctx *ctx);

/* Wait for the context's stream, then return (and clear) any latched device error. */
int gpfc_sync(gpfc_ctx *ctx);

/* Number of multiprocessors of the context's device. */
int gpfc_num_sms(const gpfc_ctx *ctx);

/* Kernel timing. With timing enabled, each call records CUDA events on the context's
 * stream around its main kernels (the fold kernel for gpfc_fold, the fold and scoring
 * kernels for gpfc_search, the scoring kernel for gpfc_score_*). gpfc_kernel_time_ms synchronises on the stop event
 * of the last recorded launch and writes its duration in milliseconds to *ms (host).
 * Returns GPFC_EINVAL if timing is off or nothing was recorded yet. */
int gpfc_set_timing(gpfc_ctx *ctx, int enable);
int gpfc_kernel_time_ms(gpfc_ctx *ctx, float *ms);
/* With timing enabled, a gpfc_search whose box search runs in the warp-per-profile
 * kernel (gpfc_set_box_path) also records events around each of its fold launches, on
 * the side stream they run on (so a launch's time includes the scorer running beside
 * it). This writes their summed duration (ms) and their number for the last such call;
 * it synchronises on the last stop event. GPFC_EINVAL if none was recorded. */
int gpfc_fold_launch_times(gpfc_ctx *ctx, float *total_ms, int32_t *launches);

/* Launch configuration of the fold kernel (gpfc_fold, gpfc_search, gpfc_search_batched).
 * Every field 0 means "automatic" (the autotuner's choice if it has one, else a default).
 * Layouts 1 and 2 give bit-identical outputs for any warps, tile and blocks_per_sm (chunk
 * changes the FP32 rounding of the per-chunk partial sums). Layout 3 sums flux quantised to
 * multiples of 2^-e (e per star, the largest with chunk x max|x| 2^e < 2^31) exactly and
 * rounds each bin once to FP32: bit-identical for any warps, streams, tile and
 * blocks_per_sm; chunk sets e.
 *   warps          warps per block, 32 trial periods per warp (1..16, capped by shared memory)
 *   layout         shared-memory bins: 1 = FP32 sum + 16-bit count (6 B per bin),
 *                  2 = FP32 sum + 32-bit count in one 64-bit word (8 B per bin),
 *                  3 = fixed-point 32-bit sum + 32-bit count updated by shared-memory
 *                  reductions (8 B per bin; flux quantised per star, see gpfc_fold)
 *   chunk          samples per compensated chunk (rounded down to a multiple of 16, 256..65520)
 *   tile           light-curve samples per bulk copy into shared memory: 512, 1024 or 2048
 *   blocks_per_sm  resident blocks per multiprocessor of the persistent grid (capped by
 *                  what fits)
 *   streams        layout 3 only: fold warps per period group (1..12 with warps x streams
 *                  <= 12). With up to three period groups the block's warps x streams warps
 *                  each fold a disjoint share of the samples into the bins of every group;
 *                  with more, each group's streams fold into that group. The box epilogue
 *                  of gpfc_search uses 1 where its streams' merge does not fit in a tile. */
typedef struct {
    int32_t warps;
    int32_t layout;
    int32_t chunk;
    int32_t tile;
    int32_t blocks_per_sm;
    int32_t streams;
} gpfc_fold_config;

/* Set (cfg != NULL) or reset to automatic (cfg == NULL) the context's fold config.
 * GPFC_EINVAL if a field is out of range. */
int gpfc_set_fold_config(gpfc_ctx *ctx, const gpfc_fold_config *cfg);

/* Largest `warps` the fold kernel fits in shared memory for nbins and layout with
 * 1024-sample tiles (0 if none). */
int gpfc_fold_max_warps(int32_t nbins, int32_t layout);

/* The launch config of the context's most recent fold launch plan (all fields filled). */
int gpfc_last_fold_plan(const gpfc_ctx *ctx, gpfc_fold_config *out);

/* Autotuner. gpfc_autotune times the fold kernel on the given star (device arrays, as
 * for gpfc_search) over its first min(n_periods, 4 * 128 * SMs) periods for every launch
 * config (layout x tile x warps, with the blocks per SM that fit) whose resident periods
 * per SM are at least half the largest, among the layouts of the same arithmetic as the
 * default (or the set) layout: 1 and 2 (FP32 partial sums), or 3 (fixed point), so a tuned
 * config gives the same results as the default one; it keeps the fastest in the context under
 * (nbins, scorer, floor(log2 n)). scorer GPFC_SCORER_BOX times the fold with its box-SNR
 * epilogue (scorer_params: gpfc_box_params*), GPFC_SCORER_CNN the fold that writes
 * profiles (scorer_params unused). The chosen config goes to *out (host, may be NULL).
 * It synchronises the context's stream (GPFC_EINVAL under stream capture) and writes
 * nothing the caller owns.
 * With autotuning enabled (the default), gpfc_fold, gpfc_search and gpfc_search_batched
 * use a tuned config with a matching key, and gpfc_search_batched tunes on its first
 * star when there is none (keyed by the average star length), unless its stream is
 * capturing. gpfc_set_autotune(ctx, 0) disables both; enable < 0 also forgets the
 * tuned configs. Fields set by gpfc_set_fold_config take precedence. */
int gpfc_autotune(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n,
                  const double *periods, int64_t n_periods, int32_t nbins, int scorer,
                  const void *scorer_params, gpfc_fold_config *out);
int gpfc_set_autotune(gpfc_ctx *ctx, int enable);

/* Self-test of the device-side failure path. Every wait in the kernels (on the
 * bulk-copy and tensor-core mbarriers) gives up after about two seconds, latches a
 * timeout bit, lets the block's own copies and MMAs land and returns, so a stuck wait
 * never hangs the GPU. This call launches one thread that waits on an mbarrier nothing
 * arrives on, with a limit of limit_cycles clock cycles (1e3 .. 4e9): the wait gives up,
 * and gpfc_sync (or the next call) returns GPFC_ETIMEOUT. The context stays usable. */
int gpfc_check_wait_timeout(gpfc_ctx *ctx, int64_t limit_cycles);

/* Device workspace (bytes) the context needs for gpfc_fold, or gpfc_search with the box
 * scorer on either box path, of one star of n samples over n_periods periods under the
 * current launch config. */
int gpfc_workspace_size(gpfc_ctx *ctx, int64_t n, int64_t n_periods, int32_t nbins, size_t *bytes);

/* ------------------------------------------------------------------ fold
 * Phase fold (Sec. 2.3: modular residual of each timestamp by the trial period, map to
 * a bin, per-bin count and flux sum, mean = sum / count), with equal-width bins and the
 * phase exact in 64-bit fixed point:
 *     tau_i = rint((times_i - t0) * 2^24)            (int64, round-to-nearest-even)
 *     F_k   = rint(2^40 / periods_k)                 (uint64)
 *     bin   = floor(((tau_i * F_k) mod 2^64) * nbins / 2^64)
 * so the bin index equals floor(frac((t - t0)/P) * nbins) up to the 2^-25 d time and
 * 2^-41 c/d frequency quanta, and is bit-identical on every run and machine.
 *
 * times   [n]            float64, days, any order
 * flux    [n]            float32
 * periods [n_periods]    float64, days, finite and > 0 (else GPFC_ERANGE, latched)
 * nbins                  2..4096
 * t0                     phase origin in days; NaN means t0 = times[0]
 * folded  [n_periods][nbins] float32 row-major, per-bin mean flux, NaN for an empty bin;
 *                        may be NULL (not written)
 * counts  [n_periods][nbins] int32 row-major, samples per bin; may be NULL
 * Sums are of x = float32(flux - mean flux); counts are exact integers. From 256 bins (fold
 * layout 3, the default) x is rounded to a multiple of 2^-e, e per star the largest with
 * max|x| 2^e <= floor((2^31 - 1) / min(chunk, n)), and the multiples are summed exactly
 * (shared-memory integer reductions, int64 across chunks), each bin rounded once to FP32:
 * a bin mean is within 2^-e / 2 of the exact mean of the x. Below 256 bins (layouts 1 and 2)
 * they are accumulated in FP32 with Kahan compensation (chunk partials in shared memory,
 * compensated across chunks). Above 1024 bins (more than a lane's shared-memory share) the
 * fold adds each sample with shared-memory atomics per period into count << 40 plus the
 * flux sum in fixed point (quantum 2^-k with n max|x| 2^k < 2^38, or up to 65,536 samples
 * two 32-bit reductions with n max|x| 2^k < 2^31): exact sums, rounded once.
 * Limits: 1 <= n <= 2^24 (n < 2^24 above 1024 bins), 1 <= n_periods <= 2^31 - 1,
 * |tau| < 2^62, F < 2^63. */
int gpfc_fold(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n,
              const double *periods, int64_t n_periods, int32_t nbins, double t0,
              float *folded, int32_t *counts);

/* ------------------------------------------------------------------ box-SNR
 * Box statistic per folded profile (the box-fitting idea of Sec. 3.1, BLS). For every
 * width w in [w_min, w_max] and start bin s, the box is bins s..s+w-1 (mod nbins); with
 * n_in, n_out the samples inside/outside and mu_in, mu_out their mean flux,
 *     snr = (mu_out - mu_in) * sqrt(n_in * n_out / N) / sigma
 * over boxes with n_in >= 1 and n_out >= 1. The score is the largest snr (ties: smaller
 * w, then smaller s); -inf with best_s = best_w = -1 when no box is valid. */
typedef struct {
    int32_t w_min;  /* >= 1 */
    int32_t w_max;  /* w_min..nbins */
    double sigma;   /* noise scale; <= 0 means 1 (standalone scoring) or the
                       population std of the light curve's flux (gpfc_search) */
} gpfc_box_params;

/* folded [n_periods][nbins] float32 means (NaN or count 0 marks an empty bin);
 * counts [n_periods][nbins] int32 (required); score [n_periods] float32;
 * best_s / best_w [n_periods] int32, may be NULL. Limits: nbins 2..4096,
 * per-profile sample count N <= 2^24. Each profile is centred on its count-weighted
 * mean (FP64) and scored by one warp (the search kernel of gpfc_set_box_path). */
int gpfc_score_box(gpfc_ctx *ctx, const float *folded, const int32_t *counts,
                   int64_t n_periods, int32_t nbins, const gpfc_box_params *params,
                   float *score, int32_t *best_s, int32_t *best_w);

/* ------------------------------------------------------------------ CNN scorer
 * Score of each folded profile by a 1-D CNN (Sec. 2.5; the noise normalisation of
 * Sec. 2.1 first scales each profile to unit standard deviation while keeping its mean):
 *   conv(1->16,k5) ReLU maxpool2, conv(16->32,k5) ReLU maxpool2, conv(32->64,k5) ReLU
 *   maxpool2, flatten (channel-major, 2048), fc(2048->256) ReLU, fc(256->1), sigmoid.
 * Convolutions are circular with padding 2. Normalisation over the non-empty bins:
 * m = their mean, s = their population std, x_b = m + (v_b - m) / s, empty bins -> m,
 * s = 0 -> every x_b = m. Computation: BF16 inputs, weights and activations, FP32
 * accumulation on the tensor cores.
 * Parameters are FP32 device tensors in PyTorch layout: conv1_w [16][1][5],
 * conv2_w [32][16][5], conv3_w [64][32][5], fc1_w [256][2048], fc2_w [1][256] and their
 * biases; they are rounded to BF16 on every call. */
typedef struct {
    const float *conv1_w, *conv1_b, *conv2_w, *conv2_b, *conv3_w, *conv3_b;
    const float *fc1_w, *fc1_b, *fc2_w, *fc2_b;
} gpfc_cnn_weights;

/* folded [n_periods][256] float32 means; counts [n_periods][256] int32 or NULL (then a
 * NaN mean marks an empty bin); nbins must be 256 (else GPFC_ENOTSUP);
 * score [n_periods] float32 in (0, 1). */
int gpfc_score_cnn(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                   int32_t nbins, const gpfc_cnn_weights *weights, float *score);

/* As gpfc_score_cnn, writing the pre-sigmoid logits z (score = 1 / (1 + exp(-z))). */
int gpfc_cnn_logits(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                    int32_t nbins, const gpfc_cnn_weights *weights, float *logit);

/* ------------------------------------------------------------------ CNN training
 * The training loop of the scorer (Sec. 2.5: Adam minimising binary cross-entropy; the
 * paper trains in TensorFlow): a forward pass that keeps its activations, the loss, the
 * backward pass and the Adam update, all on the device.
 *
 * Bytes of the activation buffer gpfc_cnn_forward_train fills for `batch` profiles. */
size_t gpfc_cnn_saved_bytes(int64_t batch);

/* Forward pass (as gpfc_cnn_logits) that also stores, in `saved` (a caller-owned device
 * buffer of gpfc_cnn_saved_bytes(batch) bytes), what the backward pass needs: the BF16
 * normalised input, pre-activations and pooled outputs, the fc1 operand and fc1's FP32
 * pre-activations. logit [batch] float32. */
int gpfc_cnn_forward_train(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t batch,
                           int32_t nbins, const gpfc_cnn_weights *weights, float *logit, void *saved);

/* Gradients of the CNN parameters, FP32 device tensors in PyTorch layout (overwritten). */
typedef struct {
    float *conv1_w, *conv1_b, *conv2_w, *conv2_b, *conv3_w, *conv3_b;
    float *fc1_w, *fc1_b, *fc2_w, *fc2_b;
} gpfc_cnn_grads;

/* Backward pass: given dL/dlogit [batch] (float32, device) for the forward that filled
 * `saved` with the same weights, write dL/dparam for every parameter. The ReLU/max-pool
 * gradient goes to the first maximum of each pooled pair; the computation is FP32 over
 * the saved BF16 activations and BF16-rounded weights. Deterministic. */
int gpfc_cnn_backward(gpfc_ctx *ctx, const float *dlogit, int64_t batch, const gpfc_cnn_weights *weights,
                      const void *saved, const gpfc_cnn_grads *grads);

/* Mean binary cross-entropy with logits over n items, loss = mean(max(z,0) - z*y +
 * log1p(exp(-|z|))), and its gradient dlogit = (sigmoid(z) - y) / n. logit, label [n]
 * float32; loss [1] and dlogit [n] float32, either may be NULL. */
int gpfc_bce_with_logits(gpfc_ctx *ctx, const float *logit, const float *label, int64_t n, float *loss,
                         float *dlogit);

/* One Adam step on n FP32 values in place (Kingma & Ba, Algorithm 1): m and v are the
 * moment buffers, step the 1-based step count used for the bias corrections. */
int gpfc_adam(gpfc_ctx *ctx, float *param, const float *grad, float *m, float *v, int64_t n, float lr,
              float beta1, float beta2, float eps, int64_t step);

/* ------------------------------------------------------------------ training profiles
 * Folded training profiles generated on the device: light curve j (global index) has
 * n_cadences samples at t_i = i * cadence (t0 = 0), flux = 1 + sigma z_i + signal, folded
 * at its true period P plus a frequency offset giving at most drift_bins bins of phase
 * drift over the baseline. Even j: a box transit (label 1). Odd j, by (j/2) mod 3: noise
 * only, a sinusoid, an eclipsing-binary-like primary + secondary box half a period
 * later (label 0). sigma log-uniform in [sigma_min, sigma_max]; P uniform in
 * [p_min, p_max] days; epoch uniform in [0, P); duration uniform in [dur_min_h,
 * dur_max_h] hours; depth (and sinusoid amplitude) log-uniform in [depth_min,
 * depth_max]; secondary depth = depth * U[0.2, 1]. Random numbers: Philox4x32-10
 * (Salmon et al. 2011) keyed by `seed`; counter (j, 0, 0, 2^32-1) and (j, 1, 0, 2^32-1)
 * for the parameters, (j, i/4, 1, 0) for the normals of samples 4(i/4)..4(i/4)+3 via
 * Box-Muller on u = (x >> 8) 2^-24. The fold is the 64-bit fixed-point fold of
 * gpfc_fold (t0 = 0), one light curve per block, bins merged within a warp with
 * __match_any_sync; the means are 1 + (sum of (flux - 1)) / count. */
typedef struct {
    int32_t n_cadences;
    double cadence;
    double sigma_min, sigma_max;
    double depth_min, depth_max;
    double dur_min_h, dur_max_h;
    double p_min, p_max;
    double drift_bins;
} gpfc_synth_params;

/* folded [n][nbins] float32 (NaN = empty bin); counts [n][nbins] int32, label [n]
 * float32, fold_period [n] float64 and flux_std [n] float32 (population std of each
 * light curve's flux, the noise scale gpfc_search uses) may be NULL. nbins 2..256. */
int gpfc_synth_profiles(gpfc_ctx *ctx, uint64_t seed, int64_t first, int64_t n, int32_t nbins,
                        const gpfc_synth_params *params, float *folded, int32_t *counts, float *label,
                        double *fold_period, float *flux_std);

/* The paper's own training-set recipe (Sec. 2.6, Sec. 2.7): vector j (global index j =
 * first + i) of length nbins stands for a folded light curve: Gaussian noise plus a
 * trapezoid transit whose depth gives a target SNR alpha by Eq. 2,
 *     alpha = (d / sigma) sqrt(n_points L / p)   =>   d = alpha sigma / sqrt(n_points q),
 * with q = L/p the duration at half depth over the period (phase units). Even j:
 * positive, alpha ~ U[alpha_pos_min, alpha_pos_max] (label 1). Odd j: negative (label 0),
 * noise only when (j / 2) is even, else a transit with alpha ~ U(0, alpha_neg_max). The
 * per-point noise sigma is log-uniform in [sigma_min, sigma_max]; a bin averages
 * n_points / nbins points, so its noise is sigma sqrt(nbins / n_points). The trapezoid's
 * short-to-long base ratio is r ~ U(0, 1) (long base 2q / (1 + r)), its centre phase
 * phi0 ~ U[0, 1); it is evaluated at the bin centres (b + 1/2) / nbins. Values are
 * 1 + noise - d * shape. Random numbers: Philox4x32-10 keyed by `seed`, counters
 * (j, 0, 2, 2^32-1) and (j, 1, 2, 2^32-1) for the parameters, (j, m, 3, 0) for the
 * normals of bins 4m..4m+3 (Box-Muller on u = (x >> 8) 2^-24).
 * The paper does not give the negatives' lower SNR bound, the split between noise-only
 * and injected negatives, the n of Eq. 2 for its 256-vectors or the trapezoid's phase:
 * these are this library's readings. */
typedef struct {
    double alpha_pos_min, alpha_pos_max;
    double alpha_neg_max;
    double q_min, q_max;
    double sigma_min, sigma_max;
    int32_t n_points;
} gpfc_vector_params;

/* folded [n][nbins] float32 (every bin non-empty); label [n], alpha [n] and sigma_bin [n]
 * float32 (the per-bin noise) may be NULL. nbins 8..1024; first + n <= 2^32. */
int gpfc_synth_vectors(gpfc_ctx *ctx, uint64_t seed, int64_t first, int64_t n, int32_t nbins,
                       const gpfc_vector_params *params, float *folded, float *label, float *alpha,
                       float *sigma_bin);

/* ------------------------------------------------------------------ best period
 * argmax over score[n_periods] (NaN never wins; ties go to the smaller index), Sec. 2.1:
 * the trial period with the strongest score. best_index [1] int64 (-1 if every score is
 * NaN), best_score [1] float32; device pointers. */
int gpfc_best_period(gpfc_ctx *ctx, const float *score, int64_t n_periods,
                     int64_t *best_index, float *best_score);

/* Allocation-free best period. The paper has no counterpart: this entry point exists
 * for callers that cannot allocate memory at the point of the call (a region where
 * cudaMalloc is not allowed, a pre-planned memory budget, a hot loop kept off the
 * allocator). They cannot call gpfc_create either, since it allocates, so this call
 * takes a cudaStream_t (NULL = legacy default stream) instead of a context and runs on
 * the current CUDA device. It computes what gpfc_best_period computes, with its only
 * scratch, one 8-byte argmax key, in a static device array that every GPU using the
 * library holds until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  - score [n_periods] float32, best_index [1] int64, best_score [1] float32: device
 *    pointers; either output may be NULL, not both.
 *  - n_periods must be 1..2^31-1 (the key stores a 32-bit index); else GPFC_EINVAL.
 *  - The first call on a device looks up the scratch address (cudaGetSymbolAddress);
 *    make that first call before any stream capture.
 *  - All calls share the one key: calls that overlap on the GPU (different streams, or
 *    different host threads without ordering) race and may return each other's result.
 *    The key is cleared at the start of every call.
 * Returns GPFC_OK, GPFC_EINVAL (checked before any CUDA call) or GPFC_ECUDA (enqueue
 * failure). If an error from earlier work is already pending in the calling thread
 * (cudaPeekAtLastError), the call returns GPFC_ECUDA at once, launches nothing and leaves
 * that error pending for its owner. */
int gpfc_best_period_noalloc(const float *score, int64_t n_periods, int64_t *best_index,
                             float *best_score, void *stream);

/* ------------------------------------------------------------------ two-tier fold
 * The paper's own fold (Sec. 2.3, Fig. 4 (a)-(e)): each sample goes to one of nfine
 * equal-width fine bins by its fixed-point phase (as in gpfc_fold); the fine bins are then
 * merged left to right into nbins final bins of exactly n / nbins samples each, the fine
 * bin that straddles a boundary giving each side the share of its flux sum that it gives
 * of its samples (the paper does not say how a boundary bin's sum is divided; this
 * proportional split is this library's reading); each output is the bin's mean flux. No
 * final bin is empty. The paper uses nfine = 4096, nbins = 256.
 *  - times [n] f64, flux [n] f32, periods [n_periods] f64: device; folded [n_periods][nbins]
 *    f32 means: device, caller-owned.
 *  - 1 <= n < 2^24; 2 <= nbins <= nfine <= 4096; t0 as for gpfc_fold.
 * Sums are exact fixed-point integers (quantum 2^-k per light curve, with
 * n max|flux - mean| 2^k < 2^38), so the result does not depend on summation order.
 * Returns GPFC_OK, GPFC_EINVAL, GPFC_ENOTSUP or GPFC_ECUDA; bad periods are reported
 * later as GPFC_ERANGE. */
int gpfc_fold_equal_count(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n,
                          const double *periods, int64_t n_periods, int32_t nfine, int32_t nbins,
                          double t0, float *folded);

/* ------------------------------------------------------------------ search
 * Fold + score (Fig. 1) without returning the profiles. scorer GPFC_SCORER_BOX takes a
 * gpfc_box_params* in scorer_params; the search runs where gpfc_set_box_path says (below).
 * GPFC_SCORER_CNN takes a gpfc_cnn_weights* (nbins must be
 * 256): periods are folded in chunks whose profiles stay in L2 for the CNN kernels.
 * score [n_periods] float32; best_index [1] int64 and best_score [1] float32 (device,
 * may be NULL). Limits as for gpfc_fold. */
typedef enum { GPFC_SCORER_BOX = 0, GPFC_SCORER_CNN = 1 } gpfc_scorer;

/* Where the box-SNR search runs. GPFC_BOX_EPILOGUE: in the fold kernel, on the profile
 * held on chip (no profile traffic, but only as many warps as the fold's bins leave room
 * for). GPFC_BOX_WARP: the fold writes each chunk's centred bin sums and counts to an
 * L2-resident buffer and a separate kernel scores them, one warp per profile, at full
 * occupancy. GPFC_BOX_FUSED: one kernel; each fold block has one more warp that scores
 * the block's previous task, one profile at a time, from a two-slot ring of sums and
 * counts in L2, and the fold warps take leftover profiles when they would otherwise wait
 * for a slot (when the extra warp's shared memory does not fit, GPFC_BOX_WARP is used; a
 * batched search whose tuned fold block leaves no room takes the default fold block).
 * GPFC_BOX_AUTO (the default) takes GPFC_BOX_FUSED from nbins >= 256, else the epilogue;
 * with fold layout 3 (the default from 256 bins) the one-kernel block does not fit beside
 * twelve fold warps, so GPFC_BOX_WARP runs.
 * The box scores of the warp and fused paths are bit-identical; a batched search and the
 * per-star search agree bit for bit whatever the path. */
typedef enum { GPFC_BOX_AUTO = 0, GPFC_BOX_EPILOGUE = 1, GPFC_BOX_WARP = 2, GPFC_BOX_FUSED = 3 } gpfc_box_path;
int gpfc_set_box_path(gpfc_ctx *ctx, int path);

int gpfc_search(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n,
                const double *periods, int64_t n_periods, int32_t nbins, double t0,
                int scorer, const void *scorer_params, float *score,
                int64_t *best_index, float *best_score);

/* ------------------------------------------------------------------ per-star decision
 * Decision over periodograms (the scores of gpfc_search / gpfc_search_batched, one per
 * trial period). For each star, over its finite scores: the mean and population standard
 * deviation; SDE = (max - mean) / sd (Eq. 3; 0 when sd is 0); peaks as in Sec. 4.2:
 * maximal runs of consecutive periods scoring above mean + k_sigma * sd that are at least
 * min_width periods wide (the paper's "height of 3 sigma and width of more than 3" is
 * k_sigma = 3, min_width = 4). A peak's height is its largest score (first occurrence).
 * The best peak is the highest (ties: smaller index). The highest max_peaks peaks are
 * listed, each with a harmonic flag against the best peak's period Pb (Fig. 14 shows
 * peaks at harmonics of the transit period): 1 for the best, +m if its period is m Pb,
 * -m if it is Pb / m (m = 2..4, within relative tolerance harmonic_tol), else 0.
 * Non-finite scores are left out of the statistics and end a run. */
typedef struct {
    double sde;
    double mean;
    double sd;
    int64_t best_index;   /* index into the star's grid of the best peak, -1 if none */
    float best_score;     /* its height (NaN if none) */
    int32_t n_peaks;      /* qualifying peaks */
    int32_t truncated;    /* 1 if more than 2048 qualified: the list covers the first 2048 found */
    int32_t n_listed;     /* entries written to the star's peak list */
} gpfc_star_summary;

typedef struct {
    int64_t index;        /* into the star's grid */
    float height;
    int32_t width;        /* periods in the run */
    int32_t harmonic;
    int32_t reserved;
} gpfc_peak;

/* score [n_periods] f32 and periods [n_periods] f64: device. grid_offsets: device [n_stars+1]
 * (as for gpfc_search_batched), or NULL with n_stars = 1 for one star. summary: device
 * [n_stars]; peaks: device [n_stars][max_peaks] or NULL (0 <= max_peaks <= 64).
 * Returns GPFC_OK, GPFC_EINVAL or GPFC_ECUDA. */
int gpfc_peaks(gpfc_ctx *ctx, const float *score, const double *periods, int32_t n_stars,
               const int64_t *grid_offsets, int64_t n_periods, double k_sigma, int32_t min_width,
               double harmonic_tol, int32_t max_peaks, gpfc_star_summary *summary, gpfc_peak *peaks);

/* ------------------------------------------------------------------ pre-processing
 * Detrending of a raw light curve before the fold (Sec. 2.2, Fig. 3): the light curve is
 * cut into segments wherever two adjacent samples are more than time_gap apart in time or
 * differ in flux by more than flux_gap_sigma times the flux's population standard
 * deviation; each segment is fitted by a least-squares cubic spline (clamped end knots,
 * interior knots `spacing` days apart) with known transits masked and outliers beyond
 * clip_sigma times the RMS residual removed iteratively (a removed point can return; up to
 * max_iter fits); the spacing is chosen per segment from `spacings` by the smallest
 * BIC = n ln(RSS / n) + p ln n; the segment is divided by its fit and its first and last
 * `edge` samples are dropped; the segments are stitched in time order. The paper names the
 * steps, not the spline or the criterion: these forms are this library's reading, and the
 * normal equations carry a tiny second-difference penalty on the spline coefficients
 * (ridge times trace(B^T B) / p) so that a knot interval emptied by clipping or masking
 * stays solvable. Fields left at 0 take the defaults. */
typedef struct {
    double time_gap;        /* days; default 30 x 0.020428 (30 Kepler cadences) */
    double flux_gap_sigma;  /* default 5 */
    double clip_sigma;      /* default 3 */
    double ridge;           /* default 1e-9 */
    int32_t edge;           /* samples dropped at each end of a segment; default 30 (set -1 for 0) */
    int32_t max_iter;       /* fits per candidate spacing; default 10 */
    int32_t n_spacings;     /* 0..8; default 5: 0.5, 1, 1.5, 2, 3 days */
    int32_t reserved;
    double spacings[8];     /* days, each > 0 */
} gpfc_detrend_params;

/*  - times [n] float64 (strictly increasing), flux [n] float32: device; 1 <= n <= 2^24.
 *  - mask [n] uint8 (device) or NULL: nonzero = a known transit, never used in a fit (its
 *    samples are still divided by the fit and returned).
 *  - times_out [n] float64, flux_out [n] float32 (flux / fit), segment_out [n] int32 (the
 *    sample's segment index, or NULL): device, caller-owned; the first *n_out entries are
 *    written. n_out [1] int64: device.
 * Everything runs in FP64 on the device; reductions run in a fixed order, so the result
 * does not depend on scheduling. Returns GPFC_OK, GPFC_EINVAL, GPFC_ENOMEM or GPFC_ECUDA. */
int gpfc_detrend(gpfc_ctx *ctx, const double *times, const float *flux, const uint8_t *mask, int64_t n,
                 const gpfc_detrend_params *params, double *times_out, float *flux_out,
                 int32_t *segment_out, int64_t *n_out);

/* ------------------------------------------------------------------ detection statistics
 * ROC statistics of a detector on labelled scores: the paper compares detectors by ROC
 * curves of stars, each star scored by its best trial period (Sec. 3.2, Figs. 10-13).
 *  - pos [n_pos], neg [n_neg] float32 scores (device), 1 <= n_pos, n_neg <= 2^30. A NaN
 *    score ranks below every number (never a detection).
 *  - u2 [1] int64 (device): sum over all (i, j) of 2 [pos_i > neg_j] + [pos_i == neg_j],
 *    twice the Mann-Whitney U statistic; AUC = u2 / (2 n_pos n_neg), exactly.
 *  - fpr [n_fpr] float64 HOST array of false-positive rates in [0, 1), 0 <= n_fpr <= 16:
 *    for each, k = floor(fpr n_neg) and thr [f] float32 (device) = the (k+1)-th largest
 *    negative score (-inf if k >= n_neg), tp [f] int64 (device) = #{pos_i > thr}; so
 *    TPR = tp / n_pos at a false-positive rate of at most fpr. thr and tp may be NULL when
 *    n_fpr = 0.
 * Every output is a count over pairs of scores: exact, independent of launch order. Cost
 * n_neg^2 + n_pos n_neg comparisons. Returns GPFC_OK, GPFC_EINVAL or GPFC_ECUDA. */
int gpfc_roc(gpfc_ctx *ctx, const float *pos, int64_t n_pos, const float *neg, int64_t n_neg,
             int32_t n_fpr, const double *fpr, int64_t *u2, float *thr, int64_t *tp);

/* ------------------------------------------------------------------ batched search
 * gpfc_search over many stars of uneven length, each with its own period grid, in one
 * sequence of persistent launches (the paper folds one light curve at a time, Sec. 2.3;
 * batching stars is this library's addition). Stars and grids are given in CSR form,
 * all arrays DEVICE pointers owned by the caller:
 *   lc_offsets   [n_stars + 1] int64: star s has samples lc_offsets[s] .. lc_offsets[s+1]-1
 *                of times [n_total] float64 and flux [n_total] float32;
 *                lc_offsets[0] = 0, lc_offsets[n_stars] = n_total, 1..2^24 samples a star
 *   grid_offsets [n_stars + 1] int64, likewise over periods [n_periods_total] float64:
 *                star s is folded at periods grid_offsets[s] .. grid_offsets[s+1]-1 (>= 1)
 *   t0s          [n_stars] float64 phase origins, or NULL (NaN / NULL: the star's first time)
 *   score        [n_periods_total] float32: the score of every (star, period), in the
 *                order of `periods`
 *   best_index   [n_stars] int64 (may be NULL): argmax of the star's scores as an index
 *                into ITS grid (0 .. grid length - 1), ties to the smallest, -1 if none
 *   best_score   [n_stars] float32 (may be NULL)
 * nbins 2..1024 (GPFC_ENOTSUP above: the fixed-point fold of larger bin counts runs one
 * star at a time through gpfc_search).
 * scorer / scorer_params as for gpfc_search. Every score equals the one gpfc_search gives
 * for that star alone (bit for bit).
 * The offsets are validated on the device (no host synchronisation): a violation is
 * latched and returned as GPFC_EINVAL by the next call or gpfc_sync, and the kernels then
 * run on clamped offsets, staying inside the arrays.
 * The launch sequence is captured into a CUDA graph on a private stream and replayed on
 * the context's stream when an identical call (same pointers, sizes, parameters and
 * workspace) follows; gpfc_set_graph(ctx, 0) enqueues the kernels directly instead. When
 * the context's stream is itself capturing, the kernels are enqueued into that capture,
 * provided the workspace is already large enough (make one identical call first).
 * The timed region of gpfc_set_timing covers the whole sequence. */
int gpfc_search_batched(gpfc_ctx *ctx, int32_t n_stars, const int64_t *lc_offsets,
                        const double *times, const float *flux, int64_t n_total,
                        const int64_t *grid_offsets, const double *periods,
                        int64_t n_periods_total, const double *t0s, int32_t nbins, int scorer,
                        const void *scorer_params, float *score, int64_t *best_index,
                        float *best_score);
int gpfc_set_graph(gpfc_ctx *ctx, int enable);

/* ------------------------------------------------------------------ measurement
 * Peak rate of the fold's binding pipe. The paper has no counterpart: it is the
 * denominator of the fold's roofline. The accumulation of Sec. 2.3 step 3 is one
 * read-modify-write of a trial period's bin record in shared memory per sample and
 * period; this call times a kernel that does only that, with each lane's records laid out
 * [bin][lane] as the fold keeps them, eight distinct bins updated per iteration, and
 * reports the rate.
 *  - word_bytes 8: op 0: FP32 sum + 32-bit count packed in 64 bits, one 64-bit load and
 *    store per update (fold layout 2); op 1: a 32-bit sum word and a 32-bit count word
 *    128 bytes apart (256 bytes per bin of a warp), two red.shared.add.u32 per update
 *    (fold layout 3); 6: FP32 sum word plus a 16-bit
 *    count, two counts per 32-bit word (op 0: 32-bit and 16-bit loads and stores; op 1:
 *    red.shared.add.f32 to the sum and red.shared.add.u32 to the paired count); 4: one
 *    32-bit word (op 0: load and store; op 1: red.shared.add.u32).
 *  - nbins (power of two, 8..4096) words per lane, warps per block (1..32), blocks_per_sm
 *    co-resident blocks per SM (the call checks they fit), iters iterations of 8 updates.
 *  - Runs on the current device and `stream` (a cudaStream_t, NULL = default stream) and
 *    synchronises on its own events; allocates two small device buffers.
 *  - updates_per_s: lane-updates per second (CUDA events); updates_per_clk_sm: per SM
 *    clock cycle (clock64 span of the slowest block). Either may be NULL.
 * Returns GPFC_OK, GPFC_EINVAL (bad sizes, or the blocks do not fit one SM together) or
 * GPFC_ECUDA. */
int gpfc_probe_smem_rmw(int32_t word_bytes, int32_t op, int32_t nbins, int32_t warps, int32_t blocks_per_sm,
                        int64_t iters, void *stream, double *updates_per_s, double *updates_per_clk_sm);

#ifdef __cplusplus
}
#endif

#endif /* GPFC_H */
