// gpfc_kernels.h -- launch parameters shared between the host API and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gpfc {

// Device error bits, OR-ed into the context's status word (host-mapped memory).
enum : uint32_t {
    kErrRange = 1u,    // period not finite/positive, or tau / F outside the fixed point
    kErrTimeout = 2u,  // a bounded wait on an mbarrier gave up
    kErrArgs = 4u,     // batched search: star or grid offsets not a valid partition
};

constexpr int kTile = 1024;            // default light-curve samples per bulk-copy tile
constexpr int kMaxTile = 2048;         // tiles are 512, 1024 or 2048 samples
constexpr int kMaxFoldWarps = 16;      // warps per fold block (32 periods each)
constexpr int kMaxNbinsLane = 1024;    // largest nbins of the lane-private fold
constexpr int kMaxRedWarps = 12;       // warps of a kLayoutRed32 block (fold warps of all
                                       // streams, plus the scorer warp of a search block)
constexpr size_t kSmemLimit = 232448;  // opt-in shared memory per block (227 KB); kernels ask
                                       // for at most kSmemLimit - 1024 dynamic bytes

// Per-star statistics written by the prep kernels.
struct StarStats {
    double f_ref;   // mean flux (FP64)
    float f_hi;     // f_ref rounded to FP32
    float f_lo;     // f_ref - f_hi rounded to FP32
    float sigma;    // population std of the flux (FP64 reduction, rounded)
    int32_t n;      // samples of the star
    long long dtau0;  // smallest positive step between consecutive quantised times (0: none)
    int32_t qexp;     // fixed-point flux: xq = rint(x 2^qexp), |xq| <= (2^31 - 1) / chunk
    int32_t pad;
};

// Samples of all stars, quantised, at 16-byte aligned per-star offsets.
struct SampleScratch {
    uint32_t *tau_lo;   // low 32 bits of tau
    int32_t *tau_hi;    // high 32 bits of tau
    float *x;           // flux - f_ref (FP32)
    int32_t *xq;        // rint(x 2^qexp): the fixed-point flux of the reduction layout
    int32_t *thg;       // one word per 16 samples: tau_hi of the group's first sample
    uint8_t *flags;     // one byte per 16 samples: regular-cadence group (see prep)
};

// kModeSearch: fold warps write each task's centred sums and counts to a per-block
// two-slot ring (sums, counts, slot_k) and one extra warp scores them (box-SNR), with the
// fold warps taking leftover profiles when they would otherwise wait for a slot.
enum FoldMode : int { kModeFold = 0, kModeBox = 1, kModeSearch = 3 };

// Shared-memory layout of the lane-private bins (see fold.cu).
// kLayoutRed32: 8 bytes per bin (a 32-bit sum word and a 32-bit count word), accumulated
// as fixed-point integer sums and counts by no-return shared reductions
// (red.shared.add.u32).
enum FoldLayout : int { kLayoutPaired16 = 1, kLayoutPacked64 = 2, kLayoutRed32 = 3 };

struct FoldParams {
    SampleScratch smp;
    const int64_t *lc_off;     // [S+1] sample offsets, or NULL (one star of n samples)
    int64_t n;
    const double *periods;
    const int64_t *grid_off;   // [S+1] period offsets, or NULL (one grid of np periods)
    int64_t np;
    const int64_t *task_off;   // [S+1] first fold task of each star, or NULL
    int64_t ntasks;            // end of this launch's task range (host bound)
    int64_t task_begin;        // first task of this launch
    const int64_t *ntasks_dev; // device task count that also bounds the range, or NULL
    int nstars;
    const StarStats *stats;
    int nbins;
    int shift;                 // 32 - log2(nbins) if nbins is a power of two, else -1
    int warps;                 // period groups per block; periods per block = 32 * warps
    int streams;               // fold warps per period group (kLayoutRed32; else 1): warp
                               // w folds group w % warps over every streams-th sample group
    int chunk;                 // samples per shared-memory chunk: multiple of 16, <= 65520
    int layout;                // FoldLayout
    int tile;                  // samples per bulk-copy tile: 512, 1024 or 2048
    float2 *ws_sc;             // [grid][nbins][32*warps] Kahan (sum, compensation), or
                               // the int64 fixed-point sums of kLayoutRed32
    uint32_t *ws_cnt;          // [grid][nbins][32*warps] counts
    // kModeFold outputs ([global period][nbins], or [slot][nbins] when slot_k is set);
    // kModeSearch uses sums, counts and slot_k as its ring, [grid][2][32 * warps] rows
    float *folded;
    float *sums;               // centred bin sums (0 for empty bins), for the separate box scorer
    int32_t *counts;
    int64_t *slot_k;           // chunk slots: slot (task - task_begin) * 32 * warps + lane of
                               // the block gets period k, or -1 (then counts 0, means NaN)
    // kModeBox outputs
    float *score;              // [global period]
    int32_t *best_s;
    int32_t *best_w;
    unsigned long long *best_key;  // [S] argmax keys (may be NULL)
    int w_min, w_max;
    float sigma_user;          // > 0: use it; else the star's flux std (1 if that is 0)
    size_t stage_off;          // kModeSearch: byte offset of the scorer staging in shared memory
    uint32_t *status;
};

// Box-SNR over profiles the fold wrote as centred sums and counts ([row][nbins]), one warp
// per profile. Row r holds period k = slot_k[r] (skipped if < 0), or k_begin + r.
struct BoxCoopParams {
    const float *sums;            // centred bin sums, or NULL when means are given
    const float *means;           // bin means (used only where the count is > 0), or NULL
    const int32_t *counts;
    const int64_t *slot_k;
    int64_t k_begin;
    int64_t rows;
    int nbins;
    int w_min, w_max;
    float sigma_user;             // > 0: use it; else the star's flux std (1 if that is 0 or stats is NULL)
    const StarStats *stats;       // may be NULL
    const int64_t *grid_off;      // [S+1] period offsets, or NULL (one star)
    int nstars;
    float *score;                 // [global period]
    int32_t *best_s;
    int32_t *best_w;
    unsigned long long *best_key; // [S] argmax keys (may be NULL)
};

// float2 (sum, count) slots one warp of the scorer stages per profile
__host__ __device__ inline int coop_pairs(int nbins) { return nbins + (nbins >> 3) + 2; }
constexpr int kCoopWarps = 8;  // warps per block of the scorer

size_t box_coop_smem(int nbins);
cudaError_t launch_box_coop(const BoxCoopParams &p, int num_sms, cudaStream_t st);

size_t fold_smem_bytes(int nbins, int warps, int layout, int tile = kTile);
int fold_max_warps(int nbins, int layout, int tile = kTile);
int fold_blocks_per_sm(int nbins, int warps, int layout, int tile, int streams = 1);
int fold_register_kernels();

cudaError_t launch_prep(const double *times, const float *flux, const int64_t *lc_off, int64_t n,
                        int nstars, int64_t max_len, const double *t0s, double t0, SampleScratch smp,
                        double *partial, int G, StarStats *stats, uint32_t *status, cudaStream_t st,
                        int chunk = 65520);
cudaError_t launch_fold(const FoldParams &p, int mode, int grid, cudaStream_t st);
// Shared memory of a kModeSearch block (0 if it does not fit or warps + 1 > 4).
size_t search_smem_bytes(int nbins, int warps, int layout, int tile, int streams = 1);
int search_blocks_per_sm(int nbins, int warps, int layout, int tile, int streams = 1);
cudaError_t launch_argmax(const float *score, int64_t np, unsigned long long *key, cudaStream_t st);
cudaError_t launch_batch_plan(const int64_t *lc_off, const int64_t *grid_off, int nstars, int64_t n_total,
                              int64_t np_total, int ppc, int64_t *lc_s, int64_t *grid_s, int64_t *task_off,
                              uint32_t *status, cudaStream_t st);
cudaError_t launch_argmax_segmented(const float *score, const int64_t *grid_off, int nstars,
                                    unsigned long long *key, int num_sms, cudaStream_t st);
cudaError_t launch_wait_selftest(long long limit, uint32_t *status, cudaStream_t st);
cudaError_t launch_argmax_finalize(const unsigned long long *key, int nstars, int64_t *best_index,
                                   float *best_score, cudaStream_t st);

inline int64_t scratch_elems(int64_t total_samples, int nstars)
{
    return 256 * ((total_samples + 255) / 256 + nstars) + 2 * kMaxTile;
}

}  // namespace gpfc
