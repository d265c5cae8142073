// gpfc_twotier.h -- launch parameters of the two-tier equal-count fold (twotier.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gpfc_kernels.h"

namespace gpfc {

constexpr int kEqMaxPeriods = 8;   // periods a block folds at a time
constexpr int kEqMaxFine = 4096;   // largest number of fine bins
constexpr int64_t kEqRed32MaxN = 65536;  // up to this many samples: 32-bit reductions

// The fine bins of a star of n samples are folded by two 32-bit shared-memory reductions
// per update (fixed-point sum and count rows) when every bin sum then fits in 32 bits with
// at least 2^15 quantisation levels; longer stars take one 64-bit atomic (count << 40 plus
// the sum).
__host__ __device__ inline bool eq_red32(int64_t n) { return n <= kEqRed32MaxN; }

struct EqParams {
    const uint32_t *tau_lo;   // quantised times of the star (sample scratch, star at offset 0)
    const int32_t *tau_hi;
    const long long *q;       // flux - f_ref in fixed point, quantum 2^-k
    int64_t n;
    const double *periods;
    int64_t np;
    int nfine, nbins;
    int fshift;               // 32 - log2(nfine) if nfine is a power of two, else -1
    int ppb;                  // periods per block pass (<= kEqMaxPeriods)
    const int *kscale;        // k (device)
    const StarStats *stats;
    int width_only;           // 1: equal-width fold into nfine (= nbins) bins, no merge
    int red32;                // eq_red32(n): the 32-bit reduction fold (set by the host)
    float *folded;            // [np][nbins] means (may be NULL when width_only)
    // width_only outputs, [np][nfine] (each may be NULL)
    int32_t *counts;          // samples per bin
    float *sums;              // sum of (flux - f_ref) per bin
    uint32_t *status;
};

size_t eq_smem_bytes(int nfine, int ppb);
int eq_periods_per_block(int nfine);
cudaError_t launch_eq_prep(const float *x, int64_t n, unsigned int *maxbits, long long *q, int *kscale,
                           int num_sms, cudaStream_t st);
cudaError_t launch_eq_fold(const EqParams &p, int num_sms, cudaStream_t st);

}  // namespace gpfc
