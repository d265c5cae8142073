// gpfc_twotier.h -- launch parameters of the two-tier equal-count fold (twotier.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gpfc_kernels.h"

namespace gpfc {

constexpr int kEqMaxPeriods = 8;   // periods a block folds at a time
constexpr int kEqMaxFine = 4096;   // largest number of fine bins

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
