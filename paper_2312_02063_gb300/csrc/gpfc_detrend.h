// gpfc_detrend.h -- launch parameters of the pre-processing kernels (detrend.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gpfc {

constexpr int kDetrendMaxSpacings = 8;

struct DetrendParams {
    const double *t;        // [n] sorted times
    const float *f;         // [n] flux
    const uint8_t *mask;    // [n] known transits (nonzero: never used in a fit), or NULL
    int64_t n;
    double time_gap, flux_gap_sigma, clip_sigma, ridge;
    int edge, max_iter, n_sp;
    double sp[kDetrendMaxSpacings];
    int blocks;             // blocks of the moment and segment-start passes
    // workspace (context-owned)
    double *partial;        // [2 * blocks]
    int64_t *blk_count;     // [blocks]
    int64_t *blk_off;       // [blocks + 1]
    int64_t *n_seg;         // [1]
    int64_t *seg_start;     // [n + 1]
    int64_t *seg_keep;      // [n]
    int64_t *seg_off;       // [n]
    double *G4, *LB;        // [n][4] banded normal matrix rows and Cholesky factor
    double *rhs, *coef, *trend, *best;  // [n]
    uint8_t *used, *used2;  // [n]
    float *det;             // [n]
    // outputs (caller-owned, device)
    double *t_out;
    float *f_out;
    int32_t *seg_out;       // or NULL
    int64_t *n_out;         // [1]
};

cudaError_t launch_detrend(const DetrendParams &p, int num_sms, cudaStream_t st);

}  // namespace gpfc
