// gpfc_decide.h -- launch parameters of the per-star decision kernel (decide.cu). The two
// output records have the layouts of gpfc_star_summary and gpfc_peak in gpfc.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gpfc {

struct PeakSummaryDev {
    double sde, mean, sd;
    long long best_index;
    float best_score;
    int n_peaks;
    int truncated;
    int n_listed;
};

struct PeakDev {
    long long index;
    float height;
    int width;
    int harmonic;
    int reserved;
};

struct PeakParams {
    const float *score;
    const double *periods;
    const int64_t *grid_off;  // [S+1] or NULL (one star of np periods)
    int64_t np;
    int nstars;
    double k_sigma;
    int min_width;
    double harm_tol;
    int max_peaks;
    PeakSummaryDev *summary;  // [S]
    PeakDev *peaks;           // [S][max_peaks] or NULL
};

cudaError_t launch_peaks(const PeakParams &p, int num_sms, cudaStream_t st);

// Detection statistics of a detector on labelled scores (gpfc_roc).
constexpr int kRocMaxFpr = 16;
struct RocParams {
    const float *pos;
    int64_t n_pos;
    const float *neg;
    int64_t n_neg;
    int n_fpr;
    int64_t k[kRocMaxFpr];        // floor(fpr * n_neg) of each requested rate
    unsigned long long *u2;       // [1]
    float *thr;                   // [n_fpr]
    unsigned long long *tp;       // [n_fpr]
};

cudaError_t launch_roc(const RocParams &p, int num_sms, cudaStream_t st);

}  // namespace gpfc
