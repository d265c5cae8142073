// gpfc_synth.h -- launch parameters of the training-profile generator (synth.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gpfc.h"

namespace gpfc {

struct SynthParams {
    uint64_t seed;
    int64_t first;          // global index of the first light curve
    int64_t n;              // light curves (= profiles) in this launch
    int nbins;              // <= 256
    gpfc_synth_params sp;
    float *folded;          // [n][nbins] means, NaN for an empty bin
    int32_t *counts;        // [n][nbins] or NULL
    float *label;           // [n] 1 transit, 0 otherwise, or NULL
    double *period_out;     // [n] fold period, or NULL
    float *sigma_out;       // [n] population std of the light curve's flux, or NULL
};

cudaError_t launch_synth(const SynthParams &p, int num_sms, cudaStream_t st);

struct VectorParams {
    uint64_t seed;
    int64_t first;
    int64_t n;
    int nbins;
    gpfc_vector_params vp;
    float *folded;          // [n][nbins]
    float *label;           // [n] or NULL
    float *alpha;           // [n] or NULL
    float *sigma_bin;       // [n] or NULL
};

cudaError_t launch_paper_vectors(const VectorParams &p, int num_sms, cudaStream_t st);

}  // namespace gpfc
