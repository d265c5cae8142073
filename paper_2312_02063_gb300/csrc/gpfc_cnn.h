// gpfc_cnn.h -- launch parameters of the CNN scorer kernels (cnn.cu, cnn_train.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gpfc_kernels.h"

namespace gpfc {

// FP32 parameters in PyTorch layout (device pointers):
// w1 [16][1][5], w2 [32][16][5], w3 [64][32][5], wf1 [256][2048], wf2 [1][256], biases.
struct CnnSrc {
    const float *w1, *b1, *w2, *b2, *w3, *b3, *wf1, *bf1, *wf2, *bf2;
};

// Device copies in the layouts the kernels read (weights rounded to BF16).
struct CnnDev {
    float *w1, *b1, *b2, *b3, *bf1, *wf2, *bf2;
    uint8_t *B1;   // conv1 weights for both pool members, operand layout (32 x 16 BF16)
    uint8_t *B2;   // conv2 weights, tensor-core operand layout (32 x 80 BF16)
    uint8_t *B3;   // conv3 weights (64 x 160 BF16)
    uint8_t *W1t;  // fc1 weights, 32 K chunks of 256 x 64 BF16
};

// The conv3 output as fc1's A operand: per tile of 128 profiles, kH3Chunks K chunks of
// 128 x 64 BF16 (16 KB), the 32 chunks of the activations' high BF16 terms followed by the 32
// chunks of their low terms (each activation is carried as hi + lo).
// The same allocation ends with the fc kernel's partial fc2 dot products, [2][tiles * 128]
// FP32 (used when a launch splits fc1's 256 outputs over two blocks).
constexpr int kH3Chunks = 64;
inline size_t cnn_h3t_tiles_bytes(int64_t np) { return (size_t)((np + 127) / 128) * kH3Chunks * 128 * 64 * 2; }
inline size_t cnn_h3t_bytes(int64_t np) { return cnn_h3t_tiles_bytes(np) + (size_t)((np + 127) / 128) * 128 * 2 * 4; }

struct CnnDevLayout {
    static constexpr size_t w1 = 0;
    static constexpr size_t b1 = 512;
    static constexpr size_t b2 = 1024;
    static constexpr size_t b3 = 1536;
    static constexpr size_t bf1 = 2048;
    static constexpr size_t wf2 = 3072;
    static constexpr size_t bf2 = 4096;
    static constexpr size_t B2 = 8192;
    static constexpr size_t B3 = B2 + 32 * 80 * 2;
    static constexpr size_t B1 = B3 + 64 * 160 * 2;
    static constexpr size_t W1t = 65536;
    static constexpr size_t total() { return W1t + (size_t)256 * 2048 * 2; }
};

struct CnnConvParams {
    const float *folded;     // [*][256] means (global profile index)
    const int32_t *counts;   // [*][256] or NULL (then NaN marks an empty bin)
    int64_t k_begin;         // first profile of this launch
    int64_t np;              // profiles in this launch
    CnnDev w;
    uint8_t *h3t;            // [ceil(np/128)][kH3Chunks][128 x 64 BF16 tile] (local profile index)
    // activations kept for the backward pass (NULL at inference), local profile index
    float *xsave;            // [np][256] normalised input as the network sees it (hi + lo)
    float *a1save;           // [np][16][256] FP32 conv1 pre-activation
    uint16_t *h1save;        // [np][16][128] BF16
    float *a2save;           // [np][32][128] FP32 conv2 pre-activation
    uint16_t *h2save;        // [np][32][64] BF16
    float *a3save;           // [np][64][64] FP32 conv3 pre-activation
    uint32_t *status;
};

struct CnnFcParams {
    const uint8_t *h3t;
    int64_t k_begin;
    int64_t np;
    CnnDev w;
    float *score;            // [global] sigmoid(logit), or NULL
    float *logit;            // [global] or NULL
    const int64_t *slot_k;   // NULL, or the output index of each profile (< 0: not written)
    float *z1save;           // [np][256] fc1 pre-activation (NULL at inference)
    uint32_t *status;
    int tiles_per_block;     // set by launch_cnn_fc: 128-profile tiles per block (1 or 2)
    int n_halves;            // set by launch_cnn_fc: 1, or 2 (a block takes one tile and half of N)
    float *zpart;            // set by launch_cnn_fc: partial fc2 dots [2][tiles * 128] (n_halves = 2)
};

// Offsets (bytes) of the activations a training forward keeps for the backward pass.
struct CnnSaved {
    size_t x, a1, h1, a2, h2, a3, h3t, z1, total;
    static CnnSaved layout(int64_t B);
};

// FP32 gradients in PyTorch layout (device), overwritten by the backward pass.
struct CnnGrads {
    float *w1, *b1, *w2, *b2, *w3, *b3, *wf1, *bf1, *wf2, *bf2;
};

size_t cnn_saved_bytes(int64_t B);
size_t cnn_backward_ws_bytes(int64_t B, int nblk, int num_sms);
cudaError_t launch_cnn_backward(const CnnSrc &w, const uint8_t *saved, int64_t B, const float *dlogit,
                                const CnnGrads &g, void *ws, int nblk, int num_sms, cudaStream_t st);
cudaError_t launch_bce(const float *z, const float *y, int64_t n, float *dlogit, float *loss, void *ws,
                       cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st);

size_t cnn_dev_bytes();
CnnDev cnn_dev_carve(void *base);
cudaError_t cnn_register_kernels();
cudaError_t launch_cnn_prep(const CnnSrc &src, const CnnDev &dst, cudaStream_t st);
cudaError_t launch_cnn_conv(const CnnConvParams &p, int num_sms, cudaStream_t st);
// fc1 + fc2 + sigmoid over the tiles at p.h3t (an allocation of cnn_h3t_bytes(p.np) bytes).
cudaError_t launch_cnn_fc(const CnnFcParams &p, int num_sms, cudaStream_t st);

}  // namespace gpfc
