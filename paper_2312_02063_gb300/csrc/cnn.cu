// cnn.cu -- the 1-D CNN scorer on 5th-generation tensor cores (tcgen05 + TMEM), sm_103a.
//
// Network (one noise-normalised folded profile of 256 bins in, one score out; the paper's
// Sec. 2.5 scores every folded profile with a CNN using circular convolutions):
//   conv1(1->16, k5) ReLU maxpool2 | conv2(16->32, k5) ReLU maxpool2 |
//   conv3(32->64, k5) ReLU maxpool2 | flatten (2048) | fc1(2048->256) ReLU | fc2(256->1) sigmoid
// Convolutions are circular with padding 2 (cross-correlation). Weights are BF16. Every
// input of a tensor-core layer (the normalised profile, the pooled conv1/conv2/conv3
// outputs) is carried as two BF16 terms, hi = bf16(a) and lo = bf16(a - hi), and the layer
// takes the MMAs of both terms against the same weights into one FP32 accumulator: BF16
// arithmetic with about 16 significant bits per activation, so the scores stay within a
// few 1e-5 of the FP64 forward on the same BF16 weights, also where many trained scores
// crowd near a decision threshold (a single BF16 term per activation moves the logit of a
// trained network by up to ~0.04).
//
// Kernels:
//  * cnn_conv_kernel: a block takes four profiles at a time. Noise normalisation (Sec. 2.1:
//    std scaled to 1, mean kept) runs on CUDA cores. conv1, conv2 and conv3 are implicit
//    GEMMs on tcgen05: conv1 from one 16-byte im2col row per pooled position (8 taps, K
//    padded to 16), conv2 and conv3 straight from the activations, which sit in shared
//    memory as even and odd position planes with a circular halo row, [channel chunk of
//    8][row][profile][8 channels] BF16, so the A window of pooled output q for pool member
//    j and tap u starts 16-byte rows apart whatever j and u are (core-matrix K step = one
//    tap), no im2col copy. conv1: M = 128 pooled positions per profile, N = 32 (pool
//    member x 16 channels), K = 16 (8 taps of the high terms, 8 of the low terms); conv2: M =
//    64 pooled positions x 2 profiles, N = 32, K = 80 per term; conv3: M = 32 pooled
//    positions x 4 profiles, N = 64, K = 160 per term; conv2 and conv3 keep one accumulator
//    per pool member. Accumulators live in TMEM; the epilogue pools
//    the two members in registers (the same TMEM lane), adds the bias, applies ReLU on
//    packed BF16 pairs and writes the next layer's input.
//    The pooled conv3 output (flattened position-major, feature = position * 64 + channel,
//    with fc1's weights permuted to match) is written to global memory pre-tiled in the
//    tensor-core operand layout, 128 profiles x 64 features per 16 KB block, high terms then
//    low terms.
//  * cnn_fc_kernel: fc1 as a tcgen05 GEMM, M = 128 profiles (two tiles per block), N = 256,
//    K = 2 x 2048 (high and low terms against the same weights), operands streamed with bulk copies through a 3-stage mbarrier pipeline by a
//    producer thread while another thread issues the MMAs. The epilogue adds fc1's bias,
//    applies ReLU, takes the fc2 dot product from TMEM and applies the sigmoid.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "gpfc_cnn.h"
#include "gpfc_common.cuh"

namespace gpfc {

// ------------------------------------------------------------------ layouts

// Activations of conv2's and conv3's inputs are stored as two planes, even and odd
// positions, each with one halo row on either side, profiles interleaved per row: the
// input window of pooled output q for pool member j and tap u starts at position
// 2q + j + u - 2, i.e. plane (j + u) & 1, row q + ((j + u) >> 1) - 1, so one MMA K step
// (one tap, 16 channels) reads rows 16 bytes apart whatever j and u are.
constexpr int kA2Rows = 66;                          // conv2 input: plane index -1..64
constexpr int kA2ChunkB = kA2Rows * 2 * 16;          // [row][profile of the pair][8 channels]
constexpr int kA2PlaneB = 2 * kA2ChunkB;             // 2 channel chunks
constexpr int kA2PairB = 2 * kA2PlaneB;              // 2 planes
constexpr int kA3Rows = 34;                          // conv3 input: plane index -1..32
constexpr int kA3ChunkB = kA3Rows * 4 * 16;          // [row][profile of the quad][8 channels]
constexpr int kA3PlaneB = 4 * kA3ChunkB;             // 4 channel chunks
constexpr int kA1ProfB = 128 * 16;                   // conv1 im2col rows: positions 2q-2 .. 2q+5
constexpr int kB1Bytes = 32 * 16 * 2;
constexpr int kB2Bytes = 32 * 80 * 2;
constexpr int kB3Bytes = 64 * 160 * 2;
constexpr int kTileBytes = 128 * 64 * 2;  // one fc1 operand block: 128 rows x 64 K
constexpr int kW1Chunk = 256 * 64 * 2;    // fc1 weights per K chunk: 256 rows x 64 K

// byte offset of element (row r, k) in a K-major no-swizzle operand whose core matrices
// along K are `lbo` bytes apart and along the rows `sbo` bytes apart
__host__ __device__ __forceinline__ uint32_t canon(int r, int k, int lbo, int sbo)
{
    return (uint32_t)((r >> 3) * sbo + (k >> 3) * lbo + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ------------------------------------------------------------------ weight preparation

// One thread per destination element. Source tensors are FP32 in PyTorch layout.
__global__ void cnn_prep_kernel(CnnSrc src, CnnDev dst)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int i = tid; i < 16 * 5; i += stride) dst.w1[i] = bf16_round(src.w1[i]);
    for (int i = tid; i < 16; i += stride) dst.b1[i] = src.b1[i];
    for (int i = tid; i < 32; i += stride) dst.b2[i] = src.b2[i];
    for (int i = tid; i < 64; i += stride) dst.b3[i] = src.b3[i];
    for (int i = tid; i < 256; i += stride) {
        dst.bf1[i] = src.bf1[i];
        dst.wf2[i] = bf16_round(src.wf2[i]);
    }
    if (tid == 0) dst.bf2[0] = src.bf2[0];
    // conv1 B operand: row n = j * 16 + co (pool member j: position 2q + j), K index u: the
    // offset into the 8-position im2col row 2q-2 .. 2q+5, of the input's high BF16 term for
    // u < 8 and of its low term for u >= 8: weight w1[co][(u & 7) - j] where it exists
    for (int i = tid; i < 32 * 16; i += stride) {
        const int n = i / 16, u = i % 16, jj = n >> 4, co = n & 15, k = (u & 7) - jj;
        const float v = (k >= 0 && k < 5) ? src.w1[co * 5 + k] : 0.f;
        *reinterpret_cast<uint16_t *>(dst.B1 + canon(n, u, 128, 256)) = bf16_bits(v);
    }
    // conv2 B operand: row n = output channel, K index q*8 + e with q = k*2 + c
    // (tap k, channel chunk c) and input channel c*8 + e
    for (int i = tid; i < 32 * 80; i += stride) {
        const int n = i / 80, kk = i % 80, q = kk >> 3, e = kk & 7, k = q >> 1, c = q & 1;
        const float v = src.w2[(n * 16 + c * 8 + e) * 5 + k];
        *reinterpret_cast<uint16_t *>(dst.B2 + canon(n, kk, 128, 1280)) = bf16_bits(v);
    }
    // conv3: q = k*4 + c
    for (int i = tid; i < 64 * 160; i += stride) {
        const int n = i / 160, kk = i % 160, q = kk >> 3, e = kk & 7, k = q >> 2, c = q & 3;
        const float v = src.w3[(n * 32 + c * 8 + e) * 5 + k];
        *reinterpret_cast<uint16_t *>(dst.B3 + canon(n, kk, 128, 2560)) = bf16_bits(v);
    }
    // fc1 weights, K chunk kc = pooled position l', K index kk = channel c:
    // device feature l' * 64 + c is PyTorch's flattened feature c * 32 + l'
    for (int i = tid; i < 256 * 2048; i += stride) {
        const int n = i / 2048, f = i % 2048, kc = f >> 6, kk = f & 63;
        const float v = src.wf1[n * 2048 + kk * 32 + kc];
        *reinterpret_cast<uint16_t *>(dst.W1t + (size_t)kc * kW1Chunk + canon(n, kk, 128, 1024)) = bf16_bits(v);
    }
}

// ------------------------------------------------------------------ conv kernel

// Every activation that feeds a tensor-core layer is held as two BF16 terms, hi = bf16(a)
// and lo = bf16(a - hi) (about 16 significant bits together), and each layer takes the MMAs
// of both against the same BF16 weights into one FP32 accumulator.
struct ConvSmem {
    uint8_t B1[kB1Bytes];
    uint8_t B2[kB2Bytes];
    uint8_t B3[kB3Bytes];
    uint8_t A1[4][kA1ProfB];      // conv1 im2col (high terms), one per profile of the quad
    uint8_t A1lo[4][kA1ProfB];    // K chunk 1 of conv1: the low terms of the same rows
    uint8_t A2[2][kA2PairB];      // conv2 input of each pair of the quad (high terms)
    uint8_t A2lo[2][kA2PairB];    // (low terms)
    union {
        uint8_t A3[2 * kA3PlaneB];  // conv3 input of the quad (high terms)
        float X[4][256];            // normalised inputs (FP32), used before A3 is written
    };
    uint8_t A3lo[2 * kA3PlaneB];  // (low terms)
    float b1[16];
    float b2[32];
    float b3[64];
    uint64_t bar;
    uint32_t tslot;
    int abort;
};

constexpr int kConvThreads = 128;
constexpr int kConvProfiles = 4;  // profiles per block iteration

// Two FP32 values as two BF16 terms each: hi packs bf16(v0), bf16(v1) (low half = first), lo
// packs the BF16 roundings of the remainders v - hi.
__device__ __forceinline__ void split_bf16x2(float v0, float v1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// ReLU(max(a0, a1) + b) of two channels in FP32 (pooling before the bias gives the same value
// as pooling the biased members: FP32 rounding is monotone), as two BF16 terms.
__device__ __forceinline__ void pool_bias_relu2(float a00, float a01, float a10, float a11, float2 b, uint32_t &hi,
                                                uint32_t &lo)
{
    split_bf16x2(fmaxf(fmaxf(a00, a01) + b.x, 0.f), fmaxf(fmaxf(a10, a11) + b.y, 0.f), hi, lo);
}

// Issue the MMAs of one stage and wait for them (thread 0 issues; everyone waits).
#define CONV_MMA_WAIT(...)                                                                         \
    do {                                                                                          \
        fence_proxy_async_smem();                                                                 \
        tc_fence_before();                                                                        \
        __syncthreads();                                                                          \
        tc_fence_after();                                                                         \
        if (tid == 0) {                                                                           \
            __VA_ARGS__;                                                                          \
            umma_commit(&S.bar);                                                                  \
        }                                                                                         \
        if (!mbar_wait_bounded(&S.bar, phase)) S.abort = 1;                                       \
        phase ^= 1u;                                                                              \
        tc_fence_after();                                                                         \
    } while (0)

__global__ void __launch_bounds__(kConvThreads, 2) cnn_conv_kernel(const CnnConvParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    ConvSmem &S = *reinterpret_cast<ConvSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // stage the weights once per block
    for (int i = tid; i < kB1Bytes / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(S.B1)[i] = reinterpret_cast<const uint4 *>(p.w.B1)[i];
    for (int i = tid; i < kB2Bytes / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(S.B2)[i] = reinterpret_cast<const uint4 *>(p.w.B2)[i];
    for (int i = tid; i < kB3Bytes / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(S.B3)[i] = reinterpret_cast<const uint4 *>(p.w.B3)[i];
    if (tid < 16) S.b1[tid] = p.w.b1[tid];
    if (tid < 32) S.b2[tid] = p.w.b2[tid];
    if (tid < 64) S.b3[tid] = p.w.b3[tid];
    if (warp == 0) tmem_alloc(&S.tslot, 128);
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
        S.abort = 0;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tslot;
    const uint32_t tlane = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0u;
    const int64_t nquads = (p.np + kConvProfiles - 1) / kConvProfiles;

    for (int64_t quad = blockIdx.x; quad < nquads; quad += gridDim.x) {
        const int64_t l0 = kConvProfiles * quad;  // local index of the quad's first profile
        {
            // pull the next quad's means and counts (8 KB) toward L2 while this quad runs
            const int64_t ln = l0 + kConvProfiles * (int64_t)gridDim.x;
            const int64_t pl = ln + (tid & 63) / 16;  // 16 lines of 128 bytes per 1 KB row
            if (pl < p.np) {
                const size_t off = (size_t)(p.k_begin + pl) * 256 + (size_t)(tid & 15) * 32;
                if (tid < 64) asm volatile("prefetch.global.L2 [%0];" ::"l"(p.folded + off));
                else if (p.counts) asm volatile("prefetch.global.L2 [%0];" ::"l"(p.counts + off));
            }
        }
        // ---- noise normalisation (Sec. 2.1): warp w takes profile w, 8 bins per lane
        {
            const int64_t kl = l0 + warp;
            const bool valid = kl < p.np;
            const int64_t k = p.k_begin + kl;
            float v[8];
            bool ne[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = 0.f;
                ne[u] = false;
            }
            if (valid) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 f = *reinterpret_cast<const float4 *>(p.folded + (size_t)k * 256 + 8 * lane + 4 * h);
                    v[4 * h] = f.x;
                    v[4 * h + 1] = f.y;
                    v[4 * h + 2] = f.z;
                    v[4 * h + 3] = f.w;
                    if (p.counts) {
                        const int4 c = *reinterpret_cast<const int4 *>(p.counts + (size_t)k * 256 + 8 * lane + 4 * h);
                        ne[4 * h] = c.x > 0;
                        ne[4 * h + 1] = c.y > 0;
                        ne[4 * h + 2] = c.z > 0;
                        ne[4 * h + 3] = c.w > 0;
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) ne[4 * h + u] = !(v[4 * h + u] != v[4 * h + u]);
                    }
                }
            }
            // FP32 throughout: the sum is compensated (TwoSum), the deviations v - m are
            // small, and one reciprocal standard deviation per profile scales them
            float sh = 0.f, sl = 0.f, cnt = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (ne[u]) {
                    const float t = sh + v[u];
                    const float bb = t - sh;
                    sl += (sh - (t - bb)) + (v[u] - bb);
                    sh = t;
                    cnt += 1.f;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
                const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                const float t = sh + oh;
                const float bb = t - sh;
                sl += ol + ((sh - (t - bb)) + (oh - bb));
                sh = t;
            }
            // The mean as a double-float pair m + ml: the deviations v - m of a folded
            // profile are ~1e-5 of its mean, so an FP32 mean alone (error up to half an ulp,
            // ~3e-8) would shift every deviation alike by up to ~0.5% of the profile's
            // standard deviation, and the network would see that shift in every bin.
            // fmaf(-m, cnt, sh) is the exact remainder of the rounded division, and v - m is
            // exact whenever v and m are within a factor of two (the case that needs it).
            float m = 0.f, ml = 0.f;
            if (cnt > 0.f) {
                m = sh / cnt;
                ml = (fmaf(-m, cnt, sh) + sl) / cnt;
            }
            float d[8], ss = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                d[u] = ne[u] ? (v[u] - m) - ml : 0.f;
                ss = fmaf(d[u], d[u], ss);
            }
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            const float var = cnt > 0.f ? ss / cnt : 0.f;
            const float inv_sd = var > 0.f ? 1.0f / sqrtf(var) : 0.f;
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = (inv_sd > 0.f && ne[u]) ? fmaf(d[u], inv_sd, m) : m;
            *reinterpret_cast<float4 *>(&S.X[warp][8 * lane]) = make_float4(x[0], x[1], x[2], x[3]);
            *reinterpret_cast<float4 *>(&S.X[warp][8 * lane + 4]) = make_float4(x[4], x[5], x[6], x[7]);
            if (p.xsave && valid) {
                // the input the network sees (hi + lo, exact in FP32), kept for the backward pass
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    uint32_t hi, lo;
                    split_bf16x2(x[u], x[u + 1], hi, lo);
                    const float2 h2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hi));
                    const float2 l2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lo));
                    p.xsave[(size_t)kl * 256 + 8 * lane + u] = h2.x + l2.x;
                    p.xsave[(size_t)kl * 256 + 8 * lane + u + 1] = h2.y + l2.y;
                }
            }
        }
        __syncthreads();
        // ---- conv1 im2col: thread q builds row q (input positions 2q-2 .. 2q+5) of each
        // profile, high terms in A1, low terms in A1lo
        {
            const int q = tid;
#pragma unroll
            for (int pp = 0; pp < kConvProfiles; ++pp) {
                uint32_t wh[4], wl[4];
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    split_bf16x2(S.X[pp][(2 * q - 2 + 2 * h) & 255], S.X[pp][(2 * q - 1 + 2 * h) & 255], wh[h], wl[h]);
                *reinterpret_cast<uint4 *>(S.A1[pp] + q * 16) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                *reinterpret_cast<uint4 *>(S.A1lo[pp] + q * 16) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
            }
        }
        // (S.X shares its memory with A3, which the conv2 epilogue writes after two more
        // block barriers)
        // ---- conv1: per profile M = 128 pooled positions, N = 32 (pool member, channel), K = 16
        CONV_MMA_WAIT({
            const uint32_t idesc = umma_idesc_bf16(128, 32);
            const uint64_t bd = umma_desc(smem_u32(S.B1), 128, 256);
#pragma unroll
            for (int pp = 0; pp < kConvProfiles; ++pp) {
                const uint32_t a = smem_u32(S.A1[pp]);
                umma_bf16(tmem + 32 * pp, umma_desc(a, smem_u32(S.A1lo[pp]) - a, 128), bd, idesc, false);
            }
        });
        // ---- conv1 epilogue: bias, ReLU, pool the two members in registers, write conv2 input
        {
            const int q = tid;  // pooled position 0..127
#pragma unroll 1
            for (int pp = 0; pp < kConvProfiles; ++pp) {
                const int64_t kl = l0 + pp;
                const bool valid = kl < p.np;
                float v[32];
                tmem_ld32(tmem + tlane + 32 * pp, v);
                uint32_t h[8], hl[8];
#pragma unroll
                for (int co = 0; co < 16; co += 2)
                    pool_bias_relu2(v[co], v[16 + co], v[co + 1], v[17 + co], *reinterpret_cast<const float2 *>(&S.b1[co]),
                                    h[co >> 1], hl[co >> 1]);
                if (p.a1save) {
#pragma unroll
                    for (int co = 0; co < 16; co += 2) {
                        const float a00 = v[co] + S.b1[co], a01 = v[16 + co] + S.b1[co];
                        const float a10 = v[co + 1] + S.b1[co + 1], a11 = v[17 + co] + S.b1[co + 1];
                        if (valid) {
                            float *a1 = p.a1save + ((size_t)kl * 16 + co) * 256 + 2 * q;
                            a1[0] = a00;
                            a1[1] = a01;
                            a1[256] = a10;
                            a1[257] = a11;
                        }
                    }
                }
                if (p.h1save && valid)
#pragma unroll
                    for (int co = 0; co < 16; ++co)
                        p.h1save[((size_t)kl * 16 + co) * 128 + q] = (uint16_t)(h[co >> 1] >> (16 * (co & 1)));
                const int row = (q >> 1) + 1;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    uint8_t *A2 = (t ? S.A2lo : S.A2)[pp >> 1] + (q & 1) * kA2PlaneB + (pp & 1) * 16;
                    const uint32_t *hw = t ? hl : h;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint4 w = make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                        *reinterpret_cast<uint4 *>(A2 + c * kA2ChunkB + row * 32) = w;
                        if (q >= 126) *reinterpret_cast<uint4 *>(A2 + c * kA2ChunkB) = w;                   // row -1
                        if (q <= 1) *reinterpret_cast<uint4 *>(A2 + c * kA2ChunkB + (kA2Rows - 1) * 32) = w;  // row 64
                    }
                }
            }
        }
        // ---- conv2: per pair, M = 64 pooled positions x 2 profiles, N = 32, K = 80, one
        // accumulator per pool member
        CONV_MMA_WAIT({
            const uint32_t idesc = umma_idesc_bf16(128, 32);
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                    for (int u = 0; u < 5; ++u) {
                        const int sft = jj + u;
                        const uint32_t off = (sft & 1) * kA2PlaneB + (sft >> 1) * 32;
                        const uint64_t bd = umma_desc(smem_u32(S.B2) + u * 256, 128, 1280);
                        umma_bf16(tmem + g * 64 + jj * 32, umma_desc(smem_u32(S.A2[g]) + off, kA2ChunkB, 128), bd, idesc,
                                  u > 0);
                        umma_bf16(tmem + g * 64 + jj * 32, umma_desc(smem_u32(S.A2lo[g]) + off, kA2ChunkB, 128), bd, idesc,
                                  true);
                    }
        });
        // ---- conv2 epilogue: row m = (pooled position m >> 1, profile m & 1 of the pair)
        {
            const int m = tid, q = m >> 1, pr = m & 1;
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                const int pp = 2 * g + pr;
                const int64_t kl = l0 + pp;
                const bool valid = kl < p.np;
                float v0[32], v1[32];
                tmem_ld32(tmem + tlane + g * 64, v0);
                tmem_ld32(tmem + tlane + g * 64 + 32, v1);
                uint32_t h[16], hl[16];
#pragma unroll
                for (int co = 0; co < 32; co += 2)
                    pool_bias_relu2(v0[co], v1[co], v0[co + 1], v1[co + 1], *reinterpret_cast<const float2 *>(&S.b2[co]),
                                    h[co >> 1], hl[co >> 1]);
                if (p.a2save) {
#pragma unroll
                    for (int co = 0; co < 32; co += 2) {
                        const float a00 = v0[co] + S.b2[co], a01 = v1[co] + S.b2[co];
                        const float a10 = v0[co + 1] + S.b2[co + 1], a11 = v1[co + 1] + S.b2[co + 1];
                        if (valid) {
                            float *a2 = p.a2save + ((size_t)kl * 32 + co) * 128 + 2 * q;
                            a2[0] = a00;
                            a2[1] = a01;
                            a2[128] = a10;
                            a2[129] = a11;
                        }
                    }
                }
                if (p.h2save && valid)
#pragma unroll
                    for (int co = 0; co < 32; ++co)
                        p.h2save[((size_t)kl * 32 + co) * 64 + q] = (uint16_t)(h[co >> 1] >> (16 * (co & 1)));
                const int row = (q >> 1) + 1;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    uint8_t *A3 = (t ? S.A3lo : S.A3) + (q & 1) * kA3PlaneB + pp * 16;
                    const uint32_t *hw = t ? hl : h;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 w = make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                        *reinterpret_cast<uint4 *>(A3 + c * kA3ChunkB + row * 64) = w;
                        if (q >= 62) *reinterpret_cast<uint4 *>(A3 + c * kA3ChunkB) = w;                   // row -1
                        if (q <= 1) *reinterpret_cast<uint4 *>(A3 + c * kA3ChunkB + (kA3Rows - 1) * 64) = w;  // row 32
                    }
                }
            }
        }
        // ---- conv3: M = 32 pooled positions x 4 profiles, N = 64, K = 160, one accumulator
        // per pool member
        CONV_MMA_WAIT({
            const uint32_t idesc = umma_idesc_bf16(128, 64);
#pragma unroll
            for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                for (int u = 0; u < 5; ++u)
#pragma unroll
                    for (int cp = 0; cp < 2; ++cp) {
                        const int sft = jj + u;
                        const uint32_t off = (sft & 1) * kA3PlaneB + 2 * cp * kA3ChunkB + (sft >> 1) * 64;
                        const uint64_t bd = umma_desc(smem_u32(S.B3) + (4 * u + 2 * cp) * 128, 128, 2560);
                        umma_bf16(tmem + jj * 64, umma_desc(smem_u32(S.A3) + off, kA3ChunkB, 128), bd, idesc,
                                  u > 0 || cp > 0);
                        umma_bf16(tmem + jj * 64, umma_desc(smem_u32(S.A3lo) + off, kA3ChunkB, 128), bd, idesc, true);
                    }
        });
        // ---- conv3 epilogue: row m = (pooled position m >> 2, profile m & 3); write the fc1
        // operand tiles of the high and the low terms (feature = position * 64 + channel)
        {
            const int m = tid, q = m >> 2, pp = m & 3;
            const int64_t kl = l0 + pp;
            const bool valid = kl < p.np;
            uint32_t h[32], hl[32];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float v0[32], v1[32];
                tmem_ld32(tmem + tlane + half * 32, v0);
                tmem_ld32(tmem + tlane + 64 + half * 32, v1);
#pragma unroll
                for (int j = 0; j < 32; j += 2)
                    pool_bias_relu2(v0[j], v1[j], v0[j + 1], v1[j + 1],
                                    *reinterpret_cast<const float2 *>(&S.b3[half * 32 + j]), h[(half * 32 + j) >> 1],
                                    hl[(half * 32 + j) >> 1]);
                if (p.a3save) {
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const int co = half * 32 + j;
                        const float a00 = v0[j] + S.b3[co], a01 = v1[j] + S.b3[co];
                        const float a10 = v0[j + 1] + S.b3[co + 1], a11 = v1[j + 1] + S.b3[co + 1];
                        if (valid) {
                            float *a3 = p.a3save + ((size_t)kl * 64 + co) * 64 + 2 * q;
                            a3[0] = a00;
                            a3[1] = a01;
                            a3[64] = a10;
                            a3[65] = a11;
                        }
                    }
                }
            }
            if (valid) {
                const int64_t mt = kl >> 7;
                const int r = (int)(kl & 127);
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    uint8_t *blk = p.h3t + ((size_t)mt * kH3Chunks + t * 32 + q) * kTileBytes;
                    const uint32_t *hw = t ? hl : h;
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc)
                        *reinterpret_cast<uint4 *>(blk + canon(r, 8 * cc, 128, 1024)) =
                            make_uint4(hw[4 * cc], hw[4 * cc + 1], hw[4 * cc + 2], hw[4 * cc + 3]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (S.abort) break;
    }
    if (S.abort && tid == 0) {
        report_error(p.status, kErrTimeout);
        // the last commit tracks every MMA this block issued: let them finish before the
        // accumulator columns are released
        mbar_wait_bounded(&S.bar, phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// ------------------------------------------------------------------ fc kernel

// Pipeline stages: three of 64 KB (two activation tiles + a weight chunk) when a block
// takes two tiles, four of 48 KB when it takes one.
constexpr int kFcMaxStages = 4;
constexpr int kFcStageMem = 3 * (2 * kTileBytes + kW1Chunk);  // 192 KB

struct FcSmem {
    uint8_t stage_mem[kFcStageMem];
    float bf1[256];
    float wf2[256];
    uint64_t full[kFcMaxStages];
    uint64_t empty[kFcMaxStages];
    uint64_t done;
    uint32_t tslot;
    int abort;
    uint32_t drain_from;  // first stage use the MMA thread did not consume (abort path)
};

__global__ void __launch_bounds__(128, 1) cnn_fc_kernel(const CnnFcParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    FcSmem &S = *reinterpret_cast<FcSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 256; i += 128) {
        S.bf1[i] = p.w.bf1[i];
        S.wf2[i] = p.w.wf2[i];
    }
    if (warp == 0) tmem_alloc(&S.tslot, 512);
    if (tid == 0) {
        for (int s = 0; s < kFcMaxStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.done, 1);
        fence_mbar_init();
        S.abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tslot;
    const float b2 = p.w.bf2[0];
    const int64_t ntiles = (p.np + 127) / 128;
    // work items: pairs (or single tiles) of 128-profile tiles with all 256 outputs, or, with
    // n_halves = 2, (tile, half of the outputs)
    const bool halves = p.n_halves == 2;
    const int64_t nitems = halves ? 2 * ntiles : (ntiles + p.tiles_per_block - 1) / p.tiles_per_block;
    uint32_t it_prod = 0, it_mma = 0, done_phase = 0;
    const int nst = (!halves && p.tiles_per_block == 2) ? 3 : 4;
    const uint32_t wbytes = halves ? kW1Chunk / 2 : kW1Chunk;            // weights per stage
    const uint32_t woff = (uint32_t)(halves ? 1 : p.tiles_per_block) * kTileBytes;  // within a stage
    const uint32_t sbytes = woff + wbytes;
    auto stage = [&](int st) { return S.stage_mem + (size_t)st * sbytes; };

    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int64_t mt0 = halves ? item >> 1 : (int64_t)p.tiles_per_block * item;
        const int nh = halves ? (int)(item & 1) : 0;  // first output of this item: 128 * nh
        const bool two = !halves && p.tiles_per_block == 2 && mt0 + 1 < ntiles;
        if (tid == 0) {
            // producer: stream the activation tiles and fc1's weights (rows of this item's
            // outputs), K chunk by chunk
            for (int kc = 0; kc < kH3Chunks && !S.abort; ++kc, ++it_prod) {
                const int s = it_prod % nst;
                const uint32_t use = it_prod / nst;
                if (use > 0 && !mbar_wait_bounded(&S.empty[s], (use - 1) & 1u)) {
                    S.abort = 1;
                    break;
                }
                const uint32_t bytes = (two ? 2u : 1u) * kTileBytes + wbytes;
                mbar_arrive_expect_tx(&S.full[s], bytes);
                bulk_g2s(stage(s), p.h3t + ((size_t)mt0 * kH3Chunks + kc) * kTileBytes, kTileBytes, &S.full[s]);
                if (two)
                    bulk_g2s(stage(s) + kTileBytes, p.h3t + ((size_t)(mt0 + 1) * kH3Chunks + kc) * kTileBytes,
                             kTileBytes, &S.full[s]);
                // rows 128 * nh .. of the chunk: 16 row groups of 1 KB
                bulk_g2s(stage(s) + woff, p.w.W1t + (size_t)(kc & 31) * kW1Chunk + (size_t)nh * (kW1Chunk / 2), wbytes,
                         &S.full[s]);
            }
        } else if (tid == 32) {
            // MMA issuer: 4 K steps of 16 per chunk, two M tiles sharing each weight chunk; the
            // chunks of the low terms (32..63) take the same weights as those of the high terms
            const uint32_t idesc = umma_idesc_bf16(128, halves ? 128 : 256);
            for (int kc = 0; kc < kH3Chunks; ++kc, ++it_mma) {
                const int s = it_mma % nst;
                const uint32_t use = it_mma / nst;
                if (S.abort || !mbar_wait_bounded(&S.full[s], use & 1u)) {
                    S.abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(stage(s));
                const uint32_t a1 = a0 + kTileBytes;
                const uint32_t bw = a0 + woff;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t bd = umma_desc(bw + ks * 256, 128, 1024);
                    umma_bf16(tmem, umma_desc(a0 + ks * 256, 128, 1024), bd, idesc, kc > 0 || ks > 0);
                    if (two) umma_bf16(tmem + 256, umma_desc(a1 + ks * 256, 128, 1024), bd, idesc, kc > 0 || ks > 0);
                }
                umma_commit(&S.empty[s]);
            }
            umma_commit(&S.done);
        }
        if (!mbar_wait_bounded(&S.done, done_phase)) S.abort = 1;
        done_phase ^= 1u;
        tc_fence_after();
        // ---- epilogue: thread = profile row of the tile. The fc2 dot product is formed as
        // two partial sums, over outputs 0..127 and 128..255, added in that order, whichever
        // way the outputs are split over blocks.
        const int r = warp * 32 + lane;
#pragma unroll 1
        for (int t = 0; t < (two ? 2 : 1); ++t) {
            const int64_t kl = (mt0 + t) * 128 + r;
            float part0 = 0.f, part1 = 0.f;
#pragma unroll 1
            for (int h = 0; h < (halves ? 1 : 2); ++h) {
                const int ho = halves ? nh : h;  // which half of the outputs
#pragma unroll 1
                for (int n0 = 0; n0 < 128; n0 += 32) {
                    const int n = 128 * ho + n0;
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + t * 256 + (halves ? n0 : n), v);
                    float dot = ho ? part1 : part0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float z = v[j] + S.bf1[n + j];
                        dot = fmaf(fmaxf(z, 0.f), S.wf2[n + j], dot);
                        if (p.z1save && kl < p.np) p.z1save[(size_t)kl * 256 + n + j] = z;
                    }
                    if (ho) part1 = dot;
                    else part0 = dot;
                }
            }
            if (kl < p.np) {
                if (halves) {
                    p.zpart[(size_t)nh * ntiles * 128 + kl] = nh ? part1 : part0;
                } else {
                    const float zz = (part0 + part1) + b2;
                    const int64_t o = p.slot_k ? p.slot_k[p.k_begin + kl] : p.k_begin + kl;
                    if (o >= 0) {
                        if (p.logit) p.logit[o] = zz;
                        if (p.score) p.score[o] = 1.f / (1.f + expf(-zz));
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (S.abort) break;
    }
    if (S.abort) {
        // let the bulk copies and MMAs this block issued land before it exits
        if (tid == 32) S.drain_from = it_mma;
        __syncthreads();
        if (tid == 0) {
            report_error(p.status, kErrTimeout);
            for (uint32_t it = S.drain_from; it < it_prod; ++it)
                if (!mbar_wait_bounded(&S.full[it % nst], (it / nst) & 1u)) break;
        }
        if (tid == 32) mbar_wait_bounded(&S.done, done_phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// Logits and scores of a launch whose fc1 outputs were split over two blocks: the two
// partial fc2 dots, added in the same order as the single-block epilogue adds them.
__global__ void cnn_fc_finalize_kernel(const CnnFcParams p)
{
    const int64_t kl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kl >= p.np) return;
    const int64_t stride = (p.np + 127) / 128 * 128;
    const float zz = (p.zpart[kl] + p.zpart[stride + kl]) + p.w.bf2[0];
    const int64_t o = p.slot_k ? p.slot_k[p.k_begin + kl] : p.k_begin + kl;
    if (o >= 0) {
        if (p.logit) p.logit[o] = zz;
        if (p.score) p.score[o] = 1.f / (1.f + expf(-zz));
    }
}

// ------------------------------------------------------------------ launches

size_t cnn_dev_bytes() { return CnnDevLayout::total(); }

CnnDev cnn_dev_carve(void *base)
{
    CnnDev d;
    uint8_t *b = static_cast<uint8_t *>(base);
    d.w1 = reinterpret_cast<float *>(b + CnnDevLayout::w1);
    d.b1 = reinterpret_cast<float *>(b + CnnDevLayout::b1);
    d.b2 = reinterpret_cast<float *>(b + CnnDevLayout::b2);
    d.b3 = reinterpret_cast<float *>(b + CnnDevLayout::b3);
    d.bf1 = reinterpret_cast<float *>(b + CnnDevLayout::bf1);
    d.wf2 = reinterpret_cast<float *>(b + CnnDevLayout::wf2);
    d.bf2 = reinterpret_cast<float *>(b + CnnDevLayout::bf2);
    d.B1 = b + CnnDevLayout::B1;
    d.B2 = b + CnnDevLayout::B2;
    d.B3 = b + CnnDevLayout::B3;
    d.W1t = b + CnnDevLayout::W1t;
    return d;
}

cudaError_t launch_cnn_prep(const CnnSrc &src, const CnnDev &dst, cudaStream_t st)
{
    cnn_prep_kernel<<<512, 256, 0, st>>>(src, dst);
    return cudaGetLastError();
}

static int g_cnn_attr = 0;
static int g_conv_blocks_per_sm = 0;

// Dynamic shared memory of the conv kernel: at least 48 KB so that no more than 4 blocks
// (4 x 128 TMEM columns) are resident on an SM.
static size_t conv_smem_bytes() { return sizeof(ConvSmem) < 48 * 1024 ? 48 * 1024 : sizeof(ConvSmem); }

cudaError_t cnn_register_kernels()
{
    if (g_cnn_attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(cnn_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cnn_conv_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cnn_fc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FcSmem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_conv_blocks_per_sm, cnn_conv_kernel, kConvThreads,
                                                          conv_smem_bytes());
    if (e == cudaSuccess) {
        // blocks that fit an SM's shared memory (1 KB reserved per block), at most 4 (each
        // takes 128 of the 512 TMEM columns); the larger of this and the occupancy query
        int dev = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int fit = (int)((size_t)smem_sm / (conv_smem_bytes() + 1024));
        g_conv_blocks_per_sm = std::min(4, std::max(g_conv_blocks_per_sm, fit));
        if (g_conv_blocks_per_sm < 1) e = cudaErrorInvalidConfiguration;
    }
    if (e == cudaSuccess) g_cnn_attr = 1;
    return e;
}

cudaError_t launch_cnn_conv(const CnnConvParams &p, int num_sms, cudaStream_t st)
{
    cudaError_t e = cnn_register_kernels();
    if (e != cudaSuccess) return e;
    const int64_t nquads = (p.np + kConvProfiles - 1) / kConvProfiles;
    // as many blocks per SM as fit in shared memory (two; each holds 128 of the SM's 512 TMEM
    // columns)
    const int64_t cap = (int64_t)num_sms * g_conv_blocks_per_sm;
    const int grid = (int)(nquads < cap ? nquads : cap);
    cnn_conv_kernel<<<grid, kConvThreads, conv_smem_bytes(), st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_cnn_fc(const CnnFcParams &p_in, int num_sms, cudaStream_t st)
{
    cudaError_t e = cnn_register_kernels();
    if (e != cudaSuccess) return e;
    CnnFcParams p = p_in;
    const int64_t ntiles = (p.np + 127) / 128;
    // two tiles per block share each streamed weight chunk; with fewer tiles than two per
    // SM, one tile per block; with fewer tiles than SMs, each tile's 256 outputs are split
    // over two blocks, whose partial fc2 dots a second kernel adds
    p.n_halves = ntiles < (int64_t)num_sms ? 2 : 1;
    p.tiles_per_block = ntiles >= 2 * (int64_t)num_sms ? 2 : 1;
    p.zpart = reinterpret_cast<float *>(const_cast<uint8_t *>(p.h3t) + cnn_h3t_tiles_bytes(p.np));
    const int64_t nitems = p.n_halves == 2 ? 2 * ntiles : (ntiles + p.tiles_per_block - 1) / p.tiles_per_block;
    const int grid = (int)(nitems < (int64_t)num_sms ? nitems : (int64_t)num_sms);
    cnn_fc_kernel<<<grid, 128, sizeof(FcSmem), st>>>(p);
    if (p.n_halves == 2) cnn_fc_finalize_kernel<<<(int)((p.np + 255) / 256), 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace gpfc
