// cnn.cu -- the 1-D CNN scorer on 5th-generation tensor cores (tcgen05 + TMEM), sm_103a.
//
// Network (one noise-normalised folded profile of 256 bins in, one score out; the paper's
// Sec. 2.5 scores every folded profile with a CNN using circular convolutions):
//   conv1(1->16, k5) ReLU maxpool2 | conv2(16->32, k5) ReLU maxpool2 |
//   conv3(32->64, k5) ReLU maxpool2 | flatten (2048) | fc1(2048->256) ReLU | fc2(256->1) sigmoid
// Convolutions are circular with padding 2 (cross-correlation). Inputs, weights and
// activations are BF16; every product is accumulated in FP32.
//
// Kernels:
//  * cnn_conv_kernel: a block takes two profiles at a time. Noise normalisation (Sec. 2.1:
//    std scaled to 1, mean kept) and conv1 run on CUDA cores. conv2 and conv3 are implicit
//    GEMMs on tcgen05: activations sit in shared memory as [channel chunk of 8][position
//    with a circular halo][8 channels] BF16, so the im2col matrix row of output position l
//    for tap k is the 16-byte row at position l + k: the MMA's A descriptor walks those rows
//    directly (core-matrix K step = one tap), no im2col copy. conv2: M = 128 positions of one
//    profile, N = 32, K = 80; conv3: M = 64 positions x 2 profiles interleaved, N = 64, K = 160.
//    Accumulators live in TMEM; the epilogue adds the bias, applies ReLU, pools neighbouring
//    TMEM lanes with warp shuffles and writes the next layer's input.
//    The pooled conv3 output (flattened position-major, feature = position * 64 + channel,
//    with fc1's weights permuted to match) is written to global memory pre-tiled in the
//    tensor-core operand layout, 128 profiles x 64 features per 16 KB block.
//  * cnn_fc_kernel: fc1 as a tcgen05 GEMM, M = 128 profiles (two tiles per block), N = 256,
//    K = 2048, operands streamed with bulk copies through a 3-stage mbarrier pipeline by a
//    producer thread while another thread issues the MMAs. The epilogue adds fc1's bias,
//    applies ReLU, takes the fc2 dot product from TMEM and applies the sigmoid.
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "gpfc_cnn.h"
#include "gpfc_common.cuh"

namespace gpfc {

// ------------------------------------------------------------------ layouts

constexpr int kA2Chunk = 132 * 16;   // conv2 input: positions -2..129, 8 channels, BF16
constexpr int kA2Prof = 2 * kA2Chunk;
constexpr int kA3Chunk = 68 * 2 * 16;  // conv3 input: positions -2..65 x 2 profiles x 8 channels
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
    // conv2 B operand: row n = output channel, K index q*8 + j with q = c*5 + k
    // (channel chunk c, tap k) and input channel c*8 + j
    for (int i = tid; i < 32 * 80; i += stride) {
        const int n = i / 80, kk = i % 80, q = kk >> 3, j = kk & 7, c = q / 5, k = q % 5;
        const float v = src.w2[(n * 16 + c * 8 + j) * 5 + k];
        *reinterpret_cast<uint16_t *>(dst.B2 + canon(n, kk, 128, 1280)) = bf16_bits(v);
    }
    for (int i = tid; i < 64 * 160; i += stride) {
        const int n = i / 160, kk = i % 160, q = kk >> 3, j = kk & 7, c = q / 5, k = q % 5;
        const float v = src.w3[(n * 32 + c * 8 + j) * 5 + k];
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

struct ConvSmem {
    uint8_t B2[kB2Bytes];
    uint8_t B3[kB3Bytes];
    uint8_t A2[2 * kA2Prof];
    uint8_t A3[4 * kA3Chunk];
    float X[2][256];
    float w1[80];
    float b1[16];
    float b2[32];
    float b3[64];
    float red[2][6];
    uint64_t bar;
    uint32_t tslot;
    int abort;
};

constexpr int kConvThreads = 128;

__global__ void __launch_bounds__(kConvThreads) cnn_conv_kernel(const CnnConvParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    ConvSmem &S = *reinterpret_cast<ConvSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // stage the weights once per block
    for (int i = tid; i < kB2Bytes / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(S.B2)[i] = reinterpret_cast<const uint4 *>(p.w.B2)[i];
    for (int i = tid; i < kB3Bytes / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(S.B3)[i] = reinterpret_cast<const uint4 *>(p.w.B3)[i];
    for (int i = tid; i < 80; i += kConvThreads) S.w1[i] = p.w.w1[i];
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
    uint32_t phase = 0u;
    const int64_t npairs = (p.np + 1) / 2;

    for (int64_t pair = blockIdx.x; pair < npairs; pair += gridDim.x) {
        const int64_t k0 = p.k_begin + 2 * pair;  // global index of the pair's first profile
        // ---- load and noise-normalise two profiles (64 threads per profile, 4 bins each)
        {
            const int prof = tid >> 6, q = tid & 63;
            const int64_t k = k0 + prof;
            const bool valid = (k - p.k_begin) < p.np;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            bool ne[4] = {false, false, false, false};
            if (valid) {
                const float4 f = *reinterpret_cast<const float4 *>(p.folded + (size_t)k * 256 + 4 * q);
                v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
                if (p.counts) {
                    const int4 c = *reinterpret_cast<const int4 *>(p.counts + (size_t)k * 256 + 4 * q);
                    ne[0] = c.x > 0; ne[1] = c.y > 0; ne[2] = c.z > 0; ne[3] = c.w > 0;
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) ne[u] = !(v[u] != v[u]);
                }
            }
            // FP32 throughout (this GPU's FP64 rate is tiny): the sum of the values is
            // compensated (TwoSum), the deviations v - m are small and exact-ish in FP32,
            // and one reciprocal standard deviation per profile scales them.
            float sh = 0.f, sl = 0.f, cnt = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u)
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
            if (lane == 0) {
                S.red[prof][(warp & 1) * 3 + 0] = sh;
                S.red[prof][(warp & 1) * 3 + 1] = sl;
                S.red[prof][(warp & 1) * 3 + 2] = cnt;
            }
            __syncthreads();
            const float n = S.red[prof][2] + S.red[prof][5];
            float m = 0.f;
            if (n > 0.f) {
                const float t = S.red[prof][0] + S.red[prof][3];
                const float bb = t - S.red[prof][0];
                const float lo = S.red[prof][1] + S.red[prof][4] + ((S.red[prof][0] - (t - bb)) + (S.red[prof][3] - bb));
                m = (t + lo) / n;
            }
            float d[4], ss = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                d[u] = ne[u] ? v[u] - m : 0.f;
                ss = fmaf(d[u], d[u], ss);
            }
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            __syncthreads();
            if (lane == 0) S.red[prof][(warp & 1) * 3] = ss;
            __syncthreads();
            const float var = n > 0.f ? (S.red[prof][0] + S.red[prof][3]) / n : 0.f;
            const float inv_sd = var > 0.f ? 1.0f / sqrtf(var) : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float x = (inv_sd > 0.f && ne[u]) ? fmaf(d[u], inv_sd, m) : m;
                S.X[prof][4 * q + u] = bf16_round(x);
            }
            if (p.xsave && valid) {
                // normalised BF16 input, kept for the backward pass
#pragma unroll
                for (int u = 0; u < 4; ++u) p.xsave[(size_t)(k - p.k_begin) * 256 + 4 * q + u] = S.X[prof][4 * q + u];
            }
        }
        __syncthreads();
        // ---- conv1 on CUDA cores: thread -> profile, pooled positions 2lp and 2lp+1
        {
            const int prof = tid >> 6, lp = tid & 63;
            float in[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) in[j] = S.X[prof][(4 * lp - 2 + j + 256) & 255];
            uint16_t h[2][16];
#pragma unroll
            for (int co = 0; co < 16; ++co) {
                float a[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    float acc = S.b1[co];
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc = fmaf(S.w1[co * 5 + k], in[l + k], acc);
                    if (p.a1save && (k0 + prof - p.k_begin) < p.np)
                        p.a1save[((size_t)(k0 + prof - p.k_begin) * 16 + co) * 256 + 4 * lp + l] = acc;
                    a[l] = fmaxf(acc, 0.f);
                }
                h[0][co] = bf16_bits(fmaxf(a[0], a[1]));
                h[1][co] = bf16_bits(fmaxf(a[2], a[3]));
            }
            uint8_t *A2 = S.A2 + prof * kA2Prof;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int lq = 2 * lp + t;  // pooled position 0..127
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    uint4 w;
                    w.x = h[t][8 * c + 0] | ((uint32_t)h[t][8 * c + 1] << 16);
                    w.y = h[t][8 * c + 2] | ((uint32_t)h[t][8 * c + 3] << 16);
                    w.z = h[t][8 * c + 4] | ((uint32_t)h[t][8 * c + 5] << 16);
                    w.w = h[t][8 * c + 6] | ((uint32_t)h[t][8 * c + 7] << 16);
                    *reinterpret_cast<uint4 *>(A2 + c * kA2Chunk + (lq + 2) * 16) = w;
                    if (lq >= 126) *reinterpret_cast<uint4 *>(A2 + c * kA2Chunk + (lq - 126) * 16) = w;
                    if (lq <= 1) *reinterpret_cast<uint4 *>(A2 + c * kA2Chunk + (lq + 130) * 16) = w;
                }
                if (p.h1save) {
                    const int64_t k = k0 + prof;
                    if ((k - p.k_begin) < p.np)
                        for (int co = 0; co < 16; ++co)
                            p.h1save[((size_t)(k - p.k_begin) * 16 + co) * 128 + lq] = h[t][co];
                }
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- conv2: two implicit GEMMs (one per profile), M = 128, N = 32, K = 80
        if (tid == 0) {
            const uint32_t idesc = umma_idesc_bf16(128, 32);
#pragma unroll
            for (int prof = 0; prof < 2; ++prof) {
                const uint32_t abase = smem_u32(S.A2 + prof * kA2Prof);
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const int q0 = 2 * i, q1 = 2 * i + 1;
                    const uint32_t o0 = (q0 / 5) * kA2Chunk + (q0 % 5) * 16;
                    const uint32_t o1 = (q1 / 5) * kA2Chunk + (q1 % 5) * 16;
                    const uint64_t ad = umma_desc(abase + o0, o1 - o0, 128);
                    const uint64_t bd = umma_desc(smem_u32(S.B2) + i * 256, 128, 1280);
                    umma_bf16(tmem + prof * 32, ad, bd, idesc, i > 0);
                }
            }
            umma_commit(&S.bar);
        }
        if (!mbar_wait_bounded(&S.bar, phase)) S.abort = 1;
        phase ^= 1u;
        tc_fence_after();
        // ---- conv2 epilogue: bias, ReLU, pool lanes (l, l+1), write conv3's input
        {
            const int l = warp * 32 + lane;  // output position 0..127
#pragma unroll 1
            for (int prof = 0; prof < 2; ++prof) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + prof * 32, v);
                uint16_t h[32];
#pragma unroll
                for (int co = 0; co < 32; ++co) {
                    const float a = fmaxf(v[co] + S.b2[co], 0.f);
                    const float o = __shfl_xor_sync(0xffffffffu, a, 1);
                    h[co] = bf16_bits(fmaxf(a, o));
                }
                if ((l & 1) == 0) {
                    const int lq = l >> 1;  // 0..63
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint4 w;
                        w.x = h[8 * c + 0] | ((uint32_t)h[8 * c + 1] << 16);
                        w.y = h[8 * c + 2] | ((uint32_t)h[8 * c + 3] << 16);
                        w.z = h[8 * c + 4] | ((uint32_t)h[8 * c + 5] << 16);
                        w.w = h[8 * c + 6] | ((uint32_t)h[8 * c + 7] << 16);
                        uint8_t *A3 = S.A3 + c * kA3Chunk + prof * 16;
                        *reinterpret_cast<uint4 *>(A3 + (lq + 2) * 32) = w;
                        if (lq >= 62) *reinterpret_cast<uint4 *>(A3 + (lq - 62) * 32) = w;
                        if (lq <= 1) *reinterpret_cast<uint4 *>(A3 + (lq + 66) * 32) = w;
                    }
                    if (p.h2save) {
                        const int64_t k = k0 + prof;
                        if ((k - p.k_begin) < p.np)
                            for (int co = 0; co < 32; ++co)
                                p.h2save[((size_t)(k - p.k_begin) * 32 + co) * 64 + lq] = h[co];
                    }
                }
                if (p.a2save) {
                    // pre-activation of conv2 (with bias), for the ReLU/pool backward
                    const int64_t k = k0 + prof;
                    if ((k - p.k_begin) < p.np)
                        for (int co = 0; co < 32; ++co)
                            p.a2save[((size_t)(k - p.k_begin) * 32 + co) * 128 + l] = v[co] + S.b2[co];
                }
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- conv3: one implicit GEMM, M = 64 positions x 2 profiles, N = 64, K = 160
        if (tid == 0) {
            const uint32_t idesc = umma_idesc_bf16(128, 64);
            const uint32_t abase = smem_u32(S.A3);
#pragma unroll
            for (int i = 0; i < 10; ++i) {
                const int q0 = 2 * i, q1 = 2 * i + 1;
                const uint32_t o0 = (q0 / 5) * kA3Chunk + (q0 % 5) * 32;
                const uint32_t o1 = (q1 / 5) * kA3Chunk + (q1 % 5) * 32;
                const uint64_t ad = umma_desc(abase + o0, o1 - o0, 128);
                const uint64_t bd = umma_desc(smem_u32(S.B3) + i * 256, 128, 2560);
                umma_bf16(tmem + 64, ad, bd, idesc, i > 0);
            }
            umma_commit(&S.bar);
        }
        if (!mbar_wait_bounded(&S.bar, phase)) S.abort = 1;
        phase ^= 1u;
        tc_fence_after();
        // ---- conv3 epilogue: row m = (position m / 2, profile m % 2); pool rows m, m ^ 2
        {
            const int m = warp * 32 + lane, l = m >> 1, prof = m & 1;
            const int64_t k = k0 + prof;
            const bool valid = (k - p.k_begin) < p.np;
            uint16_t h[64];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 64 + half * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int co = half * 32 + j;
                    const float pre = v[j] + S.b3[co];
                    const float a = fmaxf(pre, 0.f);
                    const float o = __shfl_xor_sync(0xffffffffu, a, 2);
                    h[co] = bf16_bits(fmaxf(a, o));
                    if (p.a3save && valid)
                        p.a3save[((size_t)(k - p.k_begin) * 64 + co) * 64 + l] = pre;
                }
            }
            if ((l & 1) == 0 && valid) {
                const int lq = l >> 1;  // pooled position 0..31 = fc1 K chunk
                const int64_t kl = k - p.k_begin;
                const int64_t mt = kl >> 7;
                const int r = (int)(kl & 127);
                uint8_t *blk = p.h3t + ((size_t)mt * 32 + lq) * kTileBytes;
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    uint4 w;
                    w.x = h[8 * cc + 0] | ((uint32_t)h[8 * cc + 1] << 16);
                    w.y = h[8 * cc + 2] | ((uint32_t)h[8 * cc + 3] << 16);
                    w.z = h[8 * cc + 4] | ((uint32_t)h[8 * cc + 5] << 16);
                    w.w = h[8 * cc + 6] | ((uint32_t)h[8 * cc + 7] << 16);
                    *reinterpret_cast<uint4 *>(blk + canon(r, 8 * cc, 128, 1024)) = w;
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

constexpr int kFcStages = 3;
constexpr int kFcStageBytes = 2 * kTileBytes + kW1Chunk;  // 64 KB

struct FcSmem {
    uint8_t stage[kFcStages][kFcStageBytes];
    float bf1[256];
    float wf2[256];
    uint64_t full[kFcStages];
    uint64_t empty[kFcStages];
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
        for (int s = 0; s < kFcStages; ++s) {
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
    const int64_t npairs = (ntiles + p.tiles_per_block - 1) / p.tiles_per_block;
    uint32_t it_prod = 0, it_mma = 0, done_phase = 0;

    for (int64_t pair = blockIdx.x; pair < npairs; pair += gridDim.x) {
        const int64_t mt0 = (int64_t)p.tiles_per_block * pair;
        const bool two = p.tiles_per_block == 2 && mt0 + 1 < ntiles;
        if (tid == 0) {
            // producer: stream the two activation tiles and fc1's weights, K chunk by chunk
            for (int kc = 0; kc < 32 && !S.abort; ++kc, ++it_prod) {
                const int s = it_prod % kFcStages;
                const uint32_t use = it_prod / kFcStages;
                if (use > 0 && !mbar_wait_bounded(&S.empty[s], (use - 1) & 1u)) {
                    S.abort = 1;
                    break;
                }
                const uint32_t bytes = (two ? 2u : 1u) * kTileBytes + kW1Chunk;
                mbar_arrive_expect_tx(&S.full[s], bytes);
                bulk_g2s(S.stage[s], p.h3t + ((size_t)mt0 * 32 + kc) * kTileBytes, kTileBytes, &S.full[s]);
                if (two)
                    bulk_g2s(S.stage[s] + kTileBytes, p.h3t + ((size_t)(mt0 + 1) * 32 + kc) * kTileBytes,
                             kTileBytes, &S.full[s]);
                bulk_g2s(S.stage[s] + 2 * kTileBytes, p.w.W1t + (size_t)kc * kW1Chunk, kW1Chunk, &S.full[s]);
            }
        } else if (tid == 32) {
            // MMA issuer: 4 K steps of 16 per chunk, two M tiles sharing each weight chunk
            const uint32_t idesc = umma_idesc_bf16(128, 256);
            for (int kc = 0; kc < 32; ++kc, ++it_mma) {
                const int s = it_mma % kFcStages;
                const uint32_t use = it_mma / kFcStages;
                if (S.abort || !mbar_wait_bounded(&S.full[s], use & 1u)) {
                    S.abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(S.stage[s]);
                const uint32_t a1 = a0 + kTileBytes;
                const uint32_t bw = a0 + 2 * kTileBytes;
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
        // ---- epilogue: thread = profile row of the tile
        const int r = warp * 32 + lane;
#pragma unroll 1
        for (int t = 0; t < (two ? 2 : 1); ++t) {
            const int64_t kl = (mt0 + t) * 128 + r;
            float dot = 0.f;
#pragma unroll 1
            for (int n0 = 0; n0 < 256; n0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + t * 256 + n0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float z = v[j] + S.bf1[n0 + j];
                    const float a = fmaxf(z, 0.f);
                    dot = fmaf(a, S.wf2[n0 + j], dot);
                    if (p.z1save && kl < p.np) p.z1save[(size_t)kl * 256 + n0 + j] = z;
                }
            }
            if (kl < p.np) {
                const float zz = dot + b2;
                const int64_t o = p.slot_k ? p.slot_k[p.k_begin + kl] : p.k_begin + kl;
                if (o >= 0) {
                    if (p.logit) p.logit[o] = zz;
                    if (p.score) p.score[o] = 1.f / (1.f + expf(-zz));
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
                if (!mbar_wait_bounded(&S.full[it % kFcStages], (it / kFcStages) & 1u)) break;
        }
        if (tid == 32) mbar_wait_bounded(&S.done, done_phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
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

// Dynamic shared memory of the conv kernel: at least 48 KB so that no more than 4 blocks
// (4 x 128 TMEM columns) are resident on an SM.
static size_t conv_smem_bytes() { return sizeof(ConvSmem) < 48 * 1024 ? 48 * 1024 : sizeof(ConvSmem); }

cudaError_t cnn_register_kernels()
{
    if (g_cnn_attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(cnn_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cnn_fc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FcSmem));
    if (e == cudaSuccess) g_cnn_attr = 1;
    return e;
}

cudaError_t launch_cnn_conv(const CnnConvParams &p, int num_sms, cudaStream_t st)
{
    cudaError_t e = cnn_register_kernels();
    if (e != cudaSuccess) return e;
    const int64_t npairs = (p.np + 1) / 2;
    // at most 4 blocks per SM: each holds 128 of the SM's 512 TMEM columns
    const int grid = (int)(npairs < (int64_t)num_sms * 4 ? npairs : (int64_t)num_sms * 4);
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
    // SM, one tile per block keeps every SM busy instead
    p.tiles_per_block = ntiles >= 2 * (int64_t)num_sms ? 2 : 1;
    const int64_t nblk = (ntiles + p.tiles_per_block - 1) / p.tiles_per_block;
    const int grid = (int)(nblk < (int64_t)num_sms ? nblk : (int64_t)num_sms);
    cnn_fc_kernel<<<grid, 128, sizeof(FcSmem), st>>>(p);
    return cudaGetLastError();
}

}  // namespace gpfc
