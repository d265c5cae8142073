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
//  * cnn_conv_kernel: one persistent block per SM, warp-specialised (see the conv kernel
//    section): a producer thread stages the folded means and counts of the block's coming
//    quads of four profiles with bulk copies, an MMA thread issues the layers, and eight
//    worker warps run the noise normalisation (Sec. 2.1: std scaled to 1, mean kept) and
//    the epilogues, each stage on a different quad so that the tensor cores and the CUDA
//    cores overlap. conv1, conv2 and conv3 are implicit GEMMs on tcgen05: conv1 from one
//    16-byte im2col row per pooled position and term, conv2 and conv3 straight from the
//    activations, which sit in shared memory as even and odd position planes with a
//    circular halo row, [channel chunk of 8][row][profile][8 channels] BF16, so the A
//    window of pooled output q for pool member j and tap u starts 16-byte rows apart
//    whatever j and u are (core-matrix K step = one tap), no im2col copy. conv1: M = 128
//    pooled positions per profile, N = 32 (pool member x 16 channels), K = 16 (8 taps of
//    the high terms, 8 of the low terms); conv2: M = 64 pooled positions x 2 profiles,
//    N = 32, K = 80 per term; conv3: M = 32 pooled positions x 4 profiles, N = 64, K = 160
//    per term; conv2 and conv3 keep one accumulator per pool member. Accumulators live in
//    TMEM; the epilogue pools the two members in registers (the same TMEM lane), adds the
//    bias, applies ReLU and writes the next layer's input as two BF16 terms.
//    The pooled conv3 output (flattened position-major, feature = position * 64 + channel,
//    with fc1's weights permuted to match) is written to global memory pre-tiled in the
//    tensor-core operand layout, 128 profiles x 64 features per 16 KB block, high terms then
//    low terms.
//  * cnn_fc_kernel: fc1 as a tcgen05 GEMM, M = 128 profiles (one or two tiles per block, or
//    half of a tile's N), N = 256, K = 2 x 2048 (high and low terms against the same
//    weights), operands streamed with bulk copies through a 2-4 stage mbarrier pipeline by
//    a producer thread while another thread issues the MMAs. The epilogue adds fc1's bias,
//    applies ReLU, takes the fc2 dot product from TMEM and applies the sigmoid.
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
// (+16 bytes: the odd plane's rows sit 4 banks away from the even plane's, so the conv1
// epilogue's stores to both planes take no more shared-memory wavefronts than their bytes need)
constexpr int kA2PlaneB = 2 * kA2ChunkB + 16;        // 2 channel chunks
constexpr int kA2PairB = 2 * kA2PlaneB;              // 2 planes
constexpr int kA3Rows = 34;                          // conv3 input: plane index -1..32
constexpr int kA3ChunkB = kA3Rows * 4 * 16;          // [row][profile of the quad][8 channels]
constexpr int kA3PlaneB = 4 * kA3ChunkB + 32;        // 4 channel chunks (+32 bytes, as for conv2's input)
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
//
// One persistent block per SM, three roles:
//  * warp 1 (one thread): copies the folded means and counts of the block's coming quads
//    into a ring of kInSlots slots with the bulk-copy engine;
//  * warp 0 (one thread): issues the MMAs, layer by layer, quad by quad;
//  * kConvWorkers worker warps in two halves of four (each half covers the four TMEM lane
//    quarters): stage N, noise normalisation and the conv1 im2col rows, built in registers
//    (first half, one profile a warp); the epilogues of conv1 (first half: profile 0, second
//    half: profiles 1-3), conv2 (one pair of profiles a half) and conv3 (32 channels a half).
// Each layer has one TMEM accumulator (C1, C2, C3: 3 x 128 columns) and one pair of operand
// buffers in shared memory (A1, A2, A3, high and low terms). In pipeline step j the workers
// run N(j), E1(j-1), E2(j-2), E3(j-3) and the MMA thread runs conv1(j), conv2(j-1),
// conv3(j-2), so the tensor cores work on one quad while the workers fill or drain the
// buffers of the others. mbarriers carry every hand-off (no worker barrier exists):
//   in_full/in_empty  input ring (bulk copies -> N; 128 arrivals free a slot)
//   aK_full           workers have written AK (128 arrivals for A1, 256 for A2, A3) ->
//                     convK may start
//   cK_full           tcgen05.commit after convK: CK holds quad j, and AK is free again
//   cK_empty          workers have read CK (256 arrivals) -> convK of the next quad may start
// A worker never runs two pipeline steps ahead of the MMAs it depends on, so no waiter can
// fall two phases behind a barrier. Every wait is bounded and also ends on the block's abort
// flag; after a failed wait a worker skips its work but still runs the loop to its end.
constexpr int kConvWorkers = 8;
constexpr int kConvWorkerThreads = 32 * kConvWorkers;
constexpr int kConvThreads = 32 * (2 + kConvWorkers);
constexpr int kConvProfiles = 4;  // profiles per quad
constexpr int kInSlots = 3;
constexpr int kConvTmemCols = 512;  // C1, C2, C3 (128 columns each), allocated as a power of two

struct ConvSmem {
    uint8_t B1[kB1Bytes];
    uint8_t B2[kB2Bytes];
    uint8_t B3[kB3Bytes];
    uint8_t A1[4][kA1ProfB];      // conv1 im2col (high terms), one per profile of the quad
    uint8_t A1lo[4][kA1ProfB];    // K chunk 1 of conv1: the low terms of the same rows
    uint8_t A2[2][kA2PairB];      // conv2 input of each pair of the quad (high terms)
    uint8_t A2lo[2][kA2PairB];    // (low terms)
    uint8_t A3[2 * kA3PlaneB];    // conv3 input of the quad (high terms)
    uint8_t A3lo[2 * kA3PlaneB];  // (low terms)
    float in_mean[kInSlots][kConvProfiles * 256];
    int32_t in_cnt[kInSlots][kConvProfiles * 256];
    float b1[16];
    float b2[32];
    float b3[64];
    uint64_t in_full[kInSlots], in_empty[kInSlots];
    uint64_t a_full[3], c_full[3], c_empty[3];
    uint64_t drain;
    uint32_t tslot;
    int abort;
};

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

// mbarrier try_wait with a suspend-time hint: a waiting thread sleeps in hardware until the
// phase completes or about 20 microseconds pass, instead of spinning on issue slots the
// other warps need.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase that also gives up when the block has aborted; a
// timeout sets the abort flag.
__device__ __forceinline__ bool conv_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - start > kWaitLimitCycles) {
            *abort = 1;
            return false;
        }
    }
}

__global__ void __launch_bounds__(kConvThreads, 1) cnn_conv_kernel(const CnnConvParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    ConvSmem &S = *reinterpret_cast<ConvSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    volatile int *abort = &S.abort;

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
    if (warp == 0) tmem_alloc(&S.tslot, kConvTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kInSlots; ++s) {
            mbar_init(&S.in_full[s], 1);
            mbar_init(&S.in_empty[s], kConvWorkerThreads / 2);  // the normalising half
        }
        for (int l = 0; l < 3; ++l) {
            mbar_init(&S.a_full[l], l == 0 ? kConvWorkerThreads / 2 : kConvWorkerThreads);
            mbar_init(&S.c_full[l], 1);
            mbar_init(&S.c_empty[l], kConvWorkerThreads);
        }
        mbar_init(&S.drain, 1);
        fence_mbar_init();
        S.abort = 0;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tslot;
    const uint32_t tC1 = tmem, tC2 = tmem + 128, tC3 = tmem + 256;
    const int64_t nquads_all = (p.np + kConvProfiles - 1) / kConvProfiles;
    // this block's quads: blockIdx.x + j * gridDim.x, j = 0 .. nq - 1
    const int nq = blockIdx.x < nquads_all ? (int)((nquads_all - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;
    auto quad_l0 = [&](int j) { return (int64_t)kConvProfiles * ((int64_t)blockIdx.x + (int64_t)j * gridDim.x); };

    if (warp == 1) {
        // ------------------------------------------------ input producer
        if (lane == 0) {
            int issued = 0;
            for (int j = 0; j < nq; ++j) {
                const int s = j % kInSlots;
                const uint32_t use = j / kInSlots;
                if (use > 0 && !conv_wait(&S.in_empty[s], (use - 1) & 1u, abort)) break;
                const int64_t l0 = quad_l0(j);
                const int64_t nv = min((int64_t)kConvProfiles, p.np - l0);
                const uint32_t bytes = (uint32_t)nv * 1024u;
                mbar_arrive_expect_tx(&S.in_full[s], p.counts ? 2u * bytes : bytes);
                bulk_g2s(S.in_mean[s], p.folded + (size_t)(p.k_begin + l0) * 256, bytes, &S.in_full[s]);
                if (p.counts) bulk_g2s(S.in_cnt[s], p.counts + (size_t)(p.k_begin + l0) * 256, bytes, &S.in_full[s]);
                ++issued;
            }
            // the last copy into each slot has landed before the block exits (after an abort
            // nobody else waits for it; copies complete on their own, so these waits end)
            for (int j = issued > kInSlots ? issued - kInSlots : 0; j < issued; ++j)
                mbar_wait_bounded(&S.in_full[j % kInSlots], (j / kInSlots) & 1u);
        }
    } else if (warp == 0) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            int issued = 0;
            for (int m = 0; m < nq + 2 && ok; ++m) {
                // conv1 of quad m: M = 128 pooled positions per profile, N = 32 (pool member,
                // channel), K = 16 (8 taps of the high terms, 8 of the low terms)
                if (m < nq) {
                    ok = conv_wait(&S.a_full[0], m & 1, abort) && (m == 0 || conv_wait(&S.c_empty[0], (m - 1) & 1, abort));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t idesc = umma_idesc_bf16(128, 32);
                    const uint64_t bd = umma_desc(smem_u32(S.B1), 128, 256);
#pragma unroll
                    for (int pp = 0; pp < kConvProfiles; ++pp) {
                        const uint32_t a = smem_u32(S.A1[pp]);
                        umma_bf16(tC1 + 32 * pp, umma_desc(a, smem_u32(S.A1lo[pp]) - a, 128), bd, idesc, false);
                    }
                    umma_commit(&S.c_full[0]);
                    ++issued;
                }
                // conv2 of quad m-1: per pair, M = 64 pooled positions x 2 profiles, N = 32,
                // K = 80 per term, one accumulator per pool member
                const int q2 = m - 1;
                if (q2 >= 0 && q2 < nq) {
                    ok = conv_wait(&S.a_full[1], q2 & 1, abort) && (q2 == 0 || conv_wait(&S.c_empty[1], (q2 - 1) & 1, abort));
                    if (!ok) break;
                    tc_fence_after();
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
                                umma_bf16(tC2 + g * 64 + jj * 32, umma_desc(smem_u32(S.A2[g]) + off, kA2ChunkB, 128), bd,
                                          idesc, u > 0);
                                umma_bf16(tC2 + g * 64 + jj * 32, umma_desc(smem_u32(S.A2lo[g]) + off, kA2ChunkB, 128),
                                          bd, idesc, true);
                            }
                    umma_commit(&S.c_full[1]);
                    ++issued;
                }
                // conv3 of quad m-2: M = 32 pooled positions x 4 profiles, N = 64, K = 160 per
                // term, one accumulator per pool member
                const int q3 = m - 2;
                if (q3 >= 0 && q3 < nq) {
                    ok = conv_wait(&S.a_full[2], q3 & 1, abort) && (q3 == 0 || conv_wait(&S.c_empty[2], (q3 - 1) & 1, abort));
                    if (!ok) break;
                    tc_fence_after();
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
                                umma_bf16(tC3 + jj * 64, umma_desc(smem_u32(S.A3) + off, kA3ChunkB, 128), bd, idesc,
                                          u > 0 || cp > 0);
                                umma_bf16(tC3 + jj * 64, umma_desc(smem_u32(S.A3lo) + off, kA3ChunkB, 128), bd, idesc,
                                          true);
                            }
                    umma_commit(&S.c_full[2]);
                    ++issued;
                }
            }
            // every MMA this thread issued completes before the accumulators are released
            if (issued > 0) {
                umma_commit(&S.drain);
                mbar_wait_bounded(&S.drain, 0u);
            }
        }
    } else {
        // ------------------------------------------------ workers
        const int wi = warp - 2;         // worker index 0..7
        const int qtr = warp & 3;        // TMEM lane quarter this warp may access
        const int sub = wi >> 2;         // which half of a stage's columns this warp takes
        const uint32_t tlane = (uint32_t)(qtr * 32) << 16;
        const int row = qtr * 32 + lane; // accumulator row (TMEM lane) of this thread
        bool ok = true;
        // after a failed or aborted wait a worker skips all work but still runs the loop: its
        // remaining waits return at once (the abort flag is set), and no worker barrier exists
        for (int j = 0; j < nq + 3; ++j) {
            // ---- N(j): noise normalisation (Sec. 2.1) and conv1 im2col, by the four warps of
            // the first half (warp wi takes profile wi)
            if (j < nq && sub == 0) {
                const int s = j % kInSlots;
                const int64_t l0 = quad_l0(j);
                ok = ok && conv_wait(&S.in_full[s], (j / kInSlots) & 1u, abort);
                // A1 is free once conv1 of the previous quad has completed
                ok = ok && (j == 0 || conv_wait(&S.c_full[0], (j - 1) & 1, abort));
                ok = __all_sync(0xffffffffu, ok);  // warp-uniform: shuffles follow
                if (ok) {
                    const int pp = wi;
                    const int64_t kl = l0 + pp;
                    const bool valid = kl < p.np;
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
                            const float4 f = *reinterpret_cast<const float4 *>(&S.in_mean[s][pp * 256 + 8 * lane + 4 * h]);
                            v[4 * h] = f.x;
                            v[4 * h + 1] = f.y;
                            v[4 * h + 2] = f.z;
                            v[4 * h + 3] = f.w;
                            if (p.counts) {
                                const int4 c = *reinterpret_cast<const int4 *>(&S.in_cnt[s][pp * 256 + 8 * lane + 4 * h]);
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
                    // profile are ~1e-5 of its mean, so an FP32 mean alone (error up to half an
                    // ulp, ~3e-8) would shift every deviation alike by up to ~0.5% of the
                    // profile's standard deviation, and the network would see that shift in
                    // every bin. fmaf(-m, cnt, sh) is the exact remainder of the rounded
                    // division, and v - m is exact whenever v and m are within a factor of two
                    // (the case that needs it).
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
                    // this lane's positions 8 lane .. 8 lane + 7 as four pairs of two BF16
                    // terms; the im2col rows q = 4 lane .. 4 lane + 3 (positions 2q-2 .. 2q+5)
                    // also take the last pair of the lane before and the first two pairs of
                    // the lane after (circularly: lane 0 follows lane 31)
                    uint32_t ph[7], pl[7];
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const float x0 = (inv_sd > 0.f && ne[u]) ? fmaf(d[u], inv_sd, m) : m;
                        const float x1 = (inv_sd > 0.f && ne[u + 1]) ? fmaf(d[u + 1], inv_sd, m) : m;
                        split_bf16x2(x0, x1, ph[1 + u / 2], pl[1 + u / 2]);
                    }
                    const int lp = (lane + 31) & 31, ln = (lane + 1) & 31;
                    ph[0] = __shfl_sync(0xffffffffu, ph[4], lp);
                    pl[0] = __shfl_sync(0xffffffffu, pl[4], lp);
                    ph[5] = __shfl_sync(0xffffffffu, ph[1], ln);
                    pl[5] = __shfl_sync(0xffffffffu, pl[1], ln);
                    ph[6] = __shfl_sync(0xffffffffu, ph[2], ln);
                    pl[6] = __shfl_sync(0xffffffffu, pl[2], ln);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int q = 4 * lane + r;
                        *reinterpret_cast<uint4 *>(S.A1[pp] + q * 16) = make_uint4(ph[r], ph[r + 1], ph[r + 2], ph[r + 3]);
                        *reinterpret_cast<uint4 *>(S.A1lo[pp] + q * 16) = make_uint4(pl[r], pl[r + 1], pl[r + 2], pl[r + 3]);
                    }
                    if (p.xsave && valid) {
                        // the input the network sees (hi + lo, exact in FP32), kept for the
                        // backward pass
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float2 h2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&ph[1 + u]));
                            const float2 l2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&pl[1 + u]));
                            p.xsave[(size_t)kl * 256 + 8 * lane + 2 * u] = h2.x + l2.x;
                            p.xsave[(size_t)kl * 256 + 8 * lane + 2 * u + 1] = h2.y + l2.y;
                        }
                    }
                }
                mbar_arrive(&S.in_empty[s]);
                fence_proxy_async_smem();
                mbar_arrive(&S.a_full[0]);
            }
            // ---- E1(j-1): conv1 epilogue: bias, ReLU, pool the two members, write A2
            const int e1 = j - 1;
            if (e1 >= 0 && e1 < nq) {
                ok = ok && conv_wait(&S.c_full[0], e1 & 1, abort);
                ok = ok && (e1 == 0 || conv_wait(&S.c_full[1], (e1 - 1) & 1, abort));  // A2 free
                ok = __all_sync(0xffffffffu, ok);  // warp-uniform: tcgen05.ld is warp-collective
                tc_fence_after();
                if (ok) {
                    const int q = row;  // pooled position 0..127
                    const int64_t l0 = quad_l0(e1);
                    // the first half takes profile 0, the second half (which does no
                    // normalisation) profiles 1..3
#pragma unroll 1
                    for (int pp = sub == 0 ? 0 : 1; pp < (sub == 0 ? 1 : kConvProfiles); ++pp) {
                        const int64_t kl = l0 + pp;
                        const bool valid = kl < p.np;
                        float v[32];
                        tmem_ld32(tC1 + tlane + 32 * pp, v);
                        uint32_t h[8], hl[8];
#pragma unroll
                        for (int co = 0; co < 16; co += 2)
                            pool_bias_relu2(v[co], v[16 + co], v[co + 1], v[17 + co],
                                            *reinterpret_cast<const float2 *>(&S.b1[co]), h[co >> 1], hl[co >> 1]);
                        if (p.a1save && valid) {
#pragma unroll
                            for (int co = 0; co < 16; ++co) {
                                float *a1 = p.a1save + ((size_t)kl * 16 + co) * 256 + 2 * q;
                                a1[0] = v[co] + S.b1[co];
                                a1[1] = v[16 + co] + S.b1[co];
                            }
                        }
                        if (p.h1save && valid)
#pragma unroll
                            for (int co = 0; co < 16; ++co)
                                p.h1save[((size_t)kl * 16 + co) * 128 + q] = (uint16_t)(h[co >> 1] >> (16 * (co & 1)));
                        const int r = (q >> 1) + 1;
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            uint8_t *A2 = (t ? S.A2lo : S.A2)[pp >> 1] + (q & 1) * kA2PlaneB + (pp & 1) * 16;
                            const uint32_t *hw = t ? hl : h;
#pragma unroll
                            for (int c = 0; c < 2; ++c) {
                                const uint4 w = make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                                *reinterpret_cast<uint4 *>(A2 + c * kA2ChunkB + r * 32) = w;
                                if (q >= 126) *reinterpret_cast<uint4 *>(A2 + c * kA2ChunkB) = w;                   // row -1
                                if (q <= 1) *reinterpret_cast<uint4 *>(A2 + c * kA2ChunkB + (kA2Rows - 1) * 32) = w;  // row 64
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&S.c_empty[0]);
                fence_proxy_async_smem();
                mbar_arrive(&S.a_full[1]);
            }
            // ---- E2(j-2): conv2 epilogue, row = (pooled position row >> 1, profile row & 1 of
            // the pair), write A3
            const int e2 = j - 2;
            if (e2 >= 0 && e2 < nq) {
                ok = ok && conv_wait(&S.c_full[1], e2 & 1, abort);
                ok = ok && (e2 == 0 || conv_wait(&S.c_full[2], (e2 - 1) & 1, abort));  // A3 free
                ok = __all_sync(0xffffffffu, ok);
                tc_fence_after();
                if (ok) {
                    const int q = row >> 1, pr = row & 1, g = sub;
                    const int pp = 2 * g + pr;
                    const int64_t kl = quad_l0(e2) + pp;
                    const bool valid = kl < p.np;
                    float v0[32], v1[32];
                    tmem_ld32(tC2 + tlane + g * 64, v0);
                    tmem_ld32(tC2 + tlane + g * 64 + 32, v1);
                    uint32_t h[16], hl[16];
#pragma unroll
                    for (int co = 0; co < 32; co += 2)
                        pool_bias_relu2(v0[co], v1[co], v0[co + 1], v1[co + 1], *reinterpret_cast<const float2 *>(&S.b2[co]),
                                        h[co >> 1], hl[co >> 1]);
                    if (p.a2save && valid) {
#pragma unroll
                        for (int co = 0; co < 32; ++co) {
                            float *a2 = p.a2save + ((size_t)kl * 32 + co) * 128 + 2 * q;
                            a2[0] = v0[co] + S.b2[co];
                            a2[1] = v1[co] + S.b2[co];
                        }
                    }
                    if (p.h2save && valid)
#pragma unroll
                        for (int co = 0; co < 32; ++co)
                            p.h2save[((size_t)kl * 32 + co) * 64 + q] = (uint16_t)(h[co >> 1] >> (16 * (co & 1)));
                    const int r = (q >> 1) + 1;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        uint8_t *A3 = (t ? S.A3lo : S.A3) + (q & 1) * kA3PlaneB + pp * 16;
                        const uint32_t *hw = t ? hl : h;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const uint4 w = make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                            *reinterpret_cast<uint4 *>(A3 + c * kA3ChunkB + r * 64) = w;
                            if (q >= 62) *reinterpret_cast<uint4 *>(A3 + c * kA3ChunkB) = w;                   // row -1
                            if (q <= 1) *reinterpret_cast<uint4 *>(A3 + c * kA3ChunkB + (kA3Rows - 1) * 64) = w;  // row 32
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&S.c_empty[1]);
                fence_proxy_async_smem();
                mbar_arrive(&S.a_full[2]);
            }
            // ---- E3(j-3): conv3 epilogue, row = (pooled position row >> 2, profile row & 3),
            // channels 32 * sub .. +31; write the fc1 operand tiles of the high and the low
            // terms (feature = position * 64 + channel)
            const int e3 = j - 3;
            if (e3 >= 0 && e3 < nq) {
                ok = ok && conv_wait(&S.c_full[2], e3 & 1, abort);
                ok = __all_sync(0xffffffffu, ok);
                tc_fence_after();
                if (ok) {
                    const int q = row >> 2, pp = row & 3;
                    const int64_t kl = quad_l0(e3) + pp;
                    const bool valid = kl < p.np;
                    float v0[32], v1[32];
                    tmem_ld32(tC3 + tlane + sub * 32, v0);
                    tmem_ld32(tC3 + tlane + 64 + sub * 32, v1);
                    uint32_t h[16], hl[16];
#pragma unroll
                    for (int jc = 0; jc < 32; jc += 2)
                        pool_bias_relu2(v0[jc], v1[jc], v0[jc + 1], v1[jc + 1],
                                        *reinterpret_cast<const float2 *>(&S.b3[sub * 32 + jc]), h[jc >> 1], hl[jc >> 1]);
                    if (p.a3save && valid) {
#pragma unroll
                        for (int jc = 0; jc < 32; ++jc) {
                            const int co = sub * 32 + jc;
                            float *a3 = p.a3save + ((size_t)kl * 64 + co) * 64 + 2 * q;
                            a3[0] = v0[jc] + S.b3[co];
                            a3[1] = v1[jc] + S.b3[co];
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
                            for (int cc = 0; cc < 4; ++cc)
                                *reinterpret_cast<uint4 *>(blk + canon(r, 8 * (4 * sub + cc), 128, 1024)) =
                                    make_uint4(hw[4 * cc], hw[4 * cc + 1], hw[4 * cc + 2], hw[4 * cc + 3]);
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&S.c_empty[2]);
            }
        }
        if (!ok && wi == 0 && lane == 0) report_error(p.status, kErrTimeout);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kConvTmemCols);
}

// ------------------------------------------------------------------ fc kernel

// Pipeline stages (each: the high- and low-term activation tiles of one K chunk for each
// of the block's M tiles, and the weight chunk both terms use): two of 96 KB when a block
// takes two tiles, three of 64 KB when it takes one, four of 48 KB when it takes half of a
// tile's outputs.
constexpr int kFcMaxStages = 4;
constexpr int kFcStageMem = 2 * (4 * kTileBytes + kW1Chunk);  // 192 KB

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
    // a stage holds, for K chunk kc, the high-term (chunk kc) and low-term (chunk 32 + kc)
    // activation tiles of each of the item's M tiles and one weight chunk, which both terms use
    const uint32_t wbytes = halves ? kW1Chunk / 2 : kW1Chunk;            // weights per stage
    const uint32_t woff = (uint32_t)(halves ? 1 : p.tiles_per_block) * 2u * kTileBytes;  // within a stage
    const uint32_t sbytes = woff + wbytes;
    const int nst = (int)min((uint32_t)kFcMaxStages, (uint32_t)kFcStageMem / sbytes);
    auto stage = [&](int st) { return S.stage_mem + (size_t)st * sbytes; };

    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int64_t mt0 = halves ? item >> 1 : (int64_t)p.tiles_per_block * item;
        const int nh = halves ? (int)(item & 1) : 0;  // first output of this item: 128 * nh
        const bool two = !halves && p.tiles_per_block == 2 && mt0 + 1 < ntiles;
        if (tid == 0) {
            // producer: stream the activation tiles and fc1's weights (rows of this item's
            // outputs), K chunk by chunk
            for (int kc = 0; kc < 32 && !S.abort; ++kc, ++it_prod) {
                const int s = it_prod % nst;
                const uint32_t use = it_prod / nst;
                if (use > 0 && !mbar_wait_bounded(&S.empty[s], (use - 1) & 1u)) {
                    S.abort = 1;
                    break;
                }
                const uint32_t bytes = (two ? 4u : 2u) * kTileBytes + wbytes;
                mbar_arrive_expect_tx(&S.full[s], bytes);
                for (int t = 0; t < (two ? 2 : 1); ++t)
                    for (int term = 0; term < 2; ++term)
                        bulk_g2s(stage(s) + (2 * t + term) * kTileBytes,
                                 p.h3t + ((size_t)(mt0 + t) * kH3Chunks + 32 * term + kc) * kTileBytes, kTileBytes,
                                 &S.full[s]);
                // rows 128 * nh .. of the chunk: 16 row groups of 1 KB
                bulk_g2s(stage(s) + woff, p.w.W1t + (size_t)kc * kW1Chunk + (size_t)nh * (kW1Chunk / 2), wbytes,
                         &S.full[s]);
            }
        } else if (tid == 32) {
            // MMA issuer: 4 K steps of 16 per chunk, the high and the low terms of each M tile
            // against the same weights, up to two M tiles sharing each weight chunk
            const uint32_t idesc = umma_idesc_bf16(128, halves ? 128 : 256);
            for (int kc = 0; kc < 32; ++kc, ++it_mma) {
                const int s = it_mma % nst;
                const uint32_t use = it_mma / nst;
                if (S.abort || !mbar_wait_bounded(&S.full[s], use & 1u)) {
                    S.abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(stage(s));
                const uint32_t bw = a0 + woff;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t bd = umma_desc(bw + ks * 256, 128, 1024);
                    for (int t = 0; t < (two ? 2 : 1); ++t) {
                        const uint32_t at = a0 + 2 * t * kTileBytes + ks * 256;
                        umma_bf16(tmem + 256 * t, umma_desc(at, 128, 1024), bd, idesc, kc > 0 || ks > 0);
                        umma_bf16(tmem + 256 * t, umma_desc(at + kTileBytes, 128, 1024), bd, idesc, true);
                    }
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

// Dynamic shared memory of the conv kernel (one block per SM: it takes all 512 TMEM columns).
static size_t conv_smem_bytes() { return sizeof(ConvSmem); }
static_assert(2 * (sizeof(ConvSmem) + 1024) > 228 * 1024, "two conv blocks must not fit one SM");

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
    const int64_t nquads = (p.np + kConvProfiles - 1) / kConvProfiles;
    // persistent: one block per SM, each taking every gridDim-th quad
    const int grid = (int)(nquads < (int64_t)num_sms ? nquads : (int64_t)num_sms);
    if (grid > 0) cnn_conv_kernel<<<grid, kConvThreads, conv_smem_bytes(), st>>>(p);
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
