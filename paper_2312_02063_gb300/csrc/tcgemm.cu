// tcgemm.cu -- BF16 tensor-core GEMM with FP32 accumulation for the CNN backward pass
// (Sec. 2.5 trains the network; this library runs its gradients' contractions here).
//
//   part[s][m][n] = sum over the K chunks of split s of A[m][k] B[n][k]
//
// A and B are packed beforehand (pack_tiles_kernel) into the tensor cores' K-major,
// no-swizzle operand layout: tiles of `rows` x 64 BF16 (128-byte rows of eight 16-byte core
// matrices), [row tile][K chunk]. A tiles have 128 rows, B tiles bn rows (a multiple of 16,
// at most 256). Each persistent block takes work items (M tile, N tile, K split) in turn:
// one thread streams the A and B tiles of each K chunk through a 4-stage ring of
// bulk copies, one thread issues the MMAs (M = 128, N = bn, K = 16) into a TMEM
// accumulator, and four warps write the FP32 tile to the split's partial output. The
// partials are then added in split order (deterministic).
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>

#include "gpfc_common.cuh"
#include "gpfc_tcgemm.h"

namespace gpfc {

constexpr int kGmStages = 4;
constexpr int kGmStageBytes = 128 * 128 + 256 * 128;  // A tile (16 KB) + largest B tile (32 KB)

struct GemmSmem {
    uint8_t stage[kGmStages][kGmStageBytes];
    uint64_t full[kGmStages];
    uint64_t empty[kGmStages];
    uint64_t done;
    uint32_t tslot;
    int abort;
    uint32_t drain_from;
};

__global__ void __launch_bounds__(128, 1) tcgemm_kernel(const TcGemm g)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    GemmSmem &S = *reinterpret_cast<GemmSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ncols = g.bn <= 32 ? 32u : (g.bn <= 64 ? 64u : (g.bn <= 128 ? 128u : 256u));
    if (warp == 0) tmem_alloc(&S.tslot, ncols);
    if (tid == 0) {
        for (int s = 0; s < kGmStages; ++s) {
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
    const uint32_t abytes = 128u * 128u, bbytes = (uint32_t)g.bn * 128u;
    const int64_t nitems = (int64_t)g.mtiles * g.ntiles * g.splits;
    uint32_t it_prod = 0, it_mma = 0, done_phase = 0;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int split = (int)(item % g.splits);
        const int64_t mn = item / g.splits;
        const int nt = (int)(mn % g.ntiles);
        const int64_t mt = mn / g.ntiles;
        const int kc0 = (int)((int64_t)split * g.kchunks / g.splits);
        const int kc1 = (int)((int64_t)(split + 1) * g.kchunks / g.splits);
        if (tid == 0) {
            for (int kc = kc0; kc < kc1 && !S.abort; ++kc, ++it_prod) {
                const int s = it_prod % kGmStages;
                const uint32_t use = it_prod / kGmStages;
                if (use > 0 && !mbar_wait_bounded(&S.empty[s], (use - 1) & 1u)) {
                    S.abort = 1;
                    break;
                }
                mbar_arrive_expect_tx(&S.full[s], abytes + bbytes);
                bulk_g2s(S.stage[s], g.A + ((size_t)mt * g.kchunks + kc) * abytes, abytes, &S.full[s]);
                bulk_g2s(S.stage[s] + abytes, g.B + ((size_t)nt * g.kchunks + kc) * bbytes, bbytes, &S.full[s]);
            }
        } else if (tid == 32) {
            const uint32_t idesc = umma_idesc_bf16(128, g.bn);
            for (int kc = kc0; kc < kc1; ++kc, ++it_mma) {
                const int s = it_mma % kGmStages;
                const uint32_t use = it_mma / kGmStages;
                if (S.abort || !mbar_wait_bounded(&S.full[s], use & 1u)) {
                    S.abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(S.stage[s]);
                const uint32_t b0 = a0 + abytes;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    umma_bf16(tmem, umma_desc(a0 + ks * 256, 128, 1024), umma_desc(b0 + ks * 256, 128, 1024), idesc,
                              kc > kc0 || ks > 0);
                umma_commit(&S.empty[s]);
            }
            umma_commit(&S.done);
        }
        if (!mbar_wait_bounded(&S.done, done_phase)) S.abort = 1;
        done_phase ^= 1u;
        tc_fence_after();
        // epilogue: thread = row of the M tile
        const int64_t row = mt * 128 + warp * 32 + lane;
        float *out = g.part + ((size_t)split * g.rows_out + row) * g.ldp + (size_t)nt * g.bn;
        const bool live = kc1 > kc0 && row < g.rows_out && !S.abort;
        for (int n0 = 0; n0 < g.bn; n0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + n0, v);
            if (live) {
                const int nn = min(32, g.bn - n0);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nn) out[n0 + j] = v[j];
            }
        }
        if (kc1 <= kc0 && row < g.rows_out)  // an empty split contributes zeros
            for (int j = 0; j < g.bn; ++j) out[j] = 0.f;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (S.abort) break;
    }
    if (S.abort) {
        // the bulk copies and MMAs this block issued land before it exits
        if (tid == 32) S.drain_from = it_mma;
        __syncthreads();
        if (tid == 0) {
            report_error(g.status, kErrTimeout);
            for (uint32_t it = S.drain_from; it < it_prod; ++it)
                if (!mbar_wait_bounded(&S.full[it % kGmStages], (it / kGmStages) & 1u)) break;
        }
        if (tid == 32) mbar_wait_bounded(&S.done, done_phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

static int g_gemm_attr = 0;

cudaError_t launch_tcgemm(const TcGemm &g, int num_sms, cudaStream_t st)
{
    if (g.bn < 16 || g.bn > 256 || (g.bn & 15) || g.splits < 1 || g.kchunks < 1) return cudaErrorInvalidValue;
    if (!g_gemm_attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(tcgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GemmSmem));
        if (e != cudaSuccess) return e;
        g_gemm_attr = 1;
    }
    const int64_t nitems = (int64_t)g.mtiles * g.ntiles * g.splits;
    const int grid = (int)std::min<int64_t>(nitems, (int64_t)num_sms);
    tcgemm_kernel<<<grid, 128, sizeof(GemmSmem), st>>>(g);
    return cudaGetLastError();
}

}  // namespace gpfc
