// probe.cu -- measured peak of the fold's binding pipe: lane-private shared-memory
// read-modify-writes (gpfc_probe_smem_rmw).
//
// The fold's accumulation (Sec. 2.3 step 3) is, per sample and trial period, one
// read-modify-write of that period's bin record in shared memory. This kernel does
// nothing else: every lane owns `nbins` words laid out [bin][lane] (the fold's layout, so
// a warp's 32 accesses never conflict beyond the word width), and updates eight distinct
// bins per iteration (all eight loads issued before the adds and stores, as the fold's
// regular-cadence loop does). The bin sequence is two integer adds and a mask per update;
// nothing else competes for issue. The record kinds are listed below.
#include <cstdint>

#include "gpfc.h"
#include "gpfc_common.cuh"

namespace gpfc {
namespace {

// Record kinds. LDST8: FP32 sum + 32-bit count packed in 8 bytes, one 64-bit load and
// store per update (the fold's default record). LDST6: FP32 sum word [bin][lane] plus a
// 16-bit count, two per 32-bit word [bin/2][lane] (load and store of each). LDST4: one
// 32-bit word. RED6: the 6-byte record updated by no-return shared reductions
// (red.shared.add.f32 to the sum, red.shared.add.u32 of 1 << 16 (bin & 1) to the paired
// count). RED4: red.shared.add.u32 to a 32-bit word. RED8: the reduction fold's record,
// 256 bytes per bin of a warp ([bin][sum row, count row][lane], 32-bit words), updated by
// two red.shared.add.u32 (sum, and count at +128 bytes).
enum ProbeKind { kLdSt8, kLdSt6, kLdSt4, kRed6, kRed4, kRed8 };

__host__ __device__ constexpr uint32_t probe_bytes_x2(int k)  // twice the bytes per bin
{
    return (k == kLdSt8 || k == kRed8) ? 16u : ((k == kLdSt6 || k == kRed6) ? 12u : 8u);
}

template <int KIND>
__global__ void smem_rmw_probe_kernel(int nbins, int iters, unsigned long long *cycles, uint32_t *sink)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool kSix = KIND == kLdSt6 || KIND == kRed6;
    // bytes of the word addressed per bin and lane (the 8-byte reduction record is two
    // 4-byte rows)
    constexpr uint32_t kW = (kSix || KIND == kRed8) ? 4u : probe_bytes_x2(KIND) / 2u;
    constexpr uint32_t kBinStride = KIND == kRed8 ? 256u : 32u * kW;  // bytes per bin of a warp
    const uint32_t wbase = smem_u32(sm) + (uint32_t)warp * (uint32_t)nbins * 32u * probe_bytes_x2(KIND) / 2u;
    const uint32_t base = wbase + (uint32_t)lane * kW;
    const uint32_t cbase = wbase + (uint32_t)nbins * 128u + (uint32_t)lane * 4u;  // 6-byte records: counts
    const uint32_t mask = (uint32_t)nbins - 1u;
    const uint32_t words = kSix ? nbins + nbins / 2 : (KIND == kRed8 ? 2 * nbins : nbins);
    for (uint32_t b = 0; b < words; ++b) {
        if (kW == 8) asm volatile("st.shared.v2.u32 [%0], {%1, %1};" ::"r"(base + b * 256u), "r"(0u));
        else asm volatile("st.shared.u32 [%0], %1;" ::"r"(base + b * 128u), "r"(0u));
    }
    __syncthreads();
    const long long t0 = clock64();
    uint32_t b = (uint32_t)lane * 7u;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
        uint32_t bb[8], a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            bb[u] = (b + 37u * (uint32_t)u) & mask;
            a[u] = base + bb[u] * kBinStride;
        }
        if (KIND == kRed6) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a[u]), "f"(1.0f) : "memory");
                asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(cbase + (bb[u] >> 1) * 128u),
                             "r"(1u << ((bb[u] & 1u) << 4)) : "memory");
            }
        } else if (KIND == kRed4) {
#pragma unroll
            for (int u = 0; u < 8; ++u) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a[u]), "r"(3u) : "memory");
        } else if (KIND == kRed8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a[u]), "r"(3u) : "memory");
                asm volatile("red.shared.add.u32 [%0+128], %1;" ::"r"(a[u]), "r"(1u) : "memory");
            }
        } else if (KIND == kLdSt8) {
            uint32_t s[8], c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(s[u]), "=r"(c[u]) : "r"(a[u]));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float v = __uint_as_float(s[u]) + 1.0f;
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a[u]), "r"(__float_as_uint(v)), "r"(c[u] + 1u));
            }
        } else if (KIND == kLdSt6) {
            uint32_t s[8], c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                asm volatile("ld.shared.u32 %0, [%1];" : "=r"(s[u]) : "r"(a[u]));
                asm volatile("ld.shared.u16 %0, [%1];" : "=r"(c[u]) : "r"(cbase + (bb[u] >> 1) * 128u + (bb[u] & 1u) * 2u));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float v = __uint_as_float(s[u]) + 1.0f;
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(a[u]), "r"(__float_as_uint(v)));
                asm volatile("st.shared.u16 [%0], %1;" ::"r"(cbase + (bb[u] >> 1) * 128u + (bb[u] & 1u) * 2u),
                             "h"((unsigned short)(c[u] + 1u)));
            }
        } else {
            uint32_t s[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) asm volatile("ld.shared.u32 %0, [%1];" : "=r"(s[u]) : "r"(a[u]));
#pragma unroll
            for (int u = 0; u < 8; ++u) asm volatile("st.shared.u32 [%0], %1;" ::"r"(a[u]), "r"(s[u] + 3u));
        }
        b += 13u;
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
    // keep the stores observable: one word per lane of warp 0 goes out
    if (warp == 0) {
        uint32_t v;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(base));
        if (v == 0xFFFFFFFFu) sink[lane] = v;
    }
}

}  // namespace
}  // namespace gpfc

extern "C" int gpfc_probe_smem_rmw(int32_t word_bytes, int32_t op, int32_t nbins, int32_t warps,
                                   int32_t blocks_per_sm, int64_t iters, void *stream, double *updates_per_s,
                                   double *updates_per_clk_sm)
{
    if ((word_bytes != 4 && word_bytes != 6 && word_bytes != 8) || (op != 0 && op != 1) || nbins < 8 ||
        nbins > 4096 || (nbins & (nbins - 1)) || warps < 1 || warps > 32 || blocks_per_sm < 1 ||
        blocks_per_sm > 32 || iters < 1 || iters > (1 << 30))
        return GPFC_EINVAL;
    const size_t smem = (size_t)warps * nbins * 32 * word_bytes;
    int dev = 0, sms = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GPFC_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)max_smem) return GPFC_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    using namespace gpfc;
    auto kern = word_bytes == 8 ? (op ? smem_rmw_probe_kernel<kRed8> : smem_rmw_probe_kernel<kLdSt8>)
              : word_bytes == 6 ? (op ? smem_rmw_probe_kernel<kRed6> : smem_rmw_probe_kernel<kLdSt6>)
                                : (op ? smem_rmw_probe_kernel<kRed4> : smem_rmw_probe_kernel<kLdSt4>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GPFC_ECUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem) != cudaSuccess ||
        occ < blocks_per_sm)
        return GPFC_EINVAL;  // the blocks of one SM would not all be resident at once
    unsigned long long *cyc = nullptr;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GPFC_ECUDA;
    if (cudaMalloc(&cyc, sizeof(unsigned long long)) == cudaSuccess &&
        cudaMalloc(&sink, 32 * sizeof(uint32_t)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess && cudaMemsetAsync(cyc, 0, sizeof(unsigned long long), st) == cudaSuccess) {
        const int grid = sms * blocks_per_sm;
        kern<<<grid, warps * 32, smem, st>>>(nbins, 64, cyc, sink);  // warm-up
        cudaMemsetAsync(cyc, 0, sizeof(unsigned long long), st);
        cudaEventRecord(e0, st);
        kern<<<grid, warps * 32, smem, st>>>(nbins, (int)iters, cyc, sink);
        cudaEventRecord(e1, st);
        unsigned long long cycles = 0;
        float ms = 0.f;
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaMemcpy(&cycles, cyc, sizeof(cycles), cudaMemcpyDeviceToHost) == cudaSuccess && ms > 0.f &&
            cycles > 0) {
            const double updates = (double)grid * warps * 32.0 * 8.0 * (double)iters;
            if (updates_per_s) *updates_per_s = updates / (ms * 1e-3);
            if (updates_per_clk_sm) *updates_per_clk_sm = updates / ((double)cycles * sms);
            rc = GPFC_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cyc) cudaFree(cyc);
    if (sink) cudaFree(sink);
    return rc;
}
