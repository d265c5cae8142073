// probe.cu -- measured peak of the fold's binding pipe: lane-private shared-memory
// read-modify-writes (gpfc_probe_smem_rmw).
//
// The fold's accumulation (Sec. 2.3 step 3) is, per sample and trial period, one
// read-modify-write of that period's bin record in shared memory. This kernel does
// nothing else: every lane owns `nbins` words laid out [bin][lane] (the fold's layout, so
// a warp's 32 accesses never conflict beyond the word width), and updates eight distinct
// bins per iteration (all eight loads issued before the adds and stores, as the fold's
// regular-cadence loop does). The bin sequence is two integer adds and a mask per update;
// nothing else competes for issue. The word is either 8 bytes (FP32 sum + 32-bit count,
// the fold's record) or 4 bytes (one 32-bit integer).
#include <cstdint>

#include "gpfc.h"
#include "gpfc_common.cuh"

namespace gpfc {
namespace {

template <bool W64>
__global__ void smem_rmw_probe_kernel(int nbins, int iters, unsigned long long *cycles, uint32_t *sink)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t kW = W64 ? 8u : 4u;
    const uint32_t base = smem_u32(sm) + ((uint32_t)warp * (uint32_t)nbins * 32u + (uint32_t)lane) * kW;
    const uint32_t mask = (uint32_t)nbins - 1u;
    for (int b = 0; b < nbins; ++b) {
        if (W64) asm volatile("st.shared.v2.u32 [%0], {%1, %1};" ::"r"(base + (uint32_t)b * 32u * kW), "r"(0u));
        else asm volatile("st.shared.u32 [%0], %1;" ::"r"(base + (uint32_t)b * 32u * kW), "r"(0u));
    }
    __syncthreads();
    const long long t0 = clock64();
    uint32_t b = (uint32_t)lane * 7u;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
        uint32_t a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = base + ((b + 37u * (uint32_t)u) & mask) * 32u * kW;
        if (W64) {
            uint32_t s[8], c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(s[u]), "=r"(c[u]) : "r"(a[u]));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float v = __uint_as_float(s[u]) + 1.0f;
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a[u]), "r"(__float_as_uint(v)), "r"(c[u] + 1u));
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

extern "C" int gpfc_probe_smem_rmw(int32_t word_bytes, int32_t nbins, int32_t warps, int32_t blocks_per_sm,
                                   int64_t iters, void *stream, double *updates_per_s,
                                   double *updates_per_clk_sm)
{
    if ((word_bytes != 4 && word_bytes != 8) || nbins < 8 || nbins > 4096 || (nbins & (nbins - 1)) ||
        warps < 1 || warps > 32 || blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || iters > (1 << 30))
        return GPFC_EINVAL;
    const size_t smem = (size_t)warps * nbins * 32 * word_bytes;
    int dev = 0, sms = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GPFC_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)max_smem) return GPFC_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto kern = word_bytes == 8 ? gpfc::smem_rmw_probe_kernel<true> : gpfc::smem_rmw_probe_kernel<false>;
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
