// noalloc.cu -- best-period search that allocates nothing (gpfc_best_period_noalloc).
//
// For callers that cannot allocate device or host memory at the point of the call: code
// running where a CUDA allocation is not allowed or not wanted (inside a region that
// must not call cudaMalloc, an environment whose memory is fully pre-planned, or a hot
// loop that must not touch the allocator). Such callers cannot create a gpfc_ctx either,
// because gpfc_create allocates. This entry point takes a stream instead of a context and
// keeps its only scratch, the packed (score, index) key of the argmax reduction, in a
// static device array that every GPU using the library holds until the process exits.
#include <cstdint>
#include <mutex>

#include "gpfc.h"
#include "gpfc_kernels.h"

namespace {

// Scratch of the argmax: one 64-bit key in a 256-byte aligned slot (8 bytes used).
constexpr int kNoAllocKeys = 1;
__device__ __align__(256) unsigned long long g_noalloc_key[kNoAllocKeys];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned long long *g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the static key on the current device. The first call on a device
// looks it up with cudaGetSymbolAddress (the name is only a host-side handle; passing
// &g_noalloc_key itself to a kernel would be wrong).
cudaError_t key_address(int device, unsigned long long **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_key);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = static_cast<unsigned long long *>(p);
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int gpfc_best_period_noalloc(const float *score, int64_t n_periods, int64_t *best_index,
                                        float *best_score, void *stream)
{
    if (!score || (!best_index && !best_score)) return GPFC_EINVAL;
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX) return GPFC_EINVAL;  // 32-bit index in the key
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return GPFC_ECUDA;
    unsigned long long *key = nullptr;
    if (key_address(device, &key) != cudaSuccess) return GPFC_ECUDA;
    // An error left pending by earlier work in this thread is not this call's to report or
    // clear: refuse to run and leave it pending, so the launch status checked below is only
    // this call's own.
    if (cudaPeekAtLastError() != cudaSuccess) return GPFC_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the key keeps the previous call's value: clear it before the reduction
    cudaError_t e = cudaMemsetAsync(key, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = gpfc::launch_argmax(score, n_periods, key, st);
    if (e == cudaSuccess) e = gpfc::launch_argmax_finalize(key, 1, best_index, best_score, st);
    return e == cudaSuccess ? GPFC_OK : GPFC_ECUDA;
}
