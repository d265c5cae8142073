// gpfc_tcgemm.h -- the BF16 tensor-core GEMM of the CNN backward pass (tcgemm.cu) and the
// CUDA-core kernel that packs its operands.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gpfc {

// part[s][m][n] = sum over split s's K chunks of A[m][k] B[n][k], m < rows_out, n < ntiles bn.
struct TcGemm {
    const uint8_t *A;  // [mtiles][kchunks] tiles of 128 x 64 BF16 (16 KB)
    const uint8_t *B;  // [ntiles][kchunks] tiles of bn x 64 BF16
    int64_t mtiles;
    int ntiles, kchunks, bn, splits;
    int64_t rows_out;  // rows of the output (<= 128 mtiles)
    float *part;       // [splits][rows_out][ldp] FP32
    int64_t ldp;       // = ntiles * bn
    uint32_t *status;
};

cudaError_t launch_tcgemm(const TcGemm &g, int num_sms, cudaStream_t st);

// Bytes of a packed operand of `rows` rows (padded to whole tiles of tile_rows) and K
// (padded to whole chunks of 64).
inline size_t packed_bytes(int64_t rows, int tile_rows, int64_t K)
{
    return (size_t)((rows + tile_rows - 1) / tile_rows) * (size_t)((K + 63) / 64) * (size_t)tile_rows * 128;
}

// Pack element (r, k) = ld(r, k) (zero outside rows x K) as BF16 (round to nearest even)
// into tiles [r / tile_rows][k / 64] of the K-major no-swizzle operand layout: row r's
// eight K values k..k+7 form one 16-byte core-matrix row. One thread per 8 values.
template <class LD>
__global__ void pack_tiles_kernel(int64_t rows, int tile_rows, int64_t K, LD ld, uint8_t *tiles)
{
    const int64_t kch = (K + 63) / 64;
    const int64_t rpad = (rows + tile_rows - 1) / tile_rows * tile_rows;
    const int64_t total = rpad * kch * 8;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / (kch * 8);
        const int64_t kq = e % (kch * 8);  // which 8-wide K group
        const int64_t k0 = kq * 8;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float v0 = 0.f, v1 = 0.f;
            if (r < rows) {
                if (k0 + 2 * h < K) v0 = ld(r, k0 + 2 * h);
                if (k0 + 2 * h + 1 < K) v1 = ld(r, k0 + 2 * h + 1);
            }
            const __nv_bfloat162 b = __floats2bfloat162_rn(v0, v1);
            w[h] = *reinterpret_cast<const uint32_t *>(&b);
        }
        const int64_t rt = r / tile_rows, rr = r % tile_rows;
        const int64_t kc = k0 / 64, kk = k0 % 64;
        uint8_t *tile = tiles + (size_t)(rt * kch + kc) * tile_rows * 128;
        *reinterpret_cast<uint4 *>(tile + (rr >> 3) * 1024 + (kk >> 3) * 128 + (rr & 7) * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace gpfc
