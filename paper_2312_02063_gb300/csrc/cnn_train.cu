// cnn_train.cu -- backward pass, loss and Adam update of the CNN scorer (sm_103a).
//
// The forward pass for training is the tensor-core forward of cnn.cu run with its
// activation saves switched on (FP32 pre-activations, BF16 pooled outputs, the fc1 operand
// tiles and fc1's FP32 pre-activations), so the backward takes the ReLU and max-pool
// decisions the forward took. The backward pass runs on CUDA cores in FP32
// from those saved values and from the BF16-rounded weights the forward used:
//   fc2/fc1 head (per profile), dW(fc1) and dh3 as tiled FP32 GEMMs,
//   ReLU + max-pool backward (the gradient goes to the first maximum of each pair),
//   conv weight and input gradients per layer (circular, padding 2).
// Every weight gradient is reduced deterministically: per-block partial sums, then a
// fixed-order sum over the blocks. Loss: binary cross-entropy with logits (mean).
// Adam (Kingma & Ba) updates FP32 master weights in place.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "gpfc_cnn.h"
#include "gpfc_common.cuh"

namespace gpfc {

__device__ __forceinline__ float bf2f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
__device__ __forceinline__ float rbf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ------------------------------------------------------------------ loss

// loss partials per block and dlogit = (sigmoid(z) - y) / n
__global__ void bce_kernel(const float *z, const float *y, int64_t n, float *dlogit, double *part)
{
    __shared__ double red[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float zi = z[i], yi = y[i];
        acc += (double)(fmaxf(zi, 0.f) - zi * yi + log1pf(expf(-fabsf(zi))));
        if (dlogit) dlogit[i] = (1.f / (1.f + expf(-zi)) - yi) / (float)n;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void bce_finish_kernel(const double *part, int nblk, int64_t n, float *loss)
{
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += part[b];
    *loss = (float)(t / (double)n);
}

// ------------------------------------------------------------------ head: fc2 and fc1's ReLU

// dZ1[k][j] = [z1 > 0] dz_k wf2[j]; partials of dwf2, dbf1 (256 each) and dbf2 (1)
__global__ void __launch_bounds__(256) head_bwd_kernel(const float *z1, const float *dlogit, const float *wf2,
                                                       int64_t B, float *dZ1, float *part)
{
    const int j = threadIdx.x;
    const float w = rbf(wf2[j]);
    float gw = 0.f, gb = 0.f, gb2 = 0.f;
    for (int64_t k = blockIdx.x; k < B; k += gridDim.x) {
        const float dz = dlogit[k];
        const float z = z1[k * 256 + j];
        gw += dz * fmaxf(z, 0.f);
        const float d = z > 0.f ? dz * w : 0.f;
        dZ1[k * 256 + j] = d;
        gb += d;
        gb2 += dz;
    }
    float *pp = part + (size_t)blockIdx.x * 513;
    pp[j] = gw;
    pp[256 + j] = gb;
    if (j == 0) pp[512] = gb2;
}

// ------------------------------------------------------------------ FP32 tiled GEMM

// C[m][n] = sum_k A(m, k) B(k, n); 64 x 64 tile per block, 256 threads, 4 x 4 per thread.
template <class LA, class LB, class ST>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, LA la, LB lb, ST st)
{
    constexpr int BK = 16;
    __shared__ float As[BK][64 + 4];
    __shared__ float Bs[BK][64 + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + 256 * i, kk = e >> 6, mm = e & 63;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? la(m, k) : 0.f;
            const int n = n0 + mm;
            Bs[kk][mm] = (n < N && k < K) ? lb(k, n) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + jj;
            if (m < M && n < N) st(m, n, acc[i][jj]);
        }
}

// device fc1 feature fd = position * 64 + channel <-> PyTorch feature channel * 32 + position
__host__ __device__ __forceinline__ int pt_feature(int fd) { return (fd & 63) * 32 + (fd >> 6); }

struct LoadDZ1T {  // A(m = j, k = profile) = dZ1[k][j]
    const float *dZ1;
    __device__ float operator()(int m, int k) const { return dZ1[(size_t)k * 256 + m]; }
};
struct LoadH3 {  // B(k = profile, n = fd) from the fc1 operand tiles: high + low BF16 terms
    const uint8_t *h3t;
    __device__ float operator()(int k, int fd) const
    {
        const int mt = k >> 7, r = k & 127, kc = fd >> 6, kk = fd & 63;
        const size_t off = ((size_t)mt * kH3Chunks + kc) * (128 * 64 * 2) +
                           (size_t)((r >> 3) * 1024 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2);
        const size_t lo = (size_t)32 * (128 * 64 * 2);  // the low terms' chunk kc + 32
        return bf2f(*reinterpret_cast<const uint16_t *>(h3t + off)) +
               bf2f(*reinterpret_cast<const uint16_t *>(h3t + off + lo));
    }
};
struct StoreDW1 {  // grad of fc1.w in PyTorch order
    float *g;
    __device__ void operator()(int j, int fd, float v) const { g[(size_t)j * 2048 + pt_feature(fd)] = v; }
};
struct LoadDZ1 {  // A(m = profile, k = j)
    const float *dZ1;
    __device__ float operator()(int m, int k) const { return dZ1[(size_t)m * 256 + k]; }
};
struct LoadW1 {  // B(k = j, n = fd) = BF16-rounded fc1.w[j][pt_feature(fd)]
    const float *w;
    __device__ float operator()(int k, int fd) const { return rbf(w[(size_t)k * 2048 + pt_feature(fd)]); }
};
struct StoreDH3 {
    float *d;
    __device__ void operator()(int m, int fd, float v) const { d[(size_t)m * 2048 + fd] = v; }
};

// ------------------------------------------------------------------ ReLU + max-pool backward

// da[k][c][2l+s] = g[k][c][l] if element 2l+s was the (first) maximum of relu(a) over the
// pair and a > 0 there; else 0. With FROM_H3, g is dh3 in the device feature order.
template <int C, int L, bool FROM_H3>
__global__ void poolrelu_bwd_kernel(const float *a, const float *g, float *da, int64_t B)
{
    const int64_t total = B * C * (L / 2);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int lp = (int)(e % (L / 2));
        const int64_t kc = e / (L / 2);
        const int c = (int)(kc % C);
        const int64_t k = kc / C;
        const float u = a[(kc * L) + 2 * lp], v = a[(kc * L) + 2 * lp + 1];
        const bool second = fmaxf(v, 0.f) > fmaxf(u, 0.f);
        const float gg = FROM_H3 ? g[k * 2048 + lp * 64 + c] : g[kc * (L / 2) + lp];
        da[kc * L + 2 * lp] = (!second && u > 0.f) ? gg : 0.f;
        da[kc * L + 2 * lp + 1] = (second && v > 0.f) ? gg : 0.f;
    }
}

// ------------------------------------------------------------------ conv backward

// One profile at a time per block: weight-gradient partials (kept in registers across the
// block's profiles) and, with DGRAD, the input gradient
//   dW[co][ci][t] += sum_l da[co][l] h[ci][(l + t - 2) mod L],  db[co] += sum_l da[co][l]
//   dh[ci][l] = sum_{co,t} da[co][(l - t + 2) mod L] W[co][ci][t]
template <int CIN, int COUT, int L, bool DGRAD, bool XF32>
__global__ void __launch_bounds__(256) conv_bwd_kernel(const float *da, const void *hin, const float *W,
                                                       float *dh, float *part, int64_t B)
{
    constexpr int NW = COUT * CIN * 5;
    constexpr int PER = (NW + 255) / 256;
    extern __shared__ float sm[];
    float *da_s = sm;                 // [COUT][L]
    float *h_s = da_s + COUT * L;     // [CIN][L]
    float *W_s = h_s + CIN * L;       // [COUT][CIN][5]
    const int t = threadIdx.x;
    if (DGRAD)
        for (int i = t; i < NW; i += 256) W_s[i] = rbf(W[i]);
    float acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0.f;
    float accb = 0.f;
    for (int64_t k = blockIdx.x; k < B; k += gridDim.x) {
        __syncthreads();
        for (int i = t; i < COUT * L; i += 256) da_s[i] = da[(size_t)k * COUT * L + i];
        for (int i = t; i < CIN * L; i += 256) {
            if (XF32) h_s[i] = static_cast<const float *>(hin)[(size_t)k * CIN * L + i];
            else h_s[i] = bf2f(static_cast<const uint16_t *>(hin)[(size_t)k * CIN * L + i]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int o = t + 256 * i;
            if (o < NW) {
                const int co = o / (CIN * 5), ci = (o / 5) % CIN, tap = o % 5;
                const float *dr = da_s + co * L;
                const float *hr = h_s + ci * L;
                float s = 0.f;
                for (int l = 0; l < L; ++l) s = fmaf(dr[l], hr[(l + tap - 2 + L) % L], s);
                acc[i] += s;
            }
        }
        if (t < COUT) {
            float s = 0.f;
            for (int l = 0; l < L; ++l) s += da_s[t * L + l];
            accb += s;
        }
        if (DGRAD) {
            for (int o = t; o < CIN * L; o += 256) {
                const int ci = o / L, l = o % L;
                float s = 0.f;
                for (int co = 0; co < COUT; ++co)
#pragma unroll
                    for (int tap = 0; tap < 5; ++tap)
                        s = fmaf(da_s[co * L + (l - tap + 2 + L) % L], W_s[(co * CIN + ci) * 5 + tap], s);
                dh[(size_t)k * CIN * L + o] = s;
            }
        }
    }
    float *pp = part + (size_t)blockIdx.x * (NW + COUT);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int o = t + 256 * i;
        if (o < NW) pp[o] = acc[i];
    }
    if (t < COUT) pp[NW + t] = accb;
}

// out[i] (+)= sum_b part[b][off + i] for i < n, in block order (deterministic)
__global__ void reduce_parts_kernel(const float *part, int nblk, int stride, int off, int n, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += (double)part[(size_t)b * stride + off + i];
    out[i] = (float)s;
}

// ------------------------------------------------------------------ Adam

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        p[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// ------------------------------------------------------------------ host launches

size_t cnn_saved_bytes(int64_t B)
{
    return CnnSaved::layout(B).total;
}

CnnSaved CnnSaved::layout(int64_t B)
{
    CnnSaved s{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = (o + 255) & ~(size_t)255;
        const size_t r = o;
        o += bytes;
        return r;
    };
    s.x = take((size_t)B * 256 * 4);
    s.a1 = take((size_t)B * 16 * 256 * 4);
    s.h1 = take((size_t)B * 16 * 128 * 2);
    s.a2 = take((size_t)B * 32 * 128 * 4);
    s.h2 = take((size_t)B * 32 * 64 * 2);
    s.a3 = take((size_t)B * 64 * 64 * 4);
    s.h3t = take(cnn_h3t_bytes(B));
    s.z1 = take((size_t)B * 256 * 4);
    s.total = (o + 255) & ~(size_t)255;
    return s;
}

size_t cnn_backward_ws_bytes(int64_t B, int nblk)
{
    size_t o = 0;
    auto take = [&](size_t bytes) { o = ((o + 255) & ~(size_t)255) + bytes; };
    take((size_t)B * 256 * 4);         // dZ1
    take((size_t)B * 2048 * 4);        // dH3
    take((size_t)B * 64 * 64 * 4);     // da3
    take((size_t)B * 32 * 64 * 4);     // dh2
    take((size_t)B * 32 * 128 * 4);    // da2
    take((size_t)B * 16 * 128 * 4);    // dh1
    take((size_t)B * 16 * 256 * 4);    // da1
    take((size_t)nblk * (64 * 32 * 5 + 64) * 4);  // conv partials (largest layer)
    take((size_t)nblk * 513 * 4);      // head partials
    return o + 256;
}

template <int CIN, int COUT, int L, bool DGRAD, bool XF32>
static cudaError_t run_conv_bwd(const float *da, const void *hin, const float *W, float *dh, float *part,
                                int64_t B, int nblk, float *gw, float *gb, cudaStream_t st)
{
    const size_t smem = (size_t)(COUT * L + CIN * L + (DGRAD ? COUT * CIN * 5 : 0)) * 4;
    cudaError_t e = cudaFuncSetAttribute(conv_bwd_kernel<CIN, COUT, L, DGRAD, XF32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv_bwd_kernel<CIN, COUT, L, DGRAD, XF32><<<nblk, 256, smem, st>>>(da, hin, W, dh, part, B);
    constexpr int NW = COUT * CIN * 5;
    reduce_parts_kernel<<<(NW + 255) / 256, 256, 0, st>>>(part, nblk, NW + COUT, 0, NW, gw);
    reduce_parts_kernel<<<1, 64, 0, st>>>(part, nblk, NW + COUT, NW, COUT, gb);
    return cudaGetLastError();
}

cudaError_t launch_cnn_backward(const CnnSrc &w, const uint8_t *saved, int64_t B, const float *dlogit,
                                const CnnGrads &g, void *ws, int nblk, cudaStream_t st)
{
    const CnnSaved S = CnnSaved::layout(B);
    uint8_t *base = static_cast<uint8_t *>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = (o + 255) & ~(size_t)255;
        uint8_t *p = base + o;
        o += bytes;
        return p;
    };
    float *dZ1 = reinterpret_cast<float *>(take((size_t)B * 256 * 4));
    float *dH3 = reinterpret_cast<float *>(take((size_t)B * 2048 * 4));
    float *da3 = reinterpret_cast<float *>(take((size_t)B * 64 * 64 * 4));
    float *dh2 = reinterpret_cast<float *>(take((size_t)B * 32 * 64 * 4));
    float *da2 = reinterpret_cast<float *>(take((size_t)B * 32 * 128 * 4));
    float *dh1 = reinterpret_cast<float *>(take((size_t)B * 16 * 128 * 4));
    float *da1 = reinterpret_cast<float *>(take((size_t)B * 16 * 256 * 4));
    float *cpart = reinterpret_cast<float *>(take((size_t)nblk * (64 * 32 * 5 + 64) * 4));
    float *hpart = reinterpret_cast<float *>(take((size_t)nblk * 513 * 4));

    const float *z1 = reinterpret_cast<const float *>(saved + S.z1);
    head_bwd_kernel<<<nblk, 256, 0, st>>>(z1, dlogit, w.wf2, B, dZ1, hpart);
    reduce_parts_kernel<<<1, 256, 0, st>>>(hpart, nblk, 513, 0, 256, g.wf2);
    reduce_parts_kernel<<<1, 256, 0, st>>>(hpart, nblk, 513, 256, 256, g.bf1);
    reduce_parts_kernel<<<1, 32, 0, st>>>(hpart, nblk, 513, 512, 1, g.bf2);
    {   // dW(fc1)[256][2048] = dZ1^T h3
        dim3 grid(2048 / 64, 256 / 64);
        gemm_kernel<<<grid, 256, 0, st>>>(256, 2048, (int)B, LoadDZ1T{dZ1}, LoadH3{saved + S.h3t}, StoreDW1{g.wf1});
    }
    {   // dh3[B][2048] = dZ1 W1
        dim3 grid(2048 / 64, (unsigned)((B + 63) / 64));
        gemm_kernel<<<grid, 256, 0, st>>>((int)B, 2048, 256, LoadDZ1{dZ1}, LoadW1{w.wf1}, StoreDH3{dH3});
    }
    const int eb = 256;
    const int egrid = (int)std::min<int64_t>((B * 64 * 32 + eb - 1) / eb, 65535);
    poolrelu_bwd_kernel<64, 64, true><<<egrid, eb, 0, st>>>(reinterpret_cast<const float *>(saved + S.a3), dH3,
                                                              da3, B);
    cudaError_t e = run_conv_bwd<32, 64, 64, true, false>(da3, saved + S.h2, w.w3, dh2, cpart, B, nblk, g.w3, g.b3, st);
    if (e != cudaSuccess) return e;
    poolrelu_bwd_kernel<32, 128, false><<<egrid, eb, 0, st>>>(reinterpret_cast<const float *>(saved + S.a2), dh2,
                                                                da2, B);
    e = run_conv_bwd<16, 32, 128, true, false>(da2, saved + S.h1, w.w2, dh1, cpart, B, nblk, g.w2, g.b2, st);
    if (e != cudaSuccess) return e;
    poolrelu_bwd_kernel<16, 256, false><<<egrid, eb, 0, st>>>(reinterpret_cast<const float *>(saved + S.a1), dh1,
                                                                da1, B);
    e = run_conv_bwd<1, 16, 256, false, true>(da1, saved + S.x, w.w1, nullptr, cpart, B, nblk, g.w1, g.b1, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_bce(const float *z, const float *y, int64_t n, float *dlogit, float *loss, void *ws, cudaStream_t st)
{
    const int nblk = (int)std::min<int64_t>(256, (n + 255) / 256);
    double *part = static_cast<double *>(ws);
    bce_kernel<<<nblk, 256, 0, st>>>(z, y, n, dlogit, part);
    if (loss) bce_finish_kernel<<<1, 32, 0, st>>>(part, nblk, n, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>(1024, (n + 255) / 256);
    adam_kernel<<<grid, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace gpfc
