// cnn_train.cu -- backward pass, loss and Adam update of the CNN scorer (sm_103a).
//
// The forward pass for training is the tensor-core forward of cnn.cu run with its
// activation saves switched on (FP32 pre-activations, pooled outputs, the fc1 operand
// tiles and fc1's FP32 pre-activations), so the backward takes the ReLU and max-pool
// decisions the forward took. The backward pass:
//   fc2/fc1 head (per profile, CUDA cores);
//   dW(fc1) = dZ1^T h3 and dh3 = dZ1 W1 as BF16 tensor-core GEMMs (tcgemm.cu);
//   ReLU + max-pool backward (the gradient goes to the first maximum of each pair);
//   conv3 and conv2: weight gradients dW[co][ci,tap] = sum over (profile, position) of
//   da[co][l] h[ci][l + tap - 2] and input gradients dh[(profile, position)][ci] = sum over
//   (co, tap) of da[co][m - tap + 2] W[co][ci][tap] (circular), as BF16 tensor-core GEMMs
//   on operands packed from the saved activations (im2col in the operand layout);
//   conv1's 80 weights and every bias by CUDA-core reductions.
// GEMM operands are BF16 (round to nearest even), accumulation FP32. Every gradient is
// reduced deterministically: split-K partials and per-block partials are added in a fixed
// order. Loss: binary cross-entropy with logits (mean). Adam (Kingma & Ba) updates FP32
// master weights in place.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "gpfc_cnn.h"
#include "gpfc_common.cuh"
#include "gpfc_tcgemm.h"

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

// device fc1 feature fd = position * 64 + channel <-> PyTorch feature channel * 32 + position
__host__ __device__ __forceinline__ int pt_feature(int fd) { return (fd & 63) * 32 + (fd >> 6); }

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
// ------------------------------------------------------------------ GEMM operand loaders
// (element (row, k) of a packed operand; the packer rounds to BF16)

struct LdDZ1T {  // dW(fc1): A(j, profile)
    const float *dZ1;
    __device__ float operator()(int64_t j, int64_t k) const { return dZ1[k * 256 + j]; }
};
struct LdH3T {  // dW(fc1): B(feature fd, profile) = h3 (high + low terms)
    const uint8_t *h3t;
    __device__ float operator()(int64_t fd, int64_t k) const { return LoadH3{h3t}((int)k, (int)fd); }
};
struct LdDZ1 {  // dh3: A(profile, j)
    const float *dZ1;
    __device__ float operator()(int64_t k, int64_t j) const { return dZ1[k * 256 + j]; }
};
struct LdW1T {  // dh3: B(fd, j) = fc1.w[j][pt_feature(fd)]
    const float *w;
    __device__ float operator()(int64_t fd, int64_t j) const { return w[j * 2048 + pt_feature((int)fd)]; }
};
template <int COUT, int L>
struct LdDa {  // conv weight gradient: A(co, (profile b, position l))
    const float *da;
    __device__ float operator()(int64_t co, int64_t k) const { return da[((k / L) * COUT + co) * L + (k % L)]; }
};
template <int CIN, int L>
struct LdHim {  // conv weight gradient: B((ci, tap), (b, l)) = h[b][ci][(l + tap - 2) mod L]
    const uint16_t *h;
    __device__ float operator()(int64_t n, int64_t k) const
    {
        const int ci = (int)(n / 5), tap = (int)(n % 5), l = (int)(k % L);
        return bf2f(h[((k / L) * CIN + ci) * L + ((l + tap - 2 + L) % L)]);
    }
};
template <int COUT, int L>
struct LdDaShift {  // conv input gradient: A((b, m), (co, tap)) = da[b][co][(m - tap + 2) mod L]
    const float *da;
    __device__ float operator()(int64_t r, int64_t k) const
    {
        const int m = (int)(r % L), co = (int)(k / 5), tap = (int)(k % 5);
        return da[((r / L) * COUT + co) * L + ((m - tap + 2 + L) % L)];
    }
};
template <int CIN>
struct LdWT {  // conv input gradient: B(ci, (co, tap)) = W[co][ci][tap]
    const float *W;
    __device__ float operator()(int64_t ci, int64_t k) const { return W[((k / 5) * CIN + ci) * 5 + (k % 5)]; }
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

// ------------------------------------------------------------------ backward launches

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

// per-block partial sums over the profiles of da[b][c][l] for each channel c (bias gradients)
template <int C, int L>
__global__ void __launch_bounds__(256) bias_grad_kernel(const float *da, int64_t B, float *part)
{
    __shared__ float acc[C];
    for (int c = threadIdx.x; c < C; c += blockDim.x) acc[c] = 0.f;
    __syncthreads();
    for (int64_t k = blockIdx.x; k < B; k += gridDim.x) {
        for (int c = threadIdx.x >> 5; c < C; c += blockDim.x >> 5) {
            float s = 0.f;
            for (int l = threadIdx.x & 31; l < L; l += 32) s += da[(k * C + c) * L + l];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if ((threadIdx.x & 31) == 0) acc[c] += s;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) part[(size_t)blockIdx.x * C + c] = acc[c];
}

// out(m, n) = sum over splits s (in order) of part[s][m][n], stored by st(m, n, value)
template <class ST>
__global__ void reduce_splits_kernel(const float *part, int splits, int64_t rows, int64_t cols, ST st)
{
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < splits; ++s) v += (double)part[(size_t)s * total + e];
        st(e / cols, e % cols, (float)v);
    }
}
struct StWf1 {  // dW(fc1)[j][fd] -> PyTorch order
    float *g;
    __device__ void operator()(int64_t j, int64_t fd, float v) const { g[j * 2048 + pt_feature((int)fd)] = v; }
};
struct StRowMajor {
    float *g;
    int64_t ld;
    __device__ void operator()(int64_t r, int64_t c, float v) const { g[r * ld + c] = v; }
};
template <int C, int L>
struct StDh {  // input gradient [(b, m)][ci] -> [b][ci][m]
    float *dh;
    __device__ void operator()(int64_t r, int64_t ci, float v) const { dh[((r / L) * C + ci) * L + (r % L)] = v; }
};

// The tensor-core GEMMs of one backward pass: (rows of A and of the output, rows of B = N,
// K, N tile, split-K count). Operands and partials share three workspace buffers.
struct BwdGemmShape {
    int64_t M, N, K;
    int bn, splits;
};

static BwdGemmShape bwd_shape(int which, int64_t B, int num_sms)
{
    BwdGemmShape s{};
    switch (which) {
    case 0: s = {256, 2048, B, 256, 1}; break;           // dW(fc1)
    case 1: s = {B, 2048, 256, 256, 1}; break;           // dh3
    case 2: s = {64, 160, B * 64, 160, 1}; break;        // dW(conv3)
    case 3: s = {B * 64, 32, 320, 32, 1}; break;         // dh2
    case 4: s = {32, 80, B * 128, 80, 1}; break;         // dW(conv2)
    default: s = {B * 128, 16, 160, 16, 1}; break;       // dh1
    }
    const int64_t mt = (s.M + 127) / 128, nt = (s.N + s.bn - 1) / s.bn, kch = (s.K + 63) / 64;
    if (mt * nt < num_sms) s.splits = (int)std::min<int64_t>(kch, (num_sms + mt * nt - 1) / (mt * nt));
    return s;
}

static void bwd_ws_sizes(int64_t B, int num_sms, size_t &a, size_t &b, size_t &part)
{
    a = b = part = 0;
    for (int w = 0; w < 6; ++w) {
        const BwdGemmShape s = bwd_shape(w, B, num_sms);
        a = std::max(a, packed_bytes(s.M, 128, s.K));
        b = std::max(b, packed_bytes(s.N, s.bn, s.K));
        part = std::max(part, (size_t)s.splits * (size_t)s.M * (size_t)((s.N + s.bn - 1) / s.bn * s.bn) * 4);
    }
}

size_t cnn_backward_ws_bytes(int64_t B, int nblk, int num_sms)
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
    take((size_t)nblk * (16 * 5 + 16) * 4);  // conv1 weight/bias partials
    take((size_t)nblk * 64 * 4);       // bias partials
    take((size_t)nblk * 513 * 4);      // head partials
    size_t a, b, part;
    bwd_ws_sizes(B, num_sms, a, b, part);
    take(a);
    take(b);
    take(part);
    return o + 256;
}

// pack A and B of GEMM `which`, run it and hand its partials to `store`
template <class LA, class LB, class ST>
static cudaError_t bwd_gemm(int which, int64_t B, int num_sms, LA la, LB lb, ST store, uint8_t *pa, uint8_t *pb,
                            float *part, cudaStream_t st)
{
    const BwdGemmShape s = bwd_shape(which, B, num_sms);
    const int64_t kch = (s.K + 63) / 64;
    const int64_t ga = std::min<int64_t>(65535, ((s.M + 127) / 128 * 128 * kch * 8 + 255) / 256);
    const int64_t gb = std::min<int64_t>(65535, ((s.N + s.bn - 1) / s.bn * s.bn * kch * 8 + 255) / 256);
    pack_tiles_kernel<<<(int)ga, 256, 0, st>>>(s.M, 128, s.K, la, pa);
    pack_tiles_kernel<<<(int)gb, 256, 0, st>>>(s.N, s.bn, s.K, lb, pb);
    TcGemm g{};
    g.A = pa;
    g.B = pb;
    g.mtiles = (s.M + 127) / 128;
    g.ntiles = (int)((s.N + s.bn - 1) / s.bn);
    g.kchunks = (int)kch;
    g.bn = s.bn;
    g.splits = s.splits;
    g.rows_out = s.M;
    g.ldp = (int64_t)g.ntiles * s.bn;
    g.part = part;
    cudaError_t e = launch_tcgemm(g, num_sms, st);
    if (e != cudaSuccess) return e;
    const int64_t total = s.M * g.ldp;
    reduce_splits_kernel<<<(int)std::min<int64_t>(4096, (total + 255) / 256), 256, 0, st>>>(part, s.splits, s.M,
                                                                                              g.ldp, store);
    return cudaGetLastError();
}

cudaError_t launch_cnn_backward(const CnnSrc &w, const uint8_t *saved, int64_t B, const float *dlogit,
                                const CnnGrads &g, void *ws, int nblk, int num_sms, cudaStream_t st)
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
    float *cpart = reinterpret_cast<float *>(take((size_t)nblk * (16 * 5 + 16) * 4));
    float *bpart = reinterpret_cast<float *>(take((size_t)nblk * 64 * 4));
    float *hpart = reinterpret_cast<float *>(take((size_t)nblk * 513 * 4));
    size_t sa, sb, sp;
    bwd_ws_sizes(B, num_sms, sa, sb, sp);
    uint8_t *pa = take(sa);
    uint8_t *pb = take(sb);
    float *gpart = reinterpret_cast<float *>(take(sp));
    const int sms = num_sms;

    const float *z1 = reinterpret_cast<const float *>(saved + S.z1);
    head_bwd_kernel<<<nblk, 256, 0, st>>>(z1, dlogit, w.wf2, B, dZ1, hpart);
    reduce_parts_kernel<<<1, 256, 0, st>>>(hpart, nblk, 513, 0, 256, g.wf2);
    reduce_parts_kernel<<<1, 256, 0, st>>>(hpart, nblk, 513, 256, 256, g.bf1);
    reduce_parts_kernel<<<1, 32, 0, st>>>(hpart, nblk, 513, 512, 1, g.bf2);
    // dW(fc1)[256][2048] = dZ1^T h3; dh3[B][2048] = dZ1 W1
    cudaError_t e = bwd_gemm(0, B, sms, LdDZ1T{dZ1}, LdH3T{saved + S.h3t}, StWf1{g.wf1}, pa, pb, gpart, st);
    if (e == cudaSuccess) e = bwd_gemm(1, B, sms, LdDZ1{dZ1}, LdW1T{w.wf1}, StRowMajor{dH3, 2048}, pa, pb, gpart, st);
    if (e != cudaSuccess) return e;
    const int eb = 256;
    const int egrid = (int)std::min<int64_t>((B * 64 * 32 + eb - 1) / eb, 65535);
    poolrelu_bwd_kernel<64, 64, true><<<egrid, eb, 0, st>>>(reinterpret_cast<const float *>(saved + S.a3), dH3,
                                                              da3, B);
    // conv3: dW[64][160] and dh2, bias by reduction
    e = bwd_gemm(2, B, sms, LdDa<64, 64>{da3}, LdHim<32, 64>{reinterpret_cast<const uint16_t *>(saved + S.h2)},
                 StRowMajor{g.w3, 160}, pa, pb, gpart, st);
    if (e == cudaSuccess)
        e = bwd_gemm(3, B, sms, LdDaShift<64, 64>{da3}, LdWT<32>{w.w3}, StDh<32, 64>{dh2}, pa, pb, gpart, st);
    if (e != cudaSuccess) return e;
    bias_grad_kernel<64, 64><<<nblk, 256, 0, st>>>(da3, B, bpart);
    reduce_parts_kernel<<<1, 64, 0, st>>>(bpart, nblk, 64, 0, 64, g.b3);
    poolrelu_bwd_kernel<32, 128, false><<<egrid, eb, 0, st>>>(reinterpret_cast<const float *>(saved + S.a2), dh2,
                                                                da2, B);
    // conv2: dW[32][80] and dh1, bias by reduction
    e = bwd_gemm(4, B, sms, LdDa<32, 128>{da2}, LdHim<16, 128>{reinterpret_cast<const uint16_t *>(saved + S.h1)},
                 StRowMajor{g.w2, 80}, pa, pb, gpart, st);
    if (e == cudaSuccess)
        e = bwd_gemm(5, B, sms, LdDaShift<32, 128>{da2}, LdWT<16>{w.w2}, StDh<16, 128>{dh1}, pa, pb, gpart, st);
    if (e != cudaSuccess) return e;
    bias_grad_kernel<32, 128><<<nblk, 256, 0, st>>>(da2, B, bpart);
    reduce_parts_kernel<<<1, 64, 0, st>>>(bpart, nblk, 32, 0, 32, g.b2);
    poolrelu_bwd_kernel<16, 256, false><<<egrid, eb, 0, st>>>(reinterpret_cast<const float *>(saved + S.a1), dh1,
                                                                da1, B);
    // conv1 (16 x 5 weights) on CUDA cores
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
