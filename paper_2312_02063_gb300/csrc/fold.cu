// fold.cu -- phase fold, box-SNR and best-period kernels for sm_103a.
//
// Fold (paper Sec. 2.3, Fig. 4 steps a-e, with equal-width bins):
//   tau_i = rint((t_i - t0) 2^24), F_k = rint(2^40 / P_k), phase = (tau F mod 2^64) / 2^64,
//   bin = floor(phase * nbins), then per-bin count and flux sum, mean = sum / count.
//
// Design. One lane owns one trial period for the whole light curve, so no two threads
// ever update the same bin and no atomics are needed. Each warp keeps the bins of its
// 32 periods in shared memory laid out [bin][lane]: lane l's bin b sits in bank l, so a
// warp's 32 read-modify-writes never conflict whatever bins the lanes hit. Light-curve
// tiles (tau split in two 32-bit words, flux - f_ref) are staged into shared memory by
// the bulk-copy (TMA) engine, double-buffered behind an mbarrier, and every lane reads
// the same sample (a broadcast). Each lane processes 4 consecutive samples at once; if
// two of them fall in the same bin it takes a sequential path.
//
// Shared memory holds per (bin, lane) an FP32 partial sum and a 16-bit count over a
// chunk of samples (<= 65535 samples, so the count cannot overflow). At the end of each
// chunk the partials are added into a per-block workspace with Kahan compensation
// (sum, compensation) and exact 32-bit counts; the workspace stays resident in L2.
//
// Epilogues, same kernel: write means + counts (gpfc_fold), or run the box-SNR search
// over the finished profile of each lane's period (gpfc_search, box scorer).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gpfc_common.cuh"
#include "gpfc_kernels.h"

namespace gpfc {

constexpr double kTwo24 = 16777216.0;
constexpr double kTwo40 = 1099511627776.0;
constexpr double kTwo62 = 4611686018427387904.0;
constexpr double kTwo63 = 9223372036854775808.0;

__device__ __forceinline__ void star_range(const int64_t *off, int64_t n, int s, int64_t &b,
                                           int64_t &e)
{
    if (off) {
        b = off[s];
        e = off[s + 1];
    } else {
        b = 0;
        e = n;
    }
}

// First element of star s in the sample scratch: a multiple of 4 (16 bytes), with room
// for the star's samples rounded up to a multiple of 4.
__device__ __forceinline__ int64_t scratch_start(int64_t lc_begin, int s)
{
    return 4 * ((lc_begin + 3) / 4 + s);
}

// ------------------------------------------------------------------ prep

__device__ __forceinline__ double block_sum_f64(double v, double *red)
{
    // fixed-order tree: deterministic for a given block size
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    }
    __syncthreads();
    return t;
}

// Pass 1: per-block FP64 partial sums of flux. grid = (G, stars).
__global__ void prep_sum_kernel(const float *flux, const int64_t *lc_off, int64_t n, double *partial)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    int64_t b, e;
    star_range(lc_off, n, s, b, e);
    const int64_t len = e - b;
    const int64_t per = (len + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = b + (int64_t)blockIdx.x * per;
    const int64_t i1 = min(e, i0 + per);
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += (double)flux[i];
    double t = block_sum_f64(acc, red);
    if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = t;
}

// Pass 2: f_ref = mean flux; quantise times; centre flux; partial sums of squares.
__global__ void prep_quant_kernel(const double *times, const float *flux, const int64_t *lc_off,
                                  int64_t n, const double *t0s, double t0_scalar, double *partial,
                                  SampleScratch smp, StarStats *stats, uint32_t *status)
{
    __shared__ double red[32];
    __shared__ double s_fref;
    const int s = blockIdx.y;
    const int G = gridDim.x;
    int64_t b, e;
    star_range(lc_off, n, s, b, e);
    const int64_t len = e - b;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += partial[(size_t)s * G + g];
        s_fref = tot / (double)len;
    }
    __syncthreads();
    const double f_ref = s_fref;
    double t0 = t0s ? t0s[s] : t0_scalar;
    if (t0 != t0) t0 = times[b];
    const int64_t base = scratch_start(b, s);
    const int64_t per = (len + G - 1) / G;
    const int64_t j0 = (int64_t)blockIdx.x * per;
    const int64_t j1 = min(len, j0 + per);
    double acc = 0.0;
    bool bad = false;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const double v = (times[b + j] - t0) * kTwo24;
        long long tau = 0;
        if (fabs(v) < kTwo62) tau = __double2ll_rn(v);
        else bad = true;
        smp.tau_lo[base + j] = (uint32_t)(unsigned long long)tau;
        smp.tau_hi[base + j] = (int32_t)(tau >> 32);
        const double d = (double)flux[b + j] - f_ref;
        smp.x[base + j] = (float)d;
        acc += d * d;
    }
    if (bad) report_error(status, kErrRange);
    // zero the (at most 3) padding elements after the star so tile copies read defined data
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        const int64_t j = len + threadIdx.x;
        if (j < ((len + 3) & ~(int64_t)3)) {
            smp.tau_lo[base + j] = 0u;
            smp.tau_hi[base + j] = 0;
            smp.x[base + j] = 0.f;
        }
    }
    double t = block_sum_f64(acc, red);
    __syncthreads();
    if (threadIdx.x == 0) partial[(size_t)gridDim.y * G + (size_t)s * G + blockIdx.x] = t;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[s].f_ref = f_ref;
        const float hi = (float)f_ref;
        stats[s].f_hi = hi;
        stats[s].f_lo = (float)(f_ref - (double)hi);
        stats[s].n = (int32_t)len;
    }
}

// Pass 3: sigma = sqrt(sum (flux - f_ref)^2 / n) per star. grid = stars, 32 threads.
__global__ void prep_sigma_kernel(const double *partial, int G, int nstars, StarStats *stats)
{
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int g = 0; g < G; ++g) t += partial[(size_t)nstars * G + (size_t)s * G + g];
    stats[s].sigma = (float)sqrt(t / (double)stats[s].n);
}

cudaError_t launch_prep(const double *times, const float *flux, const int64_t *lc_off, int64_t n,
                        int nstars, int64_t max_len, const double *t0s, double t0, SampleScratch smp,
                        double *partial, int G, StarStats *stats, uint32_t *status, cudaStream_t st)
{
    (void)max_len;
    dim3 grid(G, nstars);
    prep_sum_kernel<<<grid, 256, 0, st>>>(flux, lc_off, n, partial);
    prep_quant_kernel<<<grid, 256, 0, st>>>(times, flux, lc_off, n, t0s, t0, partial, smp, stats,
                                            status);
    prep_sigma_kernel<<<nstars, 32, 0, st>>>(partial, G, nstars, stats);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fold kernel

// bin = floor(((tau * F) mod 2^64) * nbins / 2^64) from 32-bit halves. Only the high
// word of the 64-bit product is formed: hi = umulhi(tl, Fl) + th*Fl + tl*Fh (mod 2^32).
template <bool POW2>
__device__ __forceinline__ uint32_t phase_bin(uint32_t tl, uint32_t th, uint32_t Fl, uint32_t Fh,
                                              uint32_t nbins, int shift)
{
    const uint32_t hi = __umulhi(tl, Fl) + th * Fl + tl * Fh;
    if (POW2) return hi >> shift;
    const uint32_t lo = tl * Fl;
    const unsigned long long t =
        (unsigned long long)hi * nbins + (unsigned long long)__umulhi(lo, nbins);
    return (uint32_t)(t >> 32);
}

// Lane-private bins. The FP32 partial sum of bin b is at accw[b * 32] (bank = lane).
// 16-bit counts are paired per lane: word (b / 2) * 32 + lane holds bins 2j and 2j+1,
// so a warp's count accesses also hit 32 distinct banks whatever the bins.
__device__ __forceinline__ uint32_t cidx(uint32_t b) { return ((b >> 1) << 6) | (b & 1u); }

template <bool POW2>
__device__ __forceinline__ void bins4(const uint32_t *__restrict__ stl, const uint32_t *__restrict__ sth,
                                      int i, uint32_t Fl, uint32_t Fh, uint32_t nbins, int shift,
                                      uint32_t (&b)[4])
{
    const uint4 a = *reinterpret_cast<const uint4 *>(stl + i);
    const uint4 h = *reinterpret_cast<const uint4 *>(sth + i);
    b[0] = phase_bin<POW2>(a.x, h.x, Fl, Fh, nbins, shift);
    b[1] = phase_bin<POW2>(a.y, h.y, Fl, Fh, nbins, shift);
    b[2] = phase_bin<POW2>(a.z, h.z, Fl, Fh, nbins, shift);
    b[3] = phase_bin<POW2>(a.w, h.w, Fl, Fh, nbins, shift);
}

__device__ __forceinline__ bool hazard4(const uint32_t (&b)[4])
{
    return (b[0] == b[1]) | (b[0] == b[2]) | (b[0] == b[3]) | (b[1] == b[2]) | (b[1] == b[3]) |
           (b[2] == b[3]);
}

// Fold nvalid samples of a staged tile into this lane's bins. Groups of 4 samples are
// software-pipelined: the bin reads of group g are issued, then the phases and bins of
// group g+1 are computed while they are in flight, then group g is written back. If two
// samples of a group share a bin the group is applied one sample at a time.
template <bool POW2>
__device__ __forceinline__ void fold_tile(const uint32_t *__restrict__ stl,
                                          const uint32_t *__restrict__ sth,
                                          const float *__restrict__ sx, int nvalid, float *accw,
                                          uint16_t *cntw, uint32_t Fl, uint32_t Fh,
                                          uint32_t nbins, int shift)
{
    const int ng = nvalid >> 2;
    if (ng > 0) {
        uint32_t b[4];
        bins4<POW2>(stl, sth, 0, Fl, Fh, nbins, shift, b);
        float4 x = *reinterpret_cast<const float4 *>(sx);
        bool haz = hazard4(b);
#pragma unroll 1
        for (int g = 0; g < ng; ++g) {
            float s[4];
            uint32_t c[4];
            if (!haz) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    s[u] = accw[b[u] << 5];
                    c[u] = cntw[cidx(b[u])];
                }
            }
            const int in = (g + 1 < ng) ? 4 * g + 4 : 4 * g;
            uint32_t nb[4];
            bins4<POW2>(stl, sth, in, Fl, Fh, nbins, shift, nb);
            const float4 nx = *reinterpret_cast<const float4 *>(sx + in);
            const bool nhaz = hazard4(nb);
            if (!haz) {
                accw[b[0] << 5] = s[0] + x.x;
                accw[b[1] << 5] = s[1] + x.y;
                accw[b[2] << 5] = s[2] + x.z;
                accw[b[3] << 5] = s[3] + x.w;
#pragma unroll
                for (int u = 0; u < 4; ++u) cntw[cidx(b[u])] = (uint16_t)(c[u] + 1u);
            } else {
                const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    accw[b[u] << 5] += xs[u];
                    cntw[cidx(b[u])] = (uint16_t)(cntw[cidx(b[u])] + 1u);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = nb[u];
            x = nx;
            haz = nhaz;
        }
    }
    for (int i = 4 * ng; i < nvalid; ++i) {
        const uint32_t bb = phase_bin<POW2>(stl[i], sth[i], Fl, Fh, nbins, shift);
        accw[bb << 5] += sx[i];
        cntw[cidx(bb)] = (uint16_t)(cntw[cidx(bb)] + 1u);
    }
}

// Fold this lane's chunk partials into the Kahan workspace (sum, compensation) and the
// exact 32-bit counts. On the last chunk the finished sums (sum - compensation) go back
// into accw and the counts into cntw, saturated at 65535 (the exact totals stay in the
// workspace). Workspace reads are batched 16 bins at a time to overlap their latency.
// Returns true if a count saturated.
__device__ __forceinline__ void flush_one(float *accw, uint16_t *cntw, float2 *wsc, uint32_t *wcn,
                                          int b, size_t idx, bool first, bool last, float2 sc,
                                          uint32_t cc, bool &over)
{
    const float p = accw[b << 5];
    const uint32_t c = cntw[cidx(b)];
    if (first) {
        sc = make_float2(p, 0.f);
        cc = c;
    } else {
        cc += c;
        const float y = p - sc.y;
        const float t = sc.x + y;
        sc.y = (t - sc.x) - y;
        sc.x = t;
    }
    if (last) {
        accw[b << 5] = sc.x - sc.y;
        cntw[cidx(b)] = (uint16_t)min(cc, 65535u);
        over |= cc > 65535u;
        if (!first) wcn[idx] = cc;
    } else {
        wsc[idx] = sc;
        wcn[idx] = cc;
        accw[b << 5] = 0.f;
        cntw[cidx(b)] = 0;
    }
}

__device__ __forceinline__ bool flush_chunk(float *accw, uint16_t *cntw, float2 *wsc, uint32_t *wcn,
                                            int nbins, int ppc, bool first, bool last)
{
    bool over = false;
    int b0 = 0;
    for (; b0 + 16 <= nbins; b0 += 16) {
        float2 sc[16];
        uint32_t cc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            sc[u] = make_float2(0.f, 0.f);
            cc[u] = 0u;
            if (!first) {
                sc[u] = wsc[(size_t)(b0 + u) * ppc];
                cc[u] = wcn[(size_t)(b0 + u) * ppc];
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
            flush_one(accw, cntw, wsc, wcn, b0 + u, (size_t)(b0 + u) * ppc, first, last, sc[u], cc[u], over);
    }
    for (; b0 < nbins; ++b0) {
        const size_t idx = (size_t)b0 * ppc;
        float2 sc = make_float2(0.f, 0.f);
        uint32_t cc = 0u;
        if (!first) {
            sc = wsc[idx];
            cc = wcn[idx];
        }
        flush_one(accw, cntw, wsc, wcn, b0, idx, first, last, sc, cc, over);
    }
    return over;
}

// Bins of one profile as seen by one lane: the fold's lane-private layout.
struct LaneBins {
    const float *S;        // accw
    const uint16_t *C;     // cntw
    const uint32_t *Cbig;  // exact counts (workspace) when a count saturated
    size_t cbs;
    bool big;
    __device__ __forceinline__ float s(int b) const { return S[b << 5]; }
    __device__ __forceinline__ float c(int b) const
    {
        return big ? (float)Cbig[(size_t)b * cbs] : (float)C[cidx((uint32_t)b)];
    }
};

// Bins of one profile staged transposed for the standalone scorer ([bin][33]).
struct StagedBins {
    const float *S;
    const uint16_t *C;
    const int32_t *Cbig;   // the caller's counts row when a count exceeds 65535
    bool big;
    __device__ __forceinline__ float s(int b) const { return S[b * 33]; }
    __device__ __forceinline__ float c(int b) const
    {
        return big ? (float)max(Cbig[b], 0) : (float)C[b * 33];
    }
};

// Box-SNR search over one profile held by this lane (bin sums centred on a reference,
// counts). For start s and width w the in-box sums come from running totals: starts
// s0..s0+7 are scored in one walk over bins s0..s0+6+w_max, so every bin read serves 8
// boxes and the 8 evaluations are independent. The search maximises
//     v = (S n_in - S_in N) / sqrt(n_in n_out)      (= snr * sigma * sqrt(N))
// in FP32; ties keep the smaller w, then the smaller s. The winning box is re-evaluated
// in FP64 from the same bin sums.
template <class Bins>
__device__ __forceinline__ void box_search(const Bins &B, int nbins, int w_min, int w_max, float sigma,
                                           float &score, int &best_s, int &best_w)
{
    constexpr int R = 8;
    float Stot = 0.f, Ntot = 0.f;
    for (int b = 0; b < nbins; ++b) {
        Stot += B.s(b);
        Ntot += B.c(b);
    }
    float bv = -INFINITY;
    int bkey = 0x7fffffff;
    auto eval = [&](float sin_, float nin, int key, bool ok) {
        const float nout = Ntot - nin;
        const float q = nin * nout;
        const float D = fmaf(Stot, nin, -(sin_ * Ntot));
        const float v = D * rsqrtf(q);
        const bool take = ok & (q >= 1.f) & ((v > bv) | ((v == bv) & (key < bkey)));
        bv = take ? v : bv;
        bkey = take ? key : bkey;
    };
    for (int s0 = 0; s0 < nbins; s0 += R) {
        const bool full = s0 + R <= nbins;
        float bS[R], bN[R];
        int cr[R];  // key = (w << 12) | s = ((t + 1) << 12) + cr[r]
#pragma unroll
        for (int r = 0; r < R; ++r) cr[r] = s0 + r - (r << 12);
        float runS = 0.f, runN = 0.f;
        int j = s0;
        // head: t = 0..R-1; start r is entered at t = r
#pragma unroll
        for (int t = 0; t < R; ++t) {
            bS[t] = runS;
            bN[t] = runN;
            runS += B.s(j);
            runN += B.c(j);
            j = (j + 1 == nbins) ? 0 : j + 1;
            const int T = (t + 1) << 12;
#pragma unroll
            for (int r = 0; r <= t; ++r) {
                const int w = t - r + 1;
                eval(runS - bS[r], runN - bN[r], T + cr[r],
                     (w >= w_min) & (w <= w_max) & (s0 + r < nbins));
            }
        }
        const int tend = R - 1 + w_max;  // exclusive
        int ta = max(R, w_min + R - 2);
        int tb = max(ta, min(w_max, tend));
        if (!full) {
            ta = R;
            tb = R;
        }
        for (int t = R; t < min(ta, tend); ++t) {
            runS += B.s(j);
            runN += B.c(j);
            j = (j + 1 == nbins) ? 0 : j + 1;
            const int T = (t + 1) << 12;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int w = t - r + 1;
                eval(runS - bS[r], runN - bN[r], T + cr[r],
                     (w >= w_min) & (w <= w_max) & (s0 + r < nbins));
            }
        }
        for (int t = ta; t < tb; ++t) {  // every (r, w) valid here
            runS += B.s(j);
            runN += B.c(j);
            j = (j + 1 == nbins) ? 0 : j + 1;
            const int T = (t + 1) << 12;
#pragma unroll
            for (int r = 0; r < R; ++r) eval(runS - bS[r], runN - bN[r], T + cr[r], true);
        }
        for (int t = max(tb, R); t < tend; ++t) {
            runS += B.s(j);
            runN += B.c(j);
            j = (j + 1 == nbins) ? 0 : j + 1;
            const int T = (t + 1) << 12;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int w = t - r + 1;
                eval(runS - bS[r], runN - bN[r], T + cr[r],
                     (w >= w_min) & (w <= w_max) & (s0 + r < nbins));
            }
        }
    }
    if (bkey == 0x7fffffff) {
        score = -INFINITY;
        best_s = -1;
        best_w = -1;
        return;
    }
    const int bw = bkey >> 12, bs = bkey & 4095;
    // FP64 re-evaluation: snr = (S n_in - S_in N) / (sigma sqrt(N n_in n_out))
    double St = 0.0, Nt = 0.0, Si = 0.0, Ni = 0.0;
    for (int b = 0; b < nbins; ++b) {
        St += (double)B.s(b);
        Nt += (double)B.c(b);
    }
    int j = bs;
    for (int w = 0; w < bw; ++w) {
        Si += (double)B.s(j);
        Ni += (double)B.c(j);
        j = (j + 1 == nbins) ? 0 : j + 1;
    }
    const double No = Nt - Ni;
    score = (float)((St * Ni - Si * Nt) / ((double)sigma * sqrt(Nt * Ni * No)));
    best_s = bs;
    best_w = bw;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

template <int MODE, bool POW2>
__global__ void __launch_bounds__(kMaxFoldWarps * 32, 1) fold_kernel(const FoldParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_abort;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nbins = p.nbins;
    const int ppc = 32 * p.warps;

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint32_t *tl_buf = reinterpret_cast<uint32_t *>(smem + 128);
    uint32_t *th_buf = tl_buf + 2 * kTile;
    float *x_buf = reinterpret_cast<float *>(th_buf + 2 * kTile);
    float *acc = x_buf + 2 * kTile;
    const int nb2 = (nbins + 1) & ~1;
    uint16_t *cnt = reinterpret_cast<uint16_t *>(acc + (size_t)p.warps * nbins * 32);
    float *accw = acc + (size_t)warp * nbins * 32 + lane;
    uint16_t *cntw = cnt + (size_t)warp * nb2 * 32 + 2 * lane;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t parity_bits = 0u;  // bit b: phase parity of buffer b
    float2 *wsc_cta = p.ws_sc + (size_t)blockIdx.x * nbins * ppc + warp * 32 + lane;
    uint32_t *wcn_cta = p.ws_cnt + (size_t)blockIdx.x * nbins * ppc + warp * 32 + lane;

    for (int64_t task = blockIdx.x; task < p.ntasks; task += gridDim.x) {
        // resolve the star of this task and its period block
        int s = 0;
        int64_t tbase = 0;
        if (p.task_off) {
            int lo = 0, hi = p.nstars - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.task_off[mid] <= task) lo = mid;
                else hi = mid - 1;
            }
            s = lo;
            tbase = p.task_off[s];
        }
        int64_t lb, le, gb, ge;
        star_range(p.lc_off, p.n, s, lb, le);
        star_range(p.grid_off, p.np, s, gb, ge);
        const int64_t nsamp = le - lb;
        const int64_t sbase = scratch_start(lb, s);
        const int64_t k = gb + (task - tbase) * ppc + warp * 32 + lane;
        const bool kvalid = k < ge;

        uint32_t Fl = 0u, Fh = 0u;
        if (kvalid) {
            const double P = p.periods[k];
            const double q = kTwo40 / P;
            if (P > 0.0 && P < INFINITY && q < kTwo63) {
                const unsigned long long F = (unsigned long long)__double2ll_rn(q);
                Fl = (uint32_t)F;
                Fh = (uint32_t)(F >> 32);
            } else {
                report_error(p.status, kErrRange);
            }
        }
        for (int b = 0; b < nbins; ++b) {
            accw[b << 5] = 0.f;
            cntw[cidx(b)] = 0;
        }
        const int ntiles = (int)((nsamp + kTile - 1) / kTile);
        auto issue = [&](int t, int buf) {
            const int64_t i0 = (int64_t)t * kTile;
            const int nv = (int)min((int64_t)kTile, nsamp - i0);
            const uint32_t bytes = (uint32_t)(((nv + 3) & ~3) * 4);
            mbar_arrive_expect_tx(&bars[buf], 3u * bytes);
            bulk_g2s(tl_buf + buf * kTile, p.smp.tau_lo + sbase + i0, bytes, &bars[buf]);
            bulk_g2s(th_buf + buf * kTile, p.smp.tau_hi + sbase + i0, bytes, &bars[buf]);
            bulk_g2s(x_buf + buf * kTile, p.smp.x + sbase + i0, bytes, &bars[buf]);
        };
        __syncthreads();  // previous task's readers are done with both buffers
        if (threadIdx.x == 0) {
            issue(0, 0);
            if (ntiles > 1) issue(1, 1);
        }
        bool over = false;
        bool first_flush = true;
        int chunk_left = p.chunk;
        for (int t = 0; t < ntiles; ++t) {
            const int buf = t & 1;
            const bool ok = mbar_wait_bounded(&bars[buf], (parity_bits >> buf) & 1u);
            parity_bits ^= 1u << buf;
            if (!ok) {
                s_abort = 1;
                report_error(p.status, kErrTimeout);
            } else {
                const int nv = (int)min((int64_t)kTile, nsamp - (int64_t)t * kTile);
                const uint32_t *stl = tl_buf + buf * kTile;
                const uint32_t *sth = th_buf + buf * kTile;
                const float *sx = x_buf + buf * kTile;
                int i = 0;
                while (i < nv) {
                    // segments end at chunk boundaries (multiples of 4 samples) or the tile end
                    const int seg = min(nv - i, chunk_left);
                    fold_tile<POW2>(stl + i, sth + i, sx + i, seg, accw, cntw, Fl, Fh, (uint32_t)nbins,
                                    p.shift);
                    i += seg;
                    chunk_left -= seg;
                    const bool last = (t == ntiles - 1) && (i == nv);
                    if (chunk_left == 0 || last) {
                        over = flush_chunk(accw, cntw, wsc_cta, wcn_cta, nbins, ppc, first_flush, last);
                        first_flush = false;
                        chunk_left = p.chunk;
                    }
                }
            }
            __syncthreads();
            if (s_abort) return;
            if (threadIdx.x == 0 && t + 2 < ntiles) issue(t + 2, buf);
        }

        // ---------------- epilogues (lane-private, no block barrier needed)
        if (MODE == kModeFold) {
            if (kvalid) {
                const float fh = p.stats[s].f_hi, fl = p.stats[s].f_lo;
                for (int b = 0; b < nbins; ++b) {
                    const uint32_t c = over ? wcn_cta[(size_t)b * ppc] : (uint32_t)cntw[cidx(b)];
                    const float S = accw[b << 5];
                    const float mean = c ? fh + (fl + S / (float)c) : __int_as_float(0x7fc00000);
                    if (p.folded) p.folded[(size_t)k * nbins + b] = mean;
                    if (p.counts) p.counts[(size_t)k * nbins + b] = (int32_t)c;
                }
            }
        } else if (MODE == kModeBox) {
            float sc = -INFINITY;
            int bs = -1, bw = -1;
            if (kvalid) {
                float sig = p.sigma_user;
                if (!(sig > 0.f)) sig = p.stats[s].sigma;
                if (!(sig > 0.f)) sig = 1.f;
                const LaneBins B{accw, cntw, wcn_cta, (size_t)ppc, over};
                box_search(B, nbins, p.w_min, p.w_max, sig, sc, bs, bw);
                p.score[k] = sc;
                if (p.best_s) p.best_s[k] = bs;
                if (p.best_w) p.best_w[k] = bw;
            }
            if (p.best_key) {
                unsigned long long key = kvalid ? argmax_key(sc, k - gb) : 0ull;
                key = warp_max_u64(key);
                if (lane == 0 && key) atomicMax(&p.best_key[s], key);
            }
        }
    }
}

template <int MODE, bool POW2>
static cudaError_t set_smem_attr()
{
    return cudaFuncSetAttribute(fold_kernel<MODE, POW2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kSmemLimit - 1024));
}

int fold_register_kernels()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_smem_attr<kModeFold, true>();
    if (e == cudaSuccess) e = set_smem_attr<kModeFold, false>();
    if (e == cudaSuccess) e = set_smem_attr<kModeBox, true>();
    if (e == cudaSuccess) e = set_smem_attr<kModeBox, false>();
    return (int)e;
}

size_t fold_smem_bytes(int nbins, int warps)
{
    const size_t nb2 = (size_t)((nbins + 1) & ~1);
    return 128 + (size_t)2 * kTile * 12 + (size_t)warps * 32 * (nbins * 4 + nb2 * 2);
}

int fold_max_warps(int nbins)
{
    int w = kMaxFoldWarps;
    while (w > 1 && fold_smem_bytes(nbins, w) > kSmemLimit - 1024) --w;
    return fold_smem_bytes(nbins, w) <= kSmemLimit - 1024 ? w : 0;
}

cudaError_t launch_fold(const FoldParams &p, int mode, int grid, cudaStream_t st)
{
    const size_t smem = fold_smem_bytes(p.nbins, p.warps);
    const int threads = 32 * p.warps;
    const bool pow2 = p.shift >= 0;
    if (mode == kModeFold) {
        if (pow2) fold_kernel<kModeFold, true><<<grid, threads, smem, st>>>(p);
        else fold_kernel<kModeFold, false><<<grid, threads, smem, st>>>(p);
    } else if (mode == kModeBox) {
        if (pow2) fold_kernel<kModeBox, true><<<grid, threads, smem, st>>>(p);
        else fold_kernel<kModeBox, false><<<grid, threads, smem, st>>>(p);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ standalone box-SNR

// Each warp scores 32 profiles, one per lane. The profiles are staged transposed into
// shared memory ([bin][33] so both the coalesced staging writes and the lane-per-
// profile reads are conflict-free), as centred sums (mean - m_ref) * count in FP32 with
// m_ref the count-weighted mean of the profile (FP64), plus 16-bit counts.
constexpr int kBoxWarps = 4;

__global__ void __launch_bounds__(kBoxWarps * 32) box_kernel(const float *__restrict__ folded,
                                                             const int32_t *__restrict__ counts,
                                                             int64_t np, int nbins, int w_min,
                                                             int w_max, float sigma, float *score,
                                                             int32_t *best_s, int32_t *best_w)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    float *Sw = reinterpret_cast<float *>(smem) + (size_t)warp * nbins * 33;
    uint16_t *Cw = reinterpret_cast<uint16_t *>(reinterpret_cast<float *>(smem) +
                                                 (size_t)nwarps * nbins * 33) +
                   (size_t)warp * nbins * 33;
    const int64_t nblocks = (np + 31) / 32;
    for (int64_t blk = (int64_t)blockIdx.x * nwarps + warp; blk < nblocks;
         blk += (int64_t)gridDim.x * nwarps) {
        const int64_t k0 = blk * 32;
        const int nk = (int)min((int64_t)32, np - k0);
        bool big_lane = false;
        // stage: for each profile j, lanes walk its bins (coalesced row reads)
        for (int j = 0; j < 32; ++j) {
            double num = 0.0, den = 0.0;
            if (j < nk) {
                const float *row = folded + (size_t)(k0 + j) * nbins;
                const int32_t *crow = counts + (size_t)(k0 + j) * nbins;
                for (int b = lane; b < nbins; b += 32) {
                    const int32_t c = crow[b];
                    if (c > 0) {
                        num += (double)row[b] * (double)c;
                        den += (double)c;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                num += __shfl_xor_sync(0xffffffffu, num, o);
                den += __shfl_xor_sync(0xffffffffu, den, o);
            }
            const float mref = den > 0.0 ? (float)(num / den) : 0.f;
            bool big = false;
            for (int b = lane; b < nbins; b += 32) {
                float sv = 0.f;
                uint32_t c = 0;
                if (j < nk) {
                    const int32_t ci = counts[(size_t)(k0 + j) * nbins + b];
                    c = ci > 0 ? (uint32_t)ci : 0u;
                    if (c) sv = (folded[(size_t)(k0 + j) * nbins + b] - mref) * (float)c;
                }
                big |= c > 65535u;
                Sw[b * 33 + j] = sv;
                Cw[b * 33 + j] = (uint16_t)min(c, 65535u);
            }
            if (__any_sync(0xffffffffu, big) && lane == j) big_lane = true;
        }
        __syncwarp();
        if (lane < nk) {
            const int64_t k = k0 + lane;
            float sc;
            int bs, bw;
            const StagedBins B{Sw + lane, Cw + lane, counts + (size_t)k * nbins, big_lane};
            box_search(B, nbins, w_min, w_max, sigma, sc, bs, bw);
            score[k] = sc;
            if (best_s) best_s[k] = bs;
            if (best_w) best_w[k] = bw;
        }
        __syncwarp();
    }
}

cudaError_t launch_box_standalone(const float *folded, const int32_t *counts, int64_t np, int nbins,
                                  int w_min, int w_max, float sigma, float *score, int32_t *best_s,
                                  int32_t *best_w, cudaStream_t st)
{
    static bool attr = false;
    int warps = kBoxWarps;
    while (warps > 1 && (size_t)warps * nbins * 33 * 6 > kSmemLimit - 1024) --warps;
    const size_t smem = (size_t)warps * nbins * 33 * 6;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(box_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kSmemLimit - 1024));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (smem > kSmemLimit - 1024) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nblocks = (np + 31) / 32;
    const int64_t want = (nblocks + warps - 1) / warps;
    const int grid = (int)(want < (int64_t)sms * 2 ? want : (int64_t)sms * 2);
    box_kernel<<<grid, warps * 32, smem, st>>>(folded, counts, np, nbins, w_min, w_max, sigma,
                                                   score, best_s, best_w);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ best period

__global__ void argmax_kernel(const float *__restrict__ score, int64_t np, unsigned long long *key)
{
    unsigned long long best = 0ull;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np;
         k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long v = argmax_key(score[k], k);
        best = v > best ? v : best;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

__global__ void argmax_finalize_kernel(const unsigned long long *key, int nstars, int64_t *best_index,
                                       float *best_score)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nstars) return;
    const unsigned long long k = key[s];
    const uint32_t ord = (uint32_t)(k >> 32);
    if (ord == 0u) {
        if (best_index) best_index[s] = -1;
        if (best_score) best_score[s] = __int_as_float(0x7fc00000);
        return;
    }
    const uint32_t u = (ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord;
    if (best_index) best_index[s] = (int64_t)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull));
    if (best_score) best_score[s] = __uint_as_float(u);
}

cudaError_t launch_argmax(const float *score, int64_t np, unsigned long long *key, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (np + 255) / 256;
    int64_t g = want < (int64_t)sms * 4 ? want : (int64_t)sms * 4;
    const int grid = (int)(g < 1 ? 1 : g);
    argmax_kernel<<<grid, 256, 0, st>>>(score, np, key);
    return cudaGetLastError();
}

cudaError_t launch_argmax_finalize(const unsigned long long *key, int nstars, int64_t *best_index,
                                   float *best_score, cudaStream_t st)
{
    argmax_finalize_kernel<<<(nstars + 127) / 128, 128, 0, st>>>(key, nstars, best_index, best_score);
    return cudaGetLastError();
}

}  // namespace gpfc
