// fold.cu -- phase fold, box-SNR and best-period kernels for sm_103a.
//
// Fold (paper Sec. 2.3, Fig. 4 steps a-e, with equal-width bins):
//   tau_i = rint((t_i - t0) 2^24), F_k = rint(2^40 / P_k), phase = (tau F mod 2^64) / 2^64,
//   bin = floor(phase * nbins), then per-bin count and flux sum, mean = sum / count.
//
// Design. One lane owns one trial period for the whole light curve; the bins of a warp's
// (or period group's) 32 periods sit in shared memory laid out [bin][lane], so the 32
// updates of one instruction never conflict whatever bins the lanes hit. Light-curve tiles
// (tau split in two 32-bit words, the flux, one regular-cadence flag byte per 16 samples)
// are staged into shared memory by the bulk-copy (TMA) engine, double-buffered behind an
// mbarrier, and every lane reads the same sample (a broadcast). Three bin layouts:
//
// * kLayoutRed32 (the default from 256 bins): per bin a row of the 32 lanes' 32-bit
//   fixed-point sums and a row of their 32-bit counts; an update is two no-return
//   red.shared.add.u32. The flux is pre-quantised per star (x_q = rint(x 2^e), e from the
//   largest |x| and the chunk length, so a chunk's bin sum fits in 32 bits), the sums are
//   exact and independent of the order of the additions, and so several warps (sample
//   streams) fold disjoint 16-sample groups of every tile into the same bins: three 64 KB
//   period groups per block at 256 bins and twelve warps, each warp one of twelve streams
//   that adds its samples into all three groups (lane l: period l of each), so a sample is
//   read from the tile once per block. (Blocks of more than three period groups give each
//   group its own streams.) Flushes and epilogues split each group's bins over its warps.
//   Chunk sums go exactly into an int64 workspace; each bin is rounded once to FP32.
// * kLayoutPacked64: FP32 partial sum and 32-bit count in one 8-byte word, a 64-bit load
//   and store per update; one warp per 32 periods.
// * kLayoutPaired16: FP32 sums with paired 16-bit counts (6 bytes a bin), the default below
//   256 bins.
// The FP32 layouts apply a group of 16 (or 8) regular samples that can never put two
// samples into one bin at the warp's periods through a software-pipelined loop without
// collision checks, other groups through a checked path; their partial sums cover a chunk
// of 128 * nbins samples and are then added into the workspace with Kahan compensation
// (sum, compensation) and exact 32-bit counts. The workspace stays resident in L2.
//
// Epilogues (kernel modes): write means and counts (gpfc_fold) or centred sums and counts
// (the separate box scorer); run the box-SNR search over each lane's finished profile
// (kModeBox, below 256 bins); or kModeSearch, where each block has one more warp that
// scores the block's previous task from a two-slot ring in L2 (the one-kernel search).
// box_coop_kernel scores profiles one warp per profile (the separate scorer, and
// gpfc_score_box).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <type_traits>

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

// First element of star s in the sample scratch: a multiple of 256 (so its per-16-sample
// flags start on a 16-byte boundary), with room for the star's samples rounded up to a
// multiple of 256.
__device__ __forceinline__ int64_t scratch_start(int64_t lc_begin, int s)
{
    return 256 * ((lc_begin + 255) / 256 + s);
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
__device__ __forceinline__ long long quantise_time(double t, double t0, bool &bad)
{
    const double v = (t - t0) * kTwo24;
    if (fabs(v) < kTwo62) return __double2ll_rn(v);
    bad = true;
    return 0;
}

__global__ void prep_quant_kernel(const double *times, const float *flux, const int64_t *lc_off,
                                  int64_t n, const double *t0s, double t0_scalar, double *partial,
                                  long long *pmin, SampleScratch smp, StarStats *stats, uint32_t *status)
{
    __shared__ double red[32];
    __shared__ long long redm[32];
    __shared__ float redx[32];
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
    if (t0 != t0) t0 = len > 0 ? times[b] : 0.0;
    const int64_t base = scratch_start(b, s);
    const int64_t per = (len + G - 1) / G;
    const int64_t j0 = (int64_t)blockIdx.x * per;
    const int64_t j1 = min(len, j0 + per);
    double acc = 0.0;
    float amax = 0.f;  // largest |x| of this block's samples
    bool bad = false;
    long long dmin = LLONG_MAX;  // smallest positive step tau_j - tau_{j-1}
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const long long tau = quantise_time(times[b + j], t0, bad);
        if (j > 0) {
            const long long d = tau - quantise_time(times[b + j - 1], t0, bad);
            if (d > 0 && d < dmin) dmin = d;
        }
        smp.tau_lo[base + j] = (uint32_t)(unsigned long long)tau;
        smp.tau_hi[base + j] = (int32_t)(tau >> 32);
        const double d = (double)flux[b + j] - f_ref;
        smp.x[base + j] = (float)d;
        amax = fmaxf(amax, fabsf((float)d));
        acc += d * d;
    }
    if (bad) report_error(status, kErrRange);
    // zero the padding after the star (up to the next multiple of 256) so tile copies read
    // defined data
    if (blockIdx.x == 0) {
        for (int64_t j = len + threadIdx.x; j < ((len + 255) & ~(int64_t)255); j += blockDim.x) {
            smp.tau_lo[base + j] = 0u;
            smp.tau_hi[base + j] = 0;
            smp.x[base + j] = 0.f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long u = __shfl_down_sync(0xffffffffu, dmin, o);
        dmin = u < dmin ? u : dmin;
    }
    if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = dmin;
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) redx[threadIdx.x >> 5] = amax;
    double t = block_sum_f64(acc, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        partial[(size_t)gridDim.y * G + (size_t)s * G + blockIdx.x] = t;
        long long m = LLONG_MAX;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = redm[w] < m ? redm[w] : m;
        pmin[(size_t)s * G + blockIdx.x] = m;
        float xm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) xm = fmaxf(xm, redx[w]);
        partial[(size_t)3 * gridDim.y * G + (size_t)s * G + blockIdx.x] = (double)xm;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[s].f_ref = f_ref;
        const float hi = (float)f_ref;
        stats[s].f_hi = hi;
        stats[s].f_lo = (float)(f_ref - (double)hi);
        stats[s].n = (int32_t)len;
    }
}

// Exponent of the fixed-point flux: the largest e (|e| <= 200) with xmax 2^e <= lim, so that
// every |rint(x 2^e)| <= lim. 0 for xmax = 0.
__device__ __forceinline__ int fixed_point_exp(double xmax, double lim)
{
    if (!(xmax > 0.0) || !(xmax < INFINITY)) return 0;
    int e = ilogb(lim) - ilogb(xmax);
    e = max(-200, min(200, e));
    while (e < 200 && ldexp(xmax, e + 1) <= lim) ++e;
    while (e > -200 && ldexp(xmax, e) > lim) --e;
    return e;
}

// Pass 3: sigma = sqrt(sum (flux - f_ref)^2 / n), the smallest positive time step and the
// fixed-point exponent per star: a chunk of min(chunk, n) samples then sums to at most
// 2^31 - 1 in magnitude in any bin. grid = stars, 32 threads.
__global__ void prep_sigma_kernel(const double *partial, const long long *pmin, int G, int nstars, int chunk,
                                  StarStats *stats)
{
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    double t = 0.0, xm = 0.0;
    long long m = LLONG_MAX;
    for (int g = 0; g < G; ++g) {
        t += partial[(size_t)nstars * G + (size_t)s * G + g];
        xm = fmax(xm, partial[(size_t)3 * nstars * G + (size_t)s * G + g]);
        const long long v = pmin[(size_t)s * G + g];
        m = v < m ? v : m;
    }
    stats[s].sigma = (float)sqrt(t / (double)stats[s].n);
    stats[s].dtau0 = m == LLONG_MAX ? 0 : m;
    // a chunk holds at most min(chunk, n) samples of the star
    const int lmax = min(chunk, max(1, stats[s].n));
    stats[s].qexp = fixed_point_exp(xm, floor(2147483647.0 / (double)lmax));
    stats[s].pad = 0;
}

constexpr int32_t kThMixed = INT32_MIN;  // per-group high word marker: the samples differ

// Pass 4: one flag byte per group of 16 samples: 1 if every step inside the group lies in
// [dtau0, dtau0 + 2] (a regular cadence up to the 2^-24 d rounding of tau) and the high
// word of tau is the same for all 16 (it changes every 2^32 units, ~256 d). The fold
// skips its per-group bin-collision check on flagged groups when the period allows it,
// and forms their phases with one th * F_lo product per group. The same pass writes the
// fixed-point flux xq = rint(x 2^qexp) when the scratch has room for it.
// grid = (G, stars).
__global__ void prep_flags_kernel(const int64_t *lc_off, int64_t n, SampleScratch smp,
                                  const StarStats *stats)
{
    const int s = blockIdx.y;
    int64_t b, e;
    star_range(lc_off, n, s, b, e);
    const int64_t len = e - b;
    const int64_t base = scratch_start(b, s);
    const long long d0 = stats[s].dtau0;
    const int64_t ngroups = (len + 255) / 256 * 16;  // every flag byte of the star's region
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ngroups;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = q * 16;
        bool reg = d0 > 0 && j0 + 16 <= len;
        if (reg) {
            const int32_t th0 = smp.tau_hi[base + j0];
            long long prev = ((long long)th0 << 32) | smp.tau_lo[base + j0];
            for (int k = 1; k < 16; ++k) {
                const int32_t th = smp.tau_hi[base + j0 + k];
                const long long cur = ((long long)th << 32) | smp.tau_lo[base + j0 + k];
                const long long d = cur - prev;
                reg &= (d >= d0) & (d <= d0 + 2) & (th == th0);
                prev = cur;
            }
        }
        smp.flags[base / 16 + q] = reg ? 1 : 0;
        if (smp.thg) {
            // the group's common tau high word, or kThMixed if its samples differ in it (a
            // valid high word is below 2^30 in magnitude: |tau| < 2^62)
            int32_t th0 = 0;
            bool same = true;
            for (int k = 0; k < 16 && j0 + k < len; ++k) {
                const int32_t th = smp.tau_hi[base + j0 + k];
                if (k == 0) th0 = th;
                same &= th == th0;
            }
            smp.thg[base / 16 + q] = same ? th0 : kThMixed;
        }
        if (smp.xq) {
            // fixed-point flux (exact: scaling by a power of two, then rounding to nearest
            // even); zero past the star's end
            const double sc = ldexp(1.0, stats[s].qexp);
            for (int k = 0; k < 16; ++k)
                smp.xq[base + j0 + k] = j0 + k < len ? __double2int_rn((double)smp.x[base + j0 + k] * sc) : 0;
        }
    }
}

cudaError_t launch_prep(const double *times, const float *flux, const int64_t *lc_off, int64_t n,
                        int nstars, int64_t max_len, const double *t0s, double t0, SampleScratch smp,
                        double *partial, int G, StarStats *stats, uint32_t *status, cudaStream_t st,
                        int chunk)
{
    (void)max_len;
    dim3 grid(G, nstars);
    long long *pmin = reinterpret_cast<long long *>(partial + (size_t)2 * nstars * G);
    prep_sum_kernel<<<grid, 256, 0, st>>>(flux, lc_off, n, partial);
    prep_quant_kernel<<<grid, 256, 0, st>>>(times, flux, lc_off, n, t0s, t0, partial, pmin, smp, stats,
                                            status);
    prep_sigma_kernel<<<nstars, 32, 0, st>>>(partial, pmin, G, nstars, chunk < 16 ? 16 : chunk, stats);
    prep_flags_kernel<<<grid, 256, 0, st>>>(lc_off, n, smp, stats);
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

// Lane-private bin stores. Element (b, lane) sits at index b * 32 + lane, so the 32
// lanes of a warp touch 32 distinct banks whatever bins they hit.
__device__ __forceinline__ uint32_t cidx(uint32_t b) { return ((b >> 1) << 6) | (b & 1u); }

// FP32 partial sums plus 16-bit counts (6 bytes per bin): counts are paired per lane,
// word (b / 2) * 32 + lane holds bins 2j and 2j+1, which keeps count accesses
// conflict-free too. Counts of one chunk stay below 65536.
struct StorePaired16 {
    uint32_t acc;  // shared address of this lane's bin-0 sum
    uint32_t cnt;  // shared address of this lane's bin-0/1 count word
    static constexpr bool kSaturates = true;
    __device__ __forceinline__ static uint32_t soff(uint32_t b) { return b << 7; }
    __device__ __forceinline__ static uint32_t coff(uint32_t b) { return ((b >> 1) << 7) | ((b & 1u) << 1); }
    __device__ __forceinline__ void load(uint32_t b, float &s, uint32_t &c) const
    {
        s = lds_f32(acc + soff(b));
        c = lds_u16(cnt + coff(b));
    }
    __device__ __forceinline__ void put(uint32_t b, float s, uint32_t c) const
    {
        sts_f32(acc + soff(b), s);
        sts_u16(cnt + coff(b), c);
    }
    __device__ __forceinline__ float sum(uint32_t b) const { return lds_f32(acc + soff(b)); }
    __device__ __forceinline__ uint32_t count(uint32_t b) const { return lds_u16(cnt + coff(b)); }
};

// FP32 sum and 32-bit count packed in one 64-bit word (8 bytes per bin): one shared
// load and one store per update.
struct StorePacked64 {
    uint32_t v;  // shared address of this lane's bin-0 word
    static constexpr bool kSaturates = false;
    __device__ __forceinline__ void load(uint32_t b, float &s, uint32_t &c) const
    {
        const uint2 t = lds_u32x2(v + (b << 8));
        s = __uint_as_float(t.x);
        c = t.y;
    }
    __device__ __forceinline__ void put(uint32_t b, float s, uint32_t c) const
    {
        sts_u32x2(v + (b << 8), make_uint2(__float_as_uint(s), c));
    }
    __device__ __forceinline__ float sum(uint32_t b) const { return __uint_as_float(lds_u32x2(v + (b << 8)).x); }
    __device__ __forceinline__ uint32_t count(uint32_t b) const { return lds_u32x2(v + (b << 8)).y; }
};

// Words accumulated by no-return shared reductions: 256 bytes per bin of a warp, the 32
// lanes' sum words then their 32-bit count words ([bin][sum row, count row][lane]), so both
// rows are free of bank conflicts and the count sits at a fixed offset (128) from the sum.
// During the fold the sum word holds the fixed-point sum (two's complement, mod 2^32); one
// update is two red.shared.add.u32 with no result to wait for. Reductions of one thread to
// one address take effect in program order, so no check for two samples in one bin is
// needed, and integer sums do not depend on the order anyway. After the last chunk's flush
// the sum word holds the FP32 sum and the count word the exact count.
struct StoreRed32 {
    uint32_t v;  // shared address of this lane's bin-0 sum word
    static constexpr bool kSaturates = false;
    __device__ __forceinline__ void add(uint32_t b, int32_t xq) const
    {
        const uint32_t a = v + (b << 8);
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"((uint32_t)xq) : "memory");
        asm volatile("red.shared.add.u32 [%0+128], %1;" ::"r"(a), "r"(1u) : "memory");
    }
    __device__ __forceinline__ void load(uint32_t b, float &s, uint32_t &c) const
    {
        s = lds_f32(v + (b << 8));
        c = lds_u32(v + (b << 8) + 128u);
    }
    __device__ __forceinline__ void put(uint32_t b, float s, uint32_t c) const
    {
        sts_f32(v + (b << 8), s);
        sts_u32(v + (b << 8) + 128u, c);
    }
    __device__ __forceinline__ float sum(uint32_t b) const { return lds_f32(v + (b << 8)); }
    __device__ __forceinline__ uint32_t count(uint32_t b) const { return lds_u32(v + (b << 8) + 128u); }
    __device__ __forceinline__ int32_t isum(uint32_t b) const { return (int32_t)lds_u32(v + (b << 8)); }
};

// Tile data of U consecutive samples, held in registers.
template <int U>
struct TileRegs {
    uint4 a[U / 4];   // tau low words
    uint4 h[U / 4];   // tau high words
    float4 f[U / 4];  // flux - f_ref
};

// Tile data (shared addresses of the tau-low, tau-high and flux words of sample 0).
template <int U>
__device__ __forceinline__ void load_tile_regs(uint32_t stl, uint32_t sth, uint32_t sx, int i, TileRegs<U> &T)
{
#pragma unroll
    for (int q = 0; q < U / 4; ++q) {
        const uint32_t o = 4u * (uint32_t)(i + 4 * q);
        T.a[q] = lds_u32x4(stl + o);
        T.h[q] = lds_u32x4(sth + o);
        T.f[q] = lds_f32x4(sx + o);
    }
}

// Tile data of U consecutive samples of a regular group. The prep pass flags a group
// regular only if the high word of tau is the same for all its samples, so only the
// first one is read, and th * F_lo is formed once per group.
template <int U>
struct TileRegsR {
    uint4 a[U / 4];   // tau low words
    float4 f[U / 4];  // flux - f_ref
    uint32_t th;      // tau high word of the group
};

template <int U>
__device__ __forceinline__ void load_tile_regs_r(uint32_t stl, uint32_t sth, uint32_t sx, int i, TileRegsR<U> &T)
{
#pragma unroll
    for (int q = 0; q < U / 4; ++q) {
        const uint32_t o = 4u * (uint32_t)(i + 4 * q);
        T.a[q] = lds_u32x4(stl + o);
        T.f[q] = lds_f32x4(sx + o);
    }
    T.th = lds_u32(sth + 4u * (uint32_t)i);
}

// phase_bin with the th * F_lo term of the phase's high word given
template <bool POW2>
__device__ __forceinline__ uint32_t phase_bin_th(uint32_t tl, uint32_t thF, uint32_t Fl, uint32_t Fh,
                                                 uint32_t nbins, int shift)
{
    const uint32_t hi = __umulhi(tl, Fl) + thF + tl * Fh;
    if (POW2) return hi >> shift;
    const uint32_t lo = tl * Fl;
    const unsigned long long t =
        (unsigned long long)hi * nbins + (unsigned long long)__umulhi(lo, nbins);
    return (uint32_t)(t >> 32);
}

template <bool POW2, int U>
__device__ __forceinline__ void bins_from_regs_r(const TileRegsR<U> &T, uint32_t Fl, uint32_t Fh, uint32_t nbins,
                                                 int shift, uint32_t (&b)[U], float (&x)[U])
{
    const uint32_t thF = T.th * Fl;
#pragma unroll
    for (int q = 0; q < U / 4; ++q) {
        b[4 * q + 0] = phase_bin_th<POW2>(T.a[q].x, thF, Fl, Fh, nbins, shift);
        b[4 * q + 1] = phase_bin_th<POW2>(T.a[q].y, thF, Fl, Fh, nbins, shift);
        b[4 * q + 2] = phase_bin_th<POW2>(T.a[q].z, thF, Fl, Fh, nbins, shift);
        b[4 * q + 3] = phase_bin_th<POW2>(T.a[q].w, thF, Fl, Fh, nbins, shift);
        x[4 * q + 0] = T.f[q].x;
        x[4 * q + 1] = T.f[q].y;
        x[4 * q + 2] = T.f[q].z;
        x[4 * q + 3] = T.f[q].w;
    }
}

template <bool POW2, int U>
__device__ __forceinline__ void bins_from_regs(const TileRegs<U> &T, uint32_t Fl, uint32_t Fh, uint32_t nbins,
                                               int shift, uint32_t (&b)[U], float (&x)[U])
{
#pragma unroll
    for (int q = 0; q < U / 4; ++q) {
        b[4 * q + 0] = phase_bin<POW2>(T.a[q].x, T.h[q].x, Fl, Fh, nbins, shift);
        b[4 * q + 1] = phase_bin<POW2>(T.a[q].y, T.h[q].y, Fl, Fh, nbins, shift);
        b[4 * q + 2] = phase_bin<POW2>(T.a[q].z, T.h[q].z, Fl, Fh, nbins, shift);
        b[4 * q + 3] = phase_bin<POW2>(T.a[q].w, T.h[q].w, Fl, Fh, nbins, shift);
        x[4 * q + 0] = T.f[q].x;
        x[4 * q + 1] = T.f[q].y;
        x[4 * q + 2] = T.f[q].z;
        x[4 * q + 3] = T.f[q].w;
    }
}

template <int U>
__device__ __forceinline__ bool hazard_u(const uint32_t (&b)[U])
{
    bool h = false;
#pragma unroll
    for (int u = 1; u < U; ++u)
#pragma unroll
        for (int v = 0; v < u; ++v) h |= (b[u] == b[v]);
    return h;
}

// Fold nvalid samples of a staged tile into this lane's bins, U samples per group, as a
// three-stage software pipeline: while the bin reads of group g are in flight, the tile
// data of group g+2 is fetched and the bins of group g+1 are computed from registers;
// then group g is written back. A group in which two samples share a bin is applied
// one sample at a time.
template <bool POW2, class St, int U>
__device__ __forceinline__ void fold_tile(uint32_t stl, uint32_t sth, uint32_t sx, int nvalid, const St &st,
                                          uint32_t Fl, uint32_t Fh, uint32_t nbins, int shift)
{
    const int ng = nvalid / U;
    if (ng > 0) {
        uint32_t b[U];
        float x[U];
        TileRegs<U> T1;
        load_tile_regs<U>(stl, sth, sx, 0, T1);
        bins_from_regs<POW2, U>(T1, Fl, Fh, nbins, shift, b, x);
        bool haz = hazard_u<U>(b);
        load_tile_regs<U>(stl, sth, sx, ng > 1 ? U : 0, T1);
#pragma unroll 1
        for (int g = 0; g < ng; ++g) {
            float s[U];
            uint32_t c[U];
            if (!haz) {
#pragma unroll
                for (int u = 0; u < U; ++u) st.load(b[u], s[u], c[u]);
            }
            TileRegs<U> T2;
            load_tile_regs<U>(stl, sth, sx, U * min(g + 2, ng - 1), T2);
            uint32_t nb[U];
            float nx[U];
            bins_from_regs<POW2, U>(T1, Fl, Fh, nbins, shift, nb, nx);
            const bool nhaz = hazard_u<U>(nb);
            if (!haz) {
#pragma unroll
                for (int u = 0; u < U; ++u) st.put(b[u], s[u] + x[u], c[u] + 1u);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    float s1;
                    uint32_t c1;
                    st.load(b[u], s1, c1);
                    st.put(b[u], s1 + x[u], c1 + 1u);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                b[u] = nb[u];
                x[u] = nx[u];
            }
            haz = nhaz;
            T1 = T2;
        }
    }
    for (int i = U * ng; i < nvalid; ++i) {
        const uint32_t bb = phase_bin<POW2>(lds_u32(stl + 4u * i), lds_u32(sth + 4u * i), Fl, Fh, nbins, shift);
        const float xi = lds_f32(sx + 4u * i);
        float s1;
        uint32_t c1;
        st.load(bb, s1, c1);
        st.put(bb, s1 + xi, c1 + 1u);
    }
}

// Largest group of consecutive regular samples (16, 8, or 0 for none) that can never put
// two of its samples into one bin at this lane's frequency F: for every distance k up to
// the group size minus one, k regular steps (each in [d0, d0 + 2] tau units) move the
// phase by at least one bin, without wrapping round to the same bin.
__device__ __forceinline__ int regular_group_size(unsigned long long F, long long d0, uint32_t nbins)
{
    if (d0 <= 0 || F == 0ull || F > 0xFFFFFFFFFFFFFFFFull / 32ull) return 0;
    for (int k = 1; k < 16; ++k) {
        const unsigned long long ph = (unsigned long long)k * (unsigned long long)d0 * F;  // mod 2^64
        const unsigned long long dist = ph < (0ull - ph) ? ph : (0ull - ph);  // circular distance
        const unsigned long long jitter = (unsigned long long)(2 * k) * F;
        if (dist <= jitter || __umul64hi(dist - jitter, (unsigned long long)nbins) == 0ull)  // < 1 bin
            return k < 8 ? 0 : 8;
    }
    return 16;
}

// Fold a run of ng consecutive groups of U samples in which no two samples of a group
// share a bin (regular-cadence groups, U within the period's safe group size), as a
// three-stage software pipeline: while the bin reads of group g are in flight, the tile
// data of group g+2 is fetched and the bins of group g+1 are computed from registers;
// then group g is written back. Each group's U reads are all issued before its U writes.
// The loop body holds two stages with swapped register roles, so no register array is
// copied from one iteration to the next.
template <bool POW2, class St, int U>
__device__ __forceinline__ void fold_run_regular(uint32_t stl, uint32_t sth, uint32_t sx, int ng, const St &st,
                                                 uint32_t Fl, uint32_t Fh, uint32_t nbins, int shift)
{
    // One pipeline stage: issue the bin reads of the group whose bins are in (cb, cx), fetch
    // the tile data of group `fetch` into Tn, compute the next group's bins from Tc into
    // (nb, nx), then write the current group back. Two stages per iteration with the
    // register roles swapped, so nothing is copied between iterations.
    auto stage = [&](const uint32_t (&cb)[U], const float (&cx)[U], const TileRegsR<U> &Tc, TileRegsR<U> &Tn,
                     uint32_t (&nb)[U], float (&nx)[U], int fetch) {
        float sm[U];
        uint32_t c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) st.load(cb[u], sm[u], c[u]);
        load_tile_regs_r<U>(stl, sth, sx, U * fetch, Tn);
        bins_from_regs_r<POW2, U>(Tc, Fl, Fh, nbins, shift, nb, nx);
#pragma unroll
        for (int u = 0; u < U; ++u) st.put(cb[u], sm[u] + cx[u], c[u] + 1u);
    };
    uint32_t b0[U], b1[U];
    float x0[U], x1[U];
    TileRegsR<U> T0, T1;
    load_tile_regs_r<U>(stl, sth, sx, 0, T0);
    bins_from_regs_r<POW2, U>(T0, Fl, Fh, nbins, shift, b0, x0);  // group 0
    load_tile_regs_r<U>(stl, sth, sx, ng > 1 ? U : 0, T1);        // group 1
    int g = 0;
#pragma unroll 1
    for (; g + 1 < ng; g += 2) {
        stage(b0, x0, T1, T0, b1, x1, min(g + 2, ng - 1));  // write g; bins of g+1; fetch g+2
        stage(b1, x1, T0, T1, b0, x0, min(g + 3, ng - 1));  // write g+1; bins of g+2; fetch g+3
    }
    if (g < ng) stage(b0, x0, T1, T0, b1, x1, g);  // the last group (odd count)
}

// Fold nvalid samples (a segment starting on a 16-sample boundary of the tile) in groups
// of 16. Runs of groups flagged regular by the prep pass go through the pipelined run
// without collision checks when the warp's group size `wg` allows it: 16-sample groups
// (wg = 16, blocks with the 255-register budget) or 8-sample halves (wg = 8, or wg = 16
// where the register budget is 128). Other groups, and the tail, go through the checked
// path.
template <bool POW2, class St, bool WIDE16>
__device__ __forceinline__ void fold_segment(uint32_t stl, uint32_t sth, uint32_t sx, unsigned long long fmask,
                                             int nvalid, const St &st, uint32_t Fl, uint32_t Fh,
                                             uint32_t nbins, int shift, int wg)
{
    const int ng = nvalid >> 4;
    if (wg == 0) fmask = 0ull;
    if (ng < 64) fmask &= (1ull << ng) - 1ull;
    int g = 0;
#pragma unroll 1
    while (g < ng) {
        const unsigned long long rest = fmask >> g;
        if (rest & 1ull) {
            // length of the run of flagged groups starting at g
            const int run = (~rest == 0ull) ? 64 - g : __ffsll((long long)~rest) - 1;
            if (WIDE16 && wg == 16)
                fold_run_regular<POW2, St, 16>(stl + 64u * g, sth + 64u * g, sx + 64u * g, run, st, Fl, Fh, nbins,
                                               shift);
            else
                fold_run_regular<POW2, St, 8>(stl + 64u * g, sth + 64u * g, sx + 64u * g, 2 * run, st, Fl, Fh,
                                              nbins, shift);
            g += run;
        } else {
            const int i = g << 4;
#pragma unroll 1
            for (int q = 0; q < 16; q += 4) {
                TileRegs<4> T;
                load_tile_regs<4>(stl, sth, sx, i + q, T);
                uint32_t b[4];
                float x[4];
                bins_from_regs<POW2, 4>(T, Fl, Fh, nbins, shift, b, x);
                if (!hazard_u<4>(b)) {
                    float sm[4];
                    uint32_t c[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) st.load(b[u], sm[u], c[u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) st.put(b[u], sm[u] + x[u], c[u] + 1u);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float s1;
                        uint32_t c1;
                        st.load(b[u], s1, c1);
                        st.put(b[u], s1 + x[u], c1 + 1u);
                    }
                }
            }
            ++g;
        }
    }
    if (nvalid & 15)
        fold_tile<POW2, St, 4>(stl + 64u * ng, sth + 64u * ng, sx + 64u * ng, nvalid & 15, st, Fl, Fh,
                               nbins, shift);
}

// Tile data of one 16-sample group for the reduction fold: tau low words, fixed-point
// flux and the tau high word of the group's first sample (all from the tile).
struct RedGroup {
    uint4 a[4];
    uint4 x[4];
    uint32_t th;
};

// sthg: shared address of the segment's per-group high words
__device__ __forceinline__ void load_red_group(uint32_t stl, uint32_t sthg, uint32_t sxq, int g, RedGroup &G)
{
    const uint32_t o = 64u * (uint32_t)g;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        G.a[q] = lds_u32x4(stl + o + 16u * q);
        G.x[q] = lds_u32x4(sxq + o + 16u * q);
    }
    G.th = lds_u32(sthg + 4u * (uint32_t)g);
}

// Bins of a group. A group whose samples share one tau high word (th) forms th * F_lo
// once; the others (marked kThMixed by the prep pass: the few that straddle a change of the
// high word, every ~256 days, or unsorted times) read every sample's high word from global
// memory.
template <bool POW2>
__device__ __forceinline__ void red_group_bins(const RedGroup &G, const int32_t *gth, int g, uint32_t Fl,
                                               uint32_t Fh, uint32_t nbins, int shift, uint32_t (&b)[16])
{
    if (G.th != (uint32_t)kThMixed) {
        const uint32_t thF = G.th * Fl;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            b[4 * q + 0] = phase_bin_th<POW2>(G.a[q].x, thF, Fl, Fh, nbins, shift);
            b[4 * q + 1] = phase_bin_th<POW2>(G.a[q].y, thF, Fl, Fh, nbins, shift);
            b[4 * q + 2] = phase_bin_th<POW2>(G.a[q].z, thF, Fl, Fh, nbins, shift);
            b[4 * q + 3] = phase_bin_th<POW2>(G.a[q].w, thF, Fl, Fh, nbins, shift);
        }
    } else {
        const uint4 *h4 = reinterpret_cast<const uint4 *>(gth + 16 * g);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 h = __ldg(h4 + q);
            b[4 * q + 0] = phase_bin<POW2>(G.a[q].x, h.x, Fl, Fh, nbins, shift);
            b[4 * q + 1] = phase_bin<POW2>(G.a[q].y, h.y, Fl, Fh, nbins, shift);
            b[4 * q + 2] = phase_bin<POW2>(G.a[q].z, h.z, Fl, Fh, nbins, shift);
            b[4 * q + 3] = phase_bin<POW2>(G.a[q].w, h.w, Fl, Fh, nbins, shift);
        }
    }
}

__device__ __forceinline__ void red_group_add(const StoreRed32 &st, const uint32_t (&b)[16], const RedGroup &G)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        st.add(b[4 * q + 0], (int32_t)G.x[q].x);
        st.add(b[4 * q + 1], (int32_t)G.x[q].y);
        st.add(b[4 * q + 2], (int32_t)G.x[q].z);
        st.add(b[4 * q + 3], (int32_t)G.x[q].w);
    }
}

// kLayoutRed32: fold this stream's share of nvalid samples (a segment starting on a
// 16-sample boundary of the tile) by reductions: the 16-sample groups g with
// g mod nstreams = stream, and the tail after the last whole group if its turn falls on this
// stream. Two-stage pipeline: the tile data of the stream's next group is loaded while
// the current group's reductions issue (the loop body holds two stages with the register
// roles swapped, so nothing is copied). stl, sthg and sxq address the tile's tau low
// words, per-group high words and fixed-point flux; gth the segment's per-sample high words
// in global memory.
template <bool POW2>
__device__ __forceinline__ void fold_segment_red(uint32_t stl, uint32_t sthg, const int32_t *gth, uint32_t sxq,
                                                 int nvalid, const StoreRed32 &st,
                                                 uint32_t Fl, uint32_t Fh, uint32_t nbins, int shift, int stream,
                                                 int nstreams)
{
    const int ng = nvalid >> 4;
    // one stage: bins of group g (data in C), load group g + nstreams into N, add group g
    auto stage = [&](const RedGroup &C, RedGroup &N, int g) {
        uint32_t b[16];
        red_group_bins<POW2>(C, gth, g, Fl, Fh, nbins, shift, b);
        if (g + nstreams < ng) load_red_group(stl, sthg, sxq, g + nstreams, N);
        red_group_add(st, b, C);
    };
    int g = stream;
    if (g < ng) {
        RedGroup G0, G1;
        load_red_group(stl, sthg, sxq, g, G0);
#pragma unroll 1
        for (; g + nstreams < ng; g += 2 * nstreams) {
            stage(G0, G1, g);
            stage(G1, G0, g + nstreams);
        }
        if (g < ng) stage(G0, G1, g);
    }
    if (ng % nstreams == stream) {
        for (int i = 16 * ng; i < nvalid; ++i) {
            const uint32_t bb = phase_bin<POW2>(lds_u32(stl + 4u * i), (uint32_t)__ldg(gth + i), Fl, Fh, nbins, shift);
            st.add(bb, (int32_t)lds_u32(sxq + 4u * i));
        }
    }
}

// Most period groups a block may hold for the cross-group reduction fold below.
constexpr int kRedCross = 3;

// kLayoutRed32 with every fold warp a sample stream of all the block's period groups: the
// stream's 16-sample groups (g mod nstreams = stream, as above) go into the bins of each of
// the G period groups (lane l: period l of each group, bin records gstride bytes apart), so
// each sample is read from the tile once per block rather than once per period group.
template <bool POW2>
__device__ __forceinline__ void fold_segment_red_x(uint32_t stl, uint32_t sthg, const int32_t *gth, uint32_t sxq,
                                                   int nvalid, const StoreRed32 &st, uint32_t gstride,
                                                   const uint32_t (&Fl)[kRedCross], const uint32_t (&Fh)[kRedCross],
                                                   int G, uint32_t nbins, int shift, int stream, int nstreams)
{
    const int ng = nvalid >> 4;
    auto one = [&](const RedGroup &C, int g, int j) {
        uint32_t b[16];
        red_group_bins<POW2>(C, gth, g, Fl[j], Fh[j], nbins, shift, b);
        red_group_add(StoreRed32{st.v + (uint32_t)j * gstride}, b, C);
    };
    // one stage: group g (data in C) into every period group, group g + nstreams loaded into N
    auto stage = [&](const RedGroup &C, RedGroup &N, int g) {
        uint32_t b[16];
        red_group_bins<POW2>(C, gth, g, Fl[0], Fh[0], nbins, shift, b);
        if (g + nstreams < ng) load_red_group(stl, sthg, sxq, g + nstreams, N);
        red_group_add(st, b, C);
#pragma unroll
        for (int j = 1; j < kRedCross; ++j)
            if (j < G) one(C, g, j);
    };
    int g = stream;
    if (g < ng) {
        RedGroup G0, G1;
        load_red_group(stl, sthg, sxq, g, G0);
#pragma unroll 1
        for (; g + nstreams < ng; g += 2 * nstreams) {
            stage(G0, G1, g);
            stage(G1, G0, g + nstreams);
        }
        if (g < ng) stage(G0, G1, g);
    }
    if (ng % nstreams == stream) {
        for (int i = 16 * ng; i < nvalid; ++i) {
            const uint32_t tl = lds_u32(stl + 4u * i), th = (uint32_t)__ldg(gth + i);
            const int32_t xq = (int32_t)lds_u32(sxq + 4u * i);
#pragma unroll
            for (int j = 0; j < kRedCross; ++j)
                if (j < G)
                    StoreRed32{st.v + (uint32_t)j * gstride}.add(phase_bin<POW2>(tl, th, Fl[j], Fh[j], nbins, shift),
                                                                 xq);
        }
    }
}

// Fold this lane's chunk partials into the Kahan workspace (sum, compensation) and the
// exact 32-bit counts. On the last chunk the finished sums (sum - compensation) go back
// into the store with the counts (16-bit stores saturate at 65535; the exact totals stay
// in the workspace). Workspace reads are batched 16 bins at a time to overlap their
// latency. Returns true if a count saturated.
template <class St>
__device__ __forceinline__ void flush_one(const St &st, float2 *wsc, uint32_t *wcn, int b, size_t idx,
                                          bool first, bool last, float2 sc, uint32_t cc, bool &over)
{
    float p;
    uint32_t c;
    st.load((uint32_t)b, p, c);
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
        if (St::kSaturates) {
            st.put((uint32_t)b, sc.x - sc.y, min(cc, 65535u));
            over |= cc > 65535u;
            if (!first) wcn[idx] = cc;
        } else {
            st.put((uint32_t)b, sc.x - sc.y, cc);
        }
    } else {
        wsc[idx] = sc;
        wcn[idx] = cc;
        st.put((uint32_t)b, 0.f, 0u);
    }
}

template <class St>
__device__ __forceinline__ bool flush_chunk(const St &st, float2 *wsc, uint32_t *wcn, int nbins, int ppc,
                                            bool first, bool last)
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
            flush_one(st, wsc, wcn, b0 + u, (size_t)(b0 + u) * ppc, first, last, sc[u], cc[u], over);
    }
    for (; b0 < nbins; ++b0) {
        const size_t idx = (size_t)b0 * ppc;
        float2 sc = make_float2(0.f, 0.f);
        uint32_t cc = 0u;
        if (!first) {
            sc = wsc[idx];
            cc = wcn[idx];
        }
        flush_one(st, wsc, wcn, b0, idx, first, last, sc, cc, over);
    }
    return over;
}

// kLayoutRed32 flush: add each bin's chunk sum and count into the exact workspace (int64
// fixed-point sum, 32-bit count). On the last chunk the bin gets its FP32 sum
// tot 2^-qexp (one rounding) and its count; otherwise it is cleared. Workspace reads are
// batched 16 bins at a time to overlap their latency. qscale_f (nonzero when
// |qexp| <= 100) is 2^-qexp as an FP32 number: then tot is rounded to FP32 and scaled
// exactly (no result of a bin sum comes near the FP32 range's ends), the same single
// rounding as in FP64 without the FP64 pipe.
__device__ __forceinline__ void flush_one_red(const StoreRed32 &st, long long *wss, uint32_t *wcn, int b,
                                              size_t idx, bool last, long long tot, uint32_t cc, double qscale,
                                              float qscale_f)
{
    tot += (long long)st.isum((uint32_t)b);
    cc += st.count((uint32_t)b);
    if (last) {
        float S;
        if (qscale_f != 0.f) S = __ll2float_rn(tot) * qscale_f;
        else S = (float)((double)tot * qscale);
        st.put((uint32_t)b, S, cc);
    } else {
        wss[idx] = tot;
        wcn[idx] = cc;
        st.put((uint32_t)b, 0.f, 0u);
    }
}

__device__ __forceinline__ void flush_chunk_red(const StoreRed32 &st, long long *wss, uint32_t *wcn, int blo,
                                                int bhi, int ppc, bool first, bool last, double qscale)
{
    const int qexp = -ilogb(qscale);
    const float qscale_f = (qexp >= -100 && qexp <= 100) ? __int_as_float((127 - qexp) << 23) : 0.f;
    int b0 = blo;
    for (; b0 + 16 <= bhi; b0 += 16) {
        long long ts[16];
        uint32_t cc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            ts[u] = first ? 0ll : wss[(size_t)(b0 + u) * ppc];
            cc[u] = first ? 0u : wcn[(size_t)(b0 + u) * ppc];
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
            flush_one_red(st, wss, wcn, b0 + u, (size_t)(b0 + u) * ppc, last, ts[u], cc[u], qscale, qscale_f);
    }
    for (; b0 < bhi; ++b0) {
        const size_t idx = (size_t)b0 * ppc;
        flush_one_red(st, wss, wcn, b0, idx, last, first ? 0ll : wss[idx], first ? 0u : wcn[idx], qscale, qscale_f);
    }
}

// kLayoutRed32, kModeFold: the last chunk's flush and the epilogue in one pass. Each bin's
// exact total (the chunk's sum and count plus, unless this is the first chunk, the
// workspace's) goes straight to the output row as in write_profile_bins, with the same
// single FP32 rounding of the sum as flush_one_red; four bins at a time, so the loads,
// conversions and divisions of four bins overlap.
__device__ __forceinline__ void finish_red_rows(const StoreRed32 &st, int blo, int bhi, const long long *wss,
                                                const uint32_t *wcn, size_t ppc, bool first, double qscale,
                                                bool kvalid, size_t rowoff, float fh, float fl, float *folded,
                                                float *sums, int32_t *counts, bool vec)
{
    const int qexp = -ilogb(qscale);
    const float qscale_f = (qexp >= -100 && qexp <= 100) ? __int_as_float((127 - qexp) << 23) : 0.f;
    // warp-uniform choice of the conversion: a single chunk's total is a 32-bit integer
    // (converted on the FP32 side); longer stars and extreme units go through FP64
    const int conv = qscale_f == 0.f ? 2 : (first ? 0 : 1);
    auto bin = [&](int b, long long tot, uint32_t c, float &m, float &sv, int32_t &cv) {
        float S;
        if (conv == 0) S = __int2float_rn((int)tot) * qscale_f;
        else if (conv == 1) S = __ll2float_rn(tot) * qscale_f;
        else S = (float)((double)tot * qscale);
        if (!kvalid) c = 0u;
        m = c ? fh + (fl + S / (float)c) : __int_as_float(0x7fc00000);
        sv = c ? S : 0.f;
        cv = (int32_t)c;
        (void)b;
    };
    auto total = [&](int b, long long &tot, uint32_t &c) {
        c = st.count((uint32_t)b);
        tot = (long long)st.isum((uint32_t)b);
        if (!first) {
            tot += wss[(size_t)b * ppc];
            c += wcn[(size_t)b * ppc];
        }
    };
    int b = blo;
    if (vec) {
        for (; b + 4 <= bhi; b += 4) {
            long long t[4];
            uint32_t c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) total(b + u, t[u], c[u]);
            float4 m, sv;
            int4 cv;
            bin(b, t[0], c[0], m.x, sv.x, cv.x);
            bin(b + 1, t[1], c[1], m.y, sv.y, cv.y);
            bin(b + 2, t[2], c[2], m.z, sv.z, cv.z);
            bin(b + 3, t[3], c[3], m.w, sv.w, cv.w);
            if (folded) *reinterpret_cast<float4 *>(folded + rowoff + b) = m;
            if (sums) *reinterpret_cast<float4 *>(sums + rowoff + b) = sv;
            if (counts) *reinterpret_cast<int4 *>(counts + rowoff + b) = cv;
        }
    }
    for (; b < bhi; ++b) {
        long long t;
        uint32_t c;
        total(b, t, c);
        float m, sv;
        int32_t cv;
        bin(b, t, c, m, sv, cv);
        if (folded) folded[rowoff + b] = m;
        if (sums) sums[rowoff + b] = sv;
        if (counts) counts[rowoff + b] = cv;
    }
}

// Bins of one profile as seen by one lane: the fold's lane-private store.
template <class St>
struct LaneBins {
    St st;
    const uint32_t *Cbig;  // exact counts (workspace) when a 16-bit count saturated
    size_t cbs;
    bool big;
    __device__ __forceinline__ float s(int b) const { return st.sum((uint32_t)b); }
    __device__ __forceinline__ uint32_t ci(int b) const
    {
        return big ? Cbig[(size_t)b * cbs] : st.count((uint32_t)b);
    }
    __device__ __forceinline__ float c(int b) const { return (float)ci(b); }
    __device__ __forceinline__ float2 sc(int b) const { return make_float2(s(b), c(b)); }
};

// Bins of one profile staged by a whole warp: (sum, count) pairs at index b + b / 8, so
// lanes reading bins 8 apart hit distinct banks. Counts are exact in FP32 (n <= 2^24).
struct PairBins {
    const float2 *B;
    __device__ __forceinline__ float2 sc(int b) const { return B[b + (b >> 3)]; }
    __device__ __forceinline__ float s(int b) const { return sc(b).x; }
    __device__ __forceinline__ float c(int b) const { return sc(b).y; }
    __device__ __forceinline__ uint32_t ci(int b) const { return (uint32_t)c(b); }
};

// a_hi + a_lo += x with an error-free transformation (Knuth's TwoSum): the pair carries
// about 48 bits of the running sum
__device__ __forceinline__ void two_sum_acc(float &a_hi, float &a_lo, float x)
{
    const float s = a_hi + x;
    const float bb = s - a_hi;
    const float err = (a_hi - (s - bb)) + (x - bb);
    a_hi = s;
    a_lo += err;
}

// Box-SNR search over one profile held by this lane (bin sums centred on a reference,
// counts). The search maximises
//     v = (S n_in - S_in N) / sqrt(n_in n_out)      (= snr * sigma * sqrt(N))
// in FP32 over every circular box of w_min..w_max bins, comparing boxes through
// v |v| = D |D| / q (D the numerator, q = n_in n_out) by cross-multiplication. With the running prefix
// A(j) = S Pn(j) - N PS(j) of the bins walked so far, the numerator of a box is
// A(end) - A(start): one subtraction. R starts s0..s0+R-1 (R = 16, or 8 under a
// 128-register budget) are scored in one walk over bins s0..s0+R-2+w_max, so every bin
// read serves R boxes and the R evaluations are independent. For a fixed start the widths
// arrive in increasing order, so a strict '>' keeps the smallest width among equal
// values; the R per-start winners are then merged
// into the profile's best with ties to the smaller w, then the smaller s. The winning
// box is re-evaluated in FP64 from the same bin sums.
// Compare to a mask and bit-select through general registers: eight evaluations in
// flight would otherwise need more predicate registers than a thread has.
__device__ __forceinline__ uint32_t mask_gt(float a, float b)
{
    uint32_t m;
    asm("set.gt.u32.f32 %0, %1, %2;" : "=r"(m) : "f"(a), "f"(b));
    return m;
}
__device__ __forceinline__ uint32_t select_bits(uint32_t m, uint32_t a, uint32_t b)  // m ? a : b, bitwise
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "r"(b), "r"(m));
    return d;
}

// Two FP32 lanes in one 64-bit register pair, and element-wise IEEE round-to-nearest
// add and multiply on both (one instruction for two boxes).
__device__ __forceinline__ unsigned long long f2pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// QCHECK false is allowed when w_max is below the number of non-empty bins: then no box
// holds every sample (n_out >= 1), and a box of empty bins has D = 0 exactly (its bins add
// exact zeros to the prefix), so it never beats anything; the q >= 1 test can go.
// PACKED: the steady state of the unchecked walk evaluates starts in pairs with f32x2
// arithmetic (the same IEEE operations, so the same results).
template <int R, bool QCHECK, class Bins, bool PACKED = false>
__device__ __forceinline__ void box_walk(const Bins &B, int nbins, int w_min, int w_max, float Stot, float Ntot,
                                         int s0_first, int s0_stride, float &bv, int &bkey)
{
    for (int s0 = s0_first; s0 < nbins; s0 += s0_stride) {
        const bool full = s0 + R <= nbins;
        float bA[R] = {}, bN[R] = {};  // prefix values at each start (set as the walk enters it)
        // best per start, kept as E = D |D| and q = n_in n_out (v = sign(E) sqrt(|E| / q), so
        // E1 q2 > E2 q1 orders two boxes as v does without a square root)
        float rE[R], rq[R];
        int rt[R];  // walk step t of the best (width = t - r + 1)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            rE[r] = -INFINITY;
            rq[r] = 1.f;
            rt[r] = -1;
        }
        float runA = 0.f, runN = 0.f;
        int j = s0;
        // the next bin's sum and count are read one step ahead of their use
        float2 pf = B.sc(j);
        auto step = [&](int t) {
            const float sv = pf.x, c = pf.y;
            j = (j + 1 == nbins) ? 0 : j + 1;
            pf = B.sc(j);
            runA = fmaf(Stot, c, fmaf(-Ntot, sv, runA));
            runN += c;
            (void)t;
        };
        auto eval = [&](int r, int t, bool ok) {
            const float nin = runN - bN[r];
            const float q = nin * (Ntot - nin);
            const float D = runA - bA[r];
            const float E = D * fabsf(D);
            const bool take = ok & (q >= 1.f) & (E * rq[r] > rE[r] * q);
            rE[r] = take ? E : rE[r];
            rq[r] = take ? q : rq[r];
            rt[r] = take ? t : rt[r];
        };
        // head: t = 0..R-1; start r is entered at t = r
#pragma unroll
        for (int t = 0; t < R; ++t) {
            bA[t] = runA;
            bN[t] = runN;
            step(t);
#pragma unroll
            for (int r = 0; r <= t; ++r) {
                const int w = t - r + 1;
                eval(r, t, (w >= w_min) & (w <= w_max) & (s0 + r < nbins));
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
            step(t);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int w = t - r + 1;
                eval(r, t, (w >= w_min) & (w <= w_max) & (s0 + r < nbins));
            }
        }
        if (QCHECK) {
            for (int t = ta; t < tb; ++t) {  // every (r, w) valid here
                step(t);
#pragma unroll
                for (int r = 0; r < R; ++r) eval(r, t, true);
            }
        } else if (PACKED) {
            unsigned long long nbN2[R / 2], cN2[R / 2], nbA2[R / 2];
#pragma unroll
            for (int h = 0; h < R / 2; ++h) {
                nbN2[h] = f2pack(-bN[2 * h], -bN[2 * h + 1]);
                cN2[h] = f2pack(Ntot + bN[2 * h], Ntot + bN[2 * h + 1]);
                nbA2[h] = f2pack(-bA[2 * h], -bA[2 * h + 1]);
            }
            for (int t = ta; t < tb; ++t) {
                step(t);
                const unsigned long long RN2 = f2pack(runN, runN), nRN2 = f2pack(-runN, -runN);
                const unsigned long long RA2 = f2pack(runA, runA);
#pragma unroll
                for (int h = 0; h < R / 2; ++h) {
                    const unsigned long long q2 = f2mul(f2add(RN2, nbN2[h]), f2add(cN2[h], nRN2));
                    float D0, D1;
                    f2unpack(f2add(RA2, nbA2[h]), D0, D1);
                    const unsigned long long E2 = f2pack(D0 * fabsf(D0), D1 * fabsf(D1));
                    float l0, l1, g0, g1, q0, q1, E0, E1;
                    f2unpack(f2mul(E2, f2pack(rq[2 * h], rq[2 * h + 1])), l0, l1);
                    f2unpack(f2mul(f2pack(rE[2 * h], rE[2 * h + 1]), q2), g0, g1);
                    f2unpack(q2, q0, q1);
                    f2unpack(E2, E0, E1);
                    const uint32_t m0 = mask_gt(l0, g0), m1 = mask_gt(l1, g1);
                    rE[2 * h] = __uint_as_float(select_bits(m0, __float_as_uint(E0), __float_as_uint(rE[2 * h])));
                    rq[2 * h] = __uint_as_float(select_bits(m0, __float_as_uint(q0), __float_as_uint(rq[2 * h])));
                    rt[2 * h] = (int)select_bits(m0, (uint32_t)t, (uint32_t)rt[2 * h]);
                    rE[2 * h + 1] =
                        __uint_as_float(select_bits(m1, __float_as_uint(E1), __float_as_uint(rE[2 * h + 1])));
                    rq[2 * h + 1] =
                        __uint_as_float(select_bits(m1, __float_as_uint(q1), __float_as_uint(rq[2 * h + 1])));
                    rt[2 * h + 1] = (int)select_bits(m1, (uint32_t)t, (uint32_t)rt[2 * h + 1]);
                }
            }
        } else {
            float cN[R];  // N + Pn(start): n_out = cN - Pn(end), exact in integers
#pragma unroll
            for (int r = 0; r < R; ++r) cN[r] = Ntot + bN[r];
            for (int t = ta; t < tb; ++t) {
                step(t);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float q = (runN - bN[r]) * (cN[r] - runN);
                    const float D = runA - bA[r];
                    const float E = D * fabsf(D);
                    const uint32_t m = mask_gt(E * rq[r], rE[r] * q);
                    rE[r] = __uint_as_float(select_bits(m, __float_as_uint(E), __float_as_uint(rE[r])));
                    rq[r] = __uint_as_float(select_bits(m, __float_as_uint(q), __float_as_uint(rq[r])));
                    rt[r] = (int)select_bits(m, (uint32_t)t, (uint32_t)rt[r]);
                }
            }
        }
        for (int t = max(tb, R); t < tend; ++t) {
            step(t);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int w = t - r + 1;
                eval(r, t, (w >= w_min) & (w <= w_max) & (s0 + r < nbins));
            }
        }
        // merge the per-start winners: larger v, then smaller w, then smaller s
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (rt[r] < 0) continue;
            const float vr = rE[r] >= 0.f ? sqrtf(rE[r] / rq[r]) : -sqrtf(-rE[r] / rq[r]);
            const int key = ((rt[r] - r + 1) << 12) | (s0 + r);
            const bool take = (vr > bv) | ((vr == bv) & (key < bkey));
            bv = take ? vr : bv;
            bkey = take ? key : bkey;
        }
    }
}

// Re-evaluation of box (bs, bw), snr = (S n_in - S_in N) / (sigma sqrt(N n_in n_out)):
// exact integer counts, double-float sums, FP64 for the last few operations.
template <class Bins>
__device__ __forceinline__ float box_reeval(const Bins &B, int nbins, int bs, int bw, float sigma)
{
    float sth = 0.f, stl = 0.f, sih = 0.f, sil = 0.f;
    uint32_t nt = 0u, ni = 0u;
    for (int b = 0; b < nbins; ++b) {
        two_sum_acc(sth, stl, B.s(b));
        nt += B.ci(b);
    }
    int j = bs;
    for (int w = 0; w < bw; ++w) {
        two_sum_acc(sih, sil, B.s(j));
        ni += B.ci(j);
        j = (j + 1 == nbins) ? 0 : j + 1;
    }
    const double St = (double)sth + (double)stl, Si = (double)sih + (double)sil;
    const double Nt = (double)nt, Ni = (double)ni, No = (double)(nt - ni);
    return (float)((St * Ni - Si * Nt) / ((double)sigma * sqrt(Nt * Ni * No)));
}

// Box-SNR of one profile held by one thread: every start, then the winner re-evaluated.
// The walk over the blocks of R starts s0_first, s0_first + s0_stride, ... of one profile:
// its best (v, key = w << 12 | s), by the walk's rule.
template <int R, class Bins>
__device__ __forceinline__ void box_search_part(const Bins &B, int nbins, int w_min, int w_max, int s0_first,
                                                int s0_stride, float &bv, int &bkey)
{
    float Stot = 0.f, Ntot = 0.f;
    int nnz = 0;
    for (int b = 0; b < nbins; ++b) {
        const float c = B.c(b);
        Stot += B.s(b);
        Ntot += c;
        nnz += c > 0.f;
    }
    bv = -INFINITY;
    bkey = 0x7fffffff;
    if (w_max < nnz) box_walk<R, false>(B, nbins, w_min, w_max, Stot, Ntot, s0_first, s0_stride, bv, bkey);
    else box_walk<R, true>(B, nbins, w_min, w_max, Stot, Ntot, s0_first, s0_stride, bv, bkey);
}

template <int R, class Bins>
__device__ __forceinline__ void box_search(const Bins &B, int nbins, int w_min, int w_max, float sigma,
                                           float &score, int &best_s, int &best_w)
{
    float bv;
    int bkey;
    box_search_part<R>(B, nbins, w_min, w_max, 0, R, bv, bkey);
    if (bkey == 0x7fffffff) {
        score = -INFINITY;
        best_s = -1;
        best_w = -1;
        return;
    }
    best_w = bkey >> 12;
    best_s = bkey & 4095;
    score = box_reeval(B, nbins, best_s, best_w, sigma);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// ------------------------------------------------------------------ box-SNR, warp per profile

// A warp scores one profile at a time from the fold's centred bin sums and counts: the
// profile is staged as PairBins, lane L walks the blocks of 8 starts L, L + 32, ... and
// the lanes' winners merge by the walk's own rule (larger v, then smaller w, then smaller
// s). The winner is re-evaluated with double-float sums spread over the warp. Unlike the
// fold's own epilogue, the search here runs at full occupancy.
constexpr int kCoopR = 8;

__device__ __forceinline__ void two_sum_merge(float &hi, float &lo, float hi2, float lo2)
{
    two_sum_acc(hi, lo, hi2);
    lo += lo2;
}

__device__ __forceinline__ int star_of(const int64_t *grid_off, int nstars, int64_t k)
{
    int lo = 0, hi = nstars - 1;
    while (lo < hi) {  // the last star whose range starts at or before k
        const int mid = (lo + hi + 1) >> 1;
        if (grid_off[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Box-SNR of row r of p's profile buffer (period k >= 0) by the calling warp, staged in Bw
// as PairBins: lane L walks the blocks of 8 starts L, L + 32, ..., the lanes' winners merge
// by the walk's own rule (larger v, then smaller w, then smaller s), and the winner is
// re-evaluated with double-float sums spread over the warp. Lane 0 writes the outputs and
// folds the period's argmax key into (cur_s, cur_key).
__device__ __forceinline__ void score_row(const BoxCoopParams &p, int64_t r, int64_t k, float2 *Bw, int lane,
                                       int &cur_s, unsigned long long &cur_key)
{
    const int nbins = p.nbins;
    const PairBins B{Bw};
    const int s = p.grid_off ? star_of(p.grid_off, p.nstars, k) : 0;
    const int64_t gb = p.grid_off ? p.grid_off[s] : 0;
    const float *srow = p.sums ? p.sums + (size_t)r * nbins : nullptr;
    const float *mrow = p.means ? p.means + (size_t)r * nbins : nullptr;
    const int32_t *crow = p.counts + (size_t)r * nbins;
    float mref = 0.f;
    if (mrow) {  // means in: centre them on the profile's count-weighted mean (FP64)
        double num = 0.0, den = 0.0;
        for (int b = lane; b < nbins; b += 32) {
            const int32_t c = crow[b];
            if (c > 0) {
                num += (double)mrow[b] * (double)c;
                den += (double)c;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        mref = den > 0.0 ? (float)(num / den) : 0.f;
    }
    __syncwarp();  // the previous profile's readers are done
    float Stot = 0.f, Ntot = 0.f;
    int nnz = 0;
    // 256 bins at a time, every load issued before any is used: one L2 round trip per
    // 256 bins (a lone warp per scheduler cannot hide eight in a row)
    for (int b0 = 0; b0 < nbins; b0 += 256) {
        float vv[8];
        int32_t cv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + 32 * u + lane;
            cv[u] = b < nbins ? crow[b] : 0;
            vv[u] = b < nbins ? (mrow ? mrow[b] : srow[b]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + 32 * u + lane;
            if (b < nbins) {
                const float c = (float)max(cv[u], 0);
                const float sv = mrow ? (c > 0.f ? (vv[u] - mref) * c : 0.f) : vv[u];
                Bw[b + (b >> 3)] = make_float2(sv, c);
                Stot += sv;
                Ntot += c;
                nnz += c > 0.f;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {  // a butterfly leaves the same totals in every lane
        Stot += __shfl_xor_sync(0xffffffffu, Stot, o);
        Ntot += __shfl_xor_sync(0xffffffffu, Ntot, o);
        nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    }
    __syncwarp();
    float bv = -INFINITY;
    int bkey = 0x7fffffff;
    if (p.w_max < nnz)
        box_walk<kCoopR, false, PairBins, true>(B, nbins, p.w_min, p.w_max, Stot, Ntot, lane * kCoopR, 32 * kCoopR,
                                               bv, bkey);
    else
        box_walk<kCoopR, true>(B, nbins, p.w_min, p.w_max, Stot, Ntot, lane * kCoopR, 32 * kCoopR, bv, bkey);
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int okey = __shfl_xor_sync(0xffffffffu, bkey, o);
        const bool take = (ov > bv) | ((ov == bv) & (okey < bkey));
        bv = take ? ov : bv;
        bkey = take ? okey : bkey;
    }
    float sc = -INFINITY;
    int bs = -1, bw = -1;
    if (bkey != 0x7fffffff) {
        bw = bkey >> 12;
        bs = bkey & 4095;
        float sth = 0.f, stl = 0.f, sih = 0.f, sil = 0.f;
        uint32_t nt = 0u, ni = 0u;
        for (int b = lane; b < nbins; b += 32) {
            const float2 v = B.sc(b);
            const uint32_t c = (uint32_t)v.y;
            two_sum_acc(sth, stl, v.x);
            nt += c;
            int d = b - bs;
            d += d < 0 ? nbins : 0;
            if (d < bw) {
                two_sum_acc(sih, sil, v.x);
                ni += c;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            two_sum_merge(sth, stl, __shfl_xor_sync(0xffffffffu, sth, o), __shfl_xor_sync(0xffffffffu, stl, o));
            two_sum_merge(sih, sil, __shfl_xor_sync(0xffffffffu, sih, o), __shfl_xor_sync(0xffffffffu, sil, o));
            nt += __shfl_xor_sync(0xffffffffu, nt, o);
            ni += __shfl_xor_sync(0xffffffffu, ni, o);
        }
        if (lane == 0) {  // the FP64 tail once per profile (only lane 0 writes the outputs)
            float sig = p.sigma_user;
            if (!(sig > 0.f) && p.stats) sig = p.stats[s].sigma;
            if (!(sig > 0.f)) sig = 1.f;
            const double St = (double)sth + (double)stl, Si = (double)sih + (double)sil;
            const double Nt = (double)nt, Ni = (double)ni, No = (double)(nt - ni);
            sc = (float)((St * Ni - Si * Nt) / ((double)sig * sqrt(Nt * Ni * No)));
        }
    }
    if (lane == 0) {
        p.score[k] = sc;
        if (p.best_s) p.best_s[k] = bs;
        if (p.best_w) p.best_w[k] = bw;
        if (p.best_key) {
            const unsigned long long key = argmax_key(sc, k - gb);
            if (s != cur_s) {
                if (cur_key) atomicMax(&p.best_key[cur_s], cur_key);
                cur_s = s;
                cur_key = key;
            } else {
                cur_key = key > cur_key ? key : cur_key;
            }
        }
    }
}

// ---------------------------------------------------------------- fold + box-SNR in one kernel

// Work of the box-SNR scorer inside a search block. Tickets number the rows of the block's
// tasks in order (ticket t = row t % ppc of the block's task t / ppc); a warp takes the next
// ticket with a compare-and-swap, never one at or past `limit`.
__device__ __forceinline__ int take_ticket(int *ticket, int limit)
{
    int t = *reinterpret_cast<volatile int *>(ticket);
    while (t < limit) {
        const int old = atomicCAS(ticket, t, t + 1);
        if (old == t) return t;
        t = old;
    }
    return -1;
}

__device__ __forceinline__ void named_bar_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Named barrier that returns the OR of the participants' predicates (the same for all).
__device__ __forceinline__ bool named_bar_or(int id, int threads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

// Shared state of a search block: the task each ring slot last received (-1: none yet),
// the rows scored in each slot since the start (slot b is free for task i once
// done[b] >= (i / 2) * ppc), and the next ticket. All three only grow.
struct SearchShared {
    int pub[2];
    int done[2];
    int ticket;
};

// Score the row of ticket t (its task already published) with the calling warp; the ring
// slot's done count goes up once the row's staging reads are over.
__device__ __forceinline__ void score_ticket(const FoldParams &p, SearchShared &sh, int t, int ppc, float2 *Bw,
                                             int lane, int &cur_s, unsigned long long &cur_key)
{
    const int task_i = t / ppc, row = t - task_i * ppc, b = task_i & 1;
    const size_t base = ((size_t)blockIdx.x * 2 + b) * ppc;
    const int64_t k = p.slot_k[base + row];
    if (k >= 0) {
        BoxCoopParams q{};
        q.sums = p.sums + base * p.nbins;
        q.counts = p.counts + base * p.nbins;
        q.nbins = p.nbins;
        q.w_min = p.w_min;
        q.w_max = p.w_max;
        q.sigma_user = p.sigma_user;
        q.stats = p.stats;
        q.grid_off = p.grid_off;
        q.nstars = p.nstars;
        q.score = p.score;
        q.best_s = p.best_s;
        q.best_w = p.best_w;
        q.best_key = p.best_key;
        score_row(q, row, k, Bw, lane, cur_s, cur_key);
    }
    __syncwarp();
    if (lane == 0) atomicAdd(&sh.done[b], 1);
}

// Wait (bounded, giving up on abort) until `*flag` >= `want`; one lane reads it.
__device__ __forceinline__ bool wait_flag(const int *flag, int want, const int *abort_flag, uint32_t *status)
{
    const long long start = clock64();
    while (*reinterpret_cast<const volatile int *>(flag) < want) {
        if (*reinterpret_cast<const volatile int *>(abort_flag)) return false;
        if (clock64() - start > kWaitLimitCycles) {
            report_error(status, kErrTimeout);
            return false;
        }
    }
    return true;
}

// Write bins [blo, bhi) of this lane's profile to its output row (row offset rowoff):
// means fh + (fl + S / c) (NaN for an empty bin), sums (0 for an empty bin) and counts;
// each output may be NULL. The lanes of a warp write 32 different rows, so every store
// touches 32 sectors: with vec (16-byte aligned outputs, nbins and blo multiples of 4) a
// lane writes four bins per store.
template <class St>
__device__ __forceinline__ void write_profile_bins(const St &st, int blo, int bhi, size_t rowoff, bool kvalid,
                                                   bool over, const uint32_t *wcn, size_t ppc, float fh, float fl,
                                                   float *folded, float *sums, int32_t *counts, bool vec)
{
    auto bin = [&](int b, float &m, float &sv, int32_t &cv) {
        float S;
        uint32_t c;
        st.load((uint32_t)b, S, c);
        if (over) c = wcn[(size_t)b * ppc];
        if (!kvalid) c = 0u;
        m = c ? fh + (fl + S / (float)c) : __int_as_float(0x7fc00000);
        sv = c ? S : 0.f;
        cv = (int32_t)c;
    };
    int b = blo;
    if (vec) {
        for (; b + 4 <= bhi; b += 4) {
            float4 m, sv;
            int4 cv;
            bin(b, m.x, sv.x, cv.x);
            bin(b + 1, m.y, sv.y, cv.y);
            bin(b + 2, m.z, sv.z, cv.z);
            bin(b + 3, m.w, sv.w, cv.w);
            if (folded) *reinterpret_cast<float4 *>(folded + rowoff + b) = m;
            if (sums) *reinterpret_cast<float4 *>(sums + rowoff + b) = sv;
            if (counts) *reinterpret_cast<int4 *>(counts + rowoff + b) = cv;
        }
    }
    for (; b < bhi; ++b) {
        float m, sv;
        int32_t cv;
        bin(b, m, sv, cv);
        if (folded) folded[rowoff + b] = m;
        if (sums) sums[rowoff + b] = sv;
        if (counts) counts[rowoff + b] = cv;
    }
}

template <int MODE, bool POW2, int LAYOUT, int MAXW>
__global__ void __launch_bounds__(MAXW * 32, 1) fold_kernel(const FoldParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_abort;
    __shared__ SearchShared sh;
    constexpr bool kRed = LAYOUT == kLayoutRed32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nbins = p.nbins;
    const int ppc = 32 * p.warps;
    const int tile = p.tile;
    // fold warps: period group gw = warp % warps, sample stream sw = warp / warps (kLayoutRed32
    // only; otherwise one stream). Stream sw finalises and writes out bins [blo, bhi).
    const int nstreams = kRed ? p.streams : 1;
    const int nfw = p.warps * nstreams;
    const int gw = warp % p.warps, sw = warp / p.warps;
    const int blo = (int)((int64_t)sw * nbins / nstreams), bhi = (int)((int64_t)(sw + 1) * nbins / nstreams);
    // kLayoutRed32 with at most kRedCross period groups: fold warp w is sample stream w of nfw
    // and folds into every group (the flushes and epilogues keep the (gw, sw) split above)
    const bool cross = kRed && p.warps <= kRedCross;
    // whether several warps add into one period group's bins (then they meet at the flushes)
    const bool shared_bins = cross ? nfw > 1 : nstreams > 1;
    // block barrier of the fold warps (in kModeSearch the scorer warp is not among them)
    auto fold_sync = [&]() {
        if (MODE == kModeSearch) named_bar_sync(1, 32 * nfw);
        else __syncthreads();
    };

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint32_t *tl_buf = reinterpret_cast<uint32_t *>(smem + 128);
    // the reduction layout's tiles hold the low words, the fixed-point flux, one high word
    // per 16-sample group and the flags (the few groups whose samples differ in their high
    // word read them from global memory)
    uint32_t *th_buf = tl_buf + 2 * tile;
    float *x_buf = reinterpret_cast<float *>(kRed ? th_buf : th_buf + 2 * tile);
    uint32_t *thg_buf = reinterpret_cast<uint32_t *>(x_buf + 2 * tile);     // kRed: [2][tile / 16]
    uint8_t *f_buf = reinterpret_cast<uint8_t *>(kRed ? thg_buf + 2 * (tile / 16)
                                                      : reinterpret_cast<uint32_t *>(x_buf + 2 * tile));  // [2][tile / 16]
    using St = typename std::conditional<LAYOUT == kLayoutPacked64, StorePacked64,
                                         typename std::conditional<kRed, StoreRed32, StorePaired16>::type>::type;
    St st;
    StoreRed32 st0{0u};  // kLayoutRed32: this lane's records of period group 0
    const uint32_t gstride = (uint32_t)nbins * 256u;  // bytes between period groups' records
    if constexpr (LAYOUT == kLayoutPacked64) {
        uint2 *v = reinterpret_cast<uint2 *>(f_buf + 2 * (tile / 16));
        st.v = smem_u32(v + (size_t)warp * nbins * 32 + lane);
    } else if constexpr (kRed) {
        uint32_t *v = reinterpret_cast<uint32_t *>(f_buf + 2 * (tile / 16));
        st.v = smem_u32(v + (size_t)gw * nbins * 64 + lane);
        st0.v = smem_u32(v + lane);
    } else {
        float *acc = reinterpret_cast<float *>(f_buf + 2 * (tile / 16));
        const int nb2 = (nbins + 1) & ~1;
        uint16_t *cnt = reinterpret_cast<uint16_t *>(acc + (size_t)p.warps * nbins * 32);
        st.acc = smem_u32(acc + (size_t)warp * nbins * 32 + lane);
        st.cnt = smem_u32(cnt + (size_t)warp * nb2 * 32 + 2 * lane);
    }

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
        sh.pub[0] = sh.pub[1] = -1;
        sh.done[0] = sh.done[1] = 0;
        sh.ticket = 0;
    }
    __syncthreads();
    uint32_t parity_bits = 0u;  // bit b: phase parity of buffer b
    // profile rows written four bins per store when the outputs allow it
    const bool vec_out = (nbins & 3) == 0 && (blo & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(p.folded) | reinterpret_cast<uintptr_t>(p.sums) |
                           reinterpret_cast<uintptr_t>(p.counts)) & 15) == 0;
    float2 *wsc_cta = p.ws_sc + (size_t)blockIdx.x * nbins * ppc + gw * 32 + lane;
    uint32_t *wcn_cta = p.ws_cnt + (size_t)blockIdx.x * nbins * ppc + gw * 32 + lane;

    int64_t task_end = p.ntasks;
    if (p.ntasks_dev) {
        const int64_t t = *p.ntasks_dev;
        task_end = t < task_end ? t : task_end;
    }
    // kModeSearch: this block's tasks, their rows as tickets, and the warps' scorer staging
    const int64_t first_task = p.task_begin + blockIdx.x;
    const int my_tasks = first_task < task_end ? (int)((task_end - first_task + gridDim.x - 1) / gridDim.x) : 0;
    // scorer staging: one slot per warp of stream 0 (the fold warps that also score
    // leftover rows) and one for the scorer warp
    float2 *Bw = reinterpret_cast<float2 *>(smem + p.stage_off) + (size_t)(warp == nfw ? p.warps : gw) * coop_pairs(nbins);
    int cur_s = -1;
    unsigned long long cur_key = 0ull;
    if (MODE == kModeSearch && warp == nfw) {
        // the scorer warp: take tickets in order, wait for each one's task to be published
        for (;;) {
            int t = 0;
            if (lane == 0) t = take_ticket(&sh.ticket, my_tasks * ppc);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t < 0) break;
            bool ok = true;
            if (lane == 0) ok = wait_flag(&sh.pub[(t / ppc) & 1], t / ppc, &s_abort, p.status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;  // the fold warps aborted, or a timeout
            __threadfence_block();
            score_ticket(p, sh, t, ppc, Bw, lane, cur_s, cur_key);
        }
        if (lane == 0 && p.best_key && cur_key) atomicMax(&p.best_key[cur_s], cur_key);
        return;
    }
    int iter = 0;  // index of the task within this block's sequence
    for (int64_t task = first_task; task < task_end; task += gridDim.x, ++iter) {
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
        // (more than 2^24 samples happens only for offsets the batch plan rejected)
        const int64_t nsamp = min(le - lb, (int64_t)1 << 24);
        const int64_t sbase = scratch_start(lb, s);
        const int64_t k = gb + (task - tbase) * ppc + gw * 32 + lane;
        const bool kvalid = k < ge;

        uint32_t Fl = 0u, Fh = 0u;
        int gsize = 16;  // lanes past the grid do not restrict the warp's group size
        if (kvalid) {
            const double P = p.periods[k];
            const double q = kTwo40 / P;
            if (P > 0.0 && P < INFINITY && q < kTwo63) {
                const unsigned long long F = (unsigned long long)__double2ll_rn(q);
                Fl = (uint32_t)F;
                Fh = (uint32_t)(F >> 32);
                // (the reduction layout needs no collision-free group size)
                if (!kRed) gsize = regular_group_size(F, p.stats[s].dtau0, (uint32_t)nbins);
            } else {
                gsize = 0;
                report_error(p.status, kErrRange);
            }
        }
        // the cross-group fold: this lane's period in each of the block's period groups
        uint32_t FlX[kRedCross], FhX[kRedCross];
#pragma unroll
        for (int j = 0; j < kRedCross; ++j) {
            FlX[j] = FhX[j] = 0u;
            const int64_t kj = gb + (task - tbase) * ppc + j * 32 + lane;
            if (cross && j < p.warps && kj < ge) {
                const double q = kTwo40 / p.periods[kj];
                if (q > 0.0 && q < kTwo63) {  // (a period outside (0, inf) is reported above)
                    const unsigned long long F = (unsigned long long)__double2ll_rn(q);
                    FlX[j] = (uint32_t)F;
                    FhX[j] = (uint32_t)(F >> 32);
                }
            }
        }
        // one group size for the whole warp, so its lanes never diverge between paths
        const int wg = __all_sync(0xffffffffu, gsize >= 16) ? 16 : (__all_sync(0xffffffffu, gsize >= 8) ? 8 : 0);
        const double qscale = kRed ? ldexp(1.0, -p.stats[s].qexp) : 1.0;  // fixed-point unit
        for (int b = blo; b < bhi; ++b) st.put((uint32_t)b, 0.f, 0u);
        const int ntiles = (int)((nsamp + tile - 1) / tile);
        auto issue = [&](int t, int buf) {
            const int64_t i0 = (int64_t)t * tile;
            const int nv = (int)min((int64_t)tile, nsamp - i0);
            const uint32_t bytes = (uint32_t)(((nv + 3) & ~3) * 4);
            const uint32_t fbytes = (uint32_t)((((nv + 15) >> 4) + 15) & ~15);
            // (the reduction layout needs no cadence flags: its groups carry their high word)
            const uint32_t gbytes = kRed ? (uint32_t)((((nv + 15) >> 4) * 4 + 15) & ~15) : 0u;
            mbar_arrive_expect_tx(&bars[buf], kRed ? 2u * bytes + gbytes : 3u * bytes + fbytes);
            bulk_g2s(tl_buf + buf * tile, p.smp.tau_lo + sbase + i0, bytes, &bars[buf]);
            if (!kRed) bulk_g2s(th_buf + buf * tile, p.smp.tau_hi + sbase + i0, bytes, &bars[buf]);
            else bulk_g2s(thg_buf + buf * (tile / 16), p.smp.thg + (sbase + i0) / 16, gbytes, &bars[buf]);
            if (kRed) bulk_g2s(x_buf + buf * tile, p.smp.xq + sbase + i0, bytes, &bars[buf]);
            else bulk_g2s(x_buf + buf * tile, p.smp.x + sbase + i0, bytes, &bars[buf]);
            if (!kRed) bulk_g2s(f_buf + buf * (tile / 16), p.smp.flags + (sbase + i0) / 16, fbytes, &bars[buf]);
        };
        fold_sync();  // previous task's readers are done with both buffers
        if (threadIdx.x == 0 && ntiles > 0) {  // a star without samples issues nothing
            issue(0, 0);
            if (ntiles > 1) issue(1, 1);
        }
        bool over = false;
        bool first_flush = true;
        bool last_first = true;  // kLayoutRed32 fold: whether the last chunk was also the first
        int chunk_left = p.chunk;
        for (int t = 0; t < ntiles; ++t) {
            const int buf = t & 1;
            bool ok = mbar_wait_bounded(&bars[buf], (parity_bits >> buf) & 1u);
            parity_bits ^= 1u << buf;
            // with several streams the fold warps meet at the chunk flushes inside a tile, so
            // before a tile that holds one they all take the same branch (every warp knows
            // whether it does: chunk boundaries and the tile count are the same for all)
            const int nv_t = (int)min((int64_t)tile, nsamp - (int64_t)t * tile);
            // (the fold mode finishes its last chunk after the tile loop; the others flush it
            // inside the last tile)
            const bool last_tile = t == ntiles - 1;
            const bool flush_inside = (chunk_left <= nv_t && !(MODE == kModeFold && chunk_left == nv_t && last_tile)) ||
                                      (last_tile && MODE != kModeFold);
            if (shared_bins && flush_inside) ok = !named_bar_or(1, 32 * nfw, !ok);
            if (!ok) {
                s_abort = 1;
                report_error(p.status, kErrTimeout);
            } else {
                const int nv = (int)min((int64_t)tile, nsamp - (int64_t)t * tile);
                // the tile in sub-tiles of up to 1024 samples, each with its 64 regular-group
                // flag bytes packed into a register bit mask
                for (int sub = 0; sub < nv; sub += 1024) {
                    const int nvs = min(1024, nv - sub);
                    const uint32_t stl = smem_u32(tl_buf + buf * tile + sub);
                    const uint32_t sth = smem_u32(th_buf + buf * tile + sub);
                    const uint32_t sx = smem_u32(x_buf + buf * tile + sub);
                    unsigned long long fmask = 0ull;
                    if (!kRed) {  // the reduction layout takes no collision-free runs
                        const uint4 *fw = reinterpret_cast<const uint4 *>(f_buf + buf * (tile / 16) + sub / 16);
                        const int nq = (nvs + 255) >> 8;  // 16-byte words holding the sub-tile's flags
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (q < nq) {
                                const uint4 w = fw[q];
                                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    // bytes (0 or 1) j = 0..3 of a word -> bits j of a nibble
                                    const unsigned long long nib = ((ww[r] * 0x01020408u) >> 24) & 0xFu;
                                    fmask |= nib << (16 * q + 4 * r);
                                }
                            }
                        }
                    }
                    int i = 0;
                    while (i < nvs) {
                        // segments end at chunk boundaries (multiples of 4 samples) or the sub-tile end
                        const int seg = min(nvs - i, chunk_left);
                        if constexpr (kRed) {
                            if (cross) {
                                // the streams' turns rotate with the segment's first group, so
                                // segments of any length share their groups out evenly
                                const int g0 = (int)((((int64_t)t * tile + sub + i) >> 4) % nfw);
                                fold_segment_red_x<POW2>(stl + 4u * i,
                                                         smem_u32(thg_buf + buf * (tile / 16) + (sub + i) / 16),
                                                         p.smp.tau_hi + sbase + (int64_t)t * tile + sub + i,
                                                         sx + 4u * i, seg, st0, gstride, FlX, FhX, p.warps,
                                                         (uint32_t)nbins, p.shift, (warp - g0 + nfw) % nfw, nfw);
                            } else
                            fold_segment_red<POW2>(stl + 4u * i,
                                                   smem_u32(thg_buf + buf * (tile / 16) + (sub + i) / 16),
                                                   p.smp.tau_hi + sbase + (int64_t)t * tile + sub + i,
                                                   sx + 4u * i, seg, st, Fl, Fh, (uint32_t)nbins, p.shift, sw,
                                                   nstreams);
                        } else
                            fold_segment<POW2, St, (MAXW <= 4)>(stl + 4u * i, sth + 4u * i, sx + 4u * i,
                                                                 fmask >> (i >> 4), seg, st, Fl, Fh, (uint32_t)nbins,
                                                                 p.shift, wg);
                        i += seg;
                        chunk_left -= seg;
                        const bool last = (t == ntiles - 1) && (sub + i == nv);
                        if (chunk_left == 0 || last) {
                            if constexpr (kRed) {
                                // every stream's reductions of the chunk land before the flush
                                // reads them, and the cleared bins before the next chunk's. The
                                // fold's last chunk is finished in the epilogue (after the tile
                                // loop's barrier), straight into the output rows.
                                if (!(MODE == kModeFold && last)) {
                                    if (shared_bins) fold_sync();
                                    flush_chunk_red(st, reinterpret_cast<long long *>(wsc_cta), wcn_cta, blo, bhi,
                                                    ppc, first_flush, last, qscale);
                                    if (shared_bins) fold_sync();
                                } else {
                                    last_first = first_flush;
                                }
                            }
                            else
                                over = flush_chunk(st, wsc_cta, wcn_cta, nbins, ppc, first_flush, last);
                            first_flush = false;
                            chunk_left = p.chunk;
                        }
                    }
                }
            }
            fold_sync();
            if (*reinterpret_cast<volatile int *>(&s_abort)) {
                if (threadIdx.x == 0) {
                    // let this block's bulk copies in flight (tiles t and t + 1) land first
                    mbar_wait_bounded(&bars[buf], ((parity_bits >> buf) & 1u) ^ 1u);
                    if (t + 1 < ntiles) mbar_wait_bounded(&bars[buf ^ 1], (parity_bits >> (buf ^ 1)) & 1u);
                }
                return;
            }
            if (threadIdx.x == 0 && t + 2 < ntiles) issue(t + 2, buf);
        }

        // ---------------- epilogues (lane-private; with several streams each writes its own
        // bins, which it also clears for the next task)
        if (MODE == kModeFold) {
            // output row: the period, or the lane's chunk slot
            const int64_t row = p.slot_k ? (task - p.task_begin) * ppc + gw * 32 + lane : k;
            if (p.slot_k && sw == 0) p.slot_k[row] = kvalid ? k : -1;
            if constexpr (kRed) {
                if ((kvalid || p.slot_k) && ntiles > 0)
                    finish_red_rows(st, blo, bhi, reinterpret_cast<const long long *>(wsc_cta), wcn_cta, (size_t)ppc,
                                    last_first, qscale, kvalid, (size_t)row * nbins, p.stats[s].f_hi,
                                    p.stats[s].f_lo, p.folded, p.sums, p.counts, vec_out);
                else if (kvalid || p.slot_k)
                    write_profile_bins(st, blo, bhi, (size_t)row * nbins, kvalid, false, wcn_cta, (size_t)ppc,
                                       p.stats[s].f_hi, p.stats[s].f_lo, p.folded, p.sums, p.counts, vec_out);
            } else if (kvalid || p.slot_k) {
                write_profile_bins(st, blo, bhi, (size_t)row * nbins, kvalid, over, wcn_cta, (size_t)ppc,
                                   p.stats[s].f_hi, p.stats[s].f_lo, p.folded, p.sums, p.counts, vec_out);
            }
        } else if (MODE == kModeSearch) {
            const int b = iter & 1;
            const int need = (iter >> 1) * ppc;  // rows of slot b that must be scored first
            bool ok = true;
            if (iter >= 2 && sw == 0) {
                // slot b still holds task iter - 2: score leftover rows of the published tasks
                // (tickets below iter * ppc) until all of iter - 2's rows are done (the
                // warps of stream 0 only: they own the fold warps' scorer staging)
                for (;;) {
                    int t = -1;
                    if (lane == 0) t = *reinterpret_cast<volatile int *>(&sh.done[b]) >= need
                                           ? -2 : take_ticket(&sh.ticket, iter * ppc);
                    t = __shfl_sync(0xffffffffu, t, 0);
                    if (t == -2) break;
                    if (t >= 0) {
                        score_ticket(p, sh, t, ppc, Bw, lane, cur_s, cur_key);
                    } else {
                        if (lane == 0) ok = wait_flag(&sh.done[b], need, &s_abort, p.status);
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                        break;
                    }
                }
            }
            // the other streams write their bins of the slot once stream 0 has found it free
            if (nstreams > 1) ok = !named_bar_or(1, 32 * nfw, !ok);
            if (ok) {
                const size_t base = ((size_t)blockIdx.x * 2 + b) * ppc + gw * 32 + lane;
                if (sw == 0) p.slot_k[base] = kvalid ? k : -1;
                write_profile_bins(st, blo, bhi, base * nbins, kvalid, over, wcn_cta, (size_t)ppc, 0.f, 0.f, nullptr,
                                   p.sums, p.counts, vec_out);
            }
            // every row of the task is written; all fold warps leave together on a failure
            if (named_bar_or(1, 32 * nfw, !ok)) {
                if (threadIdx.x == 0) *reinterpret_cast<volatile int *>(&s_abort) = 1;
                return;
            }
            if (threadIdx.x == 0) {
                __threadfence_block();
                *reinterpret_cast<volatile int *>(&sh.pub[b]) = iter;
            }
        } else if (MODE == kModeBox) {
            constexpr int kR = MAXW <= 4 ? 16 : 8;
            float sc = -INFINITY;
            int bs = -1, bw = -1;
            float sig = p.sigma_user;
            if (!(sig > 0.f)) sig = p.stats[s].sigma;
            if (!(sig > 0.f)) sig = 1.f;
            const LaneBins<St> B{st, wcn_cta, (size_t)ppc, over};
            if (nstreams == 1) {
                if (kvalid) box_search<kR>(B, nbins, p.w_min, p.w_max, sig, sc, bs, bw);
            } else {
                // the streams of a period group walk every nstreams-th block of starts of the
                // lanes' profiles; their winners meet in the idle tile buffer, and stream 0
                // keeps the best by the walk's rule and re-evaluates it
                float bv = -INFINITY;
                int bkey = 0x7fffffff;
                if (kvalid) box_search_part<kR>(B, nbins, p.w_min, p.w_max, sw * kR, nstreams * kR, bv, bkey);
                float2 *M = reinterpret_cast<float2 *>(tl_buf);  // [nstreams][ppc]
                M[sw * ppc + gw * 32 + lane] = make_float2(bv, __int_as_float(bkey));
                fold_sync();
                if (sw == 0) {
                    for (int r = 1; r < nstreams; ++r) {
                        const float2 m = M[r * ppc + gw * 32 + lane];
                        const int key = __float_as_int(m.y);
                        const bool take = (m.x > bv) | ((m.x == bv) & (key < bkey));
                        bv = take ? m.x : bv;
                        bkey = take ? key : bkey;
                    }
                    if (kvalid && bkey != 0x7fffffff) {
                        bw = bkey >> 12;
                        bs = bkey & 4095;
                        sc = box_reeval(B, nbins, bs, bw, sig);
                    }
                }
                fold_sync();  // the merge area is free before the next task's tiles
            }
            if (sw == 0) {
                if (kvalid) {
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
    if (MODE == kModeSearch && sw == 0) {
        // all tasks published: score whatever rows are left, then leave
        for (;;) {
            int t = 0;
            if (lane == 0) t = take_ticket(&sh.ticket, my_tasks * ppc);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t < 0) break;
            __threadfence_block();
            score_ticket(p, sh, t, ppc, Bw, lane, cur_s, cur_key);
        }
        if (lane == 0 && p.best_key && cur_key) atomicMax(&p.best_key[cur_s], cur_key);
    }
    if (MODE == kModeFold && p.slot_k) {
        // slots of tasks in this launch's range that lie past the device task count
        const int64_t t0 = task_end > p.task_begin ? task_end : p.task_begin;
        for (int64_t task = t0 + blockIdx.x; task < p.ntasks && (int)threadIdx.x < ppc; task += gridDim.x)
            p.slot_k[(task - p.task_begin) * ppc + threadIdx.x] = -1;
    }
}

template <int MODE, bool POW2, int LAYOUT, int MAXW>
static cudaError_t set_smem_attr()
{
    return cudaFuncSetAttribute(fold_kernel<MODE, POW2, LAYOUT, MAXW>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kSmemLimit - 1024));
}

template <int MODE, bool POW2>
static cudaError_t set_smem_attr_all()
{
    cudaError_t e = set_smem_attr<MODE, POW2, kLayoutPaired16, 4>();
    if (e == cudaSuccess) e = set_smem_attr<MODE, POW2, kLayoutPaired16, kMaxFoldWarps>();
    if (e == cudaSuccess) e = set_smem_attr<MODE, POW2, kLayoutPacked64, 4>();
    if (e == cudaSuccess) e = set_smem_attr<MODE, POW2, kLayoutPacked64, kMaxFoldWarps>();
    if (e == cudaSuccess) e = set_smem_attr<MODE, POW2, kLayoutRed32, 4>();
    if (e == cudaSuccess) e = set_smem_attr<MODE, POW2, kLayoutRed32, kMaxRedWarps>();
    return e;
}

cudaError_t box_coop_register();

int fold_register_kernels()
{
    cudaError_t e = box_coop_register();
    if (e == cudaSuccess) e = set_smem_attr<kModeSearch, true, kLayoutPacked64, 4>();
    if (e == cudaSuccess) e = set_smem_attr<kModeSearch, false, kLayoutPacked64, 4>();
    if (e == cudaSuccess) e = set_smem_attr<kModeSearch, true, kLayoutPaired16, 4>();
    if (e == cudaSuccess) e = set_smem_attr<kModeSearch, false, kLayoutPaired16, 4>();
    if (e == cudaSuccess) e = set_smem_attr<kModeSearch, true, kLayoutRed32, kMaxRedWarps>();
    if (e == cudaSuccess) e = set_smem_attr<kModeSearch, false, kLayoutRed32, kMaxRedWarps>();
    if (e == cudaSuccess) e = set_smem_attr_all<kModeFold, true>();
    if (e == cudaSuccess) e = set_smem_attr_all<kModeFold, false>();
    if (e == cudaSuccess) e = set_smem_attr_all<kModeBox, true>();
    if (e == cudaSuccess) e = set_smem_attr_all<kModeBox, false>();
    return (int)e;
}

size_t fold_smem_bytes(int nbins, int warps, int layout, int tile)
{
    const size_t nb2 = (size_t)((nbins + 1) & ~1);
    const size_t per_warp = layout == kLayoutPaired16 ? (size_t)32 * (nbins * 4 + nb2 * 2) : (size_t)32 * nbins * 8;
    // tile bytes per sample (and the reduction layout's high word per 16 samples)
    const size_t per_sample = layout == kLayoutRed32 ? 8 : 12;
    const size_t per_group = layout == kLayoutRed32 ? 4 : 0;
    return 128 + (size_t)2 * tile * per_sample + 2 * (tile / 16) * (1 + per_group) + (size_t)warps * per_warp;
}

int fold_max_warps(int nbins, int layout, int tile)
{
    int w = layout == kLayoutRed32 ? kMaxRedWarps : kMaxFoldWarps;
    while (w > 1 && fold_smem_bytes(nbins, w, layout, tile) > kSmemLimit - 1024) --w;
    return fold_smem_bytes(nbins, w, layout, tile) <= kSmemLimit - 1024 ? w : 0;
}

// Resident blocks per SM of a fold launch (0 if it does not fit).
template <int MODE, bool POW2, int LAYOUT, int MAXW>
static int occupancy_of(int threads, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fold_kernel<MODE, POW2, LAYOUT, MAXW>, threads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int search_blocks_per_sm(int nbins, int warps, int layout, int tile, int streams)
{
    const size_t smem = search_smem_bytes(nbins, warps, layout, tile, streams);
    if (smem == 0) return 0;
    const int threads = 32 * (warps * streams + 1);
    if (layout == kLayoutRed32) return occupancy_of<kModeSearch, true, kLayoutRed32, kMaxRedWarps>(threads, smem);
    return layout == kLayoutPacked64 ? occupancy_of<kModeSearch, true, kLayoutPacked64, 4>(threads, smem)
                                     : occupancy_of<kModeSearch, true, kLayoutPaired16, 4>(threads, smem);
}

int fold_blocks_per_sm(int nbins, int warps, int layout, int tile, int streams)
{
    const size_t smem = fold_smem_bytes(nbins, warps, layout, tile);
    if (smem > kSmemLimit - 1024) return 0;
    if (streams > 1 && (layout != kLayoutRed32 || warps * streams > kMaxRedWarps)) return 0;
    const int threads = 32 * warps * streams;
    if (layout == kLayoutPacked64)
        return warps <= 4 ? occupancy_of<kModeFold, true, kLayoutPacked64, 4>(threads, smem)
                          : occupancy_of<kModeFold, true, kLayoutPacked64, kMaxFoldWarps>(threads, smem);
    if (layout == kLayoutRed32)
        return warps * streams <= 4 ? occupancy_of<kModeFold, true, kLayoutRed32, 4>(threads, smem)
                                    : occupancy_of<kModeFold, true, kLayoutRed32, kMaxRedWarps>(threads, smem);
    return warps <= 4 ? occupancy_of<kModeFold, true, kLayoutPaired16, 4>(threads, smem)
                      : occupancy_of<kModeFold, true, kLayoutPaired16, kMaxFoldWarps>(threads, smem);
}

// Blocks of up to 4 warps use the instantiation with a 255-register budget (the 16-sample
// groups keep many values live); wider blocks the one capped at 128 registers.
template <int MODE, bool POW2>
static void launch_variant(const FoldParams &p, int grid, int threads, size_t smem, cudaStream_t st)
{
    if (p.layout == kLayoutPacked64) {
        if (p.warps <= 4) fold_kernel<MODE, POW2, kLayoutPacked64, 4><<<grid, threads, smem, st>>>(p);
        else fold_kernel<MODE, POW2, kLayoutPacked64, kMaxFoldWarps><<<grid, threads, smem, st>>>(p);
    } else if (p.layout == kLayoutRed32) {
        if (threads <= 128) fold_kernel<MODE, POW2, kLayoutRed32, 4><<<grid, threads, smem, st>>>(p);
        else fold_kernel<MODE, POW2, kLayoutRed32, kMaxRedWarps><<<grid, threads, smem, st>>>(p);
    } else {
        if (p.warps <= 4) fold_kernel<MODE, POW2, kLayoutPaired16, 4><<<grid, threads, smem, st>>>(p);
        else fold_kernel<MODE, POW2, kLayoutPaired16, kMaxFoldWarps><<<grid, threads, smem, st>>>(p);
    }
}

size_t search_smem_bytes(int nbins, int warps, int layout, int tile, int streams)
{
    if (streams < 1 || (streams > 1 && layout != kLayoutRed32)) return 0;
    if (warps * streams + 1 > (layout == kLayoutRed32 ? kMaxRedWarps : 4)) return 0;
    const size_t off = (fold_smem_bytes(nbins, warps, layout, tile) + 15) & ~(size_t)15;
    const size_t bytes = off + (size_t)(warps + 1) * coop_pairs(nbins) * sizeof(float2);
    return bytes <= kSmemLimit - 1024 ? bytes : 0;
}

// One fold block of `warps` warps plus the scorer warp (the 128-thread instantiation, or
// up to kMaxRedWarps warps for the reduction layout).
template <bool POW2>
static void launch_search_variant(const FoldParams &p, int grid, size_t smem, cudaStream_t st)
{
    const int threads = 32 * (p.warps * p.streams + 1);
    if (p.layout == kLayoutPacked64) fold_kernel<kModeSearch, POW2, kLayoutPacked64, 4><<<grid, threads, smem, st>>>(p);
    else if (p.layout == kLayoutRed32)
        fold_kernel<kModeSearch, POW2, kLayoutRed32, kMaxRedWarps><<<grid, threads, smem, st>>>(p);
    else fold_kernel<kModeSearch, POW2, kLayoutPaired16, 4><<<grid, threads, smem, st>>>(p);
}

cudaError_t launch_fold(const FoldParams &p_in, int mode, int grid, cudaStream_t st)
{
    FoldParams p = p_in;
    // the epilogue search of several streams merges through the tile buffer: it needs
    // nstreams x periods-per-block (v, key) pairs there
    if (mode == kModeBox && (size_t)p.streams * 32 * p.warps * 8 > (size_t)p.tile * 8) p.streams = 1;
    if (p.tile != 512 && p.tile != 1024 && p.tile != 2048) return cudaErrorInvalidValue;
    if (p.streams < 1 || (p.streams > 1 && p.layout != kLayoutRed32)) return cudaErrorInvalidValue;
    if (mode == kModeSearch) {
        const size_t smem = search_smem_bytes(p.nbins, p.warps, p.layout, p.tile, p.streams);
        if (smem == 0 || !p.sums || !p.counts || !p.slot_k || !p.score) return cudaErrorInvalidValue;
        FoldParams q = p;
        q.stage_off = (fold_smem_bytes(p.nbins, p.warps, p.layout, p.tile) + 15) & ~(size_t)15;
        if (q.shift >= 0) launch_search_variant<true>(q, grid, smem, st);
        else launch_search_variant<false>(q, grid, smem, st);
        return cudaGetLastError();
    }
    const size_t smem = fold_smem_bytes(p.nbins, p.warps, p.layout, p.tile);
    if (smem > kSmemLimit - 1024 || (p.layout == kLayoutRed32 && p.warps * p.streams > kMaxRedWarps))
        return cudaErrorInvalidValue;
    const int threads = 32 * p.warps * p.streams;
    const bool pow2 = p.shift >= 0;
    if (mode == kModeFold) {
        if (pow2) launch_variant<kModeFold, true>(p, grid, threads, smem, st);
        else launch_variant<kModeFold, false>(p, grid, threads, smem, st);
    } else if (mode == kModeBox) {
        if (pow2) launch_variant<kModeBox, true>(p, grid, threads, smem, st);
        else launch_variant<kModeBox, false>(p, grid, threads, smem, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kCoopWarps * 32, 2) box_coop_kernel(const BoxCoopParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    float2 *Bw = reinterpret_cast<float2 *>(smem) + (size_t)warp * coop_pairs(p.nbins);
    int cur_s = -1;
    unsigned long long cur_key = 0ull;
    for (int64_t r = (int64_t)blockIdx.x * nw + warp; r < p.rows; r += (int64_t)gridDim.x * nw) {
        const int64_t k = p.slot_k ? p.slot_k[r] : p.k_begin + r;
        if (k >= 0) score_row(p, r, k, Bw, lane, cur_s, cur_key);
    }
    if (lane == 0 && p.best_key && cur_key) atomicMax(&p.best_key[cur_s], cur_key);
}

// Warps per block of the scorer: 8, fewer when 8 profiles do not fit shared memory.
int box_coop_warps(int nbins)
{
    int w = kCoopWarps;
    while (w > 1 && (size_t)w * coop_pairs(nbins) * sizeof(float2) > kSmemLimit - 1024) --w;
    return w;
}

size_t box_coop_smem(int nbins) { return (size_t)box_coop_warps(nbins) * coop_pairs(nbins) * sizeof(float2); }

cudaError_t box_coop_register()
{
    return cudaFuncSetAttribute(box_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kSmemLimit - 1024));
}

cudaError_t launch_box_coop(const BoxCoopParams &p, int num_sms, cudaStream_t st)
{
    if (p.rows <= 0) return cudaSuccess;
    const size_t smem = box_coop_smem(p.nbins);
    if (smem > kSmemLimit - 1024) return cudaErrorInvalidValue;
    const int warps = box_coop_warps(p.nbins);
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, box_coop_kernel, warps * 32, smem);
    if (e != cudaSuccess) return e;
    const int64_t want = (p.rows + warps - 1) / warps;
    const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms * std::max(1, occ));
    box_coop_kernel<<<grid, warps * 32, smem, st>>>(p);
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

// ------------------------------------------------------------------ bounded-wait self-test

// One thread waits on an mbarrier that nothing arrives on, with a cycle limit, the way
// every wait of the kernels above is bounded; when the limit passes it latches the
// timeout bit and returns.
__global__ void wait_selftest_kernel(long long limit, uint32_t *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0u, limit)) report_error(status, kErrTimeout);
}

cudaError_t launch_wait_selftest(long long limit, uint32_t *status, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched search plan

constexpr int kPlanThreads = 1024;

// Inclusive block scan (Hillis-Steele) of one value per thread, with op = max or +.
template <bool MAX>
__device__ int64_t block_scan(int64_t v, int64_t *buf)
{
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        const int64_t u = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : (MAX ? INT64_MIN : 0);
        __syncthreads();
        v = MAX ? (u > v ? u : v) : v + u;
        buf[threadIdx.x] = v;
        __syncthreads();
    }
    return v;
}

// Monotone copy of the offsets off[0..S] clamped to [0, total], with 0 first and total
// last: o'[i] = max(0, max_{j <= i} min(off[j], total)). Returns true if o' == off.
__device__ bool sanitise_offsets(const int64_t *off, int S, int64_t total, int64_t *out, int64_t *buf)
{
    const int per = (S + 1 + kPlanThreads - 1) / kPlanThreads;
    const int a = threadIdx.x * per, b = min(S + 1, a + per);
    int64_t m = 0;
    for (int i = a; i < b; ++i) {
        const int64_t v = min(off[i], total);
        m = v > m ? v : m;
    }
    const int64_t incl = block_scan<true>(m, buf);
    int64_t run = threadIdx.x > 0 ? buf[threadIdx.x - 1] : 0;
    run = run > 0 ? run : 0;
    __syncthreads();
    bool same = true;
    for (int i = a; i < b; ++i) {
        const int64_t v = min(off[i], total);
        run = v > run ? v : run;
        int64_t o = i == 0 ? 0 : run;
        if (i == S) o = total;
        same &= o == off[i];
        out[i] = o;
    }
    (void)incl;
    return __syncthreads_and(same);
}

// Validated star offsets and the first fold task of every star (ceil(grid length /
// ppc) tasks each); task_off[S] is the total. One block of kPlanThreads threads.
__global__ void __launch_bounds__(kPlanThreads) batch_plan_kernel(const int64_t *lc_off, const int64_t *grid_off,
                                                                   int S, int64_t n_total, int64_t np_total, int ppc,
                                                                   int64_t *lc_s, int64_t *grid_s, int64_t *task_off,
                                                                   uint32_t *status)
{
    __shared__ int64_t buf[kPlanThreads];
    bool ok = sanitise_offsets(lc_off, S, n_total, lc_s, buf);
    ok &= sanitise_offsets(grid_off, S, np_total, grid_s, buf);
    __syncthreads();
    const int per = (S + kPlanThreads - 1) / kPlanThreads;
    const int a = threadIdx.x * per, b = min(S, a + per);
    int64_t t = 0;
    bool good = true;
    for (int i = a; i < b; ++i) {
        const int64_t len = lc_s[i + 1] - lc_s[i], np = grid_s[i + 1] - grid_s[i];
        good &= len >= 1 && len <= ((int64_t)1 << 24) && np >= 1 && np <= (int64_t)INT32_MAX;
        t += (np + ppc - 1) / ppc;
    }
    const int64_t incl = block_scan<false>(t, buf);
    int64_t run = incl - t;
    for (int i = a; i < b; ++i) {
        task_off[i] = run;
        run += (grid_s[i + 1] - grid_s[i] + ppc - 1) / ppc;
    }
    if (threadIdx.x == kPlanThreads - 1) task_off[S] = incl;
    ok &= __syncthreads_and(good);
    if (!ok && threadIdx.x == 0) report_error(status, kErrArgs);
}

cudaError_t launch_batch_plan(const int64_t *lc_off, const int64_t *grid_off, int nstars, int64_t n_total,
                              int64_t np_total, int ppc, int64_t *lc_s, int64_t *grid_s, int64_t *task_off,
                              uint32_t *status, cudaStream_t st)
{
    batch_plan_kernel<<<1, kPlanThreads, 0, st>>>(lc_off, grid_off, nstars, n_total, np_total, ppc, lc_s, grid_s,
                                                  task_off, status);
    return cudaGetLastError();
}

// Per-star argmax key over score[grid_off[s] .. grid_off[s+1]) with the star-local index;
// one block per star at a time.
__global__ void argmax_segmented_kernel(const float *__restrict__ score, const int64_t *grid_off, int S,
                                        unsigned long long *key)
{
    __shared__ unsigned long long red[8];
    for (int s = blockIdx.x; s < S; s += gridDim.x) {
        const int64_t gb = grid_off[s], ge = grid_off[s + 1];
        unsigned long long best = 0ull;
        for (int64_t k = gb + threadIdx.x; k < ge; k += blockDim.x) {
            const unsigned long long v = argmax_key(score[k], k - gb);
            best = v > best ? v : best;
        }
        best = warp_max_u64(best);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0ull;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
            key[s] = m;
        }
        __syncthreads();
    }
}

cudaError_t launch_argmax_segmented(const float *score, const int64_t *grid_off, int nstars,
                                    unsigned long long *key, int num_sms, cudaStream_t st)
{
    const int grid = nstars < num_sms * 8 ? nstars : num_sms * 8;
    argmax_segmented_kernel<<<grid, 256, 0, st>>>(score, grid_off, nstars, key);
    return cudaGetLastError();
}

cudaError_t launch_argmax_finalize(const unsigned long long *key, int nstars, int64_t *best_index,
                                   float *best_score, cudaStream_t st)
{
    argmax_finalize_kernel<<<(nstars + 127) / 128, 128, 0, st>>>(key, nstars, best_index, best_score);
    return cudaGetLastError();
}

}  // namespace gpfc
