// twotier.cu -- the paper's two-tier equal-count fold (Sec. 2.3, Fig. 4 (a)-(e)).
//
// Step 1-3: every sample goes to one of nfine equal-width fine bins by its fixed-point
// phase (the bins of fold.cu); each fine bin keeps its sample count and flux sum.
// Step 4: the fine bins are merged left to right into nbins final bins holding exactly
// n / nbins samples each; the fine bin that straddles a boundary gives each side the
// share of its flux sum that it gives of its samples. In units of 1 / nbins sample,
// final bin j covers [j n, (j+1) n) and fine bin f covers [C(f-1) nbins, C(f) nbins),
// with C the cumulative count, so bin j's sum is G((j+1) n) - G(j n) with
//     G(u) = S(f-1) + s_f (u - C(f-1) nbins) / (c_f nbins),   C(f-1) nbins < u <= C(f) nbins,
// S the cumulative flux sum.
// Step 5: mean = f_ref + sum / (n / nbins).
// With width_only set the kernel stops after step 3 and returns the fine bins themselves
// (count, sum, mean): the equal-width fold for bin counts above the lane-private fold's.
//
// Design. A fine bin is one 64-bit word, count << 40 plus the flux sum (flux - f_ref) in
// signed fixed point with a per-star quantum 2^-k, chosen so that n max|x| 2^k < 2^38:
// no sum, prefix sum or count can overflow its field, every addition is exact, and the
// fold is a single 64-bit shared-memory atomic add per sample and period, deterministic
// whatever the order. Up to 65,536 samples the fold is instead two 32-bit shared-memory
// reductions per sample and period (several times the 64-bit atomics' rate), into a row of
// 32-bit sums and a row of counts per period, with k the largest such that
// |rint(x 2^k)| <= floor((2^31 - 1) / n): still exact, at 2^31 / n levels of max|x| instead
// of 2^38 / n; the rows are then packed into the same 64-bit words. A block folds up to kEqMaxPeriods periods at a time (4096 fine
// bins x 6 periods = 192 KB of shared memory), scans each period's fine bins (exact
// integer prefix sums), and evaluates G at the boundaries by binary search on the
// cumulative counts.
#include <cmath>
#include <cstdint>

#include "gpfc_common.cuh"
#include "gpfc_kernels.h"
#include "gpfc_twotier.h"

namespace gpfc {

constexpr int kEqThreads = 512;
constexpr int kCountShift = 40;

__device__ __forceinline__ int64_t eq_count(unsigned long long P)
{
    return (int64_t)((P + (1ull << (kCountShift - 1))) >> kCountShift);
}
__device__ __forceinline__ int64_t eq_sum(unsigned long long P)
{
    return (int64_t)(P - ((unsigned long long)eq_count(P) << kCountShift));
}

// Word of fine bin f in a period's row: the low 4 bits of f XORed with bits 4-7 (rows of
// a multiple of 16 bins), so lanes whose bins are a regular stride apart spread over the
// banks instead of piling onto a few.
__device__ __forceinline__ int eq_word(int f, bool swz) { return swz ? f ^ ((f >> 4) & 15) : f; }

// max |x| over the star (as float bits: order-preserving for values >= 0)
__global__ void eq_absmax_kernel(const float *__restrict__ x, int64_t n, unsigned int *maxbits)
{
    unsigned int m = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(x[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxbits, m);
}

// Quantum exponent k, and q_i = rint(x_i 2^k). 64-bit words: n max|x| 2^k < 2^38. 32-bit
// reductions (eq_red32(n)): the largest k with max|x| 2^k <= floor((2^31 - 1) / n), so every
// |q_i| is at most that bound and no bin sum of n samples leaves 32 bits.
__device__ __forceinline__ int eq_scale(unsigned int maxbits, int64_t n)
{
    const float m = __uint_as_float(maxbits);
    if (!(m > 0.f) || !isfinite(m)) return 0;
    if (eq_red32(n)) {
        const double lim = floor(2147483647.0 / (double)n), xm = (double)m;
        int k = ilogb(lim) - ilogb(xm);
        k = max(-200, min(200, k));
        while (k < 200 && ldexp(xm, k + 1) <= lim) ++k;
        while (k > -200 && ldexp(xm, k) > lim) --k;
        return k;
    }
    int e = 0;
    frexp((double)m * (double)n, &e);  // m n < 2^e
    const int k = 38 - e;
    return k > 60 ? 60 : k;
}

__global__ void eq_quant_kernel(const float *__restrict__ x, int64_t n, const unsigned int *maxbits,
                                long long *__restrict__ q, int *kout)
{
    const int k = eq_scale(*maxbits, n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *kout = k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = __double2ll_rn(scalbn((double)x[i], k));
}

// Inclusive block scan of one 64-bit value per thread (kEqThreads threads).
__device__ __forceinline__ unsigned long long eq_block_scan(unsigned long long v, unsigned long long *warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < kEqThreads / 32 ? warp_tot[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < kEqThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const unsigned long long before = warp > 0 ? warp_tot[warp - 1] : 0ull;
    __syncthreads();
    return v + before;
}

template <bool POW2, bool RED32>
__global__ void __launch_bounds__(kEqThreads, 1) eq_fold_kernel(const EqParams p)
{
    extern __shared__ __align__(16) unsigned long long bins[];  // [ppb][nfine]
    __shared__ unsigned long long warp_tot[kEqThreads / 32];
    __shared__ uint32_t sF[2 * kEqMaxPeriods];
    const int nfine = p.nfine, nbins = p.nbins, ppb = p.ppb;
    const int k = *p.kscale;
    const double quantum = scalbn(1.0, -k);
    const double f_ref = p.stats->f_ref;
    const int64_t n = p.n;
    const int per_thread = (nfine + kEqThreads - 1) / kEqThreads;
    const bool swz = (nfine & 15) == 0;
    const int64_t ngroups = (p.np + ppb - 1) / ppb;

    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t k0 = grp * ppb;
        const int nper = (int)min((int64_t)ppb, p.np - k0);
        for (int i = threadIdx.x; i < ppb * nfine; i += kEqThreads) bins[i] = 0ull;
        if (threadIdx.x < nper) {
            const double P = p.periods[k0 + threadIdx.x];
            const double qv = 1099511627776.0 / P;
            unsigned long long F = 0ull;
            if (P > 0.0 && P < INFINITY && qv < 9223372036854775808.0) F = (unsigned long long)__double2ll_rn(qv);
            else report_error(p.status, kErrRange);
            sF[2 * threadIdx.x] = (uint32_t)F;
            sF[2 * threadIdx.x + 1] = (uint32_t)(F >> 32);
        }
        __syncthreads();
        uint32_t Fl[kEqMaxPeriods], Fh[kEqMaxPeriods];
#pragma unroll
        for (int pp = 0; pp < kEqMaxPeriods; ++pp) {
            Fl[pp] = pp < nper ? sF[2 * pp] : 0u;
            Fh[pp] = pp < nper ? sF[2 * pp + 1] : 0u;
        }
        // steps 1-3: fine bins, one 64-bit atomic add per sample and period, or (RED32) two
        // 32-bit reductions into the period's sum row and count row (2 nfine words)
        const uint32_t rows = smem_u32(bins);
        // each thread's next sample is loaded while the current one is folded (the loads
        // come from L2; their latency would otherwise stall every iteration)
        uint32_t ntl = 0u, nth = 0u;
        long long nq = 0;
        if (threadIdx.x < n) {
            ntl = p.tau_lo[threadIdx.x];
            nth = (uint32_t)p.tau_hi[threadIdx.x];
            nq = p.q[threadIdx.x];
        }
        for (int64_t i = threadIdx.x; i < n; i += kEqThreads) {
            const uint32_t tl = ntl;
            const uint32_t th = nth;
            const unsigned long long v = (1ull << kCountShift) + (unsigned long long)nq;
            if (i + kEqThreads < n) {
                ntl = p.tau_lo[i + kEqThreads];
                nth = (uint32_t)p.tau_hi[i + kEqThreads];
                nq = p.q[i + kEqThreads];
            }
#pragma unroll
            for (int pp = 0; pp < kEqMaxPeriods; ++pp) {
                if (pp < nper) {
                    const uint32_t hi = __umulhi(tl, Fl[pp]) + th * Fl[pp] + tl * Fh[pp];
                    uint32_t f;
                    if (POW2) {
                        f = hi >> p.fshift;
                    } else {
                        const uint32_t lo = tl * Fl[pp];
                        f = (uint32_t)(((unsigned long long)hi * (uint32_t)nfine +
                                        (unsigned long long)__umulhi(lo, (uint32_t)nfine)) >> 32);
                    }
                    if (RED32) {
                        const uint32_t a = rows + 4u * (uint32_t)(2 * pp * nfine + eq_word((int)f, swz));
                        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"((uint32_t)v) : "memory");
                        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a + 4u * (uint32_t)nfine), "r"(1u) : "memory");
                    } else {
                        atomicAdd(&bins[pp * nfine + eq_word((int)f, swz)], v);
                    }
                }
            }
        }
        __syncthreads();
        if (RED32) {
            // each period's rows (32-bit sums, then counts) become its 64-bit words
            // count << 40 plus the sum, in place: all of a period's reads come before a
            // barrier and its writes after it
            constexpr int kPer = kEqMaxFine / kEqThreads;
            for (int pp = 0; pp < nper; ++pp) {
                const uint32_t *R = reinterpret_cast<const uint32_t *>(bins + (size_t)pp * nfine);
                unsigned long long w[kPer];
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    const int f = threadIdx.x + u * kEqThreads;
                    w[u] = f < nfine ? ((unsigned long long)R[nfine + f] << kCountShift) +
                                           (unsigned long long)(long long)(int32_t)R[f]
                                     : 0ull;
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    const int f = threadIdx.x + u * kEqThreads;
                    if (f < nfine) bins[(size_t)pp * nfine + f] = w[u];
                }
            }
            __syncthreads();
        }
        if (p.width_only) {
            // the fine bins are the result: counts, exact sums rounded once, means
            for (int idx = threadIdx.x; idx < nper * nfine; idx += kEqThreads) {
                const int pp = idx / nfine, f = idx - pp * nfine;
                const unsigned long long w = bins[pp * nfine + eq_word(f, swz)];
                const int64_t c = eq_count(w);
                const double S = (double)eq_sum(w) * quantum;
                const size_t o = (size_t)(k0 + pp) * nfine + f;
                if (p.folded) p.folded[o] = c ? (float)(f_ref + S / (double)c) : __int_as_float(0x7fc00000);
                if (p.counts) p.counts[o] = (int32_t)c;
                if (p.sums) p.sums[o] = (float)S;
            }
            __syncthreads();
            continue;
        }
        // step 4a: inclusive prefix sums of each period's fine bins (exact integers)
        for (int pp = 0; pp < nper; ++pp) {
            unsigned long long *B = bins + (size_t)pp * nfine;
            const int f0 = threadIdx.x * per_thread;
            unsigned long long loc = 0ull;
            for (int f = f0; f < min(nfine, f0 + per_thread); ++f) loc += B[eq_word(f, swz)];
            const unsigned long long incl = eq_block_scan(loc, warp_tot);
            unsigned long long run = incl - loc;
            for (int f = f0; f < min(nfine, f0 + per_thread); ++f) {
                run += B[eq_word(f, swz)];
                B[eq_word(f, swz)] = run;
            }
            __syncthreads();
        }
        // step 4b + 5: each final bin from G at its two boundaries
        for (int idx = threadIdx.x; idx < nper * nbins; idx += kEqThreads) {
            const int pp = idx / nbins, j = idx - pp * nbins;
            const unsigned long long *B = bins + (size_t)pp * nfine;
            int64_t whole[2];
            double part[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int64_t u = (int64_t)(j + side) * n;  // boundary in units of 1/nbins sample
                whole[side] = 0;
                part[side] = 0.0;
                if (u == 0) continue;
                // smallest f with C(f) nbins >= u
                int lo = 0, hi = nfine - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (eq_count(B[eq_word(mid, swz)]) * nbins >= u) hi = mid;
                    else lo = mid + 1;
                }
                const unsigned long long Pp = lo > 0 ? B[eq_word(lo - 1, swz)] : 0ull;
                const int64_t Cp = eq_count(Pp), Sp = eq_sum(Pp);
                const int64_t cf = eq_count(B[eq_word(lo, swz)]) - Cp, sf = eq_sum(B[eq_word(lo, swz)]) - Sp;
                whole[side] = Sp;
                part[side] = (double)sf * ((double)(u - Cp * nbins) / ((double)cf * nbins));
            }
            const double sum = (double)(whole[1] - whole[0]) + (part[1] - part[0]);
            p.folded[(size_t)(k0 + pp) * nbins + j] = (float)(f_ref + sum * quantum * ((double)nbins / (double)n));
        }
        __syncthreads();
    }
}

size_t eq_smem_bytes(int nfine, int ppb) { return (size_t)nfine * ppb * sizeof(unsigned long long); }

int eq_periods_per_block(int nfine)
{
    int ppb = kEqMaxPeriods;
    while (ppb > 1 && eq_smem_bytes(nfine, ppb) > kSmemLimit - 4096) --ppb;
    return eq_smem_bytes(nfine, ppb) <= kSmemLimit - 4096 ? ppb : 0;
}

cudaError_t launch_eq_prep(const float *x, int64_t n, unsigned int *maxbits, long long *q, int *kscale,
                           int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < (int64_t)num_sms * 4 ? want : (int64_t)num_sms * 4);
    eq_absmax_kernel<<<grid, 256, 0, st>>>(x, n, maxbits);
    eq_quant_kernel<<<grid, 256, 0, st>>>(x, n, maxbits, q, kscale);
    return cudaGetLastError();
}

cudaError_t launch_eq_fold(const EqParams &p, int num_sms, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        const int lim = (int)(kSmemLimit - 4096);
        cudaError_t e = cudaFuncSetAttribute(eq_fold_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(eq_fold_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(eq_fold_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(eq_fold_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t smem = eq_smem_bytes(p.nfine, p.ppb);
    if (p.ppb < 1 || p.ppb > kEqMaxPeriods || smem > kSmemLimit - 4096) return cudaErrorInvalidValue;
    const int64_t ngroups = (p.np + p.ppb - 1) / p.ppb;
    const int grid = (int)(ngroups < (int64_t)num_sms ? ngroups : (int64_t)num_sms);
    if (p.red32 != (int)eq_red32(p.n)) return cudaErrorInvalidValue;  // must match the quantum of the prep
    if (p.red32) {
        if (p.fshift >= 0) eq_fold_kernel<true, true><<<grid, kEqThreads, smem, st>>>(p);
        else eq_fold_kernel<false, true><<<grid, kEqThreads, smem, st>>>(p);
    } else {
        if (p.fshift >= 0) eq_fold_kernel<true, false><<<grid, kEqThreads, smem, st>>>(p);
        else eq_fold_kernel<false, false><<<grid, kEqThreads, smem, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace gpfc
