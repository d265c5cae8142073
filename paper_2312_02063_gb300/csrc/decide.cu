// decide.cu -- per-star decision over a periodogram of scores.
//
// For each star's scores (one per trial period): mean and population standard deviation
// of the finite scores; SDE = (max - mean) / sd (Eq. 3; 0 when sd is 0); peaks as in
// Sec. 4.2: maximal runs of consecutive periods scoring above mean + k_sigma sd that are
// at least min_width periods wide, each with its height (largest score, first occurrence);
// the best peak (highest, ties to the smaller index) and the highest max_peaks peaks,
// each flagged against the best peak's period for harmonics (Fig. 14 notes them): 1 for
// the best, +m if P = m Pb, -m if P = Pb / m (m = 2..4), else 0.
//
// One block of kPkThreads threads per star. Statistics are FP64 block reductions. For the
// runs, thread t owns the runs that start in its contiguous chunk of periods and follows
// a run past the chunk's end until it closes; qualifying runs go to a shared candidate
// list (the first kPkCap of them; the best peak and the count are exact in any case).
#include <cmath>
#include <cstdint>

#include "gpfc_common.cuh"
#include "gpfc_decide.h"

namespace gpfc {

constexpr int kPkThreads = 1024;
constexpr int kPkCap = 2048;

template <class T>
__device__ __forceinline__ T pk_block_sum(T v, T *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = 0;
    for (int w = 0; w < kPkThreads / 32; ++w) t += red[w];
    return t;
}

__device__ __forceinline__ unsigned long long pk_block_max(unsigned long long v, unsigned long long *red)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long t = 0ull;
    for (int w = 0; w < kPkThreads / 32; ++w) t = red[w] > t ? red[w] : t;
    return t;
}

__device__ __forceinline__ float key_value(unsigned long long key)
{
    const uint32_t ord = (uint32_t)(key >> 32);
    const uint32_t u = (ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord;
    return __uint_as_float(u);
}
__device__ __forceinline__ int64_t key_index(unsigned long long key)
{
    return (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
}

__global__ void __launch_bounds__(kPkThreads) peaks_kernel(const PeakParams p)
{
    __shared__ double red_d[kPkThreads / 32];
    __shared__ float red_f[kPkThreads / 32];
    __shared__ int red_i[kPkThreads / 32];
    __shared__ unsigned long long red_k[kPkThreads / 32];
    __shared__ float c_h[kPkCap];
    __shared__ int c_i[kPkCap];
    __shared__ int c_w[kPkCap];
    __shared__ int c_n;
    for (int s = blockIdx.x; s < p.nstars; s += gridDim.x) {
        const int64_t gb = p.grid_off ? p.grid_off[s] : 0, ge = p.grid_off ? p.grid_off[s + 1] : p.np;
        const float *sc = p.score + gb;
        const int64_t len = ge - gb;
        if (threadIdx.x == 0) c_n = 0;
        // statistics of the finite scores
        double sum = 0.0;
        int cnt = 0;
        for (int64_t k = threadIdx.x; k < len; k += kPkThreads)
            if (isfinite(sc[k])) {
                sum += (double)sc[k];
                ++cnt;
            }
        sum = pk_block_sum(sum, red_d);
        const int ntot = pk_block_sum(cnt, red_i);
        const double mean = ntot > 0 ? sum / (double)ntot : NAN;
        double ss = 0.0;
        float mx = -INFINITY;
        for (int64_t k = threadIdx.x; k < len; k += kPkThreads)
            if (isfinite(sc[k])) {
                const double d = (double)sc[k] - mean;
                ss += d * d;
                mx = fmaxf(mx, sc[k]);
            }
        ss = pk_block_sum(ss, red_d);
        {
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            __syncthreads();
            if ((threadIdx.x & 31) == 0) red_f[threadIdx.x >> 5] = mx;
            __syncthreads();
            for (int w = 0; w < kPkThreads / 32; ++w) mx = fmaxf(mx, red_f[w]);
        }
        const double sd = ntot > 0 ? sqrt(ss / (double)ntot) : NAN;
        const double thr = mean + p.k_sigma * sd;
        auto above = [&](int64_t k) { return isfinite(sc[k]) && (double)sc[k] > thr; };
        // runs starting in this thread's chunk
        const int64_t chunk = (len + kPkThreads - 1) / kPkThreads;
        const int64_t a = (int64_t)threadIdx.x * chunk, b = min(len, a + chunk);
        int64_t i = a;
        if (i < b && i > 0 && above(i - 1))  // the run through a started in an earlier chunk
            while (i < len && above(i)) ++i;
        unsigned long long best = 0ull;
        int nq = 0;
        while (i < b) {
            if (!above(i)) {
                ++i;
                continue;
            }
            int64_t e = i, arg = i;
            while (e < len && above(e)) {
                if (sc[e] > sc[arg]) arg = e;
                ++e;
            }
            if (e - i >= p.min_width) {
                ++nq;
                const unsigned long long key = argmax_key(sc[arg], arg);
                best = key > best ? key : best;
                const int slot = atomicAdd(&c_n, 1);
                if (slot < kPkCap) {
                    c_h[slot] = sc[arg];
                    c_i[slot] = (int)arg;
                    c_w[slot] = (int)(e - i);
                }
            }
            i = e;
        }
        const int npk = pk_block_sum(nq, red_i);
        best = pk_block_max(best, red_k);
        const int ncand = min(c_n, kPkCap);
        // the highest max_peaks candidates, one block argmax each
        const int nlist = p.peaks ? min(p.max_peaks, ncand) : 0;
        for (int r = 0; r < nlist; ++r) {
            unsigned long long kbest = 0ull;
            int slot_best = -1;
            for (int q = threadIdx.x; q < ncand; q += kPkThreads) {
                if (c_w[q] < 0) continue;  // taken
                const unsigned long long key = argmax_key(c_h[q], c_i[q]);
                if (key > kbest) {
                    kbest = key;
                    slot_best = q;
                }
            }
            const unsigned long long kmax = pk_block_max(kbest, red_k);
            if (kbest == kmax && slot_best >= 0) {
                PeakDev &o = p.peaks[(size_t)s * p.max_peaks + r];
                o.index = c_i[slot_best];
                o.height = c_h[slot_best];
                o.width = c_w[slot_best];
                o.harmonic = 0;
                o.reserved = 0;
                c_w[slot_best] = -1;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            PeakSummaryDev &S = p.summary[s];
            S.mean = mean;
            S.sd = sd;
            S.sde = ntot > 0 ? (sd > 0.0 ? ((double)mx - mean) / sd : 0.0) : NAN;
            S.best_index = best ? key_index(best) : -1;
            S.best_score = best ? key_value(best) : NAN;
            S.n_peaks = npk;
            S.truncated = c_n > kPkCap ? 1 : 0;
            S.n_listed = nlist;
            if (p.peaks && nlist > 0) {
                const double Pb = p.periods[gb + p.peaks[(size_t)s * p.max_peaks].index];
                for (int r = 0; r < nlist; ++r) {
                    PeakDev &o = p.peaks[(size_t)s * p.max_peaks + r];
                    int h = 0;
                    if (r == 0) {
                        h = 1;
                    } else {
                        const double ratio = p.periods[gb + o.index] / Pb;
                        for (int m = 2; m <= 4 && h == 0; ++m) {
                            if (fabs(ratio - m) <= p.harm_tol * m) h = m;
                            else if (fabs(1.0 / ratio - m) <= p.harm_tol * m) h = -m;
                        }
                    }
                    o.harmonic = h;
                }
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_peaks(const PeakParams &p, int num_sms, cudaStream_t st)
{
    const int grid = p.nstars < num_sms * 2 ? p.nstars : num_sms * 2;
    peaks_kernel<<<grid, kPkThreads, 0, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ ROC

// Detection statistics of one detector over labelled scores (Sec. 3.2: ROC curves of stars
// scored by their best trial period). Every quantity is a count over pairs of scores, so it
// is exact and independent of the order of the atomics. A NaN score ranks below every
// number. Cost: n_neg^2 + n_pos * n_neg comparisons (10^8 for 10^4 of each).
constexpr int kRocThreads = 256;
constexpr int kRocTile = 2048;

__device__ __forceinline__ float roc_key(float v) { return v != v ? -INFINITY : v; }

__global__ void roc_init_kernel(RocParams p)
{
    const int t = threadIdx.x;
    if (t == 0) *p.u2 = 0ull;
    if (t < p.n_fpr) {
        p.tp[t] = 0ull;
        p.thr[t] = -INFINITY;  // the rule's value when k >= n_neg
    }
}

// thr[f] = the (k_f + 1)-th largest negative: negative j is it iff #{neg > neg_j} <= k_f <
// #{neg >= neg_j} (every such j holds the same value).
__global__ void __launch_bounds__(kRocThreads) roc_threshold_kernel(RocParams p)
{
    __shared__ float tile[kRocTile];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float v = j < p.n_neg ? roc_key(p.neg[j]) : 0.f;
    int64_t g = 0, e = 0;
    for (int64_t t0 = 0; t0 < p.n_neg; t0 += kRocTile) {
        const int nt = (int)min((int64_t)kRocTile, p.n_neg - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += blockDim.x) tile[i] = roc_key(p.neg[t0 + i]);
        __syncthreads();
        for (int i = 0; i < nt; ++i) {
            const float u = tile[i];
            g += u > v;
            e += u >= v;
        }
    }
    if (j < p.n_neg)
        for (int f = 0; f < p.n_fpr; ++f)
            if (g <= p.k[f] && p.k[f] < e) p.thr[f] = v;
}

__device__ __forceinline__ unsigned long long roc_block_sum(unsigned long long v, unsigned long long *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long t = 0ull;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRocThreads / 32; ++w) t += red[w];
    return t;
}

// u2 += 2 #{pos_i > neg_j} + #{pos_i == neg_j}; tp[f] += [pos_i > thr_f]
__global__ void __launch_bounds__(kRocThreads) roc_count_kernel(RocParams p)
{
    __shared__ float tile[kRocTile];
    __shared__ unsigned long long red[kRocThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < p.n_pos;
    const float v = live ? roc_key(p.pos[i]) : 0.f;
    unsigned long long c = 0ull;
    for (int64_t t0 = 0; t0 < p.n_neg; t0 += kRocTile) {
        const int nt = (int)min((int64_t)kRocTile, p.n_neg - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < nt; k += blockDim.x) tile[k] = roc_key(p.neg[t0 + k]);
        __syncthreads();
        if (live)
            for (int k = 0; k < nt; ++k) {
                const float u = tile[k];
                c += (v > u ? 2ull : 0ull) + (v == u ? 1ull : 0ull);
            }
    }
    const unsigned long long s = roc_block_sum(c, red);
    if (threadIdx.x == 0 && s) atomicAdd(p.u2, s);
    for (int f = 0; f < p.n_fpr; ++f) {
        const unsigned long long d = roc_block_sum(live && v > p.thr[f] ? 1ull : 0ull, red);
        if (threadIdx.x == 0 && d) atomicAdd(&p.tp[f], d);
    }
}

cudaError_t launch_roc(const RocParams &p, int num_sms, cudaStream_t st)
{
    (void)num_sms;
    roc_init_kernel<<<1, 32, 0, st>>>(p);
    if (p.n_fpr > 0)
        roc_threshold_kernel<<<(int)((p.n_neg + kRocThreads - 1) / kRocThreads), kRocThreads, 0, st>>>(p);
    roc_count_kernel<<<(int)((p.n_pos + kRocThreads - 1) / kRocThreads), kRocThreads, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace gpfc
