// detrend.cu -- the pre-processing of Sec. 2.2 (Fig. 3) on the GPU: segmentation at time
// and flux gaps, a clipped least-squares cubic spline per segment with the knot spacing
// chosen by the Bayesian Information Criterion, division by the fit, and clipping of each
// segment's edges.
//
// Readings (the paper names the steps, not the spline or the criterion's form):
//  * a segment starts at sample i when t_i - t_{i-1} > time_gap or |f_i - f_{i-1}| >
//    flux_gap_sigma times the population standard deviation of the whole light curve;
//  * the spline is cubic with clamped end knots at the segment's first and last times and
//    interior knots at t0 + spacing j strictly inside; for each candidate spacing the fit
//    solves (B^T B + lambda D^T D) c = B^T f over the used points, D the second difference
//    of the coefficients and lambda = ridge trace(B^T B) / p, so a knot interval left
//    without points takes coefficients continued from its neighbours;
//  * clipping: residuals over the whole segment, sigma = RMS over the used points; the next
//    fit uses the unmasked points with |r| <= max(clip_sigma sigma, 1e-9 RMS(f)); repeat
//    until the used set repeats or max_iter fits have been made;
//  * the spacing with the smallest BIC = n ln(RSS / n) + p ln n wins (ties: the earlier);
//    a candidate with fewer used points than coefficients, or a normal matrix that is not
//    positive definite, is skipped;
//  * the output is f / spline for every point of a segment except its first and last
//    `edge` points (segments of 2 edge points or fewer are dropped), in time order.
//
// Layout: every per-point scratch array is indexed by the point's own index, and a
// segment's p <= n_s coefficients live at the indices of its own points, so segments
// never share scratch. Every reduction runs in a fixed order: the results do not depend on
// scheduling.
#include <cmath>
#include <cstdint>

#include "gpfc_common.cuh"
#include "gpfc_detrend.h"

namespace gpfc {

constexpr int kDtThreads = 256;

// fixed-order block sum (warp shuffles, then the warp totals in order)
__device__ __forceinline__ double dt_block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kDtThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ void dt_range(int64_t n, int64_t &i0, int64_t &i1)
{
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    i0 = (int64_t)blockIdx.x * per;
    i1 = min(n, i0 + per);
    if (i0 > n) i0 = n;
}

// pass 1: per-block sums of f; pass 2: per-block sums of (f - mean)^2
__global__ void __launch_bounds__(kDtThreads) dt_moment_kernel(DetrendParams p, int pass)
{
    __shared__ double red[kDtThreads / 32];
    __shared__ double s_mean;
    if (pass == 2 && threadIdx.x == 0) {
        double tot = 0.0;
        for (int g = 0; g < (int)gridDim.x; ++g) tot += p.partial[g];
        s_mean = tot / (double)p.n;
    }
    __syncthreads();
    int64_t i0, i1;
    dt_range(p.n, i0, i1);
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kDtThreads) {
        const double v = (double)p.f[i];
        acc += pass == 1 ? v : (v - s_mean) * (v - s_mean);
    }
    const double t = dt_block_sum(acc, red);
    if (threadIdx.x == 0) p.partial[(pass - 1) * gridDim.x + blockIdx.x] = t;
}

__device__ __forceinline__ double dt_sigma(const DetrendParams &p, int G)
{
    double v = 0.0;
    for (int g = 0; g < G; ++g) v += p.partial[G + g];
    return sqrt(v / (double)p.n);
}

__device__ __forceinline__ bool dt_break(const DetrendParams &p, int64_t i, double fgap)
{
    if (i == 0) return true;
    return (p.t[i] - p.t[i - 1] > p.time_gap) || (fabs((double)p.f[i] - (double)p.f[i - 1]) > fgap);
}

// segment starts: pass 1 counts per block, pass 2 writes them in order
__global__ void __launch_bounds__(kDtThreads) dt_starts_kernel(DetrendParams p, int pass)
{
    __shared__ double s_fgap;
    __shared__ int64_t s_base;
    __shared__ int s_warp[kDtThreads / 32];
    if (threadIdx.x == 0) {
        s_fgap = p.flux_gap_sigma * dt_sigma(p, gridDim.x);
        s_base = pass == 2 ? p.blk_off[blockIdx.x] : 0;
    }
    __syncthreads();
    int64_t i0, i1;
    dt_range(p.n, i0, i1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t count = 0;
    for (int64_t c0 = i0; c0 < i1; c0 += kDtThreads) {
        const int64_t i = c0 + threadIdx.x;
        const bool br = i < i1 && dt_break(p, i, s_fgap);
        const unsigned m = __ballot_sync(0xffffffffu, br);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < kDtThreads / 32; ++w) {
            if (w < warp) before += s_warp[w];
            tot += s_warp[w];
        }
        if (pass == 2 && br) p.seg_start[s_base + count + before + __popc(m & ((1u << lane) - 1u))] = i;
        count += tot;
        __syncthreads();
    }
    if (pass == 1 && threadIdx.x == 0) p.blk_count[blockIdx.x] = count;
}

// exclusive scan over at most a few thousand block counts (one block, fixed order)
__global__ void dt_scan_kernel(const int64_t *cnt, int64_t ncnt, int64_t *off, int64_t *total)
{
    if (threadIdx.x != 0) return;
    int64_t s = 0;
    for (int64_t g = 0; g < ncnt; ++g) {
        off[g] = s;
        s += cnt[g];
    }
    off[ncnt] = s;
    if (total) *total = s;
}

__global__ void dt_close_starts_kernel(DetrendParams p)
{
    if (threadIdx.x == 0) p.seg_start[*p.n_seg] = p.n;
}

// knot j of the clamped cubic knot vector of a segment [t0, t1] with m interior knots
__device__ __forceinline__ double dt_knot(int j, double t0, double t1, double sp, int m)
{
    return j < 4 ? t0 : (j < 4 + m ? t0 + sp * (double)(j - 3) : t1);
}

// knot interval mu (3 <= mu <= p - 1) holding t: k_mu <= t < k_{mu+1}, the segment's last
// time in the last interval; and the four nonzero cubic B-splines B_{mu-3 .. mu}(t)
// (de Boor's triangular recursion)
__device__ __forceinline__ int dt_basis(double t, double t0, double t1, double sp, int m, double (&N)[4])
{
    int j = (int)floor((t - t0) / sp);  // interior knots t0 + sp i <= t: i = 1 .. j
    if (j < 0) j = 0;
    if (j > m) j = m;
    while (j > 0 && t0 + sp * (double)j > t) --j;
    while (j < m && t0 + sp * (double)(j + 1) <= t) ++j;
    const int mu = 3 + j;
    double left[4], right[4];
    N[0] = 1.0;
    for (int d = 1; d <= 3; ++d) {
        left[d] = t - dt_knot(mu + 1 - d, t0, t1, sp, m);
        right[d] = dt_knot(mu + d, t0, t1, sp, m) - t;
        double saved = 0.0;
        for (int r = 0; r < d; ++r) {
            const double den = right[r + 1] + left[d - r];
            const double temp = den != 0.0 ? N[r] / den : 0.0;
            N[r] = saved + right[r + 1] * temp;
            saved = left[d - r] * temp;
        }
        N[d] = saved;
    }
    return mu;
}

// first index in [lo, hi) with t[i] >= x
__device__ __forceinline__ int64_t dt_lower_bound(const double *t, int64_t lo, int64_t hi, double x)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (t[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kDtThreads) dt_fit_kernel(DetrendParams p)
{
    __shared__ double red[kDtThreads / 32];
    __shared__ int s_m, s_p, s_ok, s_changed;
    __shared__ double s_lambda;
    const int tid = threadIdx.x;
    const int64_t nseg = *p.n_seg;
    for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const int64_t a = p.seg_start[s], b = p.seg_start[s + 1], ns = b - a;
        if (ns <= 2 * (int64_t)p.edge) {
            if (tid == 0) p.seg_keep[s] = 0;
            continue;
        }
        const double t0 = p.t[a], t1 = p.t[b - 1];
        double best_bic = INFINITY;
        bool have = false;
        for (int c = 0; c < p.n_sp; ++c) {
            const double sp = p.sp[c];
            __syncthreads();  // every thread has read the previous candidate's s_m, s_p
            if (tid == 0) {
                int m = 0;
                while (t0 + sp * (double)(m + 1) < t1 && m < (1 << 30)) ++m;
                s_m = m;
                s_p = m + 4;
            }
            __syncthreads();
            const int m = s_m, np_ = s_p;
            if ((int64_t)np_ > ns) continue;  // fewer points than coefficients
            for (int64_t i = a + tid; i < b; i += kDtThreads) p.used[i] = p.mask ? (uint8_t)(p.mask[i] == 0) : 1;
            __syncthreads();
            bool valid = true;
            double bic = INFINITY;
            for (int it = 0; it < p.max_iter; ++it) {
                // used count
                double cu = 0.0;
                for (int64_t i = a + tid; i < b; i += kDtThreads) cu += p.used[i];
                const double nu = dt_block_sum(cu, red);
                if (nu < (double)np_) {
                    valid = false;
                    break;
                }
                // normal equations, one thread per coefficient row j: G[j][j+d], d = 0..3, and
                // (B^T f)_j, summed over the used points of B_j's support in point order
                for (int j = tid; j < np_; j += kDtThreads) {
                    const double klo = dt_knot(j, t0, t1, sp, m), khi = dt_knot(j + 4, t0, t1, sp, m);
                    const int64_t i0 = dt_lower_bound(p.t, a, b, klo);
                    const int64_t i1 = (j + 4 >= np_) ? b : dt_lower_bound(p.t, a, b, khi);
                    double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0, r = 0.0;
                    for (int64_t i = i0; i < i1; ++i) {
                        if (!p.used[i]) continue;
                        double N[4];
                        const int mu = dt_basis(p.t[i], t0, t1, sp, m, N);
                        const int q = j - (mu - 3);  // position of B_j among the four
                        if (q < 0 || q > 3) continue;
                        const double bj = N[q];
                        g0 += bj * bj;
                        if (q + 1 <= 3) g1 += bj * N[q + 1];
                        if (q + 2 <= 3) g2 += bj * N[q + 2];
                        if (q + 3 <= 3) g3 += bj * N[q + 3];
                        r += bj * (double)p.f[i];
                    }
                    double *G = p.G4 + (a + j) * 4;
                    G[0] = g0;
                    G[1] = g1;
                    G[2] = g2;
                    G[3] = g3;
                    p.rhs[a + j] = r;
                }
                __syncthreads();
                double tr = 0.0;
                for (int j = tid; j < np_; j += kDtThreads) tr += p.G4[(a + j) * 4];
                const double trace = dt_block_sum(tr, red);
                if (tid == 0) s_lambda = p.ridge * trace / (double)np_;
                __syncthreads();
                // + lambda D^T D: (D^T D)[j][j+d] = sum over rows r of D (coefficients r..r+2
                // weighted 1, -2, 1) of D[r][j] D[r][j+d]
                for (int j = tid; j < np_; j += kDtThreads) {
                    for (int d = 0; d <= 2; ++d) {
                        if (j + d >= np_) break;
                        double v = 0.0;
                        for (int r = j + d - 2; r <= j; ++r) {
                            if (r < 0 || r > np_ - 3) continue;
                            const double w1 = j - r == 0 ? 1.0 : (j - r == 1 ? -2.0 : 1.0);
                            const int e = j + d - r;
                            const double w2 = e == 0 ? 1.0 : (e == 1 ? -2.0 : 1.0);
                            v += w1 * w2;
                        }
                        p.G4[(a + j) * 4 + d] += s_lambda * v;
                    }
                }
                __syncthreads();
                // banded Cholesky G = L L^T (L[i][i-q] in LB[i][q]) and the two triangular
                // solves, by one thread
                if (tid == 0) {
                    int ok = 1;
                    for (int i = 0; i < np_ && ok; ++i) {
                        double *Li = p.LB + (a + i) * 4;
                        for (int k = (i >= 3 ? i - 3 : 0); k < i; ++k) {
                            const double *Lk = p.LB + (a + k) * 4;
                            double v = p.G4[(a + k) * 4 + (i - k)];
                            for (int l = (i >= 3 ? i - 3 : 0); l < k; ++l) v -= Li[i - l] * Lk[k - l];
                            Li[i - k] = v / Lk[0];
                        }
                        double v = p.G4[(a + i) * 4];
                        for (int l = (i >= 3 ? i - 3 : 0); l < i; ++l) v -= Li[i - l] * Li[i - l];
                        if (!(v > 0.0)) ok = 0;
                        else Li[0] = sqrt(v);
                    }
                    if (ok) {
                        for (int i = 0; i < np_; ++i) {  // L y = rhs (y kept in coef)
                            const double *Li = p.LB + (a + i) * 4;
                            double v = p.rhs[a + i];
                            for (int l = (i >= 3 ? i - 3 : 0); l < i; ++l) v -= Li[i - l] * p.coef[a + l];
                            p.coef[a + i] = v / Li[0];
                        }
                        for (int i = np_ - 1; i >= 0; --i) {  // L^T c = y
                            double v = p.coef[a + i];
                            for (int l = i + 1; l <= i + 3 && l < np_; ++l) v -= p.LB[(a + l) * 4 + (l - i)] * p.coef[a + l];
                            p.coef[a + i] = v / p.LB[(a + i) * 4];
                        }
                    }
                    s_ok = ok;
                }
                __syncthreads();
                if (!s_ok) {
                    valid = false;
                    break;
                }
                // the fit at every point of the segment, residual statistics over the used ones
                double rr = 0.0, ff = 0.0;
                for (int64_t i = a + tid; i < b; i += kDtThreads) {
                    double N[4];
                    const int mu = dt_basis(p.t[i], t0, t1, sp, m, N);
                    double v = 0.0;
                    for (int q = 0; q < 4; ++q) v += p.coef[a + mu - 3 + q] * N[q];
                    p.trend[i] = v;
                    if (p.used[i]) {
                        const double r = (double)p.f[i] - v;
                        rr += r * r;
                        ff += (double)p.f[i] * (double)p.f[i];
                    }
                }
                const double rss = dt_block_sum(rr, red);
                const double fss = dt_block_sum(ff, red);
                const double thr = fmax(p.clip_sigma * sqrt(rss / nu), 1e-9 * sqrt(fss / nu));
                if (tid == 0) s_changed = 0;
                __syncthreads();
                int ch = 0;
                for (int64_t i = a + tid; i < b; i += kDtThreads) {
                    const uint8_t free_ = p.mask ? (uint8_t)(p.mask[i] == 0) : 1;
                    const uint8_t nx = free_ && fabs((double)p.f[i] - p.trend[i]) <= thr;
                    p.used2[i] = nx;
                    ch |= nx != p.used[i];
                }
                if (ch) s_changed = 1;
                __syncthreads();
                if (!s_changed || it == p.max_iter - 1) {
                    bic = rss > 0.0 ? nu * log(rss / nu) + (double)np_ * log(nu) : -INFINITY;
                    break;  // the last fit's own point set is `used`
                }
                for (int64_t i = a + tid; i < b; i += kDtThreads) p.used[i] = p.used2[i];
                __syncthreads();
            }
            if (valid && bic < best_bic) {
                best_bic = bic;
                have = true;
                for (int64_t i = a + tid; i < b; i += kDtThreads) p.best[i] = p.trend[i];
            }
            __syncthreads();
        }
        for (int64_t i = a + tid; i < b; i += kDtThreads) p.det[i] = have ? (float)((double)p.f[i] / p.best[i]) : 0.f;
        if (tid == 0) p.seg_keep[s] = have ? ns - 2 * (int64_t)p.edge : 0;
        __syncthreads();
    }
}

// kept counts -> output offsets and the output length (one thread, fixed order)
__global__ void dt_offsets_kernel(DetrendParams p)
{
    if (threadIdx.x != 0) return;
    const int64_t nseg = *p.n_seg;
    int64_t o = 0;
    for (int64_t s = 0; s < nseg; ++s) {
        p.seg_off[s] = o;
        o += p.seg_keep[s];
    }
    *p.n_out = o;
}

__global__ void dt_write_kernel(DetrendParams p)
{
    const int64_t nseg = *p.n_seg;
    for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const int64_t keep = p.seg_keep[s];
        if (keep == 0) continue;
        const int64_t a = p.seg_start[s] + p.edge, o = p.seg_off[s];
        for (int64_t k = threadIdx.x; k < keep; k += blockDim.x) {
            p.t_out[o + k] = p.t[a + k];
            p.f_out[o + k] = p.det[a + k];
            if (p.seg_out) p.seg_out[o + k] = (int32_t)s;
        }
    }
}

cudaError_t launch_detrend(const DetrendParams &p, int num_sms, cudaStream_t st)
{
    const int G = p.blocks;
    dt_moment_kernel<<<G, kDtThreads, 0, st>>>(p, 1);
    dt_moment_kernel<<<G, kDtThreads, 0, st>>>(p, 2);
    dt_starts_kernel<<<G, kDtThreads, 0, st>>>(p, 1);
    dt_scan_kernel<<<1, 32, 0, st>>>(p.blk_count, G, p.blk_off, p.n_seg);
    dt_starts_kernel<<<G, kDtThreads, 0, st>>>(p, 2);
    dt_close_starts_kernel<<<1, 32, 0, st>>>(p);
    dt_fit_kernel<<<num_sms * 2, kDtThreads, 0, st>>>(p);
    dt_offsets_kernel<<<1, 32, 0, st>>>(p);
    dt_write_kernel<<<num_sms * 2, kDtThreads, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace gpfc
