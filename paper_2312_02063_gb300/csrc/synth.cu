// synth.cu -- training profiles: seeded light curves generated on the device and folded
// at their true period (plus a random drift of at most `drift_bins` bins over the
// baseline) by a single-period fold.
//
// Light curve j (global index) has n_cadences samples at t_i = i * cadence from t0 = 0,
// flux = 1 + sigma z_i + signal(t_i) with z_i standard normal. Even j: a box transit
// (positive). Odd j, by (j / 2) mod 3: noise only, a sinusoid, or an eclipsing-binary-like
// pair of boxes (primary + secondary half a period later) -- the negatives.
// Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the
// 64-bit seed: counter (j, 0, 0, 0xFFFFFFFF) and (j, 1, 0, 0xFFFFFFFF) give the light curve's
// parameters, counter (j, i / 4, 1, 0) the four normals of samples 4(i/4) .. 4(i/4)+3
// (Box-Muller on uniforms u = (x >> 8) 2^-24).
//
// Fold: one block per light curve. Each warp owns a private copy of the bins in shared
// memory. Lanes take four consecutive samples each; samples that land in the same bin in
// one step are merged with __match_any_sync and their sum is added, in lane order, by the
// group's lowest lane, so no two threads update a bin at once. The per-warp bins are added
// in warp order at the end (deterministic). Phases are the 64-bit fixed point of the fold.
#include <cmath>
#include <cstdint>

#include "gpfc_common.cuh"
#include "gpfc_synth.h"

namespace gpfc {

struct Philox4 {
    uint32_t v[4];
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                          uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    return Philox4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ double unif64(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
__device__ __forceinline__ float unif32(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// parameters of light curve j
struct LcParams {
    int kind;        // 0 transit, 1 noise, 2 sinusoid, 3 eclipsing binary
    double sigma, period, epoch, duration, depth, depth2, amp, fold_period;
};

__device__ LcParams lc_params(uint64_t seed, int64_t j, const gpfc_synth_params &sp)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const Philox4 a = philox4x32_10((uint32_t)j, 0u, 0u, 0xFFFFFFFFu, k0, k1);
    const Philox4 b = philox4x32_10((uint32_t)j, 1u, 0u, 0xFFFFFFFFu, k0, k1);
    LcParams p{};
    p.kind = (j & 1) ? 1 + (int)((j >> 1) % 3) : 0;
    p.sigma = exp(log(sp.sigma_min) + unif64(a.v[0]) * log(sp.sigma_max / sp.sigma_min));
    // explicit round-to-nearest operations (no fused multiply-add), so that these values
    // are bit-identical to any IEEE-754 evaluation of the same formulas
    p.period = __dadd_rn(sp.p_min, __dmul_rn(unif64(a.v[1]), __dsub_rn(sp.p_max, sp.p_min)));
    p.epoch = __dmul_rn(unif64(a.v[2]), p.period);
    p.duration = __ddiv_rn(__dadd_rn(sp.dur_min_h, __dmul_rn(unif64(a.v[3]), __dsub_rn(sp.dur_max_h, sp.dur_min_h))),
                           24.0);
    p.depth = exp(log(sp.depth_min) + unif64(b.v[0]) * log(sp.depth_max / sp.depth_min));
    p.depth2 = __dmul_rn(p.depth, __dadd_rn(0.2, __dmul_rn(0.8, unif64(b.v[1]))));
    p.amp = exp(log(sp.depth_min) + unif64(b.v[2]) * log(sp.depth_max / sp.depth_min));
    const double T = __dmul_rn((double)sp.n_cadences, sp.cadence);
    const double df = __ddiv_rn(__dmul_rn(__dsub_rn(__dmul_rn(2.0, unif64(b.v[3])), 1.0), sp.drift_bins),
                                __dmul_rn(256.0, T));
    p.fold_period = __ddiv_rn(1.0, __dadd_rn(__ddiv_rn(1.0, p.period), df));
    return p;
}

__device__ __forceinline__ bool in_box(double t, double period, double centre, double dur)
{
    const double half = __dmul_rn(0.5, period);
    const double d = fmod(__dadd_rn(__dsub_rn(t, centre), half), period);
    const double dd = __dsub_rn(d < 0.0 ? __dadd_rn(d, period) : d, half);
    return fabs(dd) < __dmul_rn(0.5, dur);
}

constexpr int kSynthWarps = 8;

__global__ void __launch_bounds__(kSynthWarps * 32) synth_fold_kernel(SynthParams P)
{
    __shared__ float s_sum[kSynthWarps][256];
    __shared__ uint32_t s_cnt[kSynthWarps][256];
    __shared__ double s_mom[kSynthWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = P.nbins;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    for (int64_t q = blockIdx.x; q < P.n; q += gridDim.x) {
        const int64_t j = P.first + q;
        const LcParams lp = lc_params(P.seed, j, P.sp);
        const double Fd = __ddiv_rn(1099511627776.0, lp.fold_period);
        const unsigned long long F = (unsigned long long)__double2ll_rn(Fd);
        for (int b = lane; b < nb; b += 32) {
            s_sum[warp][b] = 0.f;
            s_cnt[warp][b] = 0u;
        }
        __syncwarp();
        // a multiple of 128 samples per warp keeps every lane's first sample at i % 4 == 0
        const int per_warp = ((P.sp.n_cadences + kSynthWarps - 1) / kSynthWarps + 127) & ~127;
        const int i_begin = warp * per_warp;
        const int i_end = min(P.sp.n_cadences, i_begin + per_warp);
        double m1 = 0.0, m2 = 0.0;  // sum of x and x^2 over this lane's samples
        for (int base = i_begin; base < i_end; base += 128) {
            const int i0 = base + 4 * lane;  // this lane's 4 samples (i0 % 4 == 0 when base is)
            const Philox4 r = philox4x32_10((uint32_t)j, (uint32_t)(i0 >> 2), 1u, 0u, k0, k1);
            float z[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float u1 = 1.0f - unif32(r.v[2 * h]);  // (0, 1]
                const float u2 = unif32(r.v[2 * h + 1]);
                const float rad = sqrtf(-2.0f * logf(u1));
                float s, c;
                sincospif(2.0f * u2, &s, &c);
                z[2 * h] = rad * c;
                z[2 * h + 1] = rad * s;
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int i = i0 + qq;
                const bool valid = i < i_end;
                const double t = __dmul_rn((double)i, P.sp.cadence);
                float x = (float)lp.sigma * z[qq];
                if (lp.kind == 0) {
                    if (in_box(t, lp.period, lp.epoch, lp.duration)) x -= (float)lp.depth;
                } else if (lp.kind == 2) {
                    x += (float)(lp.amp * sinpi(2.0 * (t - lp.epoch) / lp.period));
                } else if (lp.kind == 3) {
                    if (in_box(t, lp.period, lp.epoch, lp.duration)) x -= (float)lp.depth;
                    if (in_box(t, lp.period, __dadd_rn(lp.epoch, __dmul_rn(0.5, lp.period)), lp.duration))
                        x -= (float)lp.depth2;
                }
                if (valid) {
                    m1 += (double)x;
                    m2 += (double)x * (double)x;
                }
                const long long tau = __double2ll_rn(__dmul_rn(t, 16777216.0));
                const unsigned long long phi = (unsigned long long)tau * F;
                const int bin = valid ? (int)__umul64hi(phi, (unsigned long long)nb) : -1;
                const unsigned m = __match_any_sync(0xffffffffu, bin);
                float gs = 0.f;
                for (int src = 0; src < 32; ++src) {
                    const float xs = __shfl_sync(0xffffffffu, x, src);
                    if ((m >> src) & 1u) gs += xs;
                }
                if (valid && (__ffs(m) - 1) == lane) {
                    s_sum[warp][bin] += gs;
                    s_cnt[warp][bin] += (uint32_t)__popc(m);
                }
                __syncwarp();
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            m1 += __shfl_xor_sync(0xffffffffu, m1, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        }
        if (lane == 0) {
            s_mom[warp][0] = m1;
            s_mom[warp][1] = m2;
        }
        __syncthreads();
        if (threadIdx.x == 0 && P.sigma_out) {
            double a = 0.0, b2 = 0.0;
            for (int w = 0; w < kSynthWarps; ++w) {
                a += s_mom[w][0];
                b2 += s_mom[w][1];
            }
            const double nn = (double)P.sp.n_cadences, mu = a / nn;
            P.sigma_out[q] = (float)sqrt(fmax(b2 / nn - mu * mu, 0.0));
        }
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            float s = 0.f;
            uint32_t c = 0u;
            for (int w = 0; w < kSynthWarps; ++w) {
                s += s_sum[w][b];
                c += s_cnt[w][b];
            }
            if (P.folded) P.folded[q * nb + b] = c ? 1.0f + s / (float)c : __int_as_float(0x7fc00000);
            if (P.counts) P.counts[q * nb + b] = (int32_t)c;
        }
        if (threadIdx.x == 0 && P.label) P.label[q] = lp.kind == 0 ? 1.f : 0.f;
        if (threadIdx.x == 0 && P.period_out) P.period_out[q] = lp.fold_period;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ the paper's vectors

// One thread per 4 bins of a vector (the 4 normals of one Philox call), 64 per vector of
// 256 bins; the vector's parameters are derived by every thread from the same counters.
__global__ void paper_vectors_kernel(VectorParams P)
{
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const int per_vec = (P.nbins + 3) / 4;
    const int64_t total = P.n * per_vec;
    const gpfc_vector_params &v = P.vp;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = g / per_vec;
        const int m = (int)(g - q * per_vec);
        const int64_t j = P.first + q;
        const Philox4 a = philox4x32_10((uint32_t)j, 0u, 2u, 0xFFFFFFFFu, k0, k1);
        const Philox4 b = philox4x32_10((uint32_t)j, 1u, 2u, 0xFFFFFFFFu, k0, k1);
        const bool positive = (j & 1) == 0;
        const bool inject = positive || ((j >> 1) & 1);
        const double sigma = exp(log(v.sigma_min) + unif64(a.v[0]) * log(v.sigma_max / v.sigma_min));
        double alpha = 0.0;
        if (positive) alpha = v.alpha_pos_min + unif64(a.v[1]) * (v.alpha_pos_max - v.alpha_pos_min);
        else if (inject) alpha = unif64(a.v[1]) * v.alpha_neg_max;
        const double qq = v.q_min + unif64(a.v[2]) * (v.q_max - v.q_min);
        const double r = unif64(a.v[3]);
        const double phi0 = unif64(b.v[0]);
        const double depth = alpha * sigma / sqrt((double)v.n_points * qq);
        const double sigma_bin = sigma * sqrt((double)P.nbins / (double)v.n_points);
        const double t14 = 2.0 * qq / (1.0 + r), t23 = r * t14;
        const Philox4 rr = philox4x32_10((uint32_t)j, (uint32_t)m, 3u, 0u, k0, k1);
        float z[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float u1 = 1.0f - unif32(rr.v[2 * h]);
            const float u2 = unif32(rr.v[2 * h + 1]);
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            z[2 * h] = rad * cs;
            z[2 * h + 1] = rad * sn;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int bin = 4 * m + u;
            if (bin >= P.nbins) break;
            const double x = ((double)bin + 0.5) / (double)P.nbins;
            double d = x - phi0;
            d = fabs(d - floor(d + 0.5));
            const double shape = d <= 0.5 * t23 ? 1.0 : (d < 0.5 * t14 ? (0.5 * t14 - d) / (0.5 * (t14 - t23)) : 0.0);
            P.folded[q * P.nbins + bin] = (float)(1.0 + sigma_bin * (double)z[u] - depth * shape);
        }
        if (m == 0) {
            if (P.label) P.label[q] = positive ? 1.f : 0.f;
            if (P.alpha) P.alpha[q] = (float)alpha;
            if (P.sigma_bin) P.sigma_bin[q] = (float)sigma_bin;
        }
    }
}

cudaError_t launch_paper_vectors(const VectorParams &p, int num_sms, cudaStream_t st)
{
    const int64_t total = p.n * ((p.nbins + 3) / 4);
    const int64_t want = (total + 255) / 256;
    const int grid = (int)(want < (int64_t)num_sms * 8 ? want : (int64_t)num_sms * 8);
    paper_vectors_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_synth(const SynthParams &p, int num_sms, cudaStream_t st)
{
    const int64_t want = p.n;
    const int grid = (int)(want < (int64_t)num_sms * 8 ? want : (int64_t)num_sms * 8);
    synth_fold_kernel<<<grid, kSynthWarps * 32, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace gpfc
