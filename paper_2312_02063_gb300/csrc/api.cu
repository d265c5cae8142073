// api.cu -- the extern "C" entry points of libgpfc.so (declared in include/gpfc.h).
//
// Host-side argument checks, workspace management and kernel launches. All work is
// enqueued on the context's stream; device-side errors are latched in a status word in
// mapped (zero-copy) host memory and reported by gpfc_sync() and the next call.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gpfc.h"
#include "gpfc_cnn.h"
#include "gpfc_kernels.h"
#include "gpfc_synth.h"
#include "gpfc_twotier.h"
#include "gpfc_decide.h"
#include "gpfc_detrend.h"

using namespace gpfc;

struct gpfc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint32_t *status_host = nullptr;  // mapped pinned memory
    uint32_t *status_dev = nullptr;
    gpfc_fold_config fold_cfg{0, 0, 0, 0, 0};
    // autotuner: tuned fold configs by (nbins, mode, floor(log2 n))
    struct Tuned {
        int nbins, mode, lg;
        gpfc_fold_config cfg;
        float ms;
    };
    std::vector<Tuned> tuned;
    bool autotune = true;
    // CUDA graph of the last batched search, replayed when the same call comes again
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint8_t> graph_key;
    gpfc_fold_config last_plan{0, 0, 0, 0, 0};
    int box_path = GPFC_BOX_AUTO;
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    // side streams of the overlapped box search: folds (high priority), box scorer (low)
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t side_ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // with timing on: event pairs around each fold launch of the last pipelined search
    std::vector<cudaEvent_t> fold_ev;
    int fold_ev_used = 0;
    char last_error[512] = {0};
};

namespace {

// Profiles scored per CNN launch pair: their fc1 operand tiles (high and low BF16 terms,
// 64 MB) stay in L2.
constexpr int64_t kCnnChunk = 8192;

// Message of the last failure that had no context to hold it (gpfc_create).
thread_local char g_create_error[512] = {0};

// Bracket the main kernel of a call with events when timing is enabled.
struct KernelTimer {
    gpfc_ctx *ctx;
    explicit KernelTimer(gpfc_ctx *c) : ctx(c)
    {
        ctx->fold_ev_used = 0;
        if (ctx->timing) cudaEventRecord(ctx->ev_start, ctx->stream);
    }
    void stop()
    {
        if (ctx->timing) {
            cudaEventRecord(ctx->ev_stop, ctx->stream);
            ctx->timed = true;
        }
    }
};

int set_err(gpfc_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->last_error, sizeof(ctx->last_error), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_err(gpfc_ctx *ctx, cudaError_t e, const char *what)
{
    return set_err(ctx, GPFC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device errors latched by earlier work (non-blocking peek of the mapped word).
int take_latched(gpfc_ctx *ctx)
{
    volatile uint32_t *w = ctx->status_host;
    const uint32_t bits = *w;
    if (!bits) return GPFC_OK;
    *w = 0u;
    if (bits & kErrTimeout) return set_err(ctx, GPFC_ETIMEOUT, "a device-side wait timed out");
    if (bits & kErrArgs)
        return set_err(ctx, GPFC_EINVAL,
                       "batched search: offsets are not a partition starting at 0 and ending at the totals, "
                       "or a star has no samples, more than 2^24 samples or no periods");
    return set_err(ctx, GPFC_ERANGE,
                   "a period is not finite and > 0, or a time/frequency overflows the 64-bit fixed point");
}

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

int ensure_ws(gpfc_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return GPFC_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamSynchronize");
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t want = bytes + bytes / 8;
    e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return set_err(ctx, GPFC_ENOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    ctx->ws_bytes = want;
    return GPFC_OK;
}

struct FoldPlan {
    int warps, ppc, grid, G, layout, chunk, tile, bps, streams;
    int64_t ntasks;
};

// At 256 bins and more the reduction layout: its updates need no load, so three period
// groups of 8-byte bins can be folded by twelve warps at once (1.3x the 64-bit
// read-modify-write layout on a Kepler-length star). Below 256 bins the box search runs
// in the fold's epilogue, one warp per 32 periods, where the 6-byte bins fit the most
// warps.
int default_layout(int nbins) { return nbins >= 256 ? kLayoutRed32 : kLayoutPaired16; }

int floor_log2(int64_t n)
{
    int l = 0;
    while (n > 1) {
        n >>= 1;
        ++l;
    }
    return l;
}

// The tuned config for (nbins, mode, n), if the autotuner has one.
const gpfc_fold_config *find_tuned(const gpfc_ctx *ctx, int nbins, int mode, int64_t n)
{
    if (!ctx->autotune) return nullptr;
    const int lg = floor_log2(n);
    for (const auto &t : ctx->tuned)
        if (t.nbins == nbins && t.mode == mode && t.lg == lg) return &t.cfg;
    return nullptr;
}

// Launch plan of a fold over np periods of stars of about n samples. Fields of the
// context's fold config that are set win; the rest come from `tuned` (if given) or the
// defaults: 1024-sample tiles, the paired 16-bit count layout, the widest block that
// still leaves one block per SM when the grid is short.
FoldPlan plan_with(const gpfc_ctx *ctx, int64_t n, int64_t np, int nbins, const gpfc_fold_config &cfg)
{
    FoldPlan pl{};
    pl.tile = cfg.tile ? cfg.tile : kTile;
    pl.layout = cfg.layout ? cfg.layout : default_layout(nbins);
    if (fold_max_warps(nbins, pl.layout, pl.tile) < 1) pl.layout = kLayoutPaired16;
    if (fold_max_warps(nbins, pl.layout, pl.tile) < 1) pl.tile = 512;
    // the reduction layout's tiles are 8 bytes a sample: 2048-sample tiles (half the
    // per-tile work) where they cost no period group
    if (!cfg.tile && pl.layout == kLayoutRed32 &&
        fold_max_warps(nbins, pl.layout, kMaxTile) >= fold_max_warps(nbins, pl.layout, pl.tile))
        pl.tile = kMaxTile;
    const int maxw = fold_max_warps(nbins, pl.layout, pl.tile);
    // enough blocks to cover the SMs when the grid is short, else the widest block
    int64_t per_sm = (np + (int64_t)32 * ctx->num_sms - 1) / ((int64_t)32 * ctx->num_sms);
    int w = (int)std::min<int64_t>(maxw, std::max<int64_t>(1, per_sm));
    if (cfg.warps > 0) w = std::min(cfg.warps, maxw);
    // ~128 samples per bin per chunk keeps the plain FP32 partials short; the chunk
    // partials are then added with Kahan compensation. Each flush costs a few L2 round
    // trips that one warp per scheduler cannot hide, so chunks are as long as precision
    // allows (the C2 search: 18.3 / 17.3 / 16.7 ms at 32 / 64 / 128 samples per bin).
    // The reduction layout's sums are exact, so its chunks are as long as allowed: one
    // chunk per star up to 65,520 samples (each flush stalls all the block's warps; the
    // fixed-point unit grows with the chunk).
    int64_t chunk = cfg.chunk > 0 ? cfg.chunk : (pl.layout == kLayoutRed32 ? (int64_t)65520 : (int64_t)128 * nbins);
    pl.chunk = (int)std::min<int64_t>(65520, std::max<int64_t>(256, chunk)) & ~15;
    pl.warps = w;
    pl.ppc = 32 * w;
    pl.ntasks = (np + pl.ppc - 1) / pl.ppc;
    // layout 3: enough sample streams for 12 fold warps (three per scheduler); a one-kernel
    // search block needs one warp fewer for its scorer
    pl.streams = 1;
    if (pl.layout == kLayoutRed32) pl.streams = cfg.streams > 0 ? cfg.streams : kMaxRedWarps / w;
    pl.streams = std::max(1, std::min(pl.streams, kMaxRedWarps / w));
    const int occ = std::max(1, fold_blocks_per_sm(nbins, w, pl.layout, pl.tile, pl.streams));
    pl.bps = cfg.blocks_per_sm > 0 ? std::min(cfg.blocks_per_sm, occ) : occ;
    pl.grid = (int)std::min<int64_t>(pl.ntasks, (int64_t)ctx->num_sms * pl.bps);
    pl.G = (int)std::min<int64_t>(256, std::max<int64_t>(1, (n + 8191) / 8192));
    return pl;
}

FoldPlan plan_fold(gpfc_ctx *ctx, int64_t n, int64_t np, int nbins, const gpfc_fold_config *tuned = nullptr)
{
    gpfc_fold_config cfg = ctx->fold_cfg;
    if (tuned) {
        if (!cfg.warps) cfg.warps = tuned->warps;
        if (!cfg.layout) cfg.layout = tuned->layout;
        if (!cfg.tile) cfg.tile = tuned->tile;
        if (!cfg.blocks_per_sm) cfg.blocks_per_sm = tuned->blocks_per_sm;
    }
    const FoldPlan pl = plan_with(ctx, n, np, nbins, cfg);
    ctx->last_plan = gpfc_fold_config{pl.warps, pl.layout, pl.chunk, pl.tile, pl.bps, pl.streams};
    return pl;
}

struct FoldBuffers {
    double *partial;
    StarStats *stats;
    SampleScratch smp;
    float2 *ws_sc;
    uint32_t *ws_cnt;
    unsigned long long *key;
};

size_t carve_fold(void *base, const FoldPlan &pl, int64_t n_total, int nstars, int nbins,
                  FoldBuffers &fb)
{
    Carver c(base);
    fb.partial = c.take<double>((size_t)4 * nstars * pl.G);  // sums, squares, min steps, max |x|
    fb.stats = c.take<StarStats>(nstars);
    const int64_t se = scratch_elems(n_total, nstars);
    fb.smp.tau_lo = c.take<uint32_t>(se);
    fb.smp.tau_hi = c.take<int32_t>(se);
    fb.smp.x = c.take<float>(se);
    fb.smp.xq = c.take<int32_t>(se);
    fb.smp.thg = c.take<int32_t>(se / 16 + 64);
    fb.smp.flags = c.take<uint8_t>(se / 16 + 64);
    fb.ws_sc = c.take<float2>((size_t)pl.grid * nbins * pl.ppc);
    fb.ws_cnt = c.take<uint32_t>((size_t)pl.grid * nbins * pl.ppc);
    fb.key = c.take<unsigned long long>(nstars);
    return c.off + 256;
}

// Bin counts above the lane-private fold's limit go through the fine-bin stage of the
// two-tier kernel (exact fixed-point shared atomics, twotier.cu).
bool wide_bins(int nbins) { return nbins > kMaxNbinsLane || fold_max_warps(nbins, kLayoutPaired16) < 1; }

int check_fold_args(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n,
                    const double *periods, int64_t np, int32_t nbins)
{
    if (!ctx) return GPFC_EINVAL;
    if (!times || !flux || !periods) return set_err(ctx, GPFC_EINVAL, "NULL input array");
    if (n < 1 || n > (int64_t)1 << 24) return set_err(ctx, GPFC_EINVAL, "n = %lld outside [1, 2^24]", (long long)n);
    if (np < 1 || np > (int64_t)INT32_MAX)
        return set_err(ctx, GPFC_EINVAL, "n_periods = %lld outside [1, 2^31-1]", (long long)np);
    if (nbins < 2 || nbins > kEqMaxFine) return set_err(ctx, GPFC_EINVAL, "nbins = %d outside [2, %d]", nbins, kEqMaxFine);
    if (wide_bins(nbins) && n >= ((int64_t)1 << 24))
        return set_err(ctx, GPFC_EINVAL, "n = %lld: above %d bins n must be below 2^24", (long long)n, kMaxNbinsLane);
    return GPFC_OK;
}

int shift_of(int nbins)
{
    if (nbins & (nbins - 1)) return -1;
    int l = 0;
    while ((1 << l) < nbins) ++l;
    return 32 - l;
}

// Buffers of the fixed-point fold of one star: prep outputs and the quantised flux.
struct WideBuffers {
    double *partial;
    StarStats *stats;
    SampleScratch smp;
    long long *q;
    unsigned int *maxbits;
    int *kscale;
};

int prep_groups(int64_t n) { return (int)std::min<int64_t>(256, std::max<int64_t>(1, (n + 8191) / 8192)); }

size_t carve_wide(void *base, int64_t n, WideBuffers &w)
{
    Carver c(base);
    w.partial = c.take<double>((size_t)4 * prep_groups(n));
    w.stats = c.take<StarStats>(1);
    const int64_t se = scratch_elems(n, 1);
    w.smp.tau_lo = c.take<uint32_t>(se);
    w.smp.tau_hi = c.take<int32_t>(se);
    w.smp.x = c.take<float>(se);
    w.smp.xq = nullptr;  // the two-tier fold quantises on its own
    w.smp.thg = nullptr;
    w.smp.flags = c.take<uint8_t>(se / 16 + 64);
    w.q = c.take<long long>(n);
    w.maxbits = c.take<unsigned int>(1);
    w.kscale = c.take<int>(1);
    return c.off;
}

cudaError_t prep_wide(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, double t0,
                      const WideBuffers &w)
{
    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, w.smp, w.partial, prep_groups(n), w.stats,
                                ctx->status_dev, ctx->stream);
    if (e == cudaSuccess) e = launch_eq_prep(w.smp.x, n, w.maxbits, w.q, w.kscale, ctx->num_sms, ctx->stream);
    return e;
}

EqParams eq_params(gpfc_ctx *ctx, const WideBuffers &w, int64_t n, const double *periods, int64_t np, int nfine,
                   int nbins)
{
    EqParams p{};
    p.tau_lo = w.smp.tau_lo;
    p.tau_hi = w.smp.tau_hi;
    p.q = w.q;
    p.n = n;
    p.periods = periods;
    p.np = np;
    p.nfine = nfine;
    p.nbins = nbins;
    p.fshift = shift_of(nfine);
    p.ppb = eq_periods_per_block(nfine);
    p.kscale = w.kscale;
    p.red32 = eq_red32(n) ? 1 : 0;
    p.stats = w.stats;
    p.status = ctx->status_dev;
    return p;
}

// Equal-width fold above the lane-private limit (means and/or counts out).
int run_fold_wide(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                  int64_t np, int32_t nbins, double t0, float *folded, int32_t *counts)
{
    WideBuffers w{};
    int rc = ensure_ws(ctx, carve_wide(nullptr, n, w) + 256);
    if (rc) return rc;
    carve_wide(ctx->ws, n, w);
    cudaError_t e = prep_wide(ctx, times, flux, n, t0, w);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    EqParams p = eq_params(ctx, w, n, periods, np, nbins, nbins);
    p.width_only = 1;
    p.folded = folded;
    p.counts = counts;
    KernelTimer timer(ctx);
    e = launch_eq_fold(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "fold kernel");
    timer.stop();
    return GPFC_OK;
}

// Chunk of the wide box search: one block pass of periods per SM.
int64_t wide_chunk(const gpfc_ctx *ctx, int64_t np, int nbins)
{
    return std::min<int64_t>(np, (int64_t)ctx->num_sms * eq_periods_per_block(nbins));
}

size_t box_wide_bytes(const gpfc_ctx *ctx, int64_t n, int64_t np, int nbins)
{
    WideBuffers w{};
    Carver c(nullptr);
    c.take<uint8_t>(carve_wide(nullptr, n, w));
    const int64_t chunk = wide_chunk(ctx, np, nbins);
    c.take<float>((size_t)chunk * nbins);
    c.take<int32_t>((size_t)chunk * nbins);
    c.take<unsigned long long>(1);
    return c.off + 256;
}

// Box-SNR search above the lane-private limit: chunks of the equal-width fixed-point fold,
// each scored by the warp-per-profile kernel from its centred sums.
int run_search_box_wide(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                        int64_t np, int32_t nbins, double t0, const gpfc_box_params *bp, float *score,
                        int64_t *best_index, float *best_score)
{
    int rc = ensure_ws(ctx, box_wide_bytes(ctx, n, np, nbins));
    if (rc) return rc;
    const int64_t chunk = wide_chunk(ctx, np, nbins);
    Carver c(ctx->ws);
    WideBuffers w{};
    carve_wide(c.take<uint8_t>(carve_wide(nullptr, n, w)), n, w);
    float *cs = c.take<float>((size_t)chunk * nbins);
    int32_t *cc = c.take<int32_t>((size_t)chunk * nbins);
    unsigned long long *key = c.take<unsigned long long>(1);
    const bool want_best = best_index || best_score;
    cudaError_t e = prep_wide(ctx, times, flux, n, t0, w);
    if (e == cudaSuccess && want_best) e = cudaMemsetAsync(key, 0, sizeof(*key), ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    KernelTimer timer(ctx);
    for (int64_t k0 = 0; k0 < np && e == cudaSuccess; k0 += chunk) {
        const int64_t nk = std::min<int64_t>(chunk, np - k0);
        EqParams p = eq_params(ctx, w, n, periods + k0, nk, nbins, nbins);
        p.width_only = 1;
        p.sums = cs;
        p.counts = cc;
        e = launch_eq_fold(p, ctx->num_sms, ctx->stream);
        if (e != cudaSuccess) break;
        BoxCoopParams q{};
        q.sums = cs;
        q.counts = cc;
        q.k_begin = k0;
        q.rows = nk;
        q.nbins = nbins;
        q.w_min = bp->w_min;
        q.w_max = bp->w_max;
        q.sigma_user = bp->sigma > 0.0 ? (float)bp->sigma : 0.f;
        q.stats = w.stats;
        q.nstars = 1;
        q.score = score;
        q.best_key = want_best ? key : nullptr;
        e = launch_box_coop(q, ctx->num_sms, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "fold and box kernels");
    timer.stop();
    if (want_best) {
        e = launch_argmax_finalize(key, 1, best_index, best_score, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "argmax finalize");
    }
    return GPFC_OK;
}

// Quantise + fold one star in `mode`; fills p.* outputs set by the caller.
int run_fold(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
             int64_t np, int32_t nbins, double t0, int mode, FoldParams p, bool want_key,
             FoldBuffers *out_fb)
{
    const FoldPlan pl = plan_fold(ctx, n, np, nbins, find_tuned(ctx, nbins, mode, n));
    FoldBuffers fb{};
    const size_t need = carve_fold(nullptr, pl, n, 1, nbins, fb);
    int rc = ensure_ws(ctx, need);
    if (rc) return rc;
    carve_fold(ctx->ws, pl, n, 1, nbins, fb);
    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, fb.smp, fb.partial, pl.G,
                                fb.stats, ctx->status_dev, ctx->stream, pl.chunk);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    p.smp = fb.smp;
    p.lc_off = nullptr;
    p.n = n;
    p.periods = periods;
    p.grid_off = nullptr;
    p.np = np;
    p.task_off = nullptr;
    p.ntasks = pl.ntasks;
    p.nstars = 1;
    p.stats = fb.stats;
    p.nbins = nbins;
    p.shift = shift_of(nbins);
    p.warps = pl.warps;
    p.chunk = pl.chunk;
    p.layout = pl.layout;
    p.streams = pl.streams;
    p.tile = pl.tile;
    p.ws_sc = fb.ws_sc;
    p.ws_cnt = fb.ws_cnt;
    p.status = ctx->status_dev;
    p.best_key = nullptr;
    if (want_key) {
        p.best_key = fb.key;
        e = cudaMemsetAsync(fb.key, 0, sizeof(unsigned long long), ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMemsetAsync");
    }
    KernelTimer timer(ctx);
    e = launch_fold(p, mode, pl.grid, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "fold kernel");
    timer.stop();
    if (out_fb) *out_fb = fb;
    return GPFC_OK;
}

// The box search runs outside the fold's epilogue: in the one-kernel search, or in the
// separate warp-per-profile kernel.
bool warp_box(const gpfc_ctx *ctx, int nbins)
{
    return ctx->box_path == GPFC_BOX_WARP || ctx->box_path == GPFC_BOX_FUSED ||
           (ctx->box_path == GPFC_BOX_AUTO && nbins >= 256);
}

// A fold-then-score search as a two-stage pipeline forked off stream st (the two-kernel
// box search, the CNN search): chunk i is folded on a high-priority side stream into
// buffer i % 2 and scored on a low-priority side stream, so the next fold's blocks take
// each SM as soon as the scorer's blocks leave it and the two stages' tails overlap. The
// fold of chunk i + 2 waits for the scoring of chunk i (same buffer). Both side streams
// are joined back into st, also on error, so that a capture stays whole.
template <class FoldFn, class BoxFn>
cudaError_t box_pipeline(gpfc_ctx *ctx, cudaStream_t st, int64_t nchunks, FoldFn fold, BoxFn box)
{
    cudaStream_t sf = ctx->side[0], sb = ctx->side[1];
    cudaEvent_t *ev = ctx->side_ev;  // fork, fold done x2, scorer done x2, join x2
    cudaError_t e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sf, ev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sb, ev[0], 0);
    for (int64_t i = 0; i < nchunks && e == cudaSuccess; ++i) {
        const int b = (int)(i & 1);
        if (i >= 2) e = cudaStreamWaitEvent(sf, ev[3 + b], 0);
        if (e == cudaSuccess) e = fold(i, b, sf);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + b], sf);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sb, ev[1 + b], 0);
        if (e == cudaSuccess) e = box(i, b, sb);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3 + b], sb);
    }
    cudaError_t j = cudaEventRecord(ev[5], sf);
    if (j == cudaSuccess) j = cudaStreamWaitEvent(st, ev[5], 0);
    if (j == cudaSuccess) j = cudaEventRecord(ev[6], sb);
    if (j == cudaSuccess) j = cudaStreamWaitEvent(st, ev[6], 0);
    return e != cudaSuccess ? e : j;
}

// Runs launch() on stream sf; with timing on, between a pair of events kept for
// gpfc_fold_launch_times.
template <class Launch>
cudaError_t timed_fold(gpfc_ctx *ctx, cudaStream_t sf, Launch launch)
{
    if (!ctx->timing) return launch();
    const size_t need = 2 * (size_t)(ctx->fold_ev_used + 1);
    while (ctx->fold_ev.size() < need) {
        cudaEvent_t ev = nullptr;
        const cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        ctx->fold_ev.push_back(ev);
    }
    cudaEvent_t *ev = &ctx->fold_ev[2 * ctx->fold_ev_used];
    cudaError_t e = cudaEventRecord(ev[0], sf);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], sf);
    if (e == cudaSuccess) ++ctx->fold_ev_used;
    return e;
}

// Plan of the one-kernel search (grid of resident search blocks), or false if its block
// does not fit.
bool fused_plan(gpfc_ctx *ctx, int64_t n, int64_t np, int nbins, FoldPlan &pl)
{
    pl = plan_fold(ctx, n, np, nbins, find_tuned(ctx, nbins, kModeFold, n));
    int bps = search_blocks_per_sm(nbins, pl.warps, pl.layout, pl.tile, pl.streams);
    if (bps < 1 && !ctx->fold_cfg.tile && pl.tile > 512) {
        // the scorer staging did not fit beside 1024-sample tiles: halve the tiles
        pl.tile = 512;
        ctx->last_plan.tile = 512;
        bps = search_blocks_per_sm(nbins, pl.warps, pl.layout, pl.tile, pl.streams);
    }
    if (bps < 1) return false;
    pl.bps = bps;
    pl.grid = (int)std::min<int64_t>(pl.ntasks, (int64_t)ctx->num_sms * bps);
    // a block numbers the rows of its tasks in 32-bit tickets
    return (pl.ntasks + pl.grid - 1) / pl.grid * pl.ppc < ((int64_t)1 << 31);
}

struct FusedBuffers {
    FoldBuffers fb;
    float *ring_s;
    int32_t *ring_c;
    int64_t *ring_k;
};

size_t carve_fused(void *base, const FoldPlan &pl, int64_t n, int nbins, FusedBuffers &B)
{
    Carver c(base);
    FoldBuffers tmp{};
    uint8_t *fold_base = c.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, tmp));
    if (base) carve_fold(fold_base, pl, n, 1, nbins, B.fb);
    const size_t rows = (size_t)pl.grid * 2 * pl.ppc;
    B.ring_s = c.take<float>(rows * nbins);
    B.ring_c = c.take<int32_t>(rows * nbins);
    B.ring_k = c.take<int64_t>(rows);
    return c.off + 256;
}

// Fold + box-SNR search of one star in one kernel (kModeSearch). Returns 1 (nothing
// enqueued) when the search block does not fit.
int run_search_box_fused(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                         int64_t np, int32_t nbins, double t0, const gpfc_box_params *bp, float *score,
                         int64_t *best_index, float *best_score)
{
    FoldPlan pl{};
    if (!fused_plan(ctx, n, np, nbins, pl)) return 1;
    FusedBuffers B{};
    int rc = ensure_ws(ctx, carve_fused(nullptr, pl, n, nbins, B));
    if (rc) return rc;
    carve_fused(ctx->ws, pl, n, nbins, B);
    const bool want_best = best_index || best_score;
    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, B.fb.smp, B.fb.partial, pl.G,
                                B.fb.stats, ctx->status_dev, ctx->stream, pl.chunk);
    if (e == cudaSuccess && want_best) e = cudaMemsetAsync(B.fb.key, 0, sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    FoldParams p{};
    p.smp = B.fb.smp;
    p.n = n;
    p.periods = periods;
    p.np = np;
    p.ntasks = pl.ntasks;
    p.nstars = 1;
    p.stats = B.fb.stats;
    p.nbins = nbins;
    p.shift = shift_of(nbins);
    p.warps = pl.warps;
    p.chunk = pl.chunk;
    p.layout = pl.layout;
    p.streams = pl.streams;
    p.tile = pl.tile;
    p.ws_sc = B.fb.ws_sc;
    p.ws_cnt = B.fb.ws_cnt;
    p.sums = B.ring_s;
    p.counts = B.ring_c;
    p.slot_k = B.ring_k;
    p.score = score;
    p.w_min = bp->w_min;
    p.w_max = bp->w_max;
    p.sigma_user = bp->sigma > 0.0 ? (float)bp->sigma : 0.f;
    p.best_key = want_best ? B.fb.key : nullptr;
    p.status = ctx->status_dev;
    KernelTimer timer(ctx);
    e = timed_fold(ctx, ctx->stream, [&] { return launch_fold(p, kModeSearch, pl.grid, ctx->stream); });
    if (e != cudaSuccess) return cuda_err(ctx, e, "search kernel");
    timer.stop();
    if (want_best) {
        e = launch_argmax_finalize(B.fb.key, 1, best_index, best_score, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "argmax finalize");
    }
    return GPFC_OK;
}

// Period groups and sample streams of the fold launch of a chunk of nk periods, and its
// grid. A chunk too short to give every SM a block of pl.warps period groups (the last chunk
// of a search) takes fewer groups per block, each with more sample streams, so that more SMs
// share it: layout 3 only, whose results do not depend on the launch shape, and only where
// the block shape was not fixed by gpfc_set_fold_config. The launch fits the workspace
// carved for pl (no more blocks, no more periods per block).
static int chunk_shape(const gpfc_ctx *ctx, const FoldPlan &pl, int64_t nk, FoldParams &p)
{
    p.warps = pl.warps;
    p.streams = pl.streams;
    if (pl.layout == kLayoutRed32 && ctx->fold_cfg.warps == 0 && ctx->fold_cfg.streams == 0) {
        const int64_t per_sm = (nk + (int64_t)32 * ctx->num_sms - 1) / ((int64_t)32 * ctx->num_sms);
        const int w = (int)std::max<int64_t>(1, std::min<int64_t>(pl.warps, per_sm));
        if (w < pl.warps) {
            p.warps = w;
            p.streams = std::max(1, std::min(kMaxRedWarps / w, pl.warps * pl.streams / w));
        }
    }
    p.ntasks = (nk + 32 * p.warps - 1) / (32 * p.warps);
    return (int)std::min<int64_t>(p.ntasks, pl.grid);
}

// Workspace of run_search_box_warp: the fold buffers, two chunks of sums and counts.
size_t box_warp_bytes(const FoldPlan &pl, int64_t n, int64_t np, int nbins)
{
    const int64_t chunk = std::min<int64_t>(np, (int64_t)pl.grid * pl.ppc);
    FoldBuffers fb{};
    Carver c(nullptr);
    c.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, fb));
    for (int b = 0; b < 2; ++b) {
        c.take<float>((size_t)chunk * nbins);
        c.take<int32_t>((size_t)chunk * nbins);
    }
    return c.off + 256;
}

// Fold + box-SNR search of one star with the search in its own kernel. Periods go
// through in chunks of one fold wave; a chunk's centred bin sums and counts stay resident
// in L2 between the fold and the warp-per-profile scorer.
int run_search_box_warp(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                        int64_t np, int32_t nbins, double t0, const gpfc_box_params *bp, float *score,
                        int64_t *best_index, float *best_score)
{
    const FoldPlan pl = plan_fold(ctx, n, np, nbins, find_tuned(ctx, nbins, kModeFold, n));
    const int64_t chunk = std::min<int64_t>(np, (int64_t)pl.grid * pl.ppc);
    FoldBuffers fb{};
    int rc = ensure_ws(ctx, box_warp_bytes(pl, n, np, nbins));
    if (rc) return rc;
    Carver w(ctx->ws);
    uint8_t *fold_base = w.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, fb));
    carve_fold(fold_base, pl, n, 1, nbins, fb);
    float *cs[2];
    int32_t *cc[2];
    for (int b = 0; b < 2; ++b) {
        cs[b] = w.take<float>((size_t)chunk * nbins);
        cc[b] = w.take<int32_t>((size_t)chunk * nbins);
    }
    const bool want_best = best_index || best_score;
    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, fb.smp, fb.partial, pl.G, fb.stats,
                                ctx->status_dev, ctx->stream, pl.chunk);
    if (e == cudaSuccess && want_best) e = cudaMemsetAsync(fb.key, 0, sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    KernelTimer timer(ctx);
    auto fold = [&](int64_t i, int b, cudaStream_t sf) {
        const int64_t k0 = i * chunk, nk = std::min<int64_t>(chunk, np - k0);
        FoldParams p{};
        p.smp = fb.smp;
        p.n = n;
        p.periods = periods + k0;
        p.np = nk;
        p.nstars = 1;
        p.stats = fb.stats;
        p.nbins = nbins;
        p.shift = shift_of(nbins);
        p.chunk = pl.chunk;
        p.layout = pl.layout;
        p.tile = pl.tile;
        p.ws_sc = fb.ws_sc;
        p.ws_cnt = fb.ws_cnt;
        p.sums = cs[b];
        p.counts = cc[b];
        p.status = ctx->status_dev;
        const int grid = chunk_shape(ctx, pl, nk, p);
        return timed_fold(ctx, sf, [&] { return launch_fold(p, kModeFold, grid, sf); });
    };
    auto box = [&](int64_t i, int b, cudaStream_t sb) {
        const int64_t k0 = i * chunk, nk = std::min<int64_t>(chunk, np - k0);
        BoxCoopParams q{};
        q.sums = cs[b];
        q.counts = cc[b];
        q.k_begin = k0;
        q.rows = nk;
        q.nbins = nbins;
        q.w_min = bp->w_min;
        q.w_max = bp->w_max;
        q.sigma_user = bp->sigma > 0.0 ? (float)bp->sigma : 0.f;
        q.stats = fb.stats;
        q.nstars = 1;
        q.score = score;
        q.best_key = want_best ? fb.key : nullptr;
        return launch_box_coop(q, ctx->num_sms, sb);
    };
    e = box_pipeline(ctx, ctx->stream, (np + chunk - 1) / chunk, fold, box);
    if (e != cudaSuccess) return cuda_err(ctx, e, "fold and box kernels");
    timer.stop();
    if (want_best) {
        e = launch_argmax_finalize(fb.key, 1, best_index, best_score, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "argmax finalize");
    }
    return GPFC_OK;
}

bool cnn_weights_ok(const gpfc_cnn_weights *wt)
{
    if (!wt) return false;
    const float *ptrs[10] = {wt->conv1_w, wt->conv1_b, wt->conv2_w, wt->conv2_b, wt->conv3_w,
                             wt->conv3_b, wt->fc1_w,   wt->fc1_b,   wt->fc2_w,   wt->fc2_b};
    for (const float *q : ptrs)
        if (!q) return false;
    return true;
}

CnnSrc cnn_src(const gpfc_cnn_weights *wt)
{
    return CnnSrc{wt->conv1_w, wt->conv1_b, wt->conv2_w, wt->conv2_b, wt->conv3_w,
                  wt->conv3_b, wt->fc1_w,   wt->fc1_b,   wt->fc2_w,   wt->fc2_b};
}

// Fold + CNN search of one star. Periods go through in chunks of one fold wave (one
// block of 4 x 32 periods per SM); each chunk's means and counts, and the CNN's fc1
// operand tiles for half a chunk at a time, stay resident in L2 between the kernels.
int run_search_cnn(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                   int64_t np, int32_t nbins, double t0, const gpfc_cnn_weights *wt, float *score,
                   int64_t *best_index, float *best_score)
{
    const FoldPlan pl = plan_fold(ctx, n, np, nbins, find_tuned(ctx, nbins, kModeFold, n));
    const int64_t wave = (int64_t)pl.grid * pl.ppc;
    const int64_t chunk = std::min<int64_t>(np, wave);
    const int64_t half = (chunk + 1) / 2;
    FoldBuffers fb{};
    Carver c(nullptr);
    c.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, fb));
    for (int b = 0; b < 2; ++b) {
        c.take<float>((size_t)chunk * nbins);
        c.take<int32_t>((size_t)chunk * nbins);
    }
    c.take<uint8_t>(cnn_dev_bytes());
    c.take<uint8_t>(cnn_h3t_bytes(half));
    c.take<unsigned long long>(1);
    int rc = ensure_ws(ctx, c.off + 256);
    if (rc) return rc;
    Carver w(ctx->ws);
    uint8_t *fold_base = w.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, fb));
    carve_fold(fold_base, pl, n, 1, nbins, fb);
    float *cf[2];
    int32_t *cc[2];
    for (int b = 0; b < 2; ++b) {
        cf[b] = w.take<float>((size_t)chunk * nbins);
        cc[b] = w.take<int32_t>((size_t)chunk * nbins);
    }
    const CnnDev dev = cnn_dev_carve(w.take<uint8_t>(cnn_dev_bytes()));
    uint8_t *h3t = w.take<uint8_t>(cnn_h3t_bytes(half));
    unsigned long long *key = w.take<unsigned long long>(1);

    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, fb.smp, fb.partial, pl.G, fb.stats,
                                ctx->status_dev, ctx->stream, pl.chunk);
    if (e == cudaSuccess) e = launch_cnn_prep(cnn_src(wt), dev, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    KernelTimer timer(ctx);
    // the same two-stream pipeline as the box search: chunk i folds on the high-priority
    // stream into buffer i % 2 while the CNN scores chunk i - 1 on the low-priority one
    // (its fc1 operand tiles are used on that stream only)
    auto fold = [&](int64_t i, int b, cudaStream_t sf) {
        const int64_t k0 = i * chunk, nk = std::min<int64_t>(chunk, np - k0);
        FoldParams p{};
        p.smp = fb.smp;
        p.n = n;
        p.periods = periods + k0;
        p.np = nk;
        p.nstars = 1;
        p.stats = fb.stats;
        p.nbins = nbins;
        p.shift = shift_of(nbins);
        p.chunk = pl.chunk;
        p.layout = pl.layout;
        p.tile = pl.tile;
        p.ws_sc = fb.ws_sc;
        p.ws_cnt = fb.ws_cnt;
        p.folded = cf[b];
        p.counts = cc[b];
        p.status = ctx->status_dev;
        return launch_fold(p, kModeFold, chunk_shape(ctx, pl, nk, p), sf);
    };
    auto cnn = [&](int64_t i, int b, cudaStream_t sb) {
        const int64_t k0 = i * chunk, nk = std::min<int64_t>(chunk, np - k0);
        cudaError_t ec = cudaSuccess;
        for (int64_t h0 = 0; h0 < nk && ec == cudaSuccess; h0 += half) {
            const int64_t nh = std::min<int64_t>(half, nk - h0);
            CnnConvParams cp{};
            cp.folded = cf[b];
            cp.counts = cc[b];
            cp.k_begin = h0;
            cp.np = nh;
            cp.w = dev;
            cp.h3t = h3t;
            cp.status = ctx->status_dev;
            ec = launch_cnn_conv(cp, ctx->num_sms, sb);
            if (ec != cudaSuccess) break;
            CnnFcParams fp{};
            fp.h3t = h3t;
            fp.k_begin = h0;
            fp.np = nh;
            fp.w = dev;
            fp.score = score + k0;
            fp.status = ctx->status_dev;
            ec = launch_cnn_fc(fp, ctx->num_sms, sb);
        }
        return ec;
    };
    e = box_pipeline(ctx, ctx->stream, (np + chunk - 1) / chunk, fold, cnn);
    if (e != cudaSuccess) return cuda_err(ctx, e, "fold and CNN kernels");
    timer.stop();
    if (best_index || best_score) {
        e = cudaMemsetAsync(key, 0, sizeof(*key), ctx->stream);
        if (e == cudaSuccess) e = launch_argmax(score, np, key, ctx->stream);
        if (e == cudaSuccess) e = launch_argmax_finalize(key, 1, best_index, best_score, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "argmax kernels");
    }
    return GPFC_OK;
}


// ------------------------------------------------------------------ autotuner

// Times the fold kernel of `mode` (kModeFold without output writes, or kModeBox) on one
// star over its first periods, for every launch config of the default layout's
// arithmetic whose resident periods per SM are at least half the largest, and keeps the
// fastest under (nbins, mode, log2 n_key).
int tune_fold(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
              int64_t np, int nbins, int mode, const gpfc_box_params *bp, int64_t n_key, gpfc_fold_config *out)
{
    const int64_t P = std::min<int64_t>(np, (int64_t)4 * ctx->num_sms * 128);
    struct Cand {
        gpfc_fold_config cfg;
        int resident;
    };
    std::vector<Cand> cands;
    int best_res = 0;
    // layouts of the default's arithmetic only (FP32 partial sums: 1 and 2; exact fixed
    // point: 3), so tuning never changes a result
    const bool fixed = (ctx->fold_cfg.layout ? ctx->fold_cfg.layout : default_layout(nbins)) == kLayoutRed32;
    for (int layout = 1; layout <= 3; ++layout) {
        if ((layout == kLayoutRed32) != fixed) continue;
        for (int tile = 512; tile <= kMaxTile; tile *= 2) {
            const int maxw = fold_max_warps(nbins, layout, tile);
            for (int w = 1; w <= maxw; ++w) {
                const int bps = fold_blocks_per_sm(nbins, w, layout, tile);
                if (bps < 1) continue;
                const int res = 32 * w * bps;
                cands.push_back(Cand{gpfc_fold_config{w, layout, 0, tile, bps}, res});
                best_res = std::max(best_res, res);
            }
        }
    }
    if (cands.empty()) return set_err(ctx, GPFC_ENOTSUP, "no fold launch config fits nbins = %d", nbins);
    // workspace: the largest carve of any candidate plus the sample score buffer
    size_t need = 0;
    for (const Cand &c : cands) {
        if (2 * c.resident < best_res) continue;
        FoldBuffers fb{};
        need = std::max(need, carve_fold(nullptr, plan_with(ctx, n, P, nbins, c.cfg), n, 1, nbins, fb));
    }
    int rc = ensure_ws(ctx, need + (size_t)P * sizeof(float) + 512);
    if (rc) return rc;
    float *score = reinterpret_cast<float *>(static_cast<char *>(ctx->ws) + ((need + 255) & ~(size_t)255));
    bool prepped = false;
    float best_ms = 0.f;
    gpfc_fold_config best{};
    for (const Cand &c : cands) {
        if (2 * c.resident < best_res) continue;
        const FoldPlan pl = plan_with(ctx, n, P, nbins, c.cfg);
        FoldBuffers fb{};
        carve_fold(ctx->ws, pl, n, 1, nbins, fb);  // the sample scratch sits at the same place for all
        cudaError_t e = cudaSuccess;
        if (!prepped) {
            // the longest chunk, so the fixed-point flux fits every candidate's chunks
            e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, NAN, fb.smp, fb.partial, pl.G, fb.stats,
                            ctx->status_dev, ctx->stream, 65520);
            if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
            prepped = true;
        }
        FoldParams p{};
        p.smp = fb.smp;
        p.n = n;
        p.periods = periods;
        p.np = P;
        p.ntasks = pl.ntasks;
        p.nstars = 1;
        p.stats = fb.stats;
        p.nbins = nbins;
        p.shift = shift_of(nbins);
        p.warps = pl.warps;
        p.chunk = pl.chunk;
        p.layout = pl.layout;
        p.streams = pl.streams;
        p.tile = pl.tile;
        p.ws_sc = fb.ws_sc;
        p.ws_cnt = fb.ws_cnt;
        p.status = ctx->status_dev;
        if (mode == kModeBox) {
            p.score = score;
            p.w_min = bp->w_min;
            p.w_max = bp->w_max;
            p.sigma_user = bp->sigma > 0.0 ? (float)bp->sigma : 0.f;
        }
        e = launch_fold(p, mode, pl.grid, ctx->stream);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_start, ctx->stream);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch_fold(p, mode, pl.grid, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_stop, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev_stop);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev_start, ctx->ev_stop);
        if (e != cudaSuccess) return cuda_err(ctx, e, "autotune launch");
        if ((rc = take_latched(ctx))) return rc;
        ms *= 0.5f;
        if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            best = gpfc_fold_config{pl.warps, pl.layout, 0, pl.tile, pl.bps};
        }
    }
    ctx->timed = false;
    const int lg = floor_log2(n_key);
    bool found = false;
    for (auto &t : ctx->tuned)
        if (t.nbins == nbins && t.mode == mode && t.lg == lg) {
            t.cfg = best;
            t.ms = best_ms;
            found = true;
        }
    if (!found) ctx->tuned.push_back(gpfc_ctx::Tuned{nbins, mode, lg, best, best_ms});
    if (out) *out = best;
    return GPFC_OK;
}

// ------------------------------------------------------------------ batched search

struct BatchArgs {
    int32_t S;
    int32_t nbins;
    int32_t scorer;
    int32_t box_warp;  // box search: 0 in the fold's epilogue, 1 separate kernel, 2 one kernel
    const int64_t *lc_off;
    const double *times;
    const float *flux;
    int64_t n_total;
    const int64_t *grid_off;
    const double *periods;
    int64_t np_total;
    const double *t0s;
    gpfc_box_params box;
    gpfc_cnn_weights wt;
    float *score;
    int64_t *best_index;
    float *best_score;
};

struct BatchBuffers {
    int64_t *lc_s, *grid_s, *task_off;
    FoldBuffers fb;
    CnnDev dev;
    uint8_t *h3t;
    // two chunks of profiles (box: centred sums; CNN: means), counts and slot maps, for the
    // fold/score pipeline
    float *chunk_f[2];
    int32_t *chunk_c[2];
    int64_t *chunk_k[2];
    // one-kernel box search: the blocks' two-slot rings
    float *ring_s;
    int32_t *ring_c;
    int64_t *ring_k;
};

// Workspace of a batched search: validated offsets and task starts, the fold buffers of
// all stars, and for the CNN one fold wave of profiles, their slot map, the CNN's weight
// copies and fc1 operand tiles for half a wave.
size_t carve_batched(void *base, const BatchArgs &A, const FoldPlan &pl, int64_t slots, BatchBuffers &B)
{
    Carver c(base);
    B.lc_s = c.take<int64_t>(A.S + 1);
    B.grid_s = c.take<int64_t>(A.S + 1);
    B.task_off = c.take<int64_t>(A.S + 1);
    FoldBuffers tmp{};
    uint8_t *fold_base = c.take<uint8_t>(carve_fold(nullptr, pl, A.n_total, A.S, A.nbins, tmp));
    carve_fold(fold_base, pl, A.n_total, A.S, A.nbins, B.fb);
    if (A.scorer == GPFC_SCORER_BOX && A.box_warp == 2) {
        const size_t rows = (size_t)pl.grid * 2 * pl.ppc;
        B.ring_s = c.take<float>(rows * A.nbins);
        B.ring_c = c.take<int32_t>(rows * A.nbins);
        B.ring_k = c.take<int64_t>(rows);
    } else if (A.scorer == GPFC_SCORER_CNN || A.box_warp) {
        for (int b = 0; b < 2; ++b) {
            B.chunk_f[b] = c.take<float>((size_t)slots * A.nbins);
            B.chunk_c[b] = c.take<int32_t>((size_t)slots * A.nbins);
            B.chunk_k[b] = c.take<int64_t>(slots);
        }
    }
    if (A.scorer == GPFC_SCORER_CNN) {
        const int64_t half = (slots + 1) / 2;
        uint8_t *d = c.take<uint8_t>(cnn_dev_bytes());
        B.dev = base ? cnn_dev_carve(d) : CnnDev{};
        B.h3t = c.take<uint8_t>(cnn_h3t_bytes(half));
    }
    return c.off + 256;
}

// Upper bound of the total fold tasks: sum_s ceil(a_s / ppc) <= (sum_s a_s + S (ppc - 1)) / ppc.
int64_t task_bound(const BatchArgs &A, int ppc) { return (A.np_total + (int64_t)A.S * (ppc - 1)) / ppc; }

// All launches of a batched search on stream st (no host synchronisation, so the
// sequence can be captured in a CUDA graph).
cudaError_t enqueue_batched(gpfc_ctx *ctx, const BatchArgs &A, const FoldPlan &pl, const BatchBuffers &B,
                            cudaStream_t st)
{
    const int64_t T = task_bound(A, pl.ppc);
    cudaError_t e = launch_batch_plan(A.lc_off, A.grid_off, A.S, A.n_total, A.np_total, pl.ppc, B.lc_s, B.grid_s,
                                      B.task_off, ctx->status_dev, st);
    if (e == cudaSuccess)
        e = launch_prep(A.times, A.flux, B.lc_s, A.n_total, A.S, 0, A.t0s, NAN, B.fb.smp, B.fb.partial, pl.G,
                        B.fb.stats, ctx->status_dev, st, pl.chunk);
    if (e != cudaSuccess) return e;
    FoldParams p{};
    p.smp = B.fb.smp;
    p.lc_off = B.lc_s;
    p.n = A.n_total;
    p.periods = A.periods;
    p.grid_off = B.grid_s;
    p.np = A.np_total;
    p.task_off = B.task_off;
    p.ntasks_dev = B.task_off + A.S;
    p.nstars = A.S;
    p.stats = B.fb.stats;
    p.nbins = A.nbins;
    p.shift = shift_of(A.nbins);
    p.warps = pl.warps;
    p.chunk = pl.chunk;
    p.layout = pl.layout;
    p.streams = pl.streams;
    p.tile = pl.tile;
    p.ws_sc = B.fb.ws_sc;
    p.ws_cnt = B.fb.ws_cnt;
    p.status = ctx->status_dev;
    const bool want_best = A.best_index || A.best_score;
    if (A.scorer == GPFC_SCORER_BOX && A.box_warp == 2) {
        // one kernel over every task: fold warps and a scorer warp per block
        if (want_best) e = cudaMemsetAsync(B.fb.key, 0, sizeof(unsigned long long) * A.S, st);
        if (e != cudaSuccess) return e;
        p.sums = B.ring_s;
        p.counts = B.ring_c;
        p.slot_k = B.ring_k;
        p.score = A.score;
        p.w_min = A.box.w_min;
        p.w_max = A.box.w_max;
        p.sigma_user = A.box.sigma > 0.0 ? (float)A.box.sigma : 0.f;
        p.best_key = want_best ? B.fb.key : nullptr;
        p.task_begin = 0;
        p.ntasks = T;
        e = launch_fold(p, kModeSearch, (int)std::min<int64_t>(T, pl.grid), st);
        if (e == cudaSuccess && want_best) e = launch_argmax_finalize(B.fb.key, A.S, A.best_index, A.best_score, st);
        return e;
    }
    if (A.scorer == GPFC_SCORER_BOX && A.box_warp) {
        // chunks of one task per resident block, each chunk's sums and counts by slot
        if (want_best) e = cudaMemsetAsync(B.fb.key, 0, sizeof(unsigned long long) * A.S, st);
        if (e != cudaSuccess) return e;
        const int64_t wave = (int64_t)pl.grid;
        auto fold = [&](int64_t i, int b, cudaStream_t sf) {
            FoldParams q = p;
            q.sums = B.chunk_f[b];
            q.counts = B.chunk_c[b];
            q.slot_k = B.chunk_k[b];
            q.task_begin = i * wave;
            q.ntasks = std::min<int64_t>(T, q.task_begin + wave);
            return launch_fold(q, kModeFold, (int)(q.ntasks - q.task_begin), sf);
        };
        auto box = [&](int64_t i, int b, cudaStream_t sb) {
            const int64_t tb = i * wave, te = std::min<int64_t>(T, tb + wave);
            BoxCoopParams q{};
            q.sums = B.chunk_f[b];
            q.counts = B.chunk_c[b];
            q.slot_k = B.chunk_k[b];
            q.rows = (te - tb) * pl.ppc;
            q.nbins = A.nbins;
            q.w_min = A.box.w_min;
            q.w_max = A.box.w_max;
            q.sigma_user = A.box.sigma > 0.0 ? (float)A.box.sigma : 0.f;
            q.stats = B.fb.stats;
            q.grid_off = B.grid_s;
            q.nstars = A.S;
            q.score = A.score;
            q.best_key = want_best ? B.fb.key : nullptr;
            return launch_box_coop(q, ctx->num_sms, sb);
        };
        e = box_pipeline(ctx, st, (T + wave - 1) / wave, fold, box);
        if (e == cudaSuccess && want_best) e = launch_argmax_finalize(B.fb.key, A.S, A.best_index, A.best_score, st);
        return e;
    }
    if (A.scorer == GPFC_SCORER_BOX) {
        p.score = A.score;
        p.w_min = A.box.w_min;
        p.w_max = A.box.w_max;
        p.sigma_user = A.box.sigma > 0.0 ? (float)A.box.sigma : 0.f;
        if (want_best) {
            p.best_key = B.fb.key;
            e = cudaMemsetAsync(B.fb.key, 0, sizeof(unsigned long long) * A.S, st);
        }
        p.task_begin = 0;
        p.ntasks = T;
        if (e == cudaSuccess) e = launch_fold(p, kModeBox, (int)std::min<int64_t>(T, pl.grid), st);
        if (e == cudaSuccess && want_best) e = launch_argmax_finalize(B.fb.key, A.S, A.best_index, A.best_score, st);
        return e;
    }
    e = launch_cnn_prep(cnn_src(&A.wt), B.dev, st);
    if (e != cudaSuccess) return e;
    // chunks of one task per resident block through the fold/score pipeline
    const int64_t wave = (int64_t)pl.grid;
    auto fold = [&](int64_t i, int b, cudaStream_t sf) {
        FoldParams q = p;
        q.folded = B.chunk_f[b];
        q.counts = B.chunk_c[b];
        q.slot_k = B.chunk_k[b];
        q.task_begin = i * wave;
        q.ntasks = std::min<int64_t>(T, q.task_begin + wave);
        return launch_fold(q, kModeFold, (int)(q.ntasks - q.task_begin), sf);
    };
    auto cnn = [&](int64_t i, int b, cudaStream_t sb) {
        const int64_t tb = i * wave, te = std::min<int64_t>(T, tb + wave);
        const int64_t slots = (te - tb) * pl.ppc, half = (slots + 1) / 2;
        cudaError_t ec = cudaSuccess;
        for (int64_t h0 = 0; h0 < slots && ec == cudaSuccess; h0 += half) {
            const int64_t nh = std::min<int64_t>(half, slots - h0);
            CnnConvParams cp{};
            cp.folded = B.chunk_f[b];
            cp.counts = B.chunk_c[b];
            cp.k_begin = h0;
            cp.np = nh;
            cp.w = B.dev;
            cp.h3t = B.h3t;
            cp.status = ctx->status_dev;
            ec = launch_cnn_conv(cp, ctx->num_sms, sb);
            if (ec != cudaSuccess) break;
            CnnFcParams fp{};
            fp.h3t = B.h3t;
            fp.k_begin = h0;
            fp.np = nh;
            fp.w = B.dev;
            fp.score = A.score;
            fp.slot_k = B.chunk_k[b];
            fp.status = ctx->status_dev;
            ec = launch_cnn_fc(fp, ctx->num_sms, sb);
        }
        return ec;
    };
    e = box_pipeline(ctx, st, (T + wave - 1) / wave, fold, cnn);
    if (e == cudaSuccess && want_best) {
        e = launch_argmax_segmented(A.score, B.grid_s, A.S, B.fb.key, ctx->num_sms, st);
        if (e == cudaSuccess) e = launch_argmax_finalize(B.fb.key, A.S, A.best_index, A.best_score, st);
    }
    return e;
}

void drop_graph(gpfc_ctx *ctx)
{
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    ctx->graph_key.clear();
}

// Capture the batched search into a CUDA graph on the context's private capture stream
// (or reuse the graph of an identical earlier call) and launch it on the context's stream.
int launch_batched_graph(gpfc_ctx *ctx, const BatchArgs &A, const FoldPlan &pl, const BatchBuffers &B)
{
    std::vector<uint8_t> key(sizeof(BatchArgs) + sizeof(FoldPlan) + 2 * sizeof(size_t));
    memcpy(key.data(), &A, sizeof(BatchArgs));
    memcpy(key.data() + sizeof(BatchArgs), &pl, sizeof(FoldPlan));
    const size_t wsinfo[2] = {reinterpret_cast<size_t>(ctx->ws), ctx->ws_bytes};
    memcpy(key.data() + sizeof(BatchArgs) + sizeof(FoldPlan), wsinfo, sizeof(wsinfo));
    cudaError_t e = cudaSuccess;
    if (!ctx->graph_exec || key != ctx->graph_key) {
        drop_graph(ctx);
        if (!ctx->cap_stream) {
            e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamCreateWithFlags");
        }
        e = cnn_register_kernels();  // attribute calls stay outside the capture
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaFuncSetAttribute");
        e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamBeginCapture");
        const cudaError_t eq = enqueue_batched(ctx, A, pl, B, ctx->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (eq != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cuda_err(ctx, eq != cudaSuccess ? eq : e, "capture of the batched search");
        }
        e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->graph_exec = nullptr;
            return cuda_err(ctx, e, "cudaGraphInstantiate");
        }
        ctx->graph_key = key;
    }
    e = cudaGraphLaunch(ctx->graph_exec, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphLaunch");
    return GPFC_OK;
}

}  // namespace

extern "C" {

int gpfc_version(void) { return 100; }

const char *gpfc_strerror(int status)
{
    switch (status) {
    case GPFC_OK: return "ok";
    case GPFC_EINVAL: return "invalid argument";
    case GPFC_ENOMEM: return "device workspace allocation failed";
    case GPFC_ECUDA: return "CUDA error";
    case GPFC_ERANGE: return "value outside the fixed-point range";
    case GPFC_ETIMEOUT: return "device-side wait timed out";
    case GPFC_ENOTSUP: return "unsupported configuration";
    default: return "unknown status";
    }
}

int gpfc_create(gpfc_ctx **out, int device, void *stream)
{
    if (!out) return GPFC_EINVAL;
    *out = nullptr;
    gpfc_ctx *ctx = new (std::nothrow) gpfc_ctx();
    if (!ctx) return GPFC_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&ctx->status_host), 64, cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *ctx->status_host = 0u;
        e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&ctx->status_dev), ctx->status_host, 0);
    }
    if (e == cudaSuccess) e = static_cast<cudaError_t>(fold_register_kernels());
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side[0], cudaStreamNonBlocking, prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side[1], cudaStreamNonBlocking, prio_least);
    for (cudaEvent_t &ev : ctx->side_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_stop);
    if (e != cudaSuccess) {
        snprintf(g_create_error, sizeof(g_create_error), "gpfc_create on device %d: %s", device,
                 cudaGetErrorString(e));
        cudaGetLastError();
        if (ctx->status_host) cudaFreeHost(ctx->status_host);
        for (cudaStream_t q : ctx->side)
            if (q) cudaStreamDestroy(q);
        for (cudaEvent_t ev : ctx->side_ev)
            if (ev) cudaEventDestroy(ev);
        if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
        delete ctx;
        return GPFC_ECUDA;
    }
    *out = ctx;
    return GPFC_OK;
}

void gpfc_destroy(gpfc_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->status_host) cudaFreeHost(ctx->status_host);
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    if (ctx->ev_stop) cudaEventDestroy(ctx->ev_stop);
    drop_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaEvent_t ev : ctx->fold_ev) cudaEventDestroy(ev);
    for (cudaStream_t q : ctx->side)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t ev : ctx->side_ev)
        if (ev) cudaEventDestroy(ev);
    delete ctx;
}

int gpfc_set_fold_config(gpfc_ctx *ctx, const gpfc_fold_config *cfg)
{
    if (!ctx) return GPFC_EINVAL;
    if (!cfg) {
        ctx->fold_cfg = gpfc_fold_config{0, 0, 0, 0, 0};
        return GPFC_OK;
    }
    if (cfg->warps < 0 || cfg->warps > kMaxFoldWarps || cfg->layout < 0 || cfg->layout > 3 ||
        cfg->chunk < 0 || cfg->chunk > 65520 || (cfg->tile != 0 && cfg->tile != 512 && cfg->tile != 1024 &&
                                                   cfg->tile != 2048) || cfg->blocks_per_sm < 0 ||
        cfg->streams < 0 || cfg->streams > kMaxRedWarps || (cfg->streams > 1 && cfg->layout != kLayoutRed32) ||
        (cfg->warps > 0 && cfg->warps * std::max(1, cfg->streams) > kMaxRedWarps))
        return set_err(ctx, GPFC_EINVAL, "fold config out of range");
    ctx->fold_cfg = *cfg;
    return GPFC_OK;
}

int gpfc_fold_max_warps(int32_t nbins, int32_t layout)
{
    if (nbins < 2 || nbins > kMaxNbinsLane || layout < 1 || layout > 3) return 0;
    return fold_max_warps(nbins, layout);
}

int gpfc_last_fold_plan(const gpfc_ctx *ctx, gpfc_fold_config *out)
{
    if (!ctx || !out) return GPFC_EINVAL;
    *out = ctx->last_plan;
    return GPFC_OK;
}

int gpfc_set_autotune(gpfc_ctx *ctx, int enable)
{
    if (!ctx) return GPFC_EINVAL;
    ctx->autotune = enable != 0;
    if (enable < 0) ctx->tuned.clear();
    return GPFC_OK;
}

int gpfc_set_box_path(gpfc_ctx *ctx, int path)
{
    if (!ctx) return GPFC_EINVAL;
    if (path < GPFC_BOX_AUTO || path > GPFC_BOX_FUSED) return set_err(ctx, GPFC_EINVAL, "box path %d unknown", path);
    ctx->box_path = path;
    return GPFC_OK;
}

int gpfc_set_graph(gpfc_ctx *ctx, int enable)
{
    if (!ctx) return GPFC_EINVAL;
    ctx->use_graph = enable != 0;
    if (!ctx->use_graph) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamSynchronize");
        drop_graph(ctx);
    }
    return GPFC_OK;
}

int gpfc_autotune(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                  int64_t n_periods, int32_t nbins, int scorer, const void *scorer_params, gpfc_fold_config *out)
{
    int rc = check_fold_args(ctx, times, flux, n, periods, n_periods, nbins);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    if ((rc = take_latched(ctx))) return rc;
    const gpfc_box_params *bp = nullptr;
    if (scorer == GPFC_SCORER_BOX) {
        bp = static_cast<const gpfc_box_params *>(scorer_params);
        if (!bp || bp->w_min < 1 || bp->w_max < bp->w_min || bp->w_max > nbins)
            return set_err(ctx, GPFC_EINVAL, "box scorer needs gpfc_box_params with 1 <= w_min <= w_max <= nbins");
    } else if (scorer != GPFC_SCORER_CNN) {
        return set_err(ctx, GPFC_ENOTSUP, "scorer %d not available", scorer);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(ctx->stream, &cs);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return set_err(ctx, GPFC_EINVAL, "autotune cannot run under stream capture");
    const int mode = scorer == GPFC_SCORER_BOX && !warp_box(ctx, nbins) ? kModeBox : kModeFold;
    return tune_fold(ctx, times, flux, n, periods, n_periods, nbins, mode, bp, n, out);
}

int gpfc_check_wait_timeout(gpfc_ctx *ctx, int64_t limit_cycles)
{
    if (!ctx) return GPFC_EINVAL;
    if (limit_cycles < 1000 || limit_cycles > 4000000000LL)
        return set_err(ctx, GPFC_EINVAL, "limit_cycles outside [1e3, 4e9]");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    cudaError_t e = launch_wait_selftest((long long)limit_cycles, ctx->status_dev, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "wait self-test kernel");
    return GPFC_OK;
}

int gpfc_workspace_size(gpfc_ctx *ctx, int64_t n, int64_t n_periods, int32_t nbins, size_t *bytes)
{
    if (!ctx || !bytes) return GPFC_EINVAL;
    if (n < 1 || n_periods < 1 || nbins < 2 || nbins > kEqMaxFine)
        return set_err(ctx, GPFC_EINVAL, "bad sizes");
    if (wide_bins(nbins)) {
        *bytes = box_wide_bytes(ctx, n, n_periods, nbins);
        return GPFC_OK;
    }
    // the largest of a fold (gpfc_fold, the epilogue search), the warp-per-profile search
    // and the one-kernel search; planning them leaves the context's last plan as it was
    const gpfc_fold_config last = ctx->last_plan;
    const FoldPlan pb = plan_fold(ctx, n, n_periods, nbins, find_tuned(ctx, nbins, kModeBox, n));
    const FoldPlan pf = plan_fold(ctx, n, n_periods, nbins, find_tuned(ctx, nbins, kModeFold, n));
    FoldBuffers fb{};
    *bytes = std::max(carve_fold(nullptr, pb, n, 1, nbins, fb), box_warp_bytes(pf, n, n_periods, nbins));
    FoldPlan ps{};
    if (fused_plan(ctx, n, n_periods, nbins, ps)) {
        FusedBuffers B{};
        *bytes = std::max(*bytes, carve_fused(nullptr, ps, n, nbins, B));
    }
    ctx->last_plan = last;
    return GPFC_OK;
}

int gpfc_set_timing(gpfc_ctx *ctx, int enable)
{
    if (!ctx) return GPFC_EINVAL;
    ctx->timing = enable != 0;
    ctx->timed = false;
    return GPFC_OK;
}

int gpfc_kernel_time_ms(gpfc_ctx *ctx, float *ms)
{
    if (!ctx || !ms) return GPFC_EINVAL;
    if (!ctx->timing || !ctx->timed) return set_err(ctx, GPFC_EINVAL, "no timed launch recorded");
    cudaError_t e = cudaEventSynchronize(ctx->ev_stop);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ctx->ev_start, ctx->ev_stop);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaEventElapsedTime");
    return GPFC_OK;
}

int gpfc_fold_launch_times(gpfc_ctx *ctx, float *total_ms, int32_t *launches)
{
    if (!ctx || !total_ms || !launches) return GPFC_EINVAL;
    if (!ctx->timing || ctx->fold_ev_used == 0) return set_err(ctx, GPFC_EINVAL, "no timed fold launch recorded");
    float sum = 0.f;
    for (int i = 0; i < ctx->fold_ev_used; ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(ctx->fold_ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->fold_ev[2 * i], ctx->fold_ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaEventElapsedTime");
        sum += ms;
    }
    *total_ms = sum;
    *launches = ctx->fold_ev_used;
    return GPFC_OK;
}

int gpfc_set_stream(gpfc_ctx *ctx, void *stream)
{
    if (!ctx) return GPFC_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamSynchronize");
    ctx->stream = static_cast<cudaStream_t>(stream);
    return GPFC_OK;
}

const char *gpfc_last_error(const gpfc_ctx *ctx) { return ctx ? ctx->last_error : g_create_error; }

int gpfc_num_sms(const gpfc_ctx *ctx) { return ctx ? ctx->num_sms : 0; }

int gpfc_sync(gpfc_ctx *ctx)
{
    if (!ctx) return GPFC_EINVAL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamSynchronize");
    return take_latched(ctx);
}

int gpfc_fold(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
              int64_t n_periods, int32_t nbins, double t0, float *folded, int32_t *counts)
{
    int rc = check_fold_args(ctx, times, flux, n, periods, n_periods, nbins);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    if ((rc = take_latched(ctx))) return rc;
    if (wide_bins(nbins)) return run_fold_wide(ctx, times, flux, n, periods, n_periods, nbins, t0, folded, counts);
    FoldParams p{};
    p.folded = folded;
    p.counts = counts;
    return run_fold(ctx, times, flux, n, periods, n_periods, nbins, t0, kModeFold, p, false, nullptr);
}

int gpfc_fold_equal_count(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                          int64_t n_periods, int32_t nfine, int32_t nbins, double t0, float *folded)
{
    if (!ctx) return GPFC_EINVAL;
    if (!times || !flux || !periods || !folded) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n < 1 || n >= ((int64_t)1 << 24)) return set_err(ctx, GPFC_EINVAL, "n = %lld outside [1, 2^24 - 1]", (long long)n);
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX)
        return set_err(ctx, GPFC_EINVAL, "n_periods = %lld outside [1, 2^31-1]", (long long)n_periods);
    if (nbins < 2 || nfine < nbins || nfine > kEqMaxFine)
        return set_err(ctx, GPFC_EINVAL, "need 2 <= nbins <= nfine <= %d (nbins %d, nfine %d)", kEqMaxFine, nbins, nfine);
    const int ppb = eq_periods_per_block(nfine);
    if (ppb < 1) return set_err(ctx, GPFC_ENOTSUP, "nfine = %d does not fit shared memory", nfine);
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    WideBuffers w{};
    rc = ensure_ws(ctx, carve_wide(nullptr, n, w) + 256);
    if (rc) return rc;
    carve_wide(ctx->ws, n, w);
    cudaError_t e = prep_wide(ctx, times, flux, n, t0, w);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    EqParams p = eq_params(ctx, w, n, periods, n_periods, nfine, nbins);
    p.folded = folded;
    KernelTimer timer(ctx);
    e = launch_eq_fold(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "two-tier fold kernel");
    timer.stop();
    return GPFC_OK;
}

int gpfc_score_box(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                   int32_t nbins, const gpfc_box_params *params, float *score, int32_t *best_s,
                   int32_t *best_w)
{
    if (!ctx) return GPFC_EINVAL;
    if (!folded || !counts || !score || !params) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX) return set_err(ctx, GPFC_EINVAL, "bad n_periods");
    if (nbins < 2 || nbins > kEqMaxFine) return set_err(ctx, GPFC_EINVAL, "nbins outside [2, %d]", kEqMaxFine);
    if (params->w_min < 1 || params->w_max < params->w_min || params->w_max > nbins)
        return set_err(ctx, GPFC_EINVAL, "box widths must satisfy 1 <= w_min <= w_max <= nbins");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    BoxCoopParams q{};
    q.means = folded;
    q.counts = counts;
    q.rows = n_periods;
    q.nbins = nbins;
    q.w_min = params->w_min;
    q.w_max = params->w_max;
    q.sigma_user = params->sigma > 0.0 ? (float)params->sigma : 1.0f;
    q.nstars = 1;
    q.score = score;
    q.best_s = best_s;
    q.best_w = best_w;
    KernelTimer timer(ctx);
    cudaError_t e = launch_box_coop(q, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "box kernel");
    timer.stop();
    return GPFC_OK;
}

static int cnn_forward(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                       int32_t nbins, const gpfc_cnn_weights *wt, float *score, float *logit)
{
    if (!ctx) return GPFC_EINVAL;
    if (!folded || (!score && !logit) || !wt) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (nbins != 256) return set_err(ctx, GPFC_ENOTSUP, "the CNN scorer takes 256-bin profiles, got %d", nbins);
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX) return set_err(ctx, GPFC_EINVAL, "bad n_periods");
    const float *ptrs[10] = {wt->conv1_w, wt->conv1_b, wt->conv2_w, wt->conv2_b, wt->conv3_w,
                             wt->conv3_b, wt->fc1_w,   wt->fc1_b,   wt->fc2_w,   wt->fc2_b};
    for (const float *q : ptrs)
        if (!q) return set_err(ctx, GPFC_EINVAL, "NULL CNN parameter");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    const int64_t chunk = std::min<int64_t>(n_periods, kCnnChunk);
    Carver c(nullptr);
    c.take<uint8_t>(cnn_dev_bytes());
    c.take<uint8_t>(cnn_h3t_bytes(chunk));
    rc = ensure_ws(ctx, c.off + 256);
    if (rc) return rc;
    Carver c2(ctx->ws);
    const CnnDev dev = cnn_dev_carve(c2.take<uint8_t>(cnn_dev_bytes()));
    uint8_t *h3t = c2.take<uint8_t>(cnn_h3t_bytes(chunk));
    const CnnSrc src{wt->conv1_w, wt->conv1_b, wt->conv2_w, wt->conv2_b, wt->conv3_w,
                     wt->conv3_b, wt->fc1_w,   wt->fc1_b,   wt->fc2_w,   wt->fc2_b};
    cudaError_t e = launch_cnn_prep(src, dev, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "CNN weight preparation");
    KernelTimer timer(ctx);
    for (int64_t k0 = 0; k0 < n_periods; k0 += chunk) {
        const int64_t nk = std::min<int64_t>(chunk, n_periods - k0);
        CnnConvParams cp{};
        cp.folded = folded;
        cp.counts = counts;
        cp.k_begin = k0;
        cp.np = nk;
        cp.w = dev;
        cp.h3t = h3t;
        cp.status = ctx->status_dev;
        e = launch_cnn_conv(cp, ctx->num_sms, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "CNN conv kernel");
        CnnFcParams fp{};
        fp.h3t = h3t;
        fp.k_begin = k0;
        fp.np = nk;
        fp.w = dev;
        fp.score = score;
        fp.logit = logit;
        fp.status = ctx->status_dev;
        e = launch_cnn_fc(fp, ctx->num_sms, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "CNN fc kernel");
    }
    timer.stop();
    return GPFC_OK;
}

int gpfc_score_cnn(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                   int32_t nbins, const gpfc_cnn_weights *wt, float *score)
{
    return cnn_forward(ctx, folded, counts, n_periods, nbins, wt, score, nullptr);
}

int gpfc_cnn_logits(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                    int32_t nbins, const gpfc_cnn_weights *wt, float *logit)
{
    return cnn_forward(ctx, folded, counts, n_periods, nbins, wt, nullptr, logit);
}

size_t gpfc_cnn_saved_bytes(int64_t batch) { return batch > 0 ? cnn_saved_bytes(batch) : 0; }

int gpfc_cnn_forward_train(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t batch,
                           int32_t nbins, const gpfc_cnn_weights *wt, float *logit, void *saved)
{
    if (!ctx) return GPFC_EINVAL;
    if (!folded || !logit || !saved || !cnn_weights_ok(wt)) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (nbins != 256) return set_err(ctx, GPFC_ENOTSUP, "the CNN scorer takes 256-bin profiles, got %d", nbins);
    if (batch < 1 || batch > (int64_t)1 << 22) return set_err(ctx, GPFC_EINVAL, "batch outside [1, 2^22]");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    rc = ensure_ws(ctx, cnn_dev_bytes() + 256);
    if (rc) return rc;
    const CnnDev dev = cnn_dev_carve(ctx->ws);
    cudaError_t e = launch_cnn_prep(cnn_src(wt), dev, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "CNN weight preparation");
    const CnnSaved S = CnnSaved::layout(batch);
    uint8_t *sv = static_cast<uint8_t *>(saved);
    KernelTimer timer(ctx);
    CnnConvParams cp{};
    cp.folded = folded;
    cp.counts = counts;
    cp.k_begin = 0;
    cp.np = batch;
    cp.w = dev;
    cp.h3t = sv + S.h3t;
    cp.xsave = reinterpret_cast<float *>(sv + S.x);
    cp.a1save = reinterpret_cast<float *>(sv + S.a1);
    cp.h1save = reinterpret_cast<uint16_t *>(sv + S.h1);
    cp.a2save = reinterpret_cast<float *>(sv + S.a2);
    cp.h2save = reinterpret_cast<uint16_t *>(sv + S.h2);
    cp.a3save = reinterpret_cast<float *>(sv + S.a3);
    cp.status = ctx->status_dev;
    e = launch_cnn_conv(cp, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "CNN conv kernel");
    CnnFcParams fp{};
    fp.h3t = sv + S.h3t;
    fp.k_begin = 0;
    fp.np = batch;
    fp.w = dev;
    fp.logit = logit;
    fp.z1save = reinterpret_cast<float *>(sv + S.z1);
    fp.status = ctx->status_dev;
    e = launch_cnn_fc(fp, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "CNN fc kernel");
    timer.stop();
    return GPFC_OK;
}

int gpfc_cnn_backward(gpfc_ctx *ctx, const float *dlogit, int64_t batch, const gpfc_cnn_weights *wt,
                      const void *saved, const gpfc_cnn_grads *gr)
{
    if (!ctx) return GPFC_EINVAL;
    if (!dlogit || !saved || !gr || !cnn_weights_ok(wt)) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    float *gp[10] = {gr->conv1_w, gr->conv1_b, gr->conv2_w, gr->conv2_b, gr->conv3_w,
                     gr->conv3_b, gr->fc1_w,   gr->fc1_b,   gr->fc2_w,   gr->fc2_b};
    for (float *q : gp)
        if (!q) return set_err(ctx, GPFC_EINVAL, "NULL gradient buffer");
    if (batch < 1 || batch > (int64_t)1 << 22) return set_err(ctx, GPFC_EINVAL, "batch outside [1, 2^22]");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    const int nblk = (int)std::min<int64_t>(batch, (int64_t)ctx->num_sms * 2);
    rc = ensure_ws(ctx, cnn_backward_ws_bytes(batch, nblk, ctx->num_sms));
    if (rc) return rc;
    const CnnGrads g{gr->conv1_w, gr->conv1_b, gr->conv2_w, gr->conv2_b, gr->conv3_w,
                     gr->conv3_b, gr->fc1_w,   gr->fc1_b,   gr->fc2_w,   gr->fc2_b};
    cudaError_t e = launch_cnn_backward(cnn_src(wt), static_cast<const uint8_t *>(saved), batch, dlogit, g, ctx->ws,
                                        nblk, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "CNN backward kernels");
    return GPFC_OK;
}

int gpfc_bce_with_logits(gpfc_ctx *ctx, const float *logit, const float *label, int64_t n, float *loss,
                         float *dlogit)
{
    if (!ctx) return GPFC_EINVAL;
    if (!logit || !label || (!loss && !dlogit)) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n < 1) return set_err(ctx, GPFC_EINVAL, "n < 1");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    rc = ensure_ws(ctx, 256 * sizeof(double) + 256);
    if (rc) return rc;
    cudaError_t e = launch_bce(logit, label, n, dlogit, loss, ctx->ws, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "loss kernel");
    return GPFC_OK;
}

int gpfc_adam(gpfc_ctx *ctx, float *param, const float *grad, float *m, float *v, int64_t n, float lr,
              float beta1, float beta2, float eps, int64_t step)
{
    if (!ctx) return GPFC_EINVAL;
    if (!param || !grad || !m || !v) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n < 1 || step < 1) return set_err(ctx, GPFC_EINVAL, "n and step must be >= 1");
    cudaSetDevice(ctx->device);
    const double c1 = 1.0 - std::pow((double)beta1, (double)step);
    const double c2 = 1.0 - std::pow((double)beta2, (double)step);
    cudaError_t e = launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, (float)c1, (float)c2, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "Adam kernel");
    return GPFC_OK;
}

int gpfc_synth_profiles(gpfc_ctx *ctx, uint64_t seed, int64_t first, int64_t n, int32_t nbins,
                        const gpfc_synth_params *params, float *folded, int32_t *counts, float *label,
                        double *fold_period, float *flux_std)
{
    if (!ctx) return GPFC_EINVAL;
    if (!params || !folded) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n < 1 || first < 0 || first + n > ((int64_t)1 << 32)) return set_err(ctx, GPFC_EINVAL, "bad index range");
    if (nbins < 2 || nbins > 256) return set_err(ctx, GPFC_EINVAL, "nbins outside [2, 256]");
    const gpfc_synth_params &sp = *params;
    if (sp.n_cadences < 1 || !(sp.cadence > 0) || !(sp.sigma_min > 0) || !(sp.sigma_max >= sp.sigma_min) ||
        !(sp.depth_min > 0) || !(sp.depth_max >= sp.depth_min) || !(sp.p_min > 0) || !(sp.p_max >= sp.p_min) ||
        sp.dur_min_h < 0 || sp.dur_max_h < sp.dur_min_h || sp.drift_bins < 0)
        return set_err(ctx, GPFC_EINVAL, "synthesis parameters out of range");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    SynthParams p{seed, first, n, nbins, sp, folded, counts, label, fold_period, flux_std};
    cudaError_t e = launch_synth(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "synthesis kernel");
    return GPFC_OK;
}

int gpfc_synth_vectors(gpfc_ctx *ctx, uint64_t seed, int64_t first, int64_t n, int32_t nbins,
                       const gpfc_vector_params *params, float *folded, float *label, float *alpha,
                       float *sigma_bin)
{
    if (!ctx) return GPFC_EINVAL;
    if (!params || !folded) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n < 1 || first < 0 || first + n > ((int64_t)1 << 32)) return set_err(ctx, GPFC_EINVAL, "bad index range");
    if (nbins < 8 || nbins > 1024) return set_err(ctx, GPFC_EINVAL, "nbins outside [8, 1024]");
    const gpfc_vector_params &v = *params;
    if (!(v.alpha_pos_min >= 0) || !(v.alpha_pos_max >= v.alpha_pos_min) || !(v.alpha_neg_max >= 0) ||
        !(v.q_min > 0) || !(v.q_max >= v.q_min) || !(v.q_max < 1) || !(v.sigma_min > 0) ||
        !(v.sigma_max >= v.sigma_min) || v.n_points < 1)
        return set_err(ctx, GPFC_EINVAL, "vector parameters out of range");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    VectorParams p{seed, first, n, nbins, v, folded, label, alpha, sigma_bin};
    cudaError_t e = launch_paper_vectors(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "vector synthesis kernel");
    return GPFC_OK;
}

int gpfc_best_period(gpfc_ctx *ctx, const float *score, int64_t n_periods, int64_t *best_index,
                     float *best_score)
{
    if (!ctx) return GPFC_EINVAL;
    if (!score || (!best_index && !best_score)) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX) return set_err(ctx, GPFC_EINVAL, "bad n_periods");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    rc = ensure_ws(ctx, 256);
    if (rc) return rc;
    auto *key = static_cast<unsigned long long *>(ctx->ws);
    cudaError_t e = cudaMemsetAsync(key, 0, sizeof(*key), ctx->stream);
    if (e == cudaSuccess) e = launch_argmax(score, n_periods, key, ctx->stream);
    if (e == cudaSuccess) e = launch_argmax_finalize(key, 1, best_index, best_score, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "argmax kernels");
    return GPFC_OK;
}

int gpfc_search(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
                int64_t n_periods, int32_t nbins, double t0, int scorer, const void *scorer_params,
                float *score, int64_t *best_index, float *best_score)
{
    int rc = check_fold_args(ctx, times, flux, n, periods, n_periods, nbins);
    if (rc) return rc;
    if (!score) return set_err(ctx, GPFC_EINVAL, "NULL score");
    cudaSetDevice(ctx->device);
    if ((rc = take_latched(ctx))) return rc;
    if (scorer == GPFC_SCORER_BOX) {
        const auto *bp = static_cast<const gpfc_box_params *>(scorer_params);
        if (!bp) return set_err(ctx, GPFC_EINVAL, "box scorer needs gpfc_box_params");
        if (bp->w_min < 1 || bp->w_max < bp->w_min || bp->w_max > nbins)
            return set_err(ctx, GPFC_EINVAL, "box widths must satisfy 1 <= w_min <= w_max <= nbins");
        FoldParams p{};
        p.score = score;
        p.w_min = bp->w_min;
        p.w_max = bp->w_max;
        p.sigma_user = bp->sigma > 0.0 ? (float)bp->sigma : 0.f;
        const bool want_best = best_index || best_score;
        if (wide_bins(nbins))
            return run_search_box_wide(ctx, times, flux, n, periods, n_periods, nbins, t0, bp, score, best_index,
                                       best_score);
        if (warp_box(ctx, nbins)) {
            if (ctx->box_path != GPFC_BOX_WARP) {
                rc = run_search_box_fused(ctx, times, flux, n, periods, n_periods, nbins, t0, bp, score, best_index,
                                          best_score);
                if (rc != 1) return rc;
            }
            return run_search_box_warp(ctx, times, flux, n, periods, n_periods, nbins, t0, bp, score, best_index,
                                       best_score);
        }
        FoldBuffers fb{};
        rc = run_fold(ctx, times, flux, n, periods, n_periods, nbins, t0, kModeBox, p, want_best, &fb);
        if (rc) return rc;
        if (want_best) {
            cudaError_t e = launch_argmax_finalize(fb.key, 1, best_index, best_score, ctx->stream);
            if (e != cudaSuccess) return cuda_err(ctx, e, "argmax finalize");
        }
        return GPFC_OK;
    }
    if (scorer == GPFC_SCORER_CNN) {
        const auto *wt = static_cast<const gpfc_cnn_weights *>(scorer_params);
        if (!cnn_weights_ok(wt)) return set_err(ctx, GPFC_EINVAL, "CNN scorer needs gpfc_cnn_weights");
        if (nbins != 256) return set_err(ctx, GPFC_ENOTSUP, "the CNN scorer takes 256 bins, got %d", nbins);
        return run_search_cnn(ctx, times, flux, n, periods, n_periods, nbins, t0, wt, score, best_index, best_score);
    }
    return set_err(ctx, GPFC_ENOTSUP, "scorer %d not available", scorer);
}

static_assert(sizeof(gpfc_star_summary) == sizeof(PeakSummaryDev), "summary layout");
static_assert(sizeof(gpfc_peak) == sizeof(PeakDev), "peak layout");

int gpfc_peaks(gpfc_ctx *ctx, const float *score, const double *periods, int32_t n_stars,
               const int64_t *grid_offsets, int64_t n_periods, double k_sigma, int32_t min_width,
               double harmonic_tol, int32_t max_peaks, gpfc_star_summary *summary, gpfc_peak *peaks)
{
    if (!ctx) return GPFC_EINVAL;
    if (!score || !periods || !summary) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n_stars < 1 || (!grid_offsets && n_stars != 1)) return set_err(ctx, GPFC_EINVAL, "bad n_stars / offsets");
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX) return set_err(ctx, GPFC_EINVAL, "bad n_periods");
    if (min_width < 1 || max_peaks < 0 || max_peaks > 64 || !(k_sigma == k_sigma) || !(harmonic_tol >= 0.0))
        return set_err(ctx, GPFC_EINVAL, "bad decision parameters");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    PeakParams p{};
    p.score = score;
    p.periods = periods;
    p.grid_off = grid_offsets;
    p.np = n_periods;
    p.nstars = n_stars;
    p.k_sigma = k_sigma;
    p.min_width = min_width;
    p.harm_tol = harmonic_tol;
    p.max_peaks = max_peaks;
    p.summary = reinterpret_cast<PeakSummaryDev *>(summary);
    p.peaks = max_peaks > 0 ? reinterpret_cast<PeakDev *>(peaks) : nullptr;
    KernelTimer timer(ctx);
    cudaError_t e = launch_peaks(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "decision kernel");
    timer.stop();
    return GPFC_OK;
}

int gpfc_detrend(gpfc_ctx *ctx, const double *times, const float *flux, const uint8_t *mask, int64_t n,
                 const gpfc_detrend_params *params, double *times_out, float *flux_out, int32_t *segment_out,
                 int64_t *n_out)
{
    if (!ctx) return GPFC_EINVAL;
    if (!times || !flux || !times_out || !flux_out || !n_out) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n < 1 || n > ((int64_t)1 << 24)) return set_err(ctx, GPFC_EINVAL, "n = %lld outside [1, 2^24]", (long long)n);
    DetrendParams p{};
    gpfc_detrend_params q{};
    if (params) q = *params;
    p.time_gap = q.time_gap > 0.0 ? q.time_gap : 30.0 * 0.020428;
    p.flux_gap_sigma = q.flux_gap_sigma > 0.0 ? q.flux_gap_sigma : 5.0;
    p.clip_sigma = q.clip_sigma > 0.0 ? q.clip_sigma : 3.0;
    p.ridge = q.ridge > 0.0 ? q.ridge : 1e-9;
    p.edge = q.edge > 0 ? q.edge : (q.edge < 0 ? 0 : 30);
    p.max_iter = q.max_iter > 0 ? q.max_iter : 10;
    if (q.n_spacings < 0 || q.n_spacings > kDetrendMaxSpacings)
        return set_err(ctx, GPFC_EINVAL, "n_spacings must be 0..%d", kDetrendMaxSpacings);
    if (q.n_spacings == 0) {
        const double d[5] = {0.5, 1.0, 1.5, 2.0, 3.0};
        p.n_sp = 5;
        for (int i = 0; i < 5; ++i) p.sp[i] = d[i];
    } else {
        p.n_sp = q.n_spacings;
        for (int i = 0; i < p.n_sp; ++i) {
            if (!(q.spacings[i] > 0.0 && q.spacings[i] < INFINITY))
                return set_err(ctx, GPFC_EINVAL, "spacings[%d] must be positive and finite", i);
            p.sp[i] = q.spacings[i];
        }
    }
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    const int G = (int)std::min<int64_t>(4 * (int64_t)ctx->num_sms, std::max<int64_t>(1, (n + 2047) / 2048));
    auto carve = [&](void *base) {
        Carver c(base);
        p.partial = c.take<double>(2 * G);
        p.blk_count = c.take<int64_t>(G);
        p.blk_off = c.take<int64_t>(G + 1);
        p.n_seg = c.take<int64_t>(1);
        p.seg_start = c.take<int64_t>(n + 1);
        p.seg_keep = c.take<int64_t>(n);
        p.seg_off = c.take<int64_t>(n);
        p.G4 = c.take<double>(4 * n);
        p.LB = c.take<double>(4 * n);
        p.rhs = c.take<double>(n);
        p.coef = c.take<double>(n);
        p.trend = c.take<double>(n);
        p.best = c.take<double>(n);
        p.used = c.take<uint8_t>(n);
        p.used2 = c.take<uint8_t>(n);
        p.det = c.take<float>(n);
        return c.off + 256;
    };
    rc = ensure_ws(ctx, carve(nullptr));
    if (rc) return rc;
    carve(ctx->ws);
    p.t = times;
    p.f = flux;
    p.mask = mask;
    p.n = n;
    p.blocks = G;
    p.t_out = times_out;
    p.f_out = flux_out;
    p.seg_out = segment_out;
    p.n_out = n_out;
    KernelTimer timer(ctx);
    cudaError_t e = launch_detrend(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "pre-processing kernels");
    timer.stop();
    return GPFC_OK;
}

int gpfc_roc(gpfc_ctx *ctx, const float *pos, int64_t n_pos, const float *neg, int64_t n_neg, int32_t n_fpr,
             const double *fpr, int64_t *u2, float *thr, int64_t *tp)
{
    if (!ctx) return GPFC_EINVAL;
    if (!pos || !neg || !u2) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n_pos < 1 || n_pos > ((int64_t)1 << 30) || n_neg < 1 || n_neg > ((int64_t)1 << 30))
        return set_err(ctx, GPFC_EINVAL, "n_pos and n_neg must be in [1, 2^30]");
    if (n_fpr < 0 || n_fpr > kRocMaxFpr || (n_fpr > 0 && (!fpr || !thr || !tp)))
        return set_err(ctx, GPFC_EINVAL, "bad false-positive rates (0..%d, host array, outputs)", kRocMaxFpr);
    RocParams p{};
    for (int f = 0; f < n_fpr; ++f) {
        if (!(fpr[f] >= 0.0 && fpr[f] < 1.0)) return set_err(ctx, GPFC_EINVAL, "fpr[%d] outside [0, 1)", f);
        p.k[f] = (int64_t)std::floor(fpr[f] * (double)n_neg);
    }
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    p.pos = pos;
    p.n_pos = n_pos;
    p.neg = neg;
    p.n_neg = n_neg;
    p.n_fpr = n_fpr;
    p.u2 = reinterpret_cast<unsigned long long *>(u2);
    p.thr = thr;
    p.tp = reinterpret_cast<unsigned long long *>(tp);
    KernelTimer timer(ctx);
    cudaError_t e = launch_roc(p, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "ROC kernels");
    timer.stop();
    return GPFC_OK;
}

int gpfc_search_batched(gpfc_ctx *ctx, int32_t n_stars, const int64_t *lc_offsets, const double *times,
                        const float *flux, int64_t n_total, const int64_t *grid_offsets, const double *periods,
                        int64_t n_periods_total, const double *t0s, int32_t nbins, int scorer,
                        const void *scorer_params, float *score, int64_t *best_index, float *best_score)
{
    if (!ctx) return GPFC_EINVAL;
    if (!lc_offsets || !times || !flux || !grid_offsets || !periods || !score)
        return set_err(ctx, GPFC_EINVAL, "NULL input or output array");
    if (n_stars < 1 || n_stars > (1 << 24)) return set_err(ctx, GPFC_EINVAL, "n_stars = %d outside [1, 2^24]", n_stars);
    if (n_total < n_stars || n_total > ((int64_t)1 << 40))
        return set_err(ctx, GPFC_EINVAL, "n_total = %lld outside [n_stars, 2^40]", (long long)n_total);
    if (n_periods_total < n_stars || n_periods_total > ((int64_t)1 << 40))
        return set_err(ctx, GPFC_EINVAL, "n_periods_total = %lld outside [n_stars, 2^40]", (long long)n_periods_total);
    if (nbins < 2) return set_err(ctx, GPFC_EINVAL, "nbins = %d < 2", nbins);
    if (nbins > kMaxNbinsLane || fold_max_warps(nbins, kLayoutPaired16) < 1)
        return set_err(ctx, GPFC_ENOTSUP, "nbins = %d > %d", nbins, kMaxNbinsLane);
    BatchArgs A;
    memset(&A, 0, sizeof(A));  // the graph cache compares the bytes, padding included
    A.S = n_stars;
    A.nbins = nbins;
    A.scorer = scorer;
    A.lc_off = lc_offsets;
    A.times = times;
    A.flux = flux;
    A.n_total = n_total;
    A.grid_off = grid_offsets;
    A.periods = periods;
    A.np_total = n_periods_total;
    A.t0s = t0s;
    A.score = score;
    A.best_index = best_index;
    A.best_score = best_score;
    int mode = kModeFold;
    if (scorer == GPFC_SCORER_BOX) {
        const auto *bp = static_cast<const gpfc_box_params *>(scorer_params);
        if (!bp) return set_err(ctx, GPFC_EINVAL, "box scorer needs gpfc_box_params");
        if (bp->w_min < 1 || bp->w_max < bp->w_min || bp->w_max > nbins)
            return set_err(ctx, GPFC_EINVAL, "box widths must satisfy 1 <= w_min <= w_max <= nbins");
        A.box = *bp;
        A.box_warp = warp_box(ctx, nbins) ? 1 : 0;
        mode = A.box_warp ? kModeFold : kModeBox;
    } else if (scorer == GPFC_SCORER_CNN) {
        const auto *wt = static_cast<const gpfc_cnn_weights *>(scorer_params);
        if (!cnn_weights_ok(wt)) return set_err(ctx, GPFC_EINVAL, "CNN scorer needs gpfc_cnn_weights");
        if (nbins != 256) return set_err(ctx, GPFC_ENOTSUP, "the CNN scorer takes 256 bins, got %d", nbins);
        A.wt = *wt;
    } else {
        return set_err(ctx, GPFC_ENOTSUP, "scorer %d not available", scorer);
    }
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(ctx->stream, &cs);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamIsCapturing");
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    const int64_t n_avg = n_total / n_stars;
    const gpfc_fold_config *tuned = find_tuned(ctx, nbins, mode, n_avg);
    if (!tuned && ctx->autotune && !capturing) {
        // tune on the first star (its offsets are read back once)
        int64_t off[2] = {0, 0};
        e = cudaMemcpyAsync(off, lc_offsets, sizeof(off), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "reading the first star's offsets");
        const int64_t n0 = off[1] - off[0];
        if (off[0] >= 0 && n0 >= 1 && n0 <= ((int64_t)1 << 24) && off[1] <= n_total) {
            rc = tune_fold(ctx, times + off[0], flux + off[0], n0, periods, n_periods_total, nbins, mode, &A.box,
                           n_avg, nullptr);
            if (rc) return rc;
            tuned = find_tuned(ctx, nbins, mode, n_avg);
        }
    }
    FoldPlan pl = plan_fold(ctx, n_avg, n_periods_total, nbins, tuned);
    if (A.box_warp && ctx->box_path != GPFC_BOX_WARP) {
        // the one-kernel search, with the tuned fold config if its block fits, else the
        // default one
        FoldPlan ps = pl;
        int bps = search_blocks_per_sm(nbins, ps.warps, ps.layout, ps.tile, ps.streams);
        if (bps < 1) {
            ps = plan_fold(ctx, n_avg, n_periods_total, nbins, nullptr);
            bps = search_blocks_per_sm(nbins, ps.warps, ps.layout, ps.tile, ps.streams);
        }
        // a block numbers the rows of its tasks in 32-bit tickets
        const int64_t rows_per_block = (task_bound(A, ps.ppc) + ctx->num_sms - 1) / ctx->num_sms * ps.ppc;
        if (bps >= 1 && rows_per_block < ((int64_t)1 << 31)) {
            ps.bps = bps;
            ps.grid = ctx->num_sms * bps;
            pl = ps;
            A.box_warp = 2;
        }
    }
    BatchBuffers B{};
    const int64_t slots = (int64_t)pl.grid * pl.ppc;
    rc = ensure_ws(ctx, carve_batched(nullptr, A, pl, slots, B));
    if (rc) return rc;
    carve_batched(ctx->ws, A, pl, slots, B);
    KernelTimer timer(ctx);
    if (ctx->use_graph && !capturing) {
        rc = launch_batched_graph(ctx, A, pl, B);
        if (rc) return rc;
    } else {
        e = enqueue_batched(ctx, A, pl, B, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched search launches");
    }
    timer.stop();
    return GPFC_OK;
}

}  // extern "C"
