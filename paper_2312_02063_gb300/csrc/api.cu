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

#include "gpfc.h"
#include "gpfc_cnn.h"
#include "gpfc_kernels.h"
#include "gpfc_synth.h"

using namespace gpfc;

struct gpfc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint32_t *status_host = nullptr;  // mapped pinned memory
    uint32_t *status_dev = nullptr;
    gpfc_fold_config fold_cfg{0, 0, 0};
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    char last_error[512] = {0};
};

namespace {

// Profiles scored per CNN launch pair: their fc1 operand tiles (64 MB) stay in L2.
constexpr int64_t kCnnChunk = 16384;

// Message of the last failure that had no context to hold it (gpfc_create).
thread_local char g_create_error[512] = {0};

// Bracket the main kernel of a call with events when timing is enabled.
struct KernelTimer {
    gpfc_ctx *ctx;
    explicit KernelTimer(gpfc_ctx *c) : ctx(c)
    {
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
    int warps, ppc, grid, G, layout, chunk;
    int64_t ntasks;
};

int default_layout(int nbins)
{
    (void)nbins;
    return kLayoutPaired16;
}

FoldPlan plan_fold(const gpfc_ctx *ctx, int64_t n, int64_t np, int nbins)
{
    FoldPlan pl{};
    const gpfc_fold_config &cfg = ctx->fold_cfg;
    pl.layout = cfg.layout ? cfg.layout : default_layout(nbins);
    if (fold_max_warps(nbins, pl.layout) < 1) pl.layout = kLayoutPaired16;
    const int maxw = fold_max_warps(nbins, pl.layout);
    // enough blocks to cover the SMs when the grid is short, else the widest block
    int64_t per_sm = (np + (int64_t)32 * ctx->num_sms - 1) / ((int64_t)32 * ctx->num_sms);
    int w = (int)std::min<int64_t>(maxw, std::max<int64_t>(1, per_sm));
    if (cfg.warps > 0) w = std::min(cfg.warps, maxw);
    // ~64 samples per bin per chunk keeps the plain FP32 partials short; the chunk
    // partials are then added with Kahan compensation
    int64_t chunk = cfg.chunk > 0 ? cfg.chunk : (int64_t)64 * nbins;
    pl.chunk = (int)std::min<int64_t>(65520, std::max<int64_t>(256, chunk)) & ~15;
    pl.warps = w;
    pl.ppc = 32 * w;
    pl.ntasks = (np + pl.ppc - 1) / pl.ppc;
    pl.grid = (int)std::min<int64_t>(pl.ntasks, (int64_t)ctx->num_sms);
    pl.G = (int)std::min<int64_t>(256, std::max<int64_t>(1, (n + 8191) / 8192));
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
    fb.partial = c.take<double>((size_t)3 * nstars * pl.G);  // sums, squares, min steps
    fb.stats = c.take<StarStats>(nstars);
    const int64_t se = scratch_elems(n_total, nstars);
    fb.smp.tau_lo = c.take<uint32_t>(se);
    fb.smp.tau_hi = c.take<int32_t>(se);
    fb.smp.x = c.take<float>(se);
    fb.smp.flags = c.take<uint8_t>(se / 16 + 64);
    fb.ws_sc = c.take<float2>((size_t)pl.grid * nbins * pl.ppc);
    fb.ws_cnt = c.take<uint32_t>((size_t)pl.grid * nbins * pl.ppc);
    fb.key = c.take<unsigned long long>(nstars);
    return c.off + 256;
}

int check_fold_args(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n,
                    const double *periods, int64_t np, int32_t nbins)
{
    if (!ctx) return GPFC_EINVAL;
    if (!times || !flux || !periods) return set_err(ctx, GPFC_EINVAL, "NULL input array");
    if (n < 1 || n > (int64_t)1 << 24) return set_err(ctx, GPFC_EINVAL, "n = %lld outside [1, 2^24]", (long long)n);
    if (np < 1 || np > (int64_t)INT32_MAX)
        return set_err(ctx, GPFC_EINVAL, "n_periods = %lld outside [1, 2^31-1]", (long long)np);
    if (nbins < 2) return set_err(ctx, GPFC_EINVAL, "nbins = %d < 2", nbins);
    if (nbins > kMaxNbinsLane || fold_max_warps(nbins, kLayoutPaired16) < 1)
        return set_err(ctx, GPFC_ENOTSUP, "nbins = %d > %d", nbins, kMaxNbinsLane);
    return GPFC_OK;
}

int shift_of(int nbins)
{
    if (nbins & (nbins - 1)) return -1;
    int l = 0;
    while ((1 << l) < nbins) ++l;
    return 32 - l;
}

// Quantise + fold one star in `mode`; fills p.* outputs set by the caller.
int run_fold(gpfc_ctx *ctx, const double *times, const float *flux, int64_t n, const double *periods,
             int64_t np, int32_t nbins, double t0, int mode, FoldParams p, bool want_key,
             FoldBuffers *out_fb)
{
    const FoldPlan pl = plan_fold(ctx, n, np, nbins);
    FoldBuffers fb{};
    const size_t need = carve_fold(nullptr, pl, n, 1, nbins, fb);
    int rc = ensure_ws(ctx, need);
    if (rc) return rc;
    carve_fold(ctx->ws, pl, n, 1, nbins, fb);
    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, fb.smp, fb.partial, pl.G,
                                fb.stats, ctx->status_dev, ctx->stream);
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
    const int64_t wave = (int64_t)ctx->num_sms * 128;
    const int64_t chunk = std::min<int64_t>(np, wave);
    const int64_t half = (chunk + 1) / 2;
    const FoldPlan pl = plan_fold(ctx, n, chunk, nbins);
    FoldBuffers fb{};
    Carver c(nullptr);
    c.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, fb));
    c.take<float>((size_t)chunk * nbins);
    c.take<int32_t>((size_t)chunk * nbins);
    c.take<uint8_t>(cnn_dev_bytes());
    c.take<uint8_t>((size_t)((half + 127) / 128) * 32 * 128 * 64 * 2);
    c.take<unsigned long long>(1);
    int rc = ensure_ws(ctx, c.off + 256);
    if (rc) return rc;
    Carver w(ctx->ws);
    uint8_t *fold_base = w.take<uint8_t>(carve_fold(nullptr, pl, n, 1, nbins, fb));
    carve_fold(fold_base, pl, n, 1, nbins, fb);
    float *cf = w.take<float>((size_t)chunk * nbins);
    int32_t *cc = w.take<int32_t>((size_t)chunk * nbins);
    const CnnDev dev = cnn_dev_carve(w.take<uint8_t>(cnn_dev_bytes()));
    uint8_t *h3t = w.take<uint8_t>((size_t)((half + 127) / 128) * 32 * 128 * 64 * 2);
    unsigned long long *key = w.take<unsigned long long>(1);

    cudaError_t e = launch_prep(times, flux, nullptr, n, 1, n, nullptr, t0, fb.smp, fb.partial, pl.G, fb.stats,
                                ctx->status_dev, ctx->stream);
    if (e == cudaSuccess) e = launch_cnn_prep(cnn_src(wt), dev, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "prep kernels");
    KernelTimer timer(ctx);
    for (int64_t k0 = 0; k0 < np; k0 += chunk) {
        const int64_t nk = std::min<int64_t>(chunk, np - k0);
        FoldParams p{};
        p.smp = fb.smp;
        p.n = n;
        p.periods = periods + k0;
        p.np = nk;
        p.ntasks = (nk + pl.ppc - 1) / pl.ppc;
        p.nstars = 1;
        p.stats = fb.stats;
        p.nbins = nbins;
        p.shift = shift_of(nbins);
        p.warps = pl.warps;
        p.chunk = pl.chunk;
        p.layout = pl.layout;
        p.ws_sc = fb.ws_sc;
        p.ws_cnt = fb.ws_cnt;
        p.folded = cf;
        p.counts = cc;
        p.status = ctx->status_dev;
        e = launch_fold(p, kModeFold, (int)std::min<int64_t>(p.ntasks, pl.grid), ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "fold kernel");
        for (int64_t h0 = 0; h0 < nk; h0 += half) {
            const int64_t nh = std::min<int64_t>(half, nk - h0);
            CnnConvParams cp{};
            cp.folded = cf;
            cp.counts = cc;
            cp.k_begin = h0;
            cp.np = nh;
            cp.w = dev;
            cp.h3t = h3t;
            cp.status = ctx->status_dev;
            e = launch_cnn_conv(cp, ctx->num_sms, ctx->stream);
            if (e != cudaSuccess) return cuda_err(ctx, e, "CNN conv kernel");
            CnnFcParams fp{};
            fp.h3t = h3t;
            fp.k_begin = h0;
            fp.np = nh;
            fp.w = dev;
            fp.score = score + k0;
            fp.status = ctx->status_dev;
            e = launch_cnn_fc(fp, ctx->num_sms, ctx->stream);
            if (e != cudaSuccess) return cuda_err(ctx, e, "CNN fc kernel");
        }
    }
    timer.stop();
    if (best_index || best_score) {
        e = cudaMemsetAsync(key, 0, sizeof(*key), ctx->stream);
        if (e == cudaSuccess) e = launch_argmax(score, np, key, ctx->stream);
        if (e == cudaSuccess) e = launch_argmax_finalize(key, 1, best_index, best_score, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "argmax kernels");
    }
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
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_stop);
    if (e != cudaSuccess) {
        snprintf(g_create_error, sizeof(g_create_error), "gpfc_create on device %d: %s", device,
                 cudaGetErrorString(e));
        cudaGetLastError();
        if (ctx->status_host) cudaFreeHost(ctx->status_host);
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
    delete ctx;
}

int gpfc_set_fold_config(gpfc_ctx *ctx, const gpfc_fold_config *cfg)
{
    if (!ctx) return GPFC_EINVAL;
    if (!cfg) {
        ctx->fold_cfg = gpfc_fold_config{0, 0, 0};
        return GPFC_OK;
    }
    if (cfg->warps < 0 || cfg->warps > kMaxFoldWarps || cfg->layout < 0 || cfg->layout > 2 ||
        cfg->chunk < 0 || cfg->chunk > 65520)
        return set_err(ctx, GPFC_EINVAL, "fold config out of range");
    ctx->fold_cfg = *cfg;
    return GPFC_OK;
}

int gpfc_fold_max_warps(int32_t nbins, int32_t layout)
{
    if (nbins < 2 || nbins > kMaxNbinsLane || layout < 1 || layout > 2) return 0;
    return fold_max_warps(nbins, layout);
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
    FoldParams p{};
    p.folded = folded;
    p.counts = counts;
    return run_fold(ctx, times, flux, n, periods, n_periods, nbins, t0, kModeFold, p, false, nullptr);
}

int gpfc_score_box(gpfc_ctx *ctx, const float *folded, const int32_t *counts, int64_t n_periods,
                   int32_t nbins, const gpfc_box_params *params, float *score, int32_t *best_s,
                   int32_t *best_w)
{
    if (!ctx) return GPFC_EINVAL;
    if (!folded || !counts || !score || !params) return set_err(ctx, GPFC_EINVAL, "NULL argument");
    if (n_periods < 1 || n_periods > (int64_t)INT32_MAX) return set_err(ctx, GPFC_EINVAL, "bad n_periods");
    if (nbins < 2 || nbins > kMaxNbinsLane) return set_err(ctx, GPFC_EINVAL, "nbins outside [2, 1024]");
    if ((size_t)nbins * 33 * 6 > kSmemLimit - 1024) return set_err(ctx, GPFC_ENOTSUP, "nbins too large for the box kernel");
    if (params->w_min < 1 || params->w_max < params->w_min || params->w_max > nbins)
        return set_err(ctx, GPFC_EINVAL, "box widths must satisfy 1 <= w_min <= w_max <= nbins");
    cudaSetDevice(ctx->device);
    int rc = take_latched(ctx);
    if (rc) return rc;
    const float sigma = params->sigma > 0.0 ? (float)params->sigma : 1.0f;
    KernelTimer timer(ctx);
    cudaError_t e = launch_box_standalone(folded, counts, n_periods, nbins, params->w_min, params->w_max,
                                          sigma, score, best_s, best_w, ctx->stream);
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
    c.take<uint8_t>((size_t)((chunk + 127) / 128) * 32 * 128 * 64 * 2);
    rc = ensure_ws(ctx, c.off + 256);
    if (rc) return rc;
    Carver c2(ctx->ws);
    const CnnDev dev = cnn_dev_carve(c2.take<uint8_t>(cnn_dev_bytes()));
    uint8_t *h3t = c2.take<uint8_t>((size_t)((chunk + 127) / 128) * 32 * 128 * 64 * 2);
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
    rc = ensure_ws(ctx, cnn_backward_ws_bytes(batch, nblk));
    if (rc) return rc;
    const CnnGrads g{gr->conv1_w, gr->conv1_b, gr->conv2_w, gr->conv2_b, gr->conv3_w,
                     gr->conv3_b, gr->fc1_w,   gr->fc1_b,   gr->fc2_w,   gr->fc2_b};
    cudaError_t e = launch_cnn_backward(cnn_src(wt), static_cast<const uint8_t *>(saved), batch, dlogit, g, ctx->ws,
                                        nblk, ctx->stream);
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

}  // extern "C"
