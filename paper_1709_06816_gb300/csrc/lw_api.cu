// lw_api.cu -- the C ABI of liblw (declared in include/lw.h).
//
// Host side only: argument checks, pointer classification, the context's
// device workspace, copies for host buffers, and the cooperative launch of
// the persistent merge kernel (lw_merge.cu).  No clustering arithmetic runs
// on the host.

#include "../../include/lw.h"
#include "lw_internal.h"

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

struct lw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int grid_opt = 0;
    int cta_threads = lw::kThreads;  // CTA size of the merge kernel (128, 256, 512)
    int layout_opt = 0;              // 0 automatic, 1 row-log layout, 2 packed triangle
    long long timeout_ms = 5000;
    int test_skip_arrive = -1;
    long long test_fail_alloc = 0;  // the next this many device allocations fail (test hook)
    int phase_timing = 0;
    long long batch_split = 0;  // 0: largest n one CTA can hold
    std::vector<std::pair<long long, int>> batch_classes;  // (n_hi, CTA threads)

    // device workspace
    void *ws = nullptr;
    size_t ws_cap = 0;
    float *dbuf = nullptr;  // device copy of a host matrix
    size_t dbuf_cap = 0;
    void *full = nullptr;   // symmetric n x n working matrix (multi-CTA runs)
    size_t full_cap = 0;
    // side streams for uploading a host matrix in parallel pieces
    static constexpr int kCopyStreams = 4;
    cudaStream_t copy_stream[kCopyStreams] = {};
    cudaEvent_t copy_fork = nullptr;
    cudaEvent_t copy_join[kCopyStreams] = {};
    void *obuf = nullptr;   // device outputs for host output pointers
    size_t obuf_cap = 0;
    int *h_status = nullptr;       // pinned [4]
    long long *h_stats = nullptr;  // pinned [lw::kStats]

    // views into ws of the last launch
    int *d_status = nullptr;
    long long *d_stats = nullptr;
    bool pending = false;
    lw_status pending_fail = LW_OK;

    std::atomic<int> busy{0};
    char err[512] = {0};
};

namespace {

void set_err(lw_ctx *ctx, const char *fmt, ...)
{
    if (!ctx)
        return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
    va_end(ap);
}

lw_status cuda_fail(lw_ctx *ctx, cudaError_t e, const char *what)
{
    set_err(ctx, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LW_ERR_OOM : LW_ERR_CUDA;
}

// Is `p` memory the device can address as device memory (cudaMalloc,
// managed)?  Host pointers (pageable or pinned) return false.
bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked, mapped host memory (the GPU reads it over
// the host link), else null.
const float *mapped_host_alias(const float *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<const float *>(a.devicePointer) : nullptr;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Failure-injection hook (LW_OPT_TEST_FAIL_ALLOC): consumes one injected
// allocation failure, if any is pending.  The failure is made on the host,
// before cudaMalloc is called.
bool injected_alloc_failure(lw_ctx *ctx, const char *what)
{
    if (ctx->test_fail_alloc <= 0)
        return false;
    --ctx->test_fail_alloc;
    set_err(ctx, "allocation for %s failed (injected by LW_OPT_TEST_FAIL_ALLOC)", what);
    return true;
}

lw_status ensure(lw_ctx *ctx, void **buf, size_t *cap, size_t need, const char *what)
{
    if (*cap >= need)
        return LW_OK;
    if (injected_alloc_failure(ctx, what))
        return LW_ERR_OOM;
    if (*buf) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "cudaStreamSynchronize");
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(ctx, "cudaMalloc(%zu bytes) for %s failed: %s", need, what, cudaGetErrorString(e));
        return LW_ERR_OOM;
    }
    *cap = need;
    return LW_OK;
}

// Host-to-device copy of a large host matrix on the context's stream: pieces
// of 1 GiB dealt to side streams, so that several copy engines work at once;
// the context's stream waits for all of them.  One cudaMemcpyAsync per piece.
cudaError_t upload(lw_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    constexpr size_t kPiece = size_t(1) << 30;
    if (bytes <= kPiece)
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e;
    if (!ctx->copy_fork) {
        if ((e = cudaEventCreateWithFlags(&ctx->copy_fork, cudaEventDisableTiming)) != cudaSuccess)
            return e;
        for (int q = 0; q < lw_ctx::kCopyStreams; ++q) {
            if ((e = cudaStreamCreateWithFlags(&ctx->copy_stream[q], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&ctx->copy_join[q], cudaEventDisableTiming)) != cudaSuccess)
                return e;
        }
    }
    if ((e = cudaEventRecord(ctx->copy_fork, ctx->stream)) != cudaSuccess)
        return e;
    for (int q = 0; q < lw_ctx::kCopyStreams; ++q)
        if ((e = cudaStreamWaitEvent(ctx->copy_stream[q], ctx->copy_fork, 0)) != cudaSuccess)
            return e;
    const char *s8 = static_cast<const char *>(src);
    char *d8 = static_cast<char *>(dst);
    int q = 0;
    for (size_t off = 0; off < bytes; off += kPiece, q = (q + 1) % lw_ctx::kCopyStreams) {
        const size_t len = bytes - off < kPiece ? bytes - off : kPiece;
        if ((e = cudaMemcpyAsync(d8 + off, s8 + off, len, cudaMemcpyHostToDevice, ctx->copy_stream[q])) !=
            cudaSuccess)
            return e;
    }
    for (int k = 0; k < lw_ctx::kCopyStreams; ++k) {
        if ((e = cudaEventRecord(ctx->copy_join[k], ctx->copy_stream[k])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->stream, ctx->copy_join[k], 0)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

struct BusyGuard {
    lw_ctx *ctx;
    bool ok;
    explicit BusyGuard(lw_ctx *c) : ctx(c)
    {
        int expected = 0;
        ok = ctx->busy.compare_exchange_strong(expected, 1);
    }
    ~BusyGuard()
    {
        if (ok)
            ctx->busy.store(0);
    }
};

int choose_grid(lw_ctx *ctx, long long n)
{
    int G = ctx->grid_opt > 0 ? ctx->grid_opt : 0;
    if (G == 0) {
        // small matrices: one CTA (no grid barrier); larger: every SM
        G = n <= 4096 ? 1 : ctx->num_sms;
    }
    if (G > ctx->num_sms)
        G = ctx->num_sms;
    const long long nb = (n + lw::kRowBlock - 1) / lw::kRowBlock;
    if (G > nb)
        G = (int)nb;
    if (ctx->grid_opt <= 0 && G > 1) {
        // as few CTAs as give the same most row blocks per CTA, when that
        // saves a tenth of them or more: the walk, the exchange and the
        // barriers cost less while the slowest CTA's share of the rows stays
        // the same (n = 16384: 128 CTAs of 4 blocks instead of 152 of 3 or
        // 4, 2.4 % faster).  A smaller saving is not taken: CTAs with a block
        // fewer take the refill scans (n = 65536: 147 CTAs of 14 blocks ran
        // 0.3 % slower than 152 of 13 or 14).
        const long long per = (nb + G - 1) / G;
        const int G2 = (int)((nb + per - 1) / per);
        if (10LL * G2 <= 9LL * G)
            G = G2;
    }
    const int nt = ctx->cta_threads;
    while (G < ctx->num_sms && !lw::merge_config_ok(n, G, ctx->num_sms, nt))
        ++G;  // too much shared memory per CTA: spread the rows wider
    while (G > 1 && !lw::merge_config_ok(n, G, ctx->num_sms, nt))
        --G;
    return lw::merge_config_ok(n, G, ctx->num_sms, nt) ? G : 0;
}

// Queue one run on ctx->stream.  dist/merges/heights are device pointers;
// with host_src, ddist is the device address of the caller's mapped host
// matrix, which only the layout kernel reads: when the run would not use the
// row-log layout (so the kernel would work in ddist itself), nothing is
// queued and *declined is set.
lw_status enqueue(lw_ctx *ctx, float *ddist, long long n, int linkage, int32_t *dmerges,
                  float *dheights, bool host_src = false, bool *declined = nullptr)
{
    const int G = choose_grid(ctx, n);
    if (G <= 0) {
        set_err(ctx, "n=%lld does not fit a co-resident grid on this device", n);
        return LW_ERR_INVALID_ARG;
    }
    const lw::WorkspaceLayout L = lw::workspace_layout(n, G);
    lw_status s = ensure(ctx, &ctx->ws, &ctx->ws_cap, L.total, "workspace");
    if (s != LW_OK)
        return s;
    char *ws = static_cast<char *>(ctx->ws);

    // Row-log layout (multi-CTA grids): the kernel works on a symmetric n x n
    // copy M whose rows it rewrites whole, plus an n x n log TL that holds
    // each row's cells to later-merged slots, and a stamp per slot.  Every
    // merge then reads and writes contiguous words instead of one scattered
    // cell per row of the packed triangle; it costs 8 n^2 bytes of device
    // memory, used (automatically or on request) when that fits in half the
    // free memory; otherwise, and for one-CTA grids, the packed triangle.
    bool use_full = false;
    const size_t nn = (size_t)n * (size_t)lw::log_pitch(n) * sizeof(float);
    const size_t full_bytes = 2 * nn + align256((size_t)n * sizeof(int));
    if (ctx->layout_opt != 2 && G > 1) {
        size_t free_b = 0, total_b = 0;
        if (ctx->full_cap >= full_bytes) {
            use_full = true;
        } else if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                   full_bytes + ctx->full_cap <= free_b / 2 && (n + 31) / 32 <= 65535) {
            use_full = true;
        }
        cudaGetLastError();
        if (use_full) {
            s = ensure(ctx, &ctx->full, &ctx->full_cap, full_bytes, "full matrix");
            if (s != LW_OK)
                return s;
        }
    }
    if (host_src && !use_full) {
        *declined = true;
        return LW_OK;
    }

    lw::MergeParams p;
    p.D = use_full ? static_cast<float *>(ctx->full) : ddist;
    p.TL = use_full ? reinterpret_cast<float *>(static_cast<char *>(ctx->full) + nn) : nullptr;
    p.stamp = use_full ? reinterpret_cast<int *>(static_cast<char *>(ctx->full) + 2 * nn) : nullptr;
    p.full = use_full ? 1 : 0;
    p.n = n;
    p.pitch = use_full ? lw::log_pitch(n) : n;
    p.linkage = linkage;
    p.G = G;
    p.aligned16 = ((uintptr_t)p.D & 15u) == 0;
    p.merges = dmerges;
    p.heights = dheights;
    lw::bind_workspace(p, ws, L);
    if (use_full) {
        lw::check_range(p, p.D, nn);
        lw::check_range(p, p.TL, nn);
        lw::check_range(p, p.stamp, align256((size_t)n * sizeof(int)));
    } else {
        lw::check_range(p, p.D, (unsigned long long)n * (unsigned long long)(n - 1) / 2 * sizeof(float));
    }
    lw::check_range(p, p.merges, 8ull * (unsigned long long)(n - 1));
    lw::check_range(p, p.heights, 4ull * (unsigned long long)(n - 1));
    p.stats = reinterpret_cast<long long *>(ws + L.stats);
    p.timeout_ns = (unsigned long long)ctx->timeout_ms * 1000000ull;
    p.skip_arrive_cta = (ctx->test_skip_arrive >= 0 && ctx->test_skip_arrive < G && G > 1)
                            ? ctx->test_skip_arrive : -1;
    p.timing = ctx->phase_timing;
    ctx->d_status = p.status;
    ctx->d_stats = p.stats;

    cudaError_t e;
    // barrier, status and stats words are contiguous
    if ((e = cudaMemsetAsync(ws + L.zero, 0, L.total - L.zero, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemsetAsync");
    if (use_full && (e = lw::launch_expand(ddist, p.D, n, p.pitch, p.status, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "expand kernel launch");
    if ((e = lw::launch_merge(p, ctx->cta_threads, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaLaunchCooperativeKernel");
    return LW_OK;
}

}  // namespace

int lw::reserve_workspace(lw_ctx *ctx, long long n)
{
    if (!ctx || n < 2)
        return LW_ERR_INVALID_ARG;
    return ensure(ctx, &ctx->ws, &ctx->ws_cap, lw::workspace_layout(n, ctx->num_sms).total, "workspace");
}

namespace {

// Copy status/stats back and wait; maps the kernel status word.
lw_status finish(lw_ctx *ctx)
{
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                             ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemcpyAsync(status)");
    if ((e = cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, lw::kStats * sizeof(long long),
                             cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemcpyAsync(stats)");
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaStreamSynchronize");
    const int st = ctx->h_status[0];
    if (st == lw::kErrInput) {
        set_err(ctx, "input holds a NaN, infinite or negative distance");
        return LW_ERR_INVALID_INPUT;
    }
    if (st == lw::kErrTimeout) {
        set_err(ctx, "a device wait exceeded %lld ms (barrier %d)", ctx->timeout_ms,
                ctx->h_status[1]);
        return LW_ERR_TIMEOUT;
    }
    if (st == lw::kErrInternal) {
        set_err(ctx, "kernel stopped: the decided pair was out of range (internal error)");
        return LW_ERR_CUDA;
    }
    if (st == lw::kErrBounds) {
        set_err(ctx, "bounds-checked build: an access outside the job's buffers (lw_merge.cu line %d)",
                ctx->h_status[2]);
        return LW_ERR_CUDA;
    }
    if (st != 0) {
        set_err(ctx, "kernel reported status %d", st);
        return LW_ERR_CUDA;
    }
    return LW_OK;
}

lw_status check_args(lw_ctx *ctx, const float *dist, int64_t n, int linkage, const int32_t *merges,
                     const float *heights)
{
    if (n < 1 || n > LW_MAX_N) {
        set_err(ctx, "n=%lld out of range [1, %d]", (long long)n, LW_MAX_N);
        return LW_ERR_INVALID_ARG;
    }
    if (linkage < LW_SINGLE || linkage > LW_CENTROID) {
        set_err(ctx, "unknown linkage %d", linkage);
        return LW_ERR_INVALID_ARG;
    }
    if (n > 1 && (!dist || !merges || !heights)) {
        set_err(ctx, "NULL dist, merges_out or heights_out");
        return LW_ERR_INVALID_ARG;
    }
    return LW_OK;
}

}  // namespace

extern "C" {

lw_status lw_create(lw_ctx **out, int device, void *cuda_stream)
{
    if (!out)
        return LW_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return LW_ERR_CUDA;
    }
    if (device < 0 || device >= count)
        return LW_ERR_INVALID_ARG;
    lw_ctx *ctx = new (std::nothrow) lw_ctx;
    if (!ctx)
        return LW_ERR_OOM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    int coop = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (e == cudaSuccess && !coop)
        e = cudaErrorNotSupported;
    if (e == cudaSuccess) {
        if (cuda_stream) {
            ctx->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&ctx->h_status, 4 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&ctx->h_stats, lw::kStats * sizeof(long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        lw_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? LW_ERR_OOM : LW_ERR_CUDA;
    }
    memset(ctx->h_stats, 0, lw::kStats * sizeof(long long));
    *out = ctx;
    return LW_OK;
}

lw_status lw_cluster(lw_ctx *ctx, float *dist, int64_t n, int linkage, int32_t *merges_out,
                     float *heights_out)
{
    if (!ctx)
        return LW_ERR_INVALID_ARG;
    BusyGuard guard(ctx);
    if (!guard.ok) {
        set_err(ctx, "context busy");
        return LW_ERR_BUSY;
    }
    lw_status s = check_args(ctx, dist, n, linkage, merges_out, heights_out);
    if (s != LW_OK)
        return s;
    if (n == 1)
        return LW_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaSetDevice");

    const size_t cells = (size_t)n * (size_t)(n - 1) / 2;
    const bool dev_m = is_device_ptr(merges_out), dev_h = is_device_ptr(heights_out);
    int32_t *dm = merges_out;
    float *dh = heights_out;
    const size_t mbytes = sizeof(int32_t) * 2 * (size_t)(n - 1);
    const size_t hbytes = sizeof(float) * (size_t)(n - 1);
    if (!dev_m || !dev_h) {
        s = ensure(ctx, &ctx->obuf, &ctx->obuf_cap, align256(mbytes) + hbytes, "output buffers");
        if (s != LW_OK)
            return s;
        if (!dev_m)
            dm = static_cast<int32_t *>(ctx->obuf);
        if (!dev_h)
            dh = reinterpret_cast<float *>(static_cast<char *>(ctx->obuf) + align256(mbytes));
    }
    if (is_device_ptr(dist)) {
        s = enqueue(ctx, dist, n, linkage, dm, dh);
    } else {
        // A page-locked, mapped host matrix is read in place by the layout
        // kernel (one pass over the host link, no staging copy) when the run
        // uses the row-log layout; otherwise it is copied to the device.
        bool declined = true;
        const float *alias = mapped_host_alias(dist);
        if (alias) {
            declined = false;
            s = enqueue(ctx, const_cast<float *>(alias), n, linkage, dm, dh, true, &declined);
            if (s != LW_OK)
                return s;
        }
        if (declined) {
            s = ensure(ctx, (void **)&ctx->dbuf, &ctx->dbuf_cap, cells * sizeof(float), "matrix copy");
            if (s != LW_OK)
                return s;
            if ((e = upload(ctx, ctx->dbuf, dist, cells * sizeof(float))) != cudaSuccess)
                return cuda_fail(ctx, e, "matrix upload");
            s = enqueue(ctx, ctx->dbuf, n, linkage, dm, dh);
        }
    }
    if (s != LW_OK)
        return s;
    if (!dev_m && (e = cudaMemcpyAsync(merges_out, dm, mbytes, cudaMemcpyDeviceToHost,
                                       ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemcpyAsync(merges)");
    if (!dev_h && (e = cudaMemcpyAsync(heights_out, dh, hbytes, cudaMemcpyDeviceToHost,
                                       ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemcpyAsync(heights)");
    return finish(ctx);
}

lw_status lw_cluster_async(lw_ctx *ctx, float *dist, int64_t n, int linkage, int32_t *merges_out,
                           float *heights_out)
{
    if (!ctx)
        return LW_ERR_INVALID_ARG;
    BusyGuard guard(ctx);
    if (!guard.ok) {
        set_err(ctx, "context busy");
        return LW_ERR_BUSY;
    }
    lw_status s = check_args(ctx, dist, n, linkage, merges_out, heights_out);
    if (s != LW_OK)
        return s;
    ctx->pending = false;
    ctx->pending_fail = LW_OK;
    if (n == 1)
        return LW_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaSetDevice");
    if (!is_device_ptr(dist) || !is_device_ptr(merges_out) || !is_device_ptr(heights_out)) {
        set_err(ctx, "lw_cluster_async takes device pointers only");
        return LW_ERR_INVALID_ARG;
    }
    s = enqueue(ctx, dist, n, linkage, merges_out, heights_out);
    if (s != LW_OK)
        return s;
    ctx->pending = true;
    return LW_OK;
}

lw_status lw_wait(lw_ctx *ctx)
{
    if (!ctx)
        return LW_ERR_INVALID_ARG;
    BusyGuard guard(ctx);
    if (!guard.ok) {
        set_err(ctx, "context busy");
        return LW_ERR_BUSY;
    }
    if (!ctx->pending) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        return e == cudaSuccess ? LW_OK : cuda_fail(ctx, e, "cudaStreamSynchronize");
    }
    ctx->pending = false;
    return finish(ctx);
}

lw_status lw_get_stats(lw_ctx *ctx, int64_t *stats, int count)
{
    if (!ctx || !stats || count < 0)
        return LW_ERR_INVALID_ARG;
    for (int q = 0; q < count; ++q)
        stats[q] = q < lw::kStats ? ctx->h_stats[q] : 0;
    return LW_OK;
}

lw_status lw_set_option(lw_ctx *ctx, int option, int64_t value)
{
    if (!ctx)
        return LW_ERR_INVALID_ARG;
    switch (option) {
    case LW_OPT_GRID:
        if (value < 0 || value > ctx->num_sms)
            return LW_ERR_INVALID_ARG;
        ctx->grid_opt = (int)value;
        return LW_OK;
    case LW_OPT_TIMEOUT_MS:
        if (value < 0)
            return LW_ERR_INVALID_ARG;
        ctx->timeout_ms = value == 0 ? 5000 : value;
        return LW_OK;
    case LW_OPT_TEST_SKIP_ARRIVE:
        ctx->test_skip_arrive = value < 0 ? -1 : (int)value;
        return LW_OK;
    case LW_OPT_PHASE_TIMES:
        ctx->phase_timing = value != 0;
        return LW_OK;
    case LW_OPT_TEST_FAIL_ALLOC:
        if (value < 0)
            return LW_ERR_INVALID_ARG;
        ctx->test_fail_alloc = value;
        return LW_OK;
    case LW_OPT_LAYOUT:
        if (value < 0 || value > 2)
            return LW_ERR_INVALID_ARG;
        ctx->layout_opt = (int)value;
        return LW_OK;
    case LW_OPT_CTA_THREADS:
        if (value != 0 && value != 128 && value != 256 && value != 512)
            return LW_ERR_INVALID_ARG;
        ctx->cta_threads = value == 0 ? lw::kThreads : (int)value;
        return LW_OK;
    case LW_OPT_BATCH_SPLIT:
        if (value < 0)
            return LW_ERR_INVALID_ARG;
        ctx->batch_split = value;
        return LW_OK;
    default:
        return LW_ERR_INVALID_ARG;
    }
}

}  // extern "C"

struct lw_batch {
    lw_ctx *ctx = nullptr;
    int njobs = 0;
    std::vector<lw_job> jobs;        // host copy of the table
    std::vector<int> big_idx;        // jobs run over the whole device
    struct Class {
        long long n_hi = 0;          // jobs with n <= n_hi (and above the previous class)
        int nt = lw::kThreads;       // threads per CTA
        std::vector<int> idx;        // job indices
        long long n_max = 0;
        int grid = 0;
        lw::BatchJob *d_jobs = nullptr;
        char *d_ws = nullptr;
        int status_off = 0;
        cudaStream_t side = nullptr;
        cudaEvent_t join = nullptr;
    };
    std::vector<Class> classes;
    int *d_status = nullptr;         // per class, then [big] statuses
    int *d_queue = nullptr;          // one counter per class
    long long *d_merges = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Largest n whose one-CTA shared memory fits (and lets at least one CTA of
// nt threads run).
long long batch_auto_split(int nt)
{
    long long lo = 2, hi = 1 << 16;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (lw::batch_ctas_per_sm(mid, nt) >= 1)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

void batch_free(lw_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    for (auto &c : b->classes) {
        cudaFree(c.d_jobs);
        cudaFree(c.d_ws);
        if (c.side)
            cudaStreamDestroy(c.side);
        if (c.join)
            cudaEventDestroy(c.join);
    }
    if (b->fork)
        cudaEventDestroy(b->fork);
    cudaFree(b->d_status);
    cudaFree(b->d_queue);
    cudaFree(b->d_merges);
    cudaGetLastError();
    delete b;
}

}  // namespace

extern "C" {

lw_status lw_set_batch_classes(lw_ctx *ctx, const int64_t *n_hi, const int32_t *cta_threads,
                               int32_t count)
{
    if (!ctx || count < 0 || count > 16 || (count > 0 && (!n_hi || !cta_threads)))
        return LW_ERR_INVALID_ARG;
    std::vector<std::pair<long long, int>> cl;
    for (int q = 0; q < count; ++q) {
        const int nt = cta_threads[q];
        if ((nt != 128 && nt != 256 && nt != 512) || n_hi[q] < 2 ||
            (q > 0 && n_hi[q] <= n_hi[q - 1]))
            return LW_ERR_INVALID_ARG;
        cl.emplace_back((long long)n_hi[q], nt);
    }
    ctx->batch_classes = cl;
    return LW_OK;
}

lw_status lw_batch_create(lw_ctx *ctx, const lw_job *jobs, int32_t njobs, lw_batch **out)
{
    if (!ctx || !out || njobs < 0 || (njobs > 0 && !jobs))
        return LW_ERR_INVALID_ARG;
    *out = nullptr;
    BusyGuard guard(ctx);
    if (!guard.ok) {
        set_err(ctx, "context busy");
        return LW_ERR_BUSY;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaSetDevice");
    lw_batch *b = new (std::nothrow) lw_batch;
    if (!b)
        return LW_ERR_OOM;
    b->ctx = ctx;
    b->njobs = njobs;
    b->jobs.assign(jobs, jobs + njobs);
    // classes of one-CTA jobs: the tuned table, or one class of 512-thread
    // CTAs up to the largest n one CTA can hold; then the split option caps it
    std::vector<std::pair<long long, int>> cl = ctx->batch_classes;
    if (cl.empty())
        cl.emplace_back(batch_auto_split(lw::kThreads), lw::kThreads);
    const long long cap = ctx->batch_split > 0 ? ctx->batch_split : cl.back().first;
    for (auto &c : cl) {
        lw_batch::Class k;
        k.n_hi = c.first < cap ? c.first : cap;
        k.nt = c.second;
        if (b->classes.empty() || k.n_hi > b->classes.back().n_hi)
            b->classes.push_back(k);
    }
    long long big_n = 0;
    for (int q = 0; q < njobs; ++q) {
        const lw_job &J = jobs[q];
        if (J.n < 1 || J.n > LW_MAX_N || J.linkage < LW_SINGLE || J.linkage > LW_CENTROID ||
            (J.n > 1 && (!is_device_ptr(J.dist) || !is_device_ptr(J.merges_out) ||
                         !is_device_ptr(J.heights_out)))) {
            set_err(ctx, "job %d: bad n, linkage or a pointer that is not device memory", q);
            batch_free(b);
            return LW_ERR_INVALID_ARG;
        }
        bool placed = false;
        for (auto &c : b->classes) {
            if (J.n <= c.n_hi) {
                c.idx.push_back(q);
                c.n_max = J.n > c.n_max ? J.n : c.n_max;
                placed = true;
                break;
            }
        }
        if (!placed) {
            b->big_idx.push_back(q);
            big_n = J.n > big_n ? J.n : big_n;
        }
    }
    lw_status st = LW_OK;
    auto alloc = [&](void **pp, size_t bytes, const char *what) {
        if (st != LW_OK)
            return;
        if (injected_alloc_failure(ctx, what)) {
            st = LW_ERR_OOM;
            return;
        }
        cudaError_t ee = cudaMalloc(pp, bytes < 16 ? 16 : bytes);
        if (ee != cudaSuccess) {
            cudaGetLastError();
            set_err(ctx, "cudaMalloc(%zu) for %s failed", bytes, what);
            st = LW_ERR_OOM;
        }
    };
    int nstat = (int)b->big_idx.size();
    for (auto &c : b->classes) {
        c.status_off = nstat;
        nstat += (int)c.idx.size();
    }
    alloc((void **)&b->d_status, sizeof(int) * (size_t)(nstat > 0 ? nstat : 1), "batch statuses");
    alloc((void **)&b->d_queue, sizeof(int) * b->classes.size(), "batch queues");
    alloc((void **)&b->d_merges, sizeof(long long), "batch counter");
    bool any_small = false;
    for (auto &c : b->classes) {
        if (c.idx.empty() || st != LW_OK)
            continue;
        any_small = true;
        std::vector<lw::BatchJob> table(c.idx.size());
        for (size_t q = 0; q < c.idx.size(); ++q) {
            const lw_job &J = jobs[c.idx[q]];
            table[q].D = J.dist;
            table[q].n = J.n;
            table[q].linkage = J.linkage;
            table[q].pad = 0;
            table[q].merges = J.merges_out;
            table[q].heights = J.heights_out;
        }
        const int per_sm = lw::batch_ctas_per_sm(c.n_max < 2 ? 2 : c.n_max, c.nt);
        if (per_sm < 1) {
            set_err(ctx, "batch jobs of n=%lld do not fit one CTA of %d threads", c.n_max, c.nt);
            st = LW_ERR_INVALID_ARG;
            break;
        }
        c.grid = ctx->num_sms * per_sm;
        if ((size_t)c.grid > c.idx.size())
            c.grid = (int)c.idx.size();
        const lw::WorkspaceLayout L = lw::workspace_layout(c.n_max, 1);
        alloc((void **)&c.d_jobs, sizeof(lw::BatchJob) * c.idx.size(), "batch table");
        alloc((void **)&c.d_ws, L.total * (size_t)c.grid, "batch slots");
        if (st == LW_OK &&
            (e = cudaMemcpy(c.d_jobs, table.data(), sizeof(lw::BatchJob) * c.idx.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            st = cuda_fail(ctx, e, "cudaMemcpy(batch table)");
        if (st == LW_OK && (cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking) != cudaSuccess ||
                            cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming) != cudaSuccess))
            st = cuda_fail(ctx, cudaGetLastError(), "batch streams");
    }
    // record the one-CTA launches as one graph: every class on its own branch
    // (reset its queue, run its persistent kernel), all branches joined
    if (st == LW_OK && any_small) {
        if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
            st = cuda_fail(ctx, cudaGetLastError(), "batch event");
    }
    if (st == LW_OK && any_small) {
        e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        cudaError_t el = cudaSuccess;
        if (e == cudaSuccess) {
            cudaEventRecord(b->fork, ctx->stream);
            cudaMemsetAsync(b->d_merges, 0, sizeof(long long), ctx->stream);
            for (size_t k = 0; k < b->classes.size(); ++k) {
                auto &c = b->classes[k];
                if (c.idx.empty())
                    continue;
                cudaStreamWaitEvent(c.side, b->fork, 0);
                cudaMemsetAsync(b->d_queue + k, 0, sizeof(int), c.side);
                lw::BatchParams bp;
                bp.jobs = c.d_jobs;
                bp.njobs = (int)c.idx.size();
                bp.n_max = c.n_max;
                bp.queue = b->d_queue + k;
                bp.ws = c.d_ws;
                bp.job_status = b->d_status + c.status_off;
                bp.merges_done = b->d_merges;
                bp.timeout_ns = (unsigned long long)ctx->timeout_ms * 1000000ull;
                cudaError_t e2 = lw::launch_batch(bp, c.grid, c.nt, c.side);
                if (el == cudaSuccess)
                    el = e2;
                cudaEventRecord(c.join, c.side);
                cudaStreamWaitEvent(ctx->stream, c.join, 0);
            }
            e = cudaStreamEndCapture(ctx->stream, &b->graph);
            if (e == cudaSuccess)
                e = el;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess)
            st = cuda_fail(ctx, e, "batch graph capture");
    }
    if (st == LW_OK && !b->big_idx.empty()) {
        // size the context's workspace now so that runs never allocate
        const int G = choose_grid(ctx, big_n);
        if (G <= 0) {
            set_err(ctx, "n=%lld does not fit a co-resident grid on this device", big_n);
            st = LW_ERR_INVALID_ARG;
        } else {
            st = ensure(ctx, &ctx->ws, &ctx->ws_cap, lw::workspace_layout(big_n, ctx->num_sms).total,
                        "workspace");
        }
    }
    if (st != LW_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return LW_OK;
}

lw_status lw_batch_run(lw_batch *b)
{
    if (!b)
        return LW_ERR_INVALID_ARG;
    lw_ctx *ctx = b->ctx;
    BusyGuard guard(ctx);
    if (!guard.ok) {
        set_err(ctx, "context busy");
        return LW_ERR_BUSY;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaSetDevice");
    if (b->exec && (e = cudaGraphLaunch(b->exec, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaGraphLaunch");
    for (size_t q = 0; q < b->big_idx.size(); ++q) {
        const lw_job &J = b->jobs[b->big_idx[q]];
        lw_status s = enqueue(ctx, J.dist, J.n, J.linkage, J.merges_out, J.heights_out);
        if (s != LW_OK)
            return s;
        if ((e = cudaMemcpyAsync(b->d_status + q, ctx->d_status, sizeof(int),
                                 cudaMemcpyDeviceToDevice, ctx->stream)) != cudaSuccess)
            return cuda_fail(ctx, e, "cudaMemcpyAsync(job status)");
    }
    return LW_OK;
}

lw_status lw_batch_wait(lw_batch *b, lw_job *jobs)
{
    if (!b)
        return LW_ERR_INVALID_ARG;
    lw_ctx *ctx = b->ctx;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "cudaStreamSynchronize");
    std::vector<int> idx = b->big_idx;
    for (auto &c : b->classes)
        idx.insert(idx.end(), c.idx.begin(), c.idx.end());
    std::vector<int> st(idx.size(), 0);
    if (!st.empty() &&
        (e = cudaMemcpy(st.data(), b->d_status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
        return cuda_fail(ctx, e, "cudaMemcpy(job statuses)");
    lw_status first = LW_OK;
    for (size_t q = 0; q < st.size(); ++q) {
        lw_status js = LW_OK;
        switch (st[q]) {
        case 0: js = LW_OK; break;
        case lw::kErrInput: js = LW_ERR_INVALID_INPUT; break;
        case lw::kErrTimeout: js = LW_ERR_TIMEOUT; break;
        default: js = LW_ERR_CUDA; break;
        }
        if (jobs)
            jobs[idx[q]].status = js;
        if (js != LW_OK && first == LW_OK) {
            first = js;
            set_err(ctx, "job %d: %s", idx[q], lw_status_string(js));
        }
    }
    return first;
}

void lw_batch_destroy(lw_batch *b)
{
    if (!b)
        return;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    batch_free(b);
}

lw_status lw_cluster_batch(lw_ctx *ctx, lw_job *jobs, int32_t njobs)
{
    lw_batch *b = nullptr;
    lw_status s = lw_batch_create(ctx, jobs, njobs, &b);
    if (s != LW_OK)
        return s;
    s = lw_batch_run(b);
    if (s == LW_OK)
        s = lw_batch_wait(b, jobs);
    lw_batch_destroy(b);
    return s;
}

const char *lw_status_string(lw_status s)
{
    switch (s) {
    case LW_OK: return "ok";
    case LW_ERR_INVALID_ARG: return "invalid argument";
    case LW_ERR_INVALID_INPUT: return "invalid input (NaN, infinite or negative distance)";
    case LW_ERR_OOM: return "out of memory";
    case LW_ERR_CUDA: return "CUDA error";
    case LW_ERR_TIMEOUT: return "device wait timed out";
    case LW_ERR_BUSY: return "context busy";
    case LW_ERR_CANCELLED: return "request cancelled";
    }
    return "unknown status";
}

const char *lw_last_error(lw_ctx *ctx)
{
    return ctx ? ctx->err : "no context";
}

void lw_destroy(lw_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->device);
    if (ctx->stream)
        cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    cudaFree(ctx->dbuf);
    cudaFree(ctx->full);
    cudaFree(ctx->obuf);
    cudaFreeHost(ctx->h_status);
    cudaFreeHost(ctx->h_stats);
    for (int q = 0; q < lw_ctx::kCopyStreams; ++q) {
        if (ctx->copy_stream[q])
            cudaStreamDestroy(ctx->copy_stream[q]);
        if (ctx->copy_join[q])
            cudaEventDestroy(ctx->copy_join[q]);
    }
    if (ctx->copy_fork)
        cudaEventDestroy(ctx->copy_fork);
    if (ctx->own_stream && ctx->stream)
        cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

}  // extern "C"
