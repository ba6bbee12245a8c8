// lw_server.cu -- continuous-batching request loop on top of the C ABI.
//
// A server owns one device memory pool of `budget` bytes and `lanes`
// execution lanes (one CUDA stream and one lw_ctx each).  Requests queue on
// the host; a scheduler thread admits a request as soon as a lane is free and
// the pool can hold its packed matrix (n(n-1)/2 floats), copies the matrix
// into the pool on the lane's stream, launches the merge kernel there and
// queues the result copies.  Lanes run concurrently, so requests that arrive
// while others are on the GPU start as soon as a lane and memory free up and
// their work overlaps on the device.  A request that does not fit the pool at
// the moment is passed over by smaller ones behind it (backfill); one that
// can never fit is refused at submission.  Every admitted kernel fits on the
// device at the same time as all the others in flight: a 512-thread CTA of
// the merge kernel fills an SM's registers and a 256-thread one half of them,
// and the admitted requests' CTAs never need more than the SMs there are.  So
// a cooperative grid is always resident as a whole: no grid waits at its
// barrier for CTAs that another grid, or a one-CTA job, keeps off the device.
// A request still in the queue can be cancelled.
//
// Large requests run with a modest grid (one CTA per 1024 objects): a merge
// of the persistent kernel is bound by barrier and memory latency far more
// than by the number of CTAs, so several large jobs side by side finish
// sooner than the same jobs one after another over the whole device
// (cooperative launches on different lanes run concurrently).

#include "../../include/lw.h"
#include "lw_internal.h"

#include <cuda_runtime.h>
#include <cmath>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

typedef std::chrono::steady_clock Clock;

struct Request {
    uint64_t ticket = 0;
    const float *dist = nullptr;
    int64_t n = 0;
    int linkage = 0;
    int32_t *merges = nullptr;
    float *heights = nullptr;
    size_t bytes = 0;
    Clock::time_point t_submit;
};

struct Result {
    bool done = false;
    lw_status status = LW_OK;
    double latency_ms = 0.0;
};

struct Lane {
    cudaStream_t stream = nullptr;
    lw_ctx *ctx = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    Request req;
    size_t block = 0;         // pool offset
    int units = 0;            // half-SM units the request's CTAs hold
    int32_t *dm = nullptr;    // device outputs when the request's are host memory
    float *dh = nullptr;
    size_t out_cap = 0;       // merges capacity (in steps)
};

bool is_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct lw_server {
    int device = 0;
    int num_sms = 0;
    long long n_max = 2;  // largest n whose packed triangle fits the pool
    char *pool = nullptr;
    size_t budget = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    size_t resident = 0;
    std::vector<Lane> lanes;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    int inflight = 0;
    int units_inflight = 0;  // half-SM units held by the admitted requests' CTAs
    bool stop = false;
    std::thread worker;

    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0;
    size_t peak_bytes = 0;
    int peak_inflight = 0;
    std::vector<double> latencies;
    bool any = false;
    Clock::time_point t_first, t_last;

    bool pool_alloc(size_t bytes, size_t *off)
    {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t roff = it->first + bytes;
                free_blocks.erase(it);
                if (rest > 0)
                    free_blocks[roff] = rest;
                return true;
            }
        }
        return false;
    }

    void pool_free(size_t off, size_t bytes)
    {
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }

    // One CTA for up to 2048 objects (256 threads up to 512 objects, so that
    // two small requests share an SM, else 512 -- the batch autotuner's
    // finding on GB300); above that, 512-thread CTAs, one per 1024 objects.
    int grid_for(int64_t n) const
    {
        if (n <= 2048)
            return 1;
        int G = (int)((n + 1023) / 1024);
        return std::min(G, num_sms);
    }

    static int threads_for(int64_t n) { return n <= 512 ? 256 : 512; }

    // Half-SM units the request's CTAs hold while it runs: two per 512-thread
    // CTA (all of an SM's registers), one per 256-thread CTA.
    int units_for(int64_t n) const { return grid_for(n) * (threads_for(n) == 512 ? 2 : 1); }

    // Launch request r on lane L (scheduler thread, mutex held).
    lw_status launch(Lane &L, const Request &r, size_t off)
    {
        float *d = reinterpret_cast<float *>(pool + off);
        const size_t cells = (size_t)r.n * (size_t)(r.n - 1) / 2;
        cudaError_t e = cudaMemcpyAsync(d, r.dist, cells * sizeof(float), cudaMemcpyDefault, L.stream);
        if (e != cudaSuccess)
            return LW_ERR_CUDA;
        const bool dev_out = is_device(r.merges) && is_device(r.heights);
        int32_t *dm = r.merges;
        float *dh = r.heights;
        if (!dev_out) {
            if (L.out_cap < (size_t)(r.n - 1)) {
                // once per lane, for the largest request the pool can hold:
                // cudaFree of a smaller buffer would wait for the whole device
                cudaFree(L.dm);
                cudaFree(L.dh);
                L.dm = nullptr;
                L.dh = nullptr;
                L.out_cap = 0;
                const size_t steps = (size_t)(n_max > r.n ? n_max : r.n) - 1;
                if (cudaMalloc(&L.dm, sizeof(int32_t) * 2 * steps) != cudaSuccess ||
                    cudaMalloc(&L.dh, sizeof(float) * steps) != cudaSuccess) {
                    cudaGetLastError();
                    return LW_ERR_OOM;
                }
                L.out_cap = steps;
            }
            dm = L.dm;
            dh = L.dh;
        }
        lw_set_option(L.ctx, LW_OPT_GRID, grid_for(r.n));
        lw_set_option(L.ctx, LW_OPT_CTA_THREADS, threads_for(r.n));
        // the pool's byte budget covers the packed matrices only
        lw_set_option(L.ctx, LW_OPT_LAYOUT, 2);
        lw_status s = lw_cluster_async(L.ctx, d, r.n, r.linkage, dm, dh);
        if (s != LW_OK)
            return s;
        if (!dev_out) {
            cudaMemcpyAsync(r.merges, dm, sizeof(int32_t) * 2 * (size_t)(r.n - 1),
                            cudaMemcpyDeviceToHost, L.stream);
            cudaMemcpyAsync(r.heights, dh, sizeof(float) * (size_t)(r.n - 1), cudaMemcpyDeviceToHost,
                            L.stream);
        }
        if (cudaEventRecord(L.done, L.stream) != cudaSuccess)
            return LW_ERR_CUDA;
        return LW_OK;
    }

    void finish(Lane &L, lw_status st)
    {
        const auto now = Clock::now();
        Result &res = results[L.req.ticket];
        res.done = true;
        res.status = st;
        res.latency_ms = std::chrono::duration<double, std::milli>(now - L.req.t_submit).count();
        latencies.push_back(res.latency_ms);
        if (st == LW_OK)
            ++completed;
        else
            ++failed;
        t_last = now;
        if (L.req.bytes) {
            pool_free(L.block, L.req.bytes);
            resident -= L.req.bytes;
        }
        L.busy = false;
        --inflight;
        units_inflight -= L.units;
        L.units = 0;
    }

    void loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progress = false;
            // completions
            for (Lane &L : lanes) {
                if (!L.busy)
                    continue;
                const cudaError_t q = cudaEventQuery(L.done);
                if (q == cudaErrorNotReady)
                    continue;
                lw_status st = q == cudaSuccess ? lw_wait(L.ctx) : LW_ERR_CUDA;
                cudaGetLastError();
                finish(L, st);
                progress = true;
            }
            // admissions, in arrival order, passing over requests that do not fit now
            for (auto it = queue.begin(); it != queue.end();) {
                Lane *free_lane = nullptr;
                for (Lane &L : lanes)
                    if (!L.busy) {
                        free_lane = &L;
                        break;
                    }
                if (!free_lane)
                    break;
                // every admitted kernel must fit the device together with the
                // others in flight, so that no cooperative grid is ever only
                // partly resident
                const int units = it->n > 1 ? units_for(it->n) : 0;
                if (units_inflight + units > 2 * num_sms) {
                    ++it;
                    continue;
                }
                size_t off = 0;
                if (it->n > 1 && !pool_alloc(it->bytes, &off)) {
                    ++it;
                    continue;
                }
                Lane &L = *free_lane;
                L.req = *it;
                L.block = off;
                L.busy = true;
                L.units = units;
                units_inflight += units;
                ++inflight;
                if (it->n > 1) {
                    resident += it->bytes;
                    peak_bytes = std::max(peak_bytes, resident);
                }
                peak_inflight = std::max(peak_inflight, inflight);
                it = queue.erase(it);
                lw_status s = L.req.n > 1 ? launch(L, L.req, off) : LW_OK;
                if (s != LW_OK || L.req.n <= 1)
                    finish(L, s);
                progress = true;
            }
            if (stop && queue.empty() && inflight == 0)
                break;
            if (!progress) {
                if (inflight == 0 && queue.empty())
                    cv.wait(lk, [&] { return stop || !queue.empty(); });
                else
                    cv.wait_for(lk, std::chrono::microseconds(20));
            }
        }
    }
};

extern "C" {

lw_status lw_server_create(int device, int64_t budget_bytes, int32_t lanes, lw_server **out)
{
    if (!out || budget_bytes <= 0 || lanes < 1 || lanes > 256)
        return LW_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return LW_ERR_INVALID_ARG;
    }
    lw_server *s = new (std::nothrow) lw_server;
    if (!s)
        return LW_ERR_OOM;
    s->device = device;
    cudaSetDevice(device);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
    s->budget = (size_t)budget_bytes & ~(size_t)255;
    if (cudaMalloc(&s->pool, s->budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return LW_ERR_OOM;
    }
    s->free_blocks[0] = s->budget;
    long long n_max = (long long)std::sqrt(2.0 * (double)(s->budget / sizeof(float))) + 2;
    while (n_max > 2 && up256((size_t)n_max * (size_t)(n_max - 1) / 2 * sizeof(float)) > s->budget)
        --n_max;
    if (n_max > LW_MAX_N)
        n_max = LW_MAX_N;
    s->n_max = n_max;
    s->lanes.resize((size_t)lanes);
    for (Lane &L : s->lanes) {
        lw_status st = LW_OK;
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess)
            st = LW_ERR_CUDA;
        if (st == LW_OK)
            st = lw_create(&L.ctx, device, L.stream);
        // the workspace for the largest request the pool can hold, now: a
        // lane that grew it later would free the old one, and cudaFree
        // waits for the whole device (every other lane's work)
        if (st == LW_OK)
            st = (lw_status)lw::reserve_workspace(L.ctx, n_max);
        if (st != LW_OK) {
            cudaGetLastError();
            lw_server_destroy(s);
            return st;
        }
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return LW_OK;
}

lw_status lw_server_submit(lw_server *s, const float *dist, int64_t n, int linkage,
                           int32_t *merges_out, float *heights_out, uint64_t *ticket)
{
    if (!s || !ticket || n < 1 || n > LW_MAX_N || linkage < LW_SINGLE || linkage > LW_CENTROID ||
        (n > 1 && (!dist || !merges_out || !heights_out)))
        return LW_ERR_INVALID_ARG;
    Request r;
    r.dist = dist;
    r.n = n;
    r.linkage = linkage;
    r.merges = merges_out;
    r.heights = heights_out;
    r.bytes = n > 1 ? up256((size_t)n * (size_t)(n - 1) / 2 * sizeof(float)) : 0;
    if (r.bytes > s->budget)
        return LW_ERR_INVALID_ARG;  // could never be admitted
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.ticket = s->next_ticket++;
        r.t_submit = Clock::now();
        if (!s->any) {
            s->any = true;
            s->t_first = r.t_submit;
        }
        ++s->submitted;
        s->results[r.ticket] = Result();
        s->queue.push_back(r);
        *ticket = r.ticket;
    }
    s->cv.notify_one();
    return LW_OK;
}

lw_status lw_server_poll(lw_server *s, uint64_t ticket, int32_t *done, lw_status *status,
                         double *latency_ms)
{
    if (!s || !done)
        return LW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end())
        return LW_ERR_INVALID_ARG;
    *done = it->second.done ? 1 : 0;
    if (status)
        *status = it->second.status;
    if (latency_ms)
        *latency_ms = it->second.latency_ms;
    return LW_OK;
}

lw_status lw_server_cancel(lw_server *s, uint64_t ticket)
{
    if (!s)
        return LW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto res = s->results.find(ticket);
    if (res == s->results.end())
        return LW_ERR_INVALID_ARG;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if (it->ticket != ticket)
            continue;
        const auto now = Clock::now();
        res->second.done = true;
        res->second.status = LW_ERR_CANCELLED;
        res->second.latency_ms = std::chrono::duration<double, std::milli>(now - it->t_submit).count();
        ++s->cancelled;
        s->queue.erase(it);
        return LW_OK;
    }
    return LW_ERR_BUSY;  // admitted already (running or finished)
}

lw_status lw_server_drain(lw_server *s)
{
    if (!s)
        return LW_ERR_INVALID_ARG;
    while (true) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty() && s->inflight == 0)
                break;
        }
        s->cv.notify_one();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    return s->failed ? LW_ERR_CUDA : LW_OK;
}

lw_status lw_server_get_stats(lw_server *s, lw_server_stats *st)
{
    if (!s || !st)
        return LW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->peak_bytes = (int64_t)s->peak_bytes;
    st->peak_inflight = s->peak_inflight;
    st->cancelled = (int32_t)s->cancelled;
    st->budget_bytes = (int64_t)s->budget;
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty())
            return 0.0;
        size_t k = (size_t)(q * (double)(v.size() - 1) + 0.5);
        return v[std::min(k, v.size() - 1)];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double sum = 0.0;
    for (double x : v)
        sum += x;
    st->mean_ms = v.empty() ? 0.0 : sum / (double)v.size();
    st->wall_s = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    return LW_OK;
}

void lw_server_destroy(lw_server *s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_one();
    if (s->worker.joinable())
        s->worker.join();
    cudaSetDevice(s->device);
    for (Lane &L : s->lanes) {
        if (L.stream)
            cudaStreamSynchronize(L.stream);
        lw_destroy(L.ctx);
        if (L.done)
            cudaEventDestroy(L.done);
        if (L.stream)
            cudaStreamDestroy(L.stream);
        cudaFree(L.dm);
        cudaFree(L.dh);
    }
    cudaFree(s->pool);
    cudaGetLastError();
    delete s;
}

}  // extern "C"
