// lw_internal.h -- declarations shared by the CUDA translation units of liblw.
// Not part of the public C ABI (include/lw.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lw {

constexpr int kThreads = 512;            // default threads per CTA of the merge kernel
constexpr int kRowBlock = 32;            // rows per ownership block (one warp)
constexpr int kCacheKeys = 4;            // smallest keys cached per row
constexpr int kRefillAt = 2;             // ask for a refill at this many keys or fewer
constexpr int kMaxReq = 32;              // refill requests served per merge
constexpr int kReqPerCta = 4;            // refill requests one CTA may make per merge
constexpr int kStats = 16;
constexpr uint64_t kNoKey = ~0ull;

// Status words written by the kernel (values match lw_status).
enum : int { kOk = 0, kErrInput = 2, kErrInternal = 4, kErrTimeout = 5 };

// One CTA's record for the next merge, 32 bytes: its candidate for the
// global minimum, A = (bits(value) << 32) | row and c = column of its
// smallest cell, and the rows (at most kReqPerCta) that ask for a refill.
struct __align__(16) Rec {
    unsigned long long A;
    unsigned int c;
    unsigned int nreq;
    int req[kReqPerCta];
};

struct MergeParams {
    float *D;                      // packed upper triangle, rewritten in place
    long long n;
    int linkage;                   // 0 single, 1 complete, 2 average, 3 Ward
    int G;                         // CTAs in the persistent grid
    int aligned16;                 // D is 16-byte aligned (128-bit loads allowed)
    int32_t *merges;               // [2(n-1)] device
    float *heights;                // [n-1]    device
    int *size_g;                   // [n] cluster sizes
    Rec *cand;                     // [2][G] candidates (double-buffered by merge parity)
    unsigned long long *islice;    // [2][G][kCacheKeys] survivor-row partial top-K
    unsigned long long *parts;     // [3][G][kMaxReq][kCacheKeys] refill partial top-K
    unsigned int *bar;             // grid barrier counter (zero at launch)
    int *status;                   // [4] status word [0]; barrier that gave up [1]
    long long *stats;              // [kStats] counters, see lw_get_stats
    unsigned long long timeout_ns; // bound of every device wait
    int skip_arrive_cta;           // failure-detection test: this CTA never reaches the
                                   // first barrier (-1 = off), so the others' bounded
                                   // wait runs out and reports LW_ERR_TIMEOUT
    int timing;                    // accumulate per-phase wall-clock time in stats[8..13]
};

// Byte offsets of the merge kernel's global scratch inside one workspace
// block (every part 256-byte aligned).  The words from `zero` to `total`
// (barrier, status, stats) must be zero at launch.
struct WorkspaceLayout {
    size_t size, cand, islice, parts, zero, bar, status, stats, total;
};

__host__ __device__ inline WorkspaceLayout workspace_layout(long long n, int G)
{
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    WorkspaceLayout L;
    size_t off = 0;
    L.size = off;   off = up(off + sizeof(int) * (size_t)n);
    L.cand = off;   off = up(off + sizeof(Rec) * 2 * (size_t)G);
    L.islice = off; off = up(off + 8 * kCacheKeys * 2 * (size_t)G);
    L.parts = off;  off = up(off + 8 * kCacheKeys * (size_t)kMaxReq * 3 * (size_t)G);
    L.zero = off;
    L.bar = off;    off = up(off + 256);
    L.status = off; off = up(off + 4 * sizeof(int));
    L.stats = off;  off = up(off + kStats * sizeof(long long));
    L.total = off;
    return L;
}

// One job of a batch (device table entry).
struct BatchJob {
    float *D;                      // packed upper triangle (device), rewritten in place
    long long n;
    int linkage;
    int pad;
    int32_t *merges;               // [2(n-1)] device
    float *heights;                // [n-1]    device
};

struct BatchParams {
    const BatchJob *jobs;          // [njobs] device
    int njobs;
    long long n_max;               // largest n in the table (sizes shared memory and slots)
    int *queue;                    // next job to take (zero at launch)
    char *ws;                      // one workspace slot per CTA, workspace_layout(n_max, 1)
    int *job_status;               // [njobs] lw_status of each job
    long long *merges_done;        // total merges performed (optional)
    unsigned long long timeout_ns;
};

// Bytes of dynamic shared memory the merge kernel needs for (n, G).
size_t merge_smem_bytes(long long n, int G);
// CTA sizes the kernels are built for: 128, 256 or 512 threads (4, 2 or 1
// CTAs per SM by registers).
// True if a grid of G CTAs of nt threads for n objects fits co-resident on
// the current device.
bool merge_config_ok(long long n, int G, int num_sms, int nt = kThreads);
// Launch the persistent kernel (CTAs of nt threads) cooperatively on `stream`.
cudaError_t launch_merge(const MergeParams &p, int nt, cudaStream_t stream);
// CTAs of nt threads of the batch kernel that fit on one SM for jobs up to n_max.
int batch_ctas_per_sm(long long n_max, int nt = kThreads);
// Launch the batch kernel (grid CTAs of nt threads, one workspace slot each) on
// `stream`; call batch_ctas_per_sm(bp.n_max, nt) first (it sets the
// shared-memory limit).
cudaError_t launch_batch(const BatchParams &bp, int grid, int nt, cudaStream_t stream);

}  // namespace lw
