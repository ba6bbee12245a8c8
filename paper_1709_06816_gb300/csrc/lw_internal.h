// lw_internal.h -- declarations shared by the CUDA translation units of liblw.
// Not part of the public C ABI (include/lw.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct lw_ctx;

namespace lw {

constexpr int kThreads = 512;            // default threads per CTA of the merge kernel
constexpr int kRowBlock = 32;            // rows per ownership block (one warp)
constexpr int kCacheKeys = 4;            // smallest keys cached per row
constexpr int kPub = 4;                  // entries a CTA of a multi-CTA grid publishes per round
constexpr int kPubOne = 16;              // entries a job's only CTA publishes per round
constexpr int kRound = 32;               // most merges one round of a multi-CTA grid certifies
constexpr int kRoundOne = 16;            // the same for a job's only CTA
constexpr int kRefillAt = 0;             // ask for a refill when the cache holds this many keys or fewer
constexpr int kSurvivorRefillAt = 1;     // the same for a survivor row right after its merge
constexpr int kMaxReq = 256;             // refill requests served per round
constexpr int kReqPerCta = 8;            // refill requests one CTA may make per round
constexpr int kStats = 33;
constexpr uint64_t kNoKey = ~0ull;

// Column word of a published entry: the column, or one of two stop marks.
constexpr unsigned kColMask = 0x3fffffffu;
constexpr unsigned kRowStop = 0x80000000u;   // the row's cache ends here (cells beyond unknown)
constexpr unsigned kHardStop = 0x40000000u;  // the CTA published no entries beyond this one

// Status words written by the kernel (values match lw_status).
enum : int { kOk = 0, kErrInput = 2, kErrInternal = 4, kErrTimeout = 5, kErrBounds = 6 };

// Bounds-checked build (-DLW_CHECKED): every global load and store of the
// merge kernel is checked against the job's buffers; one outside them is
// skipped (a load reads zero) and sets the status to kErrBounds with the
// source line in status[2].  For testing: it replaces a memory checker.
constexpr int kCheckRanges = 8;
struct CheckRange {
    const char *base;
    unsigned long long bytes;
};

// One CTA's record at the start of a round, 240 bytes: its smallest cache
// entries (kPub of them, kPubOne for a one-CTA job; key = (bits(value) << 32)
// | (row << 3) | rank, column word beside it) and the rows (at most
// kReqPerCta) that ask for a refill.
struct __align__(16) RecA {
    unsigned long long key[kPubOne];
    unsigned int col[kPubOne];
    int nreq;
    int req[kReqPerCta];
    int pad[3];
};
static_assert(sizeof(RecA) == 240, "record layout");

struct MergeParams {
    float *D;                      // working matrix, rewritten in place: the packed
                                   // upper triangle, or (full = 1) the row-log layout:
                                   // D is an n x n row-major matrix M whose row x is
                                   // current for every column y with stamp[y] <= stamp[x]
    float *TL;                     // full = 1: n x n; TL[x * n + t] = the cell between x
                                   // and the survivor of merge t, written at merge t
    int *stamp;                    // full = 1: [n] merge that last rewrote each slot's
                                   // row (-1: never); cell {x, y} lives in the row of the
                                   // later-stamped slot, and in TL of the other one
    int full;
    long long n;
    long long pitch;               // full = 1: words per row of M and TL (n rounded up
                                   // to a multiple of 4: rows start 16-byte aligned)
    int linkage;                   // Table 1 row: 0 single, 1 complete, 2 group average,
                                   // 3 Ward, 4 weighted average, 5 centroid
    int G;                         // CTAs in the persistent grid
    int aligned16;                 // D is 16-byte aligned (128-bit loads allowed)
    int32_t *merges;               // [2(n-1)] device
    float *heights;                // [n-1]    device
    int *size_g;                   // [n] cluster sizes
    RecA *recA;                    // [G] published entries and refill requests
    unsigned long long *recB;      // [G][2][kRound] per-pair minima of the new cells
    unsigned long long *parts;     // [2][kMaxReq][kCacheKeys] refill lists (top-K of a row)
    unsigned int *bar;             // grid barrier counter (zero at launch)
    int *status;                   // [4] status word [0]; barrier that gave up [1]
    long long *stats;              // [kStats] counters, see lw_get_stats
    unsigned long long timeout_ns; // bound of every device wait
    int skip_arrive_cta;           // failure-detection test: this CTA never reaches the
                                   // first barrier (-1 = off), so the others' bounded
                                   // wait runs out and reports LW_ERR_TIMEOUT
    int timing;                    // accumulate per-phase wall-clock time in stats[8..13]
#ifdef LW_CHECKED
    CheckRange ck[kCheckRanges];   // the job's buffers (checked build only)
    int nck;
#endif
};

// Registers [base, base + bytes) as a buffer the checked kernel may touch
// (no effect in the normal build).
__host__ __device__ inline void check_range(MergeParams &p, const void *base, unsigned long long bytes)
{
#ifdef LW_CHECKED
    if (p.nck < kCheckRanges && base)
        p.ck[p.nck++] = CheckRange{static_cast<const char *>(base), bytes};
#else
    (void)p;
    (void)base;
    (void)bytes;
#endif
}

// Byte offsets of the merge kernel's global scratch inside one workspace
// block (every part 256-byte aligned).  The words from `zero` to `total`
// (barrier, status, stats) must be zero at launch.
struct WorkspaceLayout {
    size_t size, recA, recB, parts, zero, bar, status, stats, total;
};

__host__ __device__ inline WorkspaceLayout workspace_layout(long long n, int G)
{
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    WorkspaceLayout L;
    size_t off = 0;
    L.size = off;   off = up(off + sizeof(int) * (size_t)n);
    L.recA = off;   off = up(off + sizeof(RecA) * (size_t)G);
    L.recB = off;   off = up(off + 8 * 2 * kRound * (size_t)G);
    L.parts = off;  off = up(off + 8 * kCacheKeys * (size_t)kMaxReq * 2);
    L.zero = off;
    L.bar = off;    off = up(off + 256);
    L.status = off; off = up(off + 4 * sizeof(int));
    L.stats = off;  off = up(off + kStats * sizeof(long long));
    L.total = off;
    return L;
}

// Points p's scratch pointers into a workspace block laid out by L.
__host__ __device__ inline void bind_workspace(MergeParams &p, char *ws, const WorkspaceLayout &L)
{
    p.size_g = reinterpret_cast<int *>(ws + L.size);
    p.recA = reinterpret_cast<RecA *>(ws + L.recA);
    p.recB = reinterpret_cast<unsigned long long *>(ws + L.recB);
    p.parts = reinterpret_cast<unsigned long long *>(ws + L.parts);
    p.bar = reinterpret_cast<unsigned int *>(ws + L.bar);
    p.status = reinterpret_cast<int *>(ws + L.status);
#ifdef LW_CHECKED
    p.nck = 0;
#endif
    check_range(p, ws, L.total);
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

// Writes the symmetric n x n matrix `full` (row-major, rows `pitch` words
// apart, diagonal untouched) from the packed upper triangle `packed`, with
// -0 cells as +0; a NaN, infinite or negative cell sets *status to kErrInput.
cudaError_t launch_expand(const float *packed, float *full, long long n, long long pitch, int *status,
                          cudaStream_t stream);

// Row pitch (words) of the row-log layout's n x n matrices.
inline long long log_pitch(long long n) { return (n + 3) & ~3LL; }

// Bytes of dynamic shared memory the merge kernel needs for (n, G) with CTAs
// of nt threads.
size_t merge_smem_bytes(long long n, int G, int nt);
// CTA sizes the kernels are built for: 128, 256 or 512 threads (4, 2 or 1
// CTAs per SM by registers).
// True if a grid of G CTAs of nt threads for n objects fits co-resident on
// the current device.
bool merge_config_ok(long long n, int G, int num_sms, int nt = kThreads);
// Size the context's device workspace for every run of up to n objects, so
// that later runs never allocate (the serving loop reserves its lanes' at
// creation: growing a workspace frees the old one, and cudaFree waits for
// the whole device).  Returns LW_OK or LW_ERR_OOM.
int reserve_workspace(struct ::lw_ctx *ctx, long long n);

// Launch the persistent kernel (CTAs of nt threads) cooperatively on `stream`.
cudaError_t launch_merge(const MergeParams &p, int nt, cudaStream_t stream);
// CTAs of nt threads of the batch kernel that fit on one SM for jobs up to n_max.
int batch_ctas_per_sm(long long n_max, int nt = kThreads);
// Launch the batch kernel (grid CTAs of nt threads, one workspace slot each) on
// `stream`; call batch_ctas_per_sm(bp.n_max, nt) first (it sets the
// shared-memory limit).
cudaError_t launch_batch(const BatchParams &bp, int grid, int nt, cudaStream_t stream);

}  // namespace lw
