// lw_merge.cu -- the persistent cooperative Lance-Williams merge kernel.
//
// One launch performs all n - 1 merges of one matrix (Section 4, "Lance-William
// Algorithm", steps 1-4) so that no merge pays a kernel launch.  The paper
// spreads the packed upper triangle over MPI processes and exchanges local
// minima and (i, j, distance) triples by messages (Section 5.3 steps 1-6b); on
// one GB300 the whole triangle sits in HBM, so the "processors" become CTAs,
// the broadcast of local minima becomes one 32-byte record per CTA read after
// a grid barrier, and the triple exchange disappears: every CTA addresses row
// and column i and j directly.
//
// Work split.  Rows are dealt to CTAs in blocks of 32 consecutive rows,
// round-robin (block q -> CTA q mod G); a CTA "owns" those rows and, by the
// same map, those columns.  The owner of row k
//   - keeps, in shared memory, the kCacheKeys smallest keys of row k
//     (key = (value bits << 32) | column, over live columns c > k) and a bound
//     B: every live cell of the row outside the cache has a key above B
//     (B = "none" when the cache holds every live cell of the row);
//   - applies the update of Section 4 step 3 for k at every merge: reads D(k,i),
//     D(k,j), writes D(k,i+j) into D(k,i), and maintains row k's cache
//     (drops columns i and j, inserts the new cell (k,i) when it is <= B).
// The row minimum is exact while the cache is not empty.  A row whose cache
// runs low asks for a refill; in the barrier window of the NEXT merge (after
// a CTA has arrived at the grid barrier and before it waits) one warp of
// every CTA scans that CTA's columns of the row and publishes a partial
// top-K list, and two merges after the request the owner merges the lists
// and replays the two updates that happened meanwhile.  So row scans stay
// off the critical path; only a row whose cache empties before its refill
// lands is rescanned at once by its owner.
//
// The survivor row i is rewritten by every CTA (one cell per owned k > i);
// each CTA folds its part of row i into its candidate and publishes its
// partial top-K of row i, and the owner of i merges those lists after the
// barrier.
//
// One grid barrier per merge:
//   [wait] read G candidates (+ survivor lists, refill lists, requests)
//   -> global minimum (value, i, j) -> emit step -> update + cache upkeep
//   -> publish candidate and survivor list -> [arrive] serve refills [wait]
//
// Exact arithmetic: every product and sum of the update uses __fmul_rn /
// __fadd_rn / __fsub_rn (never contracted into FMA), the coefficient
// divisions __fdiv_rn; the four terms are added left to right.  The minimum
// is the smallest (value, row, column); values are non-negative floats, so
// their bit patterns order like the values and a 64-bit integer compare of
// (bits << 32 | index) gives the lexicographic order.
//
// Memory model.  L1 is not coherent across SMs, so every load of data that
// another CTA may have written (matrix cells, records, sizes) is an L2 load
// (ld.global.cg) and every store bypasses L1 (st.global.cg).  The barrier:
// __syncthreads, then one thread arrives with a release add (cumulative over
// the CTA's writes ordered before it by the __syncthreads) and later spins
// with acquire loads.  Each spin is bounded by a wall-clock limit after which
// the kernel records LW_ERR_TIMEOUT and returns.

#include "lw_internal.h"

#include <cstdint>

namespace lw {
namespace {

typedef unsigned long long u64;
constexpr int K = kCacheKeys;

__device__ __forceinline__ long long tri_off(long long r, long long n)
{
    return r * n - ((r * (r + 1)) >> 1);
}

__device__ __forceinline__ long long pair_idx(long long a, long long b, long long n)
{
    return a < b ? tri_off(a, n) + (b - a - 1) : tri_off(b, n) + (a - b - 1);
}

__device__ __forceinline__ u64 make_key(float v, unsigned c)
{
    return ((u64)__float_as_uint(v) << 32) | (u64)c;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// sorted key lists (ascending, padded with kNoKey)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cswap(u64 &a, u64 &b)
{
    const u64 lo = a < b ? a : b;
    b = a < b ? b : a;
    a = lo;
}

// Insert x into the K smallest: a compare-swap pass; the largest falls off.
__device__ __forceinline__ void list_insert(u64 (&L)[K], u64 x)
{
#pragma unroll
    for (int q = 0; q < K; ++q)
        cswap(L[q], x);
}

// Re-sort a sorted list in which at most two entries were replaced by kNoKey:
// two bubble passes carry both holes to the end.
__device__ __forceinline__ void close_holes(u64 (&L)[K])
{
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int q = 0; q + 1 < K; ++q)
            cswap(L[q], L[q + 1]);
    }
}

__device__ __forceinline__ int list_count(const u64 *L)
{
    int c = 0;
#pragma unroll
    for (int q = 0; q < K; ++q)
        c += L[q] != kNoKey;
    return c;
}

// Warp-wide minimum of 64-bit keys with two hardware warp reductions: the
// smallest high word, then the smallest low word among the lanes holding it.
__device__ __forceinline__ u64 warp_u64_min(u64 v)
{
    const unsigned hi = (unsigned)(v >> 32);
    const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? (unsigned)v : 0xffffffffu);
    return ((u64)mhi << 32) | mlo;
}

// K smallest keys over the lists of a warp (keys are distinct or kNoKey).
__device__ __forceinline__ void warp_topk(u64 (&L)[K], u64 (&out)[K])
{
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const u64 m = warp_u64_min(L[0]);
        out[q] = m;
        if (m != kNoKey && L[0] == m) {
#pragma unroll
            for (int s = 0; s + 1 < K; ++s)
                L[s] = L[s + 1];
            L[K - 1] = kNoKey;
        }
    }
}

// Candidate of the global minimum: (value, row) and column.
struct Cand {
    u64 A;       // (bits(v) << 32) | row
    unsigned c;  // column
};

__device__ __forceinline__ void cand_min(Cand &x, const Cand &y)
{
    if (y.A < x.A || (y.A == x.A && y.c < x.c))
        x = y;
}

// Warp-wide lexicographic minimum of (value bits, row, column) with three
// hardware warp reductions, each over the lanes that tie on the words before.
__device__ __forceinline__ Cand warp_cand_min(Cand v)
{
    const unsigned h = (unsigned)(v.A >> 32), r = (unsigned)v.A;
    const unsigned mh = __reduce_min_sync(0xffffffffu, h);
    const unsigned mr = __reduce_min_sync(0xffffffffu, h == mh ? r : 0xffffffffu);
    const unsigned mc =
        __reduce_min_sync(0xffffffffu, (h == mh && r == mr) ? v.c : 0xffffffffu);
    Cand out;
    out.A = ((u64)mh << 32) | mr;
    out.c = mc;
    return out;
}

template <int NT>
struct Shared {
    Cand red[(NT / 32) + 1];
    u64 tk[(NT / 32)][K];
    u64 tko[K];
    int wcnt[(NT / 32)];        // per-warp request counts (prefix sums)
    int flag;
    int nresc;               // rows to rescan at once this merge
    int nexec;               // refill rows served this merge
    int exec_row[kMaxReq];
    int my_off;              // where this CTA's requests landed in the list
    int nmyreq[2];           // this CTA's requests, by merge parity
    int myreq_l[2][kReqPerCta];
    int ninst;               // refills to install at the start of the next merge
    int inst_slot[kMaxReq];  // owned slots of those rows
};

// After the barrier: the global minimum over the G candidates, and the list
// of rows to refill in this merge -- every CTA's requests in CTA order
// (deterministic, the same in every CTA), cut at kMaxReq.  Thread t holds
// CTA t's record (cnt requests in rq).  Sets sh.exec_row, sh.nexec and
// sh.my_off (the position of this CTA's first request).
template <int NT>
__device__ Cand exchange_reduce(Cand v, int cnt, const int (&rq)[kReqPerCta], int b, Shared<NT> &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off)
            inc += o;
    }
    v = warp_cand_min(v);
    if (lane == 31)
        sh.wcnt[warp] = inc;
    if (lane == 0)
        sh.red[warp] = v;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w)
        base += sh.wcnt[w];
    const int off0 = base + inc - cnt;
#pragma unroll
    for (int q = 0; q < kReqPerCta; ++q) {
        if (q < cnt && off0 + q < kMaxReq)
            sh.exec_row[off0 + q] = rq[q];
    }
    if ((int)threadIdx.x == b)
        sh.my_off = off0;
    if (warp == 0) {
        Cand w = {kNoKey, 0xffffffffu};
        if (lane < (NT / 32))
            w = sh.red[lane];
        w = warp_cand_min(w);
        int tot = lane < (NT / 32) ? sh.wcnt[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            tot += __shfl_xor_sync(0xffffffffu, tot, off);
        if (lane == 0) {
            sh.red[(NT / 32)] = w;
            sh.nexec = tot < kMaxReq ? tot : kMaxReq;
        }
    }
    __syncthreads();
    return sh.red[(NT / 32)];
}

template <int NT>
__device__ Cand block_cand_min(Cand v, Shared<NT> &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_cand_min(v);
    if (lane == 0)
        sh.red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        Cand w = {kNoKey, 0xffffffffu};
        if (lane < (NT / 32))
            w = sh.red[lane];
        w = warp_cand_min(w);
        if (lane == 0)
            sh.red[(NT / 32)] = w;
    }
    __syncthreads();
    return sh.red[(NT / 32)];
}

// K smallest keys over every thread's list; result in sh.tko (all threads).
template <int NT>
__device__ void block_topk(u64 (&L)[K], Shared<NT> &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 w[K];
    warp_topk(L, w);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q)
            sh.tk[warp][q] = w[q];
    }
    __syncthreads();
    if (warp == 0) {
        u64 M[K];
#pragma unroll
        for (int q = 0; q < K; ++q)
            M[q] = lane < (NT / 32) ? sh.tk[lane][q] : kNoKey;
        warp_topk(M, w);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < K; ++q)
                sh.tko[q] = w[q];
        }
    }
    __syncthreads();
}

// Both reductions a CTA publishes, in one pass: the candidate minimum (in
// sh.red[(NT / 32)]) and the K smallest survivor-row keys (in sh.tko).
template <int NT>
__device__ void block_publish(Cand c, u64 (&L)[K], Shared<NT> &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 w[K];
    warp_topk(L, w);
    c = warp_cand_min(c);
    if (lane == 0) {
        sh.red[warp] = c;
#pragma unroll
        for (int q = 0; q < K; ++q)
            sh.tk[warp][q] = w[q];
    }
    __syncthreads();
    if (warp == 0) {
        Cand x = {kNoKey, 0xffffffffu};
        u64 M[K];
#pragma unroll
        for (int q = 0; q < K; ++q)
            M[q] = lane < (NT / 32) ? sh.tk[lane][q] : kNoKey;
        if (lane < (NT / 32))
            x = sh.red[lane];
        warp_topk(M, w);
        x = warp_cand_min(x);
        if (lane == 0) {
            sh.red[(NT / 32)] = x;
#pragma unroll
            for (int q = 0; q < K; ++q)
                sh.tko[q] = w[q];
        }
    }
    __syncthreads();
}

// Grid-wide barrier, split in two so that a CTA can do work that nobody
// waits for between arriving and waiting.  arrive: __syncthreads, then one
// thread adds to the counter with release semantics (the CTA's writes so far
// are published).  wait: that thread spins with acquire loads until every
// CTA has arrived, bounded by a wall-clock limit; returns false when the run
// must stop (this CTA gave up, or another CTA flagged an error).
__device__ __forceinline__ void grid_arrive(const MergeParams &p, unsigned &epoch)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        if (p.G > 1)
            red_release_add(p.bar, 1u);
    }
}

template <int NT>
__device__ bool grid_wait(const MergeParams &p, unsigned epoch, Shared<NT> &sh)
{
    if (threadIdx.x == 0) {
        int st = 0;
        if (p.G > 1) {
            const unsigned target = epoch * (unsigned)p.G;
            const u64 t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(p.bar) < target) {
                if ((++spins & 255u) == 0) {
                    st = ld_relaxed_s32(p.status);
                    if (st != 0)
                        break;
                    if (global_ns() - t0 > p.timeout_ns) {
                        atomicCAS(p.status, 0, kErrTimeout);
                        atomicCAS(p.status + 1, 0, (int)epoch);
                        st = kErrTimeout;
                        break;
                    }
                }
            }
        }
        sh.flag = st;
    }
    __syncthreads();
    return sh.flag == 0;
}

// Live-column test against the CTA's copy of the liveness bitmap.
__device__ __forceinline__ bool live(const unsigned *bitmap, long long c)
{
    return (bitmap[c >> 5] >> (c & 31)) & 1u;
}

// Adds one input cell to a per-lane list during the initial scan: checks it
// (finite and >= 0), rewrites -0 as +0 in memory, and keeps the K smallest.
__device__ __forceinline__ void init_cell(float v, long long q, unsigned c, const MergeParams &p,
                                          u64 (&L)[K], int &bad)
{
    unsigned u = __float_as_uint(v);
    if (u > 0x7f7fffffu) {
        if (u == 0x80000000u) {
            __stcg(p.D + q, 0.0f);
            u = 0u;
        } else {
            bad = 1;
            return;
        }
    }
    // cells above the list's largest value cannot enter it
    if (u > (unsigned)(L[K - 1] >> 32))
        return;
    list_insert(L, ((u64)u << 32) | (u64)c);
}

// K smallest keys of row r (all columns are live at launch), computed by one
// warp that also validates every cell of the row.
__device__ void warp_row_topk(const MergeParams &p, long long r, u64 (&out)[K], int &bad)
{
    const long long n = p.n;
    const int lane = threadIdx.x & 31;
    const long long start = tri_off(r, n);
    const long long end = start + (n - r - 1);
    const long long base_c = r + 1 - start;  // column of flat index q is q + base_c
    u64 L[K];
#pragma unroll
    for (int q = 0; q < K; ++q)
        L[q] = kNoKey;
    long long a0 = p.aligned16 ? ((start + 3) & ~3LL) : end;
    if (a0 > end)
        a0 = end;
    const long long a1 = a0 + ((end - a0) & ~3LL);
    for (long long q = start + lane; q < a0; q += 32)
        init_cell(__ldcg(p.D + q), q, (unsigned)(q + base_c), p, L, bad);
    for (long long q = a1 + lane; q < end; q += 32)
        init_cell(__ldcg(p.D + q), q, (unsigned)(q + base_c), p, L, bad);
    // 128-bit body, four loads in flight per lane
    long long q = a0 + 4 * lane;
    for (; q + 3 * 128 < a1; q += 4 * 128) {
        float4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            x[u] = __ldcg(reinterpret_cast<const float4 *>(p.D + q + 128 * u));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long qq = q + 128 * u;
            const unsigned c = (unsigned)(qq + base_c);
            init_cell(x[u].x, qq, c, p, L, bad);
            init_cell(x[u].y, qq + 1, c + 1, p, L, bad);
            init_cell(x[u].z, qq + 2, c + 2, p, L, bad);
            init_cell(x[u].w, qq + 3, c + 3, p, L, bad);
        }
    }
    for (; q < a1; q += 128) {
        const float4 x = __ldcg(reinterpret_cast<const float4 *>(p.D + q));
        const unsigned c = (unsigned)(q + base_c);
        init_cell(x.x, q, c, p, L, bad);
        init_cell(x.y, q + 1, c + 1, p, L, bad);
        init_cell(x.z, q + 2, c + 2, p, L, bad);
        init_cell(x.w, q + 3, c + 3, p, L, bad);
    }
    warp_topk(L, out);
}

// K smallest keys of row r over live columns, computed by the whole CTA
// (for a row whose cache empties before its refill arrives).  Adds the live
// cells read to `live_cells`.  Result in sh.tko.
template <int NT>
__device__ void block_row_topk(const MergeParams &p, long long r, const unsigned *bitmap, Shared<NT> &sh,
                               long long &live_cells)
{
    const long long n = p.n;
    const long long start = tri_off(r, n);
    const long long end = start + (n - r - 1);
    const long long base_c = r + 1 - start;
    u64 L[K];
#pragma unroll
    for (int q = 0; q < K; ++q)
        L[q] = kNoKey;
    long long cnt = 0;
    for (long long q = start + threadIdx.x; q < end; q += NT) {
        const long long c = q + base_c;
        if (live(bitmap, c)) {
            list_insert(L, make_key(__ldcg(p.D + q), (unsigned)c));
            ++cnt;
        }
    }
    live_cells += cnt;
    block_topk(L, sh);
}

__device__ __forceinline__ void load_list(u64 (&L)[K], const u64 *src)
{
    const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src);
#pragma unroll
    for (int q = 0; q < K / 2; ++q) {
        const ulonglong2 v = __ldcg(s2 + q);
        L[2 * q] = v.x;
        L[2 * q + 1] = v.y;
    }
}

__device__ __forceinline__ void publish_list(u64 *dst, const u64 *src, int tid)
{
    if (tid < K / 2)
        __stcg(reinterpret_cast<ulonglong2 *>(dst) + tid, make_ulonglong2(src[2 * tid], src[2 * tid + 1]));
}

// All n - 1 merges of one job, run by CTA b of the job's G CTAs (every CTA
// of the job calls this with the same p).  smem_raw: merge_smem_bytes(n, G)
// bytes of dynamic shared memory.
template <int NT>
__device__ void merge_job(const MergeParams &p, const int b, unsigned char *smem_raw, Shared<NT> &sh)
{
    const long long n = p.n;
    const int G = p.G;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const long long nb = (n + kRowBlock - 1) / kRowBlock;      // row blocks
    const long long my_blocks = b < nb ? (nb - b + G - 1) / G : 0;
    const int R = (int)(my_blocks * kRowBlock);                 // owned row slots
    const long long Rmax = ((nb + G - 1) / G) * kRowBlock;
    const long long nwords = (n + 31) / 32;

    // dynamic shared memory: liveness bitmap, then per owned slot l: cache
    // keys (key q of slot l at ck[q * Rmax + l]: consecutive threads read
    // consecutive words), bound, the new key of cell (k, i) of the last two
    // merges (by merge parity), size, key count, pending refill (merge, list
    // position), and the list of rows to rescan at once
    unsigned *bitmap = reinterpret_cast<unsigned *>(smem_raw);
    u64 *ck = reinterpret_cast<u64 *>(smem_raw + ((nwords * 4 + 15) & ~15LL));
    u64 *cB = ck + Rmax * K;
    u64 *upd = cB + Rmax;  // [2][Rmax]
    int *rsize = reinterpret_cast<int *>(upd + 2 * Rmax);
    int *ccnt = rsize + Rmax;
    int *pend_t = ccnt + Rmax;
    int *pend_s = pend_t + Rmax;
    int *rlist = pend_s + Rmax;

    auto row_of = [&](int l) -> long long {
        return (long long)((long long)b + (long long)G * (l >> 5)) * kRowBlock + (l & 31);
    };
    auto owner_of = [&](long long r) -> int { return (int)((r / kRowBlock) % G); };
    auto slot_of = [&](long long r) -> int {
        return (int)(((r / kRowBlock) / G) * kRowBlock + (r & 31));
    };
    auto cache_load = [&](u64 (&L)[K], int l) {
#pragma unroll
        for (int q = 0; q < K; ++q)
            L[q] = ck[(size_t)q * Rmax + l];
    };
    auto cache_store = [&](int l, const u64 *L) {
#pragma unroll
        for (int q = 0; q < K; ++q)
            ck[(size_t)q * Rmax + l] = L[q];
    };

    // per-phase wall-clock totals of this CTA (thread 0), when timing is on
    u64 ph0 = 0, ph1 = 0, ph2 = 0, ph3 = 0, ph4 = 0, ph5 = 0;
    u64 tmark = 0;
    auto lap = [&](u64 &acc) {
        if (p.timing && threadIdx.x == 0) {
            const u64 now = global_ns();
            acc += now - tmark;
            tmark = now;
        }
    };

    // ---- setup
    for (long long w = tid; w < nwords; w += NT) {
        const long long live_n = n - w * 32;
        bitmap[w] = live_n >= 32 ? 0xffffffffu : ((1u << live_n) - 1u);
    }
    for (int l = tid; l < R; l += NT) {
        rsize[l] = 1;
        pend_t[l] = -1;
        upd[l] = kNoKey;
        upd[Rmax + l] = kNoKey;
    }
    for (long long r = (long long)b * NT + tid; r < n; r += (long long)G * NT)
        p.size_g[r] = 1;
    if (tid == 0) {
        sh.nresc = 0;
        sh.ninst = 0;
        sh.nexec = 0;
        sh.nmyreq[0] = 0;
        sh.nmyreq[1] = 0;
    }

    // ---- phase 0: validate the matrix and fill the caches of owned rows
    // (one warp per owned row; the rows of a CTA are spread over the whole
    // triangle, so every CTA reads about the same number of cells)
    {
        int bad = 0;
        for (int l = warp; l < R; l += (NT / 32)) {
            const long long r = row_of(l);
            u64 top[K];
#pragma unroll
            for (int q = 0; q < K; ++q)
                top[q] = kNoKey;
            if (r < n - 1)
                warp_row_topk(p, r, top, bad);
            if (lane == 0) {
                cache_store(l, top);
                const int c = list_count(top);
                ccnt[l] = c;
                cB[l] = c == K ? top[K - 1] : kNoKey;
            }
        }
        if (bad)
            atomicCAS(p.status, 0, kErrInput);
    }
    __syncthreads();

    long long st_updates = 0, st_resc_cells = 0, st_fill_cells = 0;
    long long st_rescans = 0, st_fills = 0, st_installs = 0;

    // first records: each CTA's smallest cached key, no refill requests
    {
        Cand c = {kNoKey, 0xffffffffu};
        for (int l = tid; l < R; l += NT) {
            if (ccnt[l] > 0) {
                const u64 k = ck[l];
                Cand o = {(k & 0xffffffff00000000ull) | (u64)row_of(l), (unsigned)k};
                cand_min(c, o);
            }
        }
        c = block_cand_min(c, sh);
        if (tid == 0) {
            ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(p.cand + b);
            __stcg(dst, make_ulonglong2(c.A, (u64)c.c));
            __stcg(dst + 1, make_ulonglong2(0ull, 0ull));
        }
    }
    unsigned epoch = 0;
    if (b == p.skip_arrive_cta)
        return;
    grid_arrive(p, epoch);
    if (!grid_wait(p, epoch, sh))
        return;
    if (tid == 0)
        sh.flag = ld_relaxed_s32(p.status);
    __syncthreads();
    if (sh.flag != 0)
        return;
    if (p.timing && tid == 0)
        tmark = global_ns();

    // the pair merged in merge t-1
    long long i1 = -1, j1 = -1;
    int carried = 0;  // size of the cluster in slot i1 after merge t-1

    for (long long t = 0; t < n - 1; ++t) {
        const int par = (int)(t & 1);

        // ---- exchange: every CTA's record (candidate + refill requests),
        // the survivor row's partial lists, the first refill to install --
        // one round of loads, then one reduction
        const bool own_prev = i1 >= 0 && owner_of(i1) == b;
        const int ninst = sh.ninst;
        const int pbuf = (int)((t + 1) % 3);  // refills served two merges ago
        Cand mine = {kNoKey, 0xffffffffu};
        int rcnt = 0;
        int rq[kReqPerCta];
#pragma unroll
        for (int q = 0; q < kReqPerCta; ++q)
            rq[q] = -1;
        u64 sl[K], il0[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            sl[q] = kNoKey;
            il0[q] = kNoKey;
        }
        if (tid < G) {
            const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(p.cand + par * G + tid);
            const ulonglong2 w0 = __ldcg(src);
            const ulonglong2 w1 = __ldcg(src + 1);
            mine.A = w0.x;
            mine.c = (unsigned)w0.y;
            rcnt = (int)(w0.y >> 32);
            rq[0] = (int)(unsigned)w1.x;
            rq[1] = (int)(unsigned)(w1.x >> 32);
            rq[2] = (int)(unsigned)w1.y;
            rq[3] = (int)(unsigned)(w1.y >> 32);
            if (own_prev)
                load_list(sl, p.islice + ((size_t)par * G + tid) * K);
            if (ninst > 0)
                load_list(il0, p.parts + (((size_t)pbuf * G + tid) * kMaxReq +
                                          pend_s[sh.inst_slot[0]]) * K);
        }
        const Cand best = exchange_reduce(mine, rcnt, rq, b, sh);
        const long long i = (long long)(best.A & 0xffffffffull);
        const long long j = (long long)best.c;
        const float h = __uint_as_float((unsigned)(best.A >> 32));
        // every CTA read the same records, so every CTA takes this exit together
        if (i >= n || j >= n || i >= j) {
            if (tid == 0)
                atomicCAS(p.status, 0, kErrInternal);
            return;
        }
        // this CTA's requests of merge t-1 now have list positions
        {
            const int pq = par ^ 1;
            const int nmy = sh.nmyreq[pq];
            if (tid < nmy) {
                const int l = sh.myreq_l[pq][tid];
                const int pos = sh.my_off + tid;
                if (pos < kMaxReq)
                    pend_s[l] = pos;
                else
                    pend_t[l] = -1;  // not served: the row may ask again
            }
        }
        lap(ph1);

        // survivor of the previous merge: merge the G partial lists of its row
        if (own_prev) {
            block_topk(sl, sh);
            if (tid == 0) {
                const int l = slot_of(i1);
                cache_store(l, sh.tko);
                const int c = list_count(sh.tko);
                ccnt[l] = c;
                cB[l] = c == K ? sh.tko[K - 1] : kNoKey;
                __stcg(p.size_g + i1, carried);  // deferred size write
            }
        }

        // refills served two merges ago (in the barrier window of merge t-2):
        // merge the partial lists, then replay merges t-2 and t-1 on the row:
        // the served scan left out column i of merge t-2 and may have seen
        // either value of the cells merge t-1 touched
        for (int s = 0; s < ninst; ++s) {
            const int l = sh.inst_slot[s];
            u64 L[K];
#pragma unroll
            for (int q = 0; q < K; ++q)
                L[q] = il0[q];
            if (s > 0) {
#pragma unroll
                for (int q = 0; q < K; ++q)
                    L[q] = kNoKey;
                if (tid < G)
                    load_list(L, p.parts + (((size_t)pbuf * G + tid) * kMaxReq + pend_s[l]) * K);
            }
            block_topk(L, sh);
            if (tid == 0) {
                u64 M[K];
#pragma unroll
                for (int q = 0; q < K; ++q)
                    M[q] = sh.tko[q];
                int c = list_count(M);
                u64 B = c == K ? M[K - 1] : kNoKey;
                // merge t-2: the new cell (r, i_{t-2})
                u64 x = upd[(size_t)par * Rmax + l];
                if (x != kNoKey && x <= B) {
                    list_insert(M, x);
                    if (c == K)
                        B = M[K - 1];
                    else
                        ++c;
                }
                // merge t-1: column j1 left, cell (r, i1) changed
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    const unsigned col = (unsigned)M[q];
                    if (M[q] != kNoKey && (col == (unsigned)i1 || col == (unsigned)j1))
                        M[q] = kNoKey;
                }
                close_holes(M);
                c = list_count(M);
                x = upd[(size_t)(par ^ 1) * Rmax + l];
                if (x != kNoKey && x <= B) {
                    list_insert(M, x);
                    if (c == K)
                        B = M[K - 1];
                    else
                        ++c;
                }
                cache_store(l, M);
                ccnt[l] = c;
                cB[l] = B;
                pend_t[l] = -1;
                if (c == 0 && B != kNoKey) {
                    // every cached key left: rescan the row after the update
                    rlist[atomicAdd(&sh.nresc, 1)] = l;
                    pend_t[l] = -2;
                }
            }
        }
        st_installs += ninst;

        if (tid == 0) {
            if (b == 0) {
                p.merges[2 * t] = (int32_t)i;
                p.merges[2 * t + 1] = (int32_t)j;
                p.heights[t] = h;
            }
            bitmap[j >> 5] &= ~(1u << (j & 31));  // Section 4 step 2: slot j retires
            sh.ninst = 0;
            sh.nmyreq[par] = 0;
        }
        int ni = 1, nj = 1;
        if (p.linkage >= 2) {
            ni = (i == i1) ? carried : __ldcg(p.size_g + i);
            nj = (j == i1) ? carried : __ldcg(p.size_g + j);
        }
        __syncthreads();
        lap(ph2);

        // ---- Section 4 step 3: D(k, i+j) for every live k owned here
        float ai = 0.5f, aj = 0.5f, be = 0.0f, ga = 0.0f;
        if (p.linkage == 0) {
            ga = -0.5f;
        } else if (p.linkage == 1) {
            ga = 0.5f;
        } else if (p.linkage == 2) {
            const float sum = (float)(ni + nj);
            ai = __fdiv_rn((float)ni, sum);
            aj = __fdiv_rn((float)nj, sum);
        }
        u64 il[K];  // this thread's smallest new cells of the survivor row
#pragma unroll
        for (int q = 0; q < K; ++q)
            il[q] = kNoKey;
        u64 *updt = upd + (size_t)par * Rmax;
        for (int l = tid; l < R; l += NT) {
            const long long k = row_of(l);
            if (k >= n || k == i || k == j || !live(bitmap, k))
                continue;
            const long long pki = pair_idx(k, i, n);
            const long long pkj = pair_idx(k, j, n);
            const float a = __ldcg(p.D + pki);
            const float bb = __ldcg(p.D + pkj);
            if (p.linkage == 3) {
                const int nk = rsize[l];
                const float T = (float)(ni + nj + nk);
                ai = __fdiv_rn((float)(ni + nk), T);
                aj = __fdiv_rn((float)(nj + nk), T);
                be = -__fdiv_rn((float)nk, T);
            }
            float s = __fmul_rn(ai, a);
            s = __fadd_rn(s, __fmul_rn(aj, bb));
            s = __fadd_rn(s, __fmul_rn(be, h));
            s = __fadd_rn(s, __fmul_rn(ga, fabsf(__fsub_rn(a, bb))));
            __stcg(p.D + pki, s);
            ++st_updates;
            if (k > i) {
                // cell (i,k) belongs to the survivor row i
                list_insert(il, make_key(s, (unsigned)k));
                updt[l] = kNoKey;
                if (k > j)
                    continue;  // row k holds neither column i nor column j
            }
            // row k loses column j; if k < i its cell (k,i) changed as well
            u64 C[K];
            cache_load(C, l);
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const unsigned col = (unsigned)C[q];
                if (col == (unsigned)j || (k < i && col == (unsigned)i))
                    C[q] = kNoKey;
            }
            close_holes(C);
            int c = list_count(C);
            u64 B = cB[l];
            if (k < i) {
                const u64 x = make_key(s, (unsigned)i);
                updt[l] = x;
                if (x <= B) {
                    list_insert(C, x);
                    if (c == K)
                        B = C[K - 1];
                    else
                        ++c;
                }
            }
            cache_store(l, C);
            ccnt[l] = c;
            cB[l] = B;
            if (c == 0 && B != kNoKey) {
                // live cells remain but none is cached: rescan (once)
                if (pend_t[l] != -2)
                    rlist[atomicAdd(&sh.nresc, 1)] = l;
                pend_t[l] = -2;
            } else if (c <= kRefillAt && B != kNoKey && pend_t[l] < 0) {
                // (a cache that holds every live cell of its row needs no refill)
                const int q = atomicAdd(&sh.nmyreq[par], 1);
                if (q < kReqPerCta) {
                    sh.myreq_l[par][q] = l;
                    pend_t[l] = (int)t;
                }
            }
        }
        if (tid == 0) {
            if (owner_of(j) == b) {
                const int l = slot_of(j);
                ccnt[l] = 0;
                pend_t[l] = -1;
            }
            if (owner_of(i) == b) {
                const int l = slot_of(i);
                ccnt[l] = 0;  // rebuilt from the partial lists after the barrier
                pend_t[l] = -1;
                rsize[l] = ni + nj;
            }
        }
        __syncthreads();
        lap(ph3);

        // ---- rows whose cache emptied before a refill arrived
        const int nresc = sh.nresc;
        for (int q = 0; q < nresc; ++q) {
            const int l = rlist[q];
            block_row_topk(p, row_of(l), bitmap, sh, st_resc_cells);
            if (tid == 0) {
                cache_store(l, sh.tko);
                const int c = list_count(sh.tko);
                ccnt[l] = c;
                cB[l] = c == K ? sh.tko[K - 1] : kNoKey;
                pend_t[l] = -1;
            }
        }
        st_rescans += nresc;
        if (nresc > 0)
            __syncthreads();  // the rescanned caches (written by thread 0) before anyone reads them

        // ---- publish: this CTA's candidate, its refill requests and its
        // part of the survivor row
        {
            Cand c = {kNoKey, 0xffffffffu};
            for (int l = tid; l < R; l += NT) {
                if (ccnt[l] > 0) {
                    const u64 k = ck[l];
                    Cand o = {(k & 0xffffffff00000000ull) | (u64)row_of(l), (unsigned)k};
                    cand_min(c, o);
                }
                // a refill asked for in merge t-2 was served in the barrier
                // window of merge t-1 and is installed at merge t+1 (pend_t
                // is negative when no refill is pending)
                if (t >= 2 && pend_t[l] == (int)t - 2) {
                    const int s = atomicAdd(&sh.ninst, 1);
                    sh.inst_slot[s] = l;
                }
            }
            block_publish(c, il, sh);
            if (tid == 0) {
                Cand x = sh.red[(NT / 32)];
                const u64 h0 = sh.tko[0];
                if (h0 != kNoKey) {
                    const Cand o = {(h0 & 0xffffffff00000000ull) | (u64)i, (unsigned)h0};
                    cand_min(x, o);
                }
                int nq = sh.nmyreq[par];
                nq = nq < kReqPerCta ? nq : kReqPerCta;
                sh.nmyreq[par] = nq;
                unsigned rr[kReqPerCta];
#pragma unroll
                for (int q = 0; q < kReqPerCta; ++q)
                    rr[q] = q < nq ? (unsigned)row_of(sh.myreq_l[par][q]) : 0xffffffffu;
                ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(p.cand + (par ^ 1) * G + b);
                __stcg(dst, make_ulonglong2(x.A, (u64)x.c | ((u64)nq << 32)));
                __stcg(dst + 1, make_ulonglong2((u64)rr[0] | ((u64)rr[1] << 32),
                                                (u64)rr[2] | ((u64)rr[3] << 32)));
                sh.nresc = 0;
            }
            publish_list(p.islice + ((size_t)(par ^ 1) * G + b) * K, sh.tko, tid);
        }
        lap(ph4);
        i1 = i;
        j1 = j;
        carried = ni + nj;
        if (t + 2 >= n)
            break;  // that was the last merge
        grid_arrive(p, epoch);

        // ---- barrier window: serve the refills asked for in the previous
        // merge, one warp per row: the K smallest keys of the row over this
        // CTA's live columns, leaving out column i (its cells were rewritten
        // by other CTAs in this merge and may not be visible yet).  The
        // lists are read two merges later, after the next barrier.
        {
            const int nexec = sh.nexec;
            const int sbuf = (int)(t % 3);
            for (int s = warp; s < nexec; s += (NT / 32)) {
                const long long r = sh.exec_row[s];
                if (r < 0 || r >= n || r == i || r == j)
                    continue;  // the owner drops this refill
                u64 L[K];
#pragma unroll
                for (int q = 0; q < K; ++q)
                    L[q] = kNoKey;
                const long long base = tri_off(r, n) - r - 1;  // cell (r, c) at base + c
                long long cnt = 0;
                for (long long qb0 = 0; qb0 < my_blocks; qb0 += 16) {
                    float v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const long long qb = qb0 + u;
                        const long long c = ((long long)b + (long long)G * qb) * kRowBlock + lane;
                        v[u] = -1.0f;  // marks "no cell"; real cells are >= 0
                        if (qb < my_blocks && c > r && c < n && c != i && live(bitmap, c))
                            v[u] = __ldcg(p.D + base + c);
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        if (v[u] >= 0.0f) {
                            const long long c = ((long long)b + (long long)G * (qb0 + u)) * kRowBlock + lane;
                            list_insert(L, make_key(v[u], (unsigned)c));
                            ++cnt;
                        }
                    }
                }
                st_fill_cells += cnt;
                u64 w[K];
                warp_topk(L, w);
                if (lane < K / 2) {
                    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(
                        p.parts + (((size_t)sbuf * G + b) * kMaxReq + s) * K);
                    __stcg(dst + lane, make_ulonglong2(w[2 * lane], w[2 * lane + 1]));
                }
            }
            st_fills += nexec;
        }
        lap(ph5);
        if (!grid_wait(p, epoch, sh))
            return;
        lap(ph0);
    }

    if (p.stats) {
        u64 *S = reinterpret_cast<u64 *>(p.stats);
        atomicAdd(S + 1, (u64)st_resc_cells);
        atomicAdd(S + 2, (u64)st_updates);
        atomicAdd(S + 5, (u64)st_fill_cells);
        if (tid == 0) {
            atomicAdd(S + 0, (u64)st_rescans);
            atomicAdd(S + 6, (u64)st_installs);
            if (b == 0) {
                S[3] = (u64)G;
                S[4] = (u64)st_fills;
            }
            if (p.timing) {
                atomicAdd(S + 8, ph0);
                atomicAdd(S + 9, ph1);
                atomicAdd(S + 10, ph2);
                atomicAdd(S + 11, ph3);
                atomicAdd(S + 12, ph4);
                atomicAdd(S + 13, ph5);
            }
        }
    }
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) merge_kernel(MergeParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<NT> sh;
    merge_job<NT>(p, blockIdx.x, smem_raw, sh);
}

// Many independent jobs in one persistent launch: each CTA takes the next job
// from a queue (atomicAdd on a counter) and runs all its merges alone (a
// one-CTA job needs no grid barrier), then takes another, until the queue is
// empty.  CTA c keeps its scratch in workspace slot c.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) batch_kernel(BatchParams bp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<NT> sh;
    __shared__ int job;
    const WorkspaceLayout L = workspace_layout(bp.n_max, 1);
    char *ws = bp.ws + (size_t)blockIdx.x * L.total;
    long long merges_done = 0;
    while (true) {
        if (threadIdx.x == 0)
            job = atomicAdd(bp.queue, 1);
        __syncthreads();
        const int jb = job;
        if (jb >= bp.njobs)
            break;
        const BatchJob J = bp.jobs[jb];
        MergeParams p;
        p.D = J.D;
        p.n = J.n;
        p.linkage = J.linkage;
        p.G = 1;
        p.aligned16 = ((uintptr_t)J.D & 15u) == 0;
        p.merges = J.merges;
        p.heights = J.heights;
        p.size_g = reinterpret_cast<int *>(ws + L.size);
        p.cand = reinterpret_cast<Rec *>(ws + L.cand);
        p.islice = reinterpret_cast<unsigned long long *>(ws + L.islice);
        p.parts = reinterpret_cast<unsigned long long *>(ws + L.parts);
        p.bar = reinterpret_cast<unsigned *>(ws + L.bar);
        p.status = reinterpret_cast<int *>(ws + L.status);
        p.stats = nullptr;
        p.timeout_ns = bp.timeout_ns;
        p.skip_arrive_cta = -1;
        p.timing = 0;
        // the slot keeps the previous job's words: clear the ones that must start at zero
        for (size_t q = threadIdx.x; q < (L.total - L.zero) / 4; q += NT)
            reinterpret_cast<int *>(ws + L.zero)[q] = 0;
        __syncthreads();
        if (J.n > 1)
            merge_job<NT>(p, 0, smem_raw, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            bp.job_status[jb] = J.n > 1 ? __ldcg(p.status) : 0;
            merges_done += J.n > 1 ? J.n - 1 : 0;
        }
    }
    if (threadIdx.x == 0 && bp.merges_done)
        atomicAdd(reinterpret_cast<unsigned long long *>(bp.merges_done), (unsigned long long)merges_done);
}

}  // namespace

size_t merge_smem_bytes(long long n, int G)
{
    const long long nb = (n + kRowBlock - 1) / kRowBlock;
    const long long Rmax = ((nb + G - 1) / G) * kRowBlock;
    const long long nwords = (n + 31) / 32;
    return (size_t)(((nwords * 4 + 15) & ~15LL) + Rmax * (8 * K + 8 + 16 + 4 * 5));
}

namespace {

// The kernel instantiations: CTA size nt and the CTAs per SM its registers allow.
const void *merge_fn(int nt)
{
    switch (nt) {
    case 128: return (const void *)merge_kernel<128, 4>;
    case 256: return (const void *)merge_kernel<256, 2>;
    default: return (const void *)merge_kernel<512, 1>;
    }
}

const void *batch_fn(int nt)
{
    switch (nt) {
    case 128: return (const void *)batch_kernel<128, 4>;
    case 256: return (const void *)batch_kernel<256, 2>;
    default: return (const void *)batch_kernel<512, 1>;
    }
}

size_t static_smem(int nt)
{
    switch (nt) {
    case 128: return sizeof(Shared<128>);
    case 256: return sizeof(Shared<256>);
    default: return sizeof(Shared<512>);
    }
}

int fit_per_sm(const void *fn, int nt, size_t smem)
{
    int dev = 0, limit = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    if (smem + static_smem(nt) > (size_t)limit)
        return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem) != cudaSuccess)
        return 0;
    return per_sm;
}

}  // namespace

bool merge_config_ok(long long n, int G, int num_sms, int nt)
{
    // the first G threads read the CTAs' records
    if (G < 1 || G > num_sms || G > nt)
        return false;
    return fit_per_sm(merge_fn(nt), nt, merge_smem_bytes(n, G)) >= 1;
}

int batch_ctas_per_sm(long long n_max, int nt)
{
    return fit_per_sm(batch_fn(nt), nt, merge_smem_bytes(n_max, 1));
}

cudaError_t launch_batch(const BatchParams &bp, int grid, int nt, cudaStream_t stream)
{
    // batch_ctas_per_sm(bp.n_max, nt) has set the kernel's shared-memory limit
    // (this launch may be recorded into a graph, where no attribute is set)
    const size_t smem = merge_smem_bytes(bp.n_max, 1);
    BatchParams q = bp;
    void *args[] = {&q};
    return cudaLaunchKernel(batch_fn(nt), dim3(grid), dim3(nt), args, smem, stream);
}

cudaError_t launch_merge(const MergeParams &p, int nt, cudaStream_t stream)
{
    const size_t smem = merge_smem_bytes(p.n, p.G);
    const void *fn = merge_fn(nt);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    MergeParams q = p;
    void *args[] = {&q};
    return cudaLaunchCooperativeKernel(fn, dim3(p.G), dim3(nt), args, smem, stream);
}

}  // namespace lw
