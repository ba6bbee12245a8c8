// lw_merge.cu -- the persistent cooperative Lance-Williams merge kernel.
//
// One launch performs all n - 1 merges of one matrix (Section 4, "Lance-William
// Algorithm", steps 1-4) so that no merge pays a kernel launch.  The paper
// spreads the packed upper triangle over MPI processes and exchanges local
// minima and (i, j, distance) triples by messages (Section 5.3 steps 1-6b); on
// one GB300 the whole triangle sits in HBM, so the "processors" become CTAs,
// the broadcast of local minima becomes a small record per CTA read after a
// grid barrier, and the triple exchange disappears: every CTA addresses rows
// and columns i and j directly.
//
// Work split.  Rows are dealt to CTAs in blocks of 32 consecutive rows,
// round-robin (block q -> CTA q mod G); a CTA "owns" those rows.  The owner
// of row k keeps, in shared memory, the kCacheKeys smallest keys of row k
// (key = (value bits << 32) | column, over live columns c > k) and a bound B:
// every live cell of the row outside the cache has a key above B (B = "none"
// when the cache holds every live cell of the row).
//
// Rounds.  A grid barrier costs about a microsecond on GB300, more than the
// arithmetic of one merge, so the kernel certifies several consecutive merges
// of the sequential iteration per pair of barriers (up to 32 for a grid, 16
// for a job's only CTA).  The merges are exactly those of the step-by-step
// algorithm (same pairs, same order, same rounded values); only the
// bookkeeping differs.  One round:
//
//   A  every CTA publishes its smallest cache entries (kPub of them, kPubOne
//      for a job's only CTA), each row's entries followed by a stop mark at
//      its bound B.  After the barrier every CTA walks the union of all
//      published entries in (value, row, column) order and proposes a chain
//      of disjoint pairs P_1..P_s: an entry whose row or column already
//      belongs to a proposed pair is skipped, a stop mark of an untouched row
//      (or the last entry of a CTA that had more) ends the walk.  P_{p+1} is
//      then the smallest cell among those no earlier proposal touches.
//   pass 1 (reads only): for every live k outside the chain and every pair a,
//      the new distance D(k, i_a + j_a) of Section 4 step 3; each CTA
//      publishes, per pair, its smallest new cell over all k and over k > i_a.
//      The cells between members of two proposed pairs are computed by every
//      CTA, in the order the sequential algorithm would write them.
//   B  after the barrier, every CTA finds the longest prefix P_1..P_L such
//      that each P_{p+1} is smaller than every cell the merges P_1..P_p have
//      rewritten: then P_{p+1} is the global minimum after merge p, so the
//      prefix is what the sequential algorithm does.  P_1 always qualifies.
//   pass 2: the L merges are emitted and applied: D(k, i_a) rewritten, caches
//      kept (column j_a leaves, the new cell (k, i_a) enters when <= B), the
//      survivor rows get their new caches from the published minima.
//
// Refills.  A row whose cache empties (a survivor row: right after its merge)
// asks for a refill; in the window of the next round's barrier B (after a CTA
// has arrived and before it waits) one CTA scans the whole row, all threads,
// and publishes its top-K; at the start of the round after that the owner
// takes the list and replays the merges of the round in between.  A row that
// empties while its bound sits at the front of the merges is rescanned at
// once by its owner.  A job's only CTA sees every write after pass 2 and
// refreshes survivor and emptied rows itself, a warp per row.
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

// Global loads and stores of the merge kernel: L2 only (see "Memory model"),
// and in the bounds-checked build (-DLW_CHECKED) checked against the job's
// buffers first (an address outside them is skipped, a load reads zero, and
// the status records kErrBounds and the source line).
#ifdef LW_CHECKED
__device__ __noinline__ bool check_ok(const MergeParams &p, const void *a, unsigned bytes, int line)
{
    const char *c = static_cast<const char *>(a);
    for (int q = 0; q < p.nck; ++q)
        if (c >= p.ck[q].base && c + bytes <= p.ck[q].base + p.ck[q].bytes)
            return true;
    if (atomicCAS(p.status, 0, kErrBounds) == 0)
        atomicExch(p.status + 2, line);
    return false;
}
template <class T>
struct same_type {
    typedef T type;
};
template <class T>
__device__ __forceinline__ T ld_checked(const MergeParams &p, const T *a, int line)
{
    return check_ok(p, a, sizeof(T), line) ? __ldcg(a) : T();
}
template <class T>
__device__ __forceinline__ void st_checked(const MergeParams &p, T *a, typename same_type<T>::type v, int line)
{
    if (check_ok(p, a, sizeof(T), line))
        __stcg(a, v);
}
#define LDCG(a) ld_checked(p, (a), __LINE__)
#define STCG(a, v) st_checked(p, (a), (v), __LINE__)
#define CHECKED_16(a) check_ok(p, (a), 16, __LINE__)
#else
#define LDCG(a) __ldcg(a)
#define STCG(a, v) __stcg((a), (v))
#define CHECKED_16(a) true
#endif

__device__ __forceinline__ long long tri_off(long long r, long long n)
{
    return r * n - ((r * (r + 1)) >> 1);
}

__device__ __forceinline__ long long pair_idx(long long a, long long b, long long n)
{
    return a < b ? tri_off(a, n) + (b - a - 1) : tri_off(b, n) + (a - b - 1);
}

// Row r of the working matrix: cell (r, c) at row_base + c (packed: c > r only).
__device__ __forceinline__ long long row_base(const MergeParams &p, long long r)
{
    return p.full ? r * p.pitch : tri_off(r, p.n) - r - 1;
}


// Cell {x, y} read directly (the cells between members of a round's chain),
// the slots' stamps sx, sy given.  Row-log layout: the cell is current in the
// row of M whose slot was stamped later (both rows hold the input value
// while neither slot has merged).
__device__ __forceinline__ float member_cell(const MergeParams &p, long long x, int sx, long long y, int sy)
{
    if (!p.full)
        return LDCG(p.D + pair_idx(x, y, p.n));
    return sx >= sy ? LDCG(p.D + x * p.pitch + y) : LDCG(p.D + y * p.pitch + x);
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

__device__ __forceinline__ unsigned atom_release_add(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// 16 bytes global -> shared, cached in L2 only (the words read are written by
// other CTAs between grid barriers, so L1 must not hold them).  The copy
// writes no register: a warp that issues one per step does not wait for the
// previous one.
__device__ __forceinline__ void copy16_async(void *dst_smem, const void *src_gmem)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src_gmem) : "memory");
}

__device__ __forceinline__ void copy_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
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

// KK smallest keys over the sorted lists of a warp (keys are distinct or kNoKey).
template <int KK>
__device__ __forceinline__ void warp_topk(u64 (&L)[KK], u64 (&out)[KK])
{
#pragma unroll
    for (int q = 0; q < KK; ++q) {
        const u64 m = warp_u64_min(L[0]);
        out[q] = m;
        if (m != kNoKey && L[0] == m) {
#pragma unroll
            for (int s = 0; s + 1 < KK; ++s)
                L[s] = L[s + 1];
            L[KK - 1] = kNoKey;
        }
    }
}

// Insert x into a sorted list of KK keys; the largest falls off.
template <int KK>
__device__ __forceinline__ void list_insert_n(u64 (&L)[KK], u64 x)
{
#pragma unroll
    for (int q = 0; q < KK; ++q)
        cswap(L[q], x);
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

// Most merges one round certifies: a one-CTA job publishes kPubOne entries
// and walks at most kRoundOne pairs; a grid walks up to kRound.
__host__ __device__ constexpr int round_of(int pub) { return pub == kPubOne ? kRoundOne : kRound; }
constexpr unsigned kFull = 0xffffffffu;
constexpr u64 kHi = 0xffffffff00000000ull;
static_assert(kPub <= kPubOne && kPub % 4 == 0 && kPubOne % 4 == 0, "record layout");
static_assert(K == 4, "sort_list is a 4-input network");
static_assert(kRound <= 32 && (32 % kRound) == 0 && (32 % kRoundOne) == 0,
              "certification and pair minima use lane groups of the round size");

// Sort a K-list in which any entries were replaced by kNoKey.
__device__ __forceinline__ void sort_list(u64 (&L)[K])
{
    cswap(L[0], L[1]);
    cswap(L[2], L[3]);
    cswap(L[0], L[2]);
    cswap(L[1], L[3]);
    cswap(L[1], L[2]);
}

// The update of Section 4 step 3 with the Table 1 coefficients for clusters
// of sizes ni, nj (merged) and nk (the other one); terms added in printed
// order, every operation rounded once.
__device__ __forceinline__ float lw_cell(int linkage, float dki, float dkj, float dij, int ni, int nj,
                                         int nk)
{
    float ai = 0.5f, aj = 0.5f, be = 0.0f, ga = 0.0f;
    if (linkage == 0) {
        ga = -0.5f;
    } else if (linkage == 1) {
        ga = 0.5f;
    } else if (linkage == 2 || linkage == 5) {
        // group average; centroid adds beta = -n_i n_j / (n_i + n_j)^2 (exact
        // integers, each converted to float once, one division)
        const float sum = (float)(ni + nj);
        ai = __fdiv_rn((float)ni, sum);
        aj = __fdiv_rn((float)nj, sum);
        if (linkage == 5)
            be = -__fdiv_rn(__ll2float_rn((long long)ni * nj),
                            __ll2float_rn((long long)(ni + nj) * (ni + nj)));
    } else if (linkage == 3) {
        const float T = (float)(ni + nj + nk);
        ai = __fdiv_rn((float)(ni + nk), T);
        aj = __fdiv_rn((float)(nj + nk), T);
        be = -__fdiv_rn((float)nk, T);
    }
    // linkage 4, weighted average: 1/2, 1/2, 0, 0
    float s = __fmul_rn(ai, dki);
    s = __fadd_rn(s, __fmul_rn(aj, dkj));
    s = __fadd_rn(s, __fmul_rn(be, dij));
    s = __fadd_rn(s, __fmul_rn(ga, fabsf(__fsub_rn(dki, dkj))));
    return s;
}

// Order key of the cell between clusters x and y holding value bits vb.
__device__ __forceinline__ Cand cell_cand(unsigned vb, unsigned x, unsigned y)
{
    Cand c;
    c.A = ((u64)vb << 32) | (x < y ? x : y);
    c.c = x < y ? y : x;
    return c;
}

template <int NT, int S>
struct Shared {
    static constexpr int W = NT / 32;
    u64 tk[W][kPubOne];
    u64 tko[kPubOne];
    int wcnt[W];
    int flag;
    int nexec;                   // refill rows served this round
    int exec_row[kMaxReq];
    int nmyreq[2];               // this CTA's requests, by round parity
    int myreq_l[2][kReqPerCta];
    int ninst;                   // refills to install at the start of the next round
    int inst_slot[kReqPerCta];
    // the round's chain of proposed merges and the cells between its members
    int np, nacc;
    unsigned front;              // value bits where this round's walk stopped
    int okp[S];
    int pi[S], pj[S];
    float ph[S];
    int szi[S], szj[S];
    long long bi[S], bj[S];      // row bases of the members: cell (x, c) at b + c
    int si[S], sj[S];            // row-log layout: the members' stamps before the round
    // the 16-byte words holding size_g[i_a], size_g[j_a], stamp[i_a], stamp[j_a]
    alignas(16) int qw[S][16];
    u64 wam[W][S], whm[W][S];    // per warp: smallest new cell per pair (all k, k > i)
    u64 gamin[S], ghmin[S];      // the same over all CTAs
    // (rows padded by one word: the certification reads a column of these
    // per warp, one row per lane, which would otherwise hit a single bank)
    alignas(16) float Dm[2 * S][2 * S + 1];  // D between members (2a = i_a, 2a + 1 = j_a)
    float X[S][S + 1];           // cell (i_a, i_b) after merge a alone
    float Y[S][S + 1];           // cell (i_a, j_b) after merge a alone
    float C[S][S + 1];           // cell (i_a, i_b) after merges a then b (a < b)
    // the previous round's merges, replayed on installed refills
    int ppi[S], ppj[S];
    int nprev;
    int nresc;                   // rows to rescan at once this round
    // phase timers and the counters one thread keeps (thread 0, thread 32 for
    // the refill team): here rather than in registers of the round loop
    struct {
        u64 ph[6], xs[8], xscan[2], xwalk, xlast, tmark;
        long long fills, installs, rounds, idle, walk, rescans;
        long long nlast, nlast_b, nlast_b_scan, nlast_a_scan;
    } ty;
};

// After barrier A: the list of rows to refill in this round -- every CTA's
// requests in CTA order (deterministic, the same in every CTA), cut at
// kMaxReq.  Thread t holds CTA t's request count and rows.  Sets
// sh.exec_row and sh.nexec; thread b gives this CTA's own requests (list
// pq) their list positions.
template <int NT, int S>
__device__ void exchange_requests(int cnt, const int (&rq)[kReqPerCta], int b, Shared<NT, S> &sh, int pq,
                                  int *pend_t, int *pend_s)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(kFull, inc, off);
        if (lane >= off)
            inc += o;
    }
    if (lane == 31)
        sh.wcnt[warp] = inc;
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
    if ((int)threadIdx.x == b) {
        // this CTA's own requests (list pq) get their positions
        for (int q = 0; q < cnt; ++q) {
            const int l = sh.myreq_l[pq][q];
            if (off0 + q < kMaxReq)
                pend_s[l] = off0 + q;
            else
                pend_t[l] = -1;  // not served: the row may ask again
        }
    }
    if (warp == 0) {
        int tot = lane < (NT / 32) ? sh.wcnt[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            tot += __shfl_xor_sync(kFull, tot, off);
        if (lane == 0)
            sh.nexec = tot < kMaxReq ? tot : kMaxReq;
    }
    __syncthreads();
}

// KK smallest keys over every thread's sorted list; result in sh.tko (all threads).
// Barrier of the threads that work together: the whole CTA (TB == NT), or
// its last TB threads (named barrier 1) while warp 0 does something else.
template <int NT, int TB>
__device__ __forceinline__ void team_sync()
{
    static_assert(TB % 32 == 0 && TB <= NT, "a team is whole warps");
    if constexpr (TB == NT)
        __syncthreads();
    else
        asm volatile("bar.sync 1, %0;" ::"n"(TB) : "memory");
}

// KK smallest keys over every thread's sorted list, for a team of the CTA's
// last TB threads (default: all of them); result in sh.tko (team threads).
template <int NT, int S, int KK, int TB = NT>
__device__ void block_topk(u64 (&L)[KK], Shared<NT, S> &sh)
{
    constexpr int W0 = (NT - TB) / 32;  // first warp of the team
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 w[KK];
    warp_topk(L, w);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < KK; ++q)
            sh.tk[warp][q] = w[q];
    }
    team_sync<NT, TB>();
    if (warp == W0) {
        u64 M[KK];
#pragma unroll
        for (int q = 0; q < KK; ++q)
            M[q] = lane < TB / 32 ? sh.tk[W0 + lane][q] : kNoKey;
        warp_topk(M, w);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < KK; ++q)
                sh.tko[q] = w[q];
        }
    }
    team_sync<NT, TB>();
}

// Grid-wide barrier, split in two so that a CTA can do work that nobody
// waits for between arriving and waiting.  arrive: __syncthreads, then one
// thread adds to the counter with release semantics (the CTA's writes so far
// are published).  wait: that thread spins with acquire loads until every
// CTA has arrived, bounded by a wall-clock limit; returns false when the run
// must stop (this CTA gave up, or another CTA flagged an error).
// With `last` given (phase timing), thread 0 also learns whether its CTA
// was the last to arrive.
__device__ __forceinline__ void grid_arrive(const MergeParams &p, unsigned &epoch, bool *last = nullptr)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        if (p.G > 1) {
            if (last)
                *last = atom_release_add(p.bar, 1u) + 1u == epoch * (unsigned)p.G;
            else
                red_release_add(p.bar, 1u);
        }
    }
}

template <int NT, int S>
__device__ bool grid_wait(const MergeParams &p, unsigned epoch, Shared<NT, S> &sh)
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
            STCG(p.D + q, 0.0f);
            u = 0u;
        } else {
            bad = 1;
            return;
        }
    }
    // a key not below the list's largest cannot enter it (an exact test of
    // the whole key: cells tying on the value are common and go no further)
    const u64 key = ((u64)u << 32) | (u64)c;
    if (key >= L[K - 1])
        return;
    list_insert(L, key);
}

// K smallest keys of row r (all columns are live at launch), computed by one
// warp that also validates every cell of the row.
__device__ void warp_row_topk(const MergeParams &p, long long r, u64 (&out)[K], int &bad)
{
    const long long n = p.n;
    const int lane = threadIdx.x & 31;
    const long long start = row_base(p, r) + r + 1;
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
        init_cell(LDCG(p.D + q), q, (unsigned)(q + base_c), p, L, bad);
    for (long long q = a1 + lane; q < end; q += 32)
        init_cell(LDCG(p.D + q), q, (unsigned)(q + base_c), p, L, bad);
    // 128-bit body, four loads in flight per lane
    long long q = a0 + 4 * lane;
    for (; q + 3 * 128 < a1; q += 4 * 128) {
        float4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            x[u] = LDCG(reinterpret_cast<const float4 *>(p.D + q + 128 * u));
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
        const float4 x = LDCG(reinterpret_cast<const float4 *>(p.D + q));
        const unsigned c = (unsigned)(q + base_c);
        init_cell(x.x, q, c, p, L, bad);
        init_cell(x.y, q + 1, c + 1, p, L, bad);
        init_cell(x.z, q + 2, c + 2, p, L, bad);
        init_cell(x.w, q + 3, c + 3, p, L, bad);
    }
    warp_topk(L, out);
}

// K smallest keys of row r over live columns, computed by the whole CTA (a
// refill, or a row whose cache emptied).  Adds the live cells read to
// `live_cells`.  Result in sh.tko.
// (Row scans are kept out of line: inside the round loop's register
// allocation their loads in flight would be spilled.)
template <int NT, int S, int TB = NT>
__device__ __noinline__ void block_row_topk(const MergeParams &p, long long r, const unsigned *bitmap,
                                            Shared<NT, S> &sh, long long &live_cells)
{
    const int ts = threadIdx.x - (NT - TB);  // thread of the team
    const long long n = p.n;
    const long long start = row_base(p, r) + r + 1;
    const long long end = start + (n - r - 1);
    const long long base_c = r + 1 - start;
    u64 L[K];
#pragma unroll
    for (int q = 0; q < K; ++q)
        L[q] = kNoKey;
    long long cnt = 0;
    auto take = [&](float v, long long q) {
        const long long c = q + base_c;
        if (live(bitmap, c)) {
            ++cnt;
            const u64 key = make_key(v, (unsigned)c);
            if (key < L[K - 1])  // the whole key: ties on the value stop here
                list_insert(L, key);
        }
    };
    // unaligned head and tail one word per thread; the body as 16-byte loads,
    // eight in flight per thread (dead cells are read and dropped: the row is
    // contiguous, latency and not bandwidth bounds the scan)
    long long a0 = p.aligned16 ? ((start + 3) & ~3LL) : end;
    if (a0 > end)
        a0 = end;
    const long long a1 = a0 + ((end - a0) & ~3LL);
    for (long long q = start + ts; q < a0; q += TB)
        take(LDCG(p.D + q), q);
    for (long long q = a1 + ts; q < end; q += TB)
        take(LDCG(p.D + q), q);
    const float4 *D4 = reinterpret_cast<const float4 *>(p.D);
    const long long j1 = a1 >> 2;
    for (long long j0 = (a0 >> 2) + ts; j0 < j1; j0 += 8 * TB) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long j = j0 + (long long)u * TB;
            v[u] = j < j1 ? LDCG(D4 + j) : make_float4(-1.0f, -1.0f, -1.0f, -1.0f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (v[u].x >= 0.0f) {
                const long long q = (j0 + (long long)u * TB) << 2;
                take(v[u].x, q);
                take(v[u].y, q + 1);
                take(v[u].z, q + 2);
                take(v[u].w, q + 3);
            }
        }
    }
    live_cells += cnt;
    block_topk<NT, S, K, TB>(L, sh);
}

// block_row_topk in the row-log layout.  Row r's current cells are (a) r's
// log at every merge q after r's stamp whose survivor c is still live and
// has not merged again (vpos: this CTA's bitmap of such "latest" merges),
// and (b) row r of M at every other live column.  Part (a) marks its columns
// in the scratch bitmap `newer`, part (b) skips them; only c > r count.
// Merges t0 .. t0 + L0 - 1 (the current round, L0 > 0 only after this CTA's
// own pass 2) take their survivors from the round's chain in shared memory,
// older ones from the merge list.  Used by the owner's immediate rescans,
// which run in the round they are needed (refill scans, which read the state
// a whole round left, go column by column: block_row_topk_cols).  Result in
// sh.tko.
template <int NT, int S, int TB = NT>
__device__ __noinline__ void block_row_topk_log(const MergeParams &p, long long r, const unsigned *bitmap,
                                   const unsigned *vpos, unsigned *newer, Shared<NT, S> &sh, long long t0,
                                   int L0, long long &live_cells, u64 *tlog = nullptr)
{
    const int ts = threadIdx.x - (NT - TB);  // thread of the team
    // with phase timing on, the team's first thread adds the time of the log
    // part to tlog[0] and of the matrix part (and the top-K) to tlog[1]
    u64 tm0 = tlog && ts == 0 ? global_ns() : 0;
    const long long n = p.n;
    const long long nwords = (n + 31) / 32;
    const int sr = LDCG(p.stamp + r);
    u64 L[K];
#pragma unroll
    for (int q = 0; q < K; ++q)
        L[q] = kNoKey;
    long long cnt = 0;
    auto take = [&](float v, long long c) {
        ++cnt;
        const u64 key = make_key(v, (unsigned)c);
        if (key < L[K - 1])  // the whole key: ties on the value stop here
            list_insert(L, key);
    };
    for (long long w = ts; w < nwords; w += TB)
        newer[w] = 0u;
    team_sync<NT, TB>();
    // (a) the log: latest merges after r's stamp, eight positions in flight
    const float *log = p.TL + r * p.pitch;
    const long long t1 = t0 + L0;
    {
        constexpr int U = 8;
        for (long long q0 = (long long)sr + 1 + ts; q0 < t1; q0 += U * TB) {
            float v[U];
            int c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long q = q0 + (long long)u * TB;
                c[u] = -1;
                if (q < t1 && ((vpos[q >> 5] >> (q & 31)) & 1u)) {
                    c[u] = q < t0 ? LDCG(p.merges + 2 * q) : sh.pi[q - t0];
                    v[u] = LDCG(log + q);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (c[u] >= 0) {
                    atomicOr(&newer[c[u] >> 5], 1u << (c[u] & 31));
                    if (c[u] > r)
                        take(v[u], c[u]);
                }
            }
        }
    }
    team_sync<NT, TB>();
    if (tlog && ts == 0) {
        const u64 now = global_ns();
        tlog[0] += now - tm0;
        tm0 = now;
    }
    // (b) row r of M at live columns c > r not found in the log: 16-byte
    // pieces (rows start 16-byte aligned), eight in flight per thread.  The
    // first batch also gives a bound: the 4th smallest of the team's
    // per-thread minima is the key of a real cell with at least three real
    // cells below it, so no cell above it can be among the row's four
    // smallest; after it only cells at or below it reach the lists.
    const float *row = p.D + r * p.pitch;
    auto cur = [&](long long c) { return ((bitmap[c >> 5] & ~newer[c >> 5]) >> (c & 31)) & 1u; };
    long long c_a = (r + 4) & ~3LL;  // first multiple of 4 above r
    if (c_a > n)
        c_a = n;
    const long long c_b = c_a + ((n - c_a) & ~3LL);
    for (long long c = r + 1 + ts; c < c_a; c += TB)
        if (cur(c))
            take(LDCG(row + c), c);
    for (long long c = c_b + ts; c < n; c += TB)
        if (cur(c))
            take(LDCG(row + c), c);
    {
        constexpr int U = 8;
        const float4 *R4 = reinterpret_cast<const float4 *>(row);
        const long long j1 = c_b >> 2;
        u64 thr = kNoKey;
        bool first = true;
        for (long long j0 = (c_a >> 2) + ts;; j0 += U * TB) {
            if (!first && j0 >= j1)
                break;  // (every thread of the team runs the first batch: it holds a barrier)
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long j = j0 + (long long)u * TB;
                v[u] = j < j1 ? LDCG(R4 + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            if (first) {
                u64 mn = kNoKey;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long j = j0 + (long long)u * TB;
                    if (j < j1) {
                        const long long c = j << 2;
                        const unsigned m4 = ((bitmap[c >> 5] & ~newer[c >> 5]) >> (c & 31)) & 15u;
                        const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const u64 k = make_key(vv[e], (unsigned)(c + e));
                            if (((m4 >> e) & 1u) && k < mn)
                                mn = k;
                        }
                    }
                }
                u64 M4[K] = {mn, kNoKey, kNoKey, kNoKey};
                block_topk<NT, S, K, TB>(M4, sh);
                thr = sh.tko[K - 1];
                first = false;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long j = j0 + (long long)u * TB;
                if (j < j1) {
                    const long long c = j << 2;
                    const unsigned m4 = ((bitmap[c >> 5] & ~newer[c >> 5]) >> (c & 31)) & 15u;
                    cnt += __popc(m4);
                    const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const u64 k = make_key(vv[e], (unsigned)(c + e));
                        if (((m4 >> e) & 1u) && k <= thr && k < L[K - 1])
                            list_insert(L, k);
                    }
                }
            }
        }
    }
    live_cells += cnt;
    block_topk<NT, S, K, TB>(L, sh);
    if (tlog && ts == 0)
        tlog[1] += global_ns() - tm0;
}

// block_row_topk in the row-log layout, column by column: live column c > r
// holds its current cell in row r of M when c's stamp is not after r's, and
// otherwise in r's log at c's stamp (written by that merge).  The stamps are
// read beside the row (16-byte pieces of both, two of each per thread and
// batch), then the log cells of the columns stamped after r: two dependent
// reads per batch and no pass over the merge list.  (A deeper batch holds
// more registers across the call, and the caller, the round loop, then
// spills: two pieces measured fastest.)  Needs p.D and p.stamp 16-byte
// aligned (rows are, the pitch being a multiple of 4).  The first batch
// gives a bound when the row has more than one batch (see
// block_row_topk_log).  Result in sh.tko.
template <int NT, int S, int TB = NT>
__device__ __noinline__ void block_row_topk_cols(const MergeParams &p, long long r, const unsigned *bitmap,
                                                 Shared<NT, S> &sh, long long &live_cells, u64 *tlog = nullptr)
{
    const int ts = threadIdx.x - (NT - TB);  // thread of the team
    const u64 tm0 = tlog && ts == 0 ? global_ns() : 0;
    const long long n = p.n;
    const int sr = LDCG(p.stamp + r);
    const float *row = p.D + r * p.pitch;
    const float *log = p.TL + r * p.pitch;
    u64 L[K];
#pragma unroll
    for (int q = 0; q < K; ++q)
        L[q] = kNoKey;
    long long cnt = 0;
    auto one = [&](long long c) {
        if (live(bitmap, c)) {
            ++cnt;
            const int sc = LDCG(p.stamp + c);
            const float v = sc > sr ? LDCG(log + sc) : LDCG(row + c);
            const u64 key = make_key(v, (unsigned)c);
            if (key < L[K - 1])
                list_insert(L, key);
        }
    };
    long long c_a = (r + 4) & ~3LL;  // first multiple of 4 above r
    if (c_a > n)
        c_a = n;
    const long long c_b = c_a + ((n - c_a) & ~3LL);
    for (long long c = r + 1 + ts; c < c_a; c += TB)
        one(c);
    for (long long c = c_b + ts; c < n; c += TB)
        one(c);
    {
        constexpr int U = 2;
        const float4 *R4 = reinterpret_cast<const float4 *>(row);
        const int4 *S4 = reinterpret_cast<const int4 *>(p.stamp);
        const long long j0a = c_a >> 2, j1 = c_b >> 2;
        // a bound from the first batch only pays when more batches follow
        bool first = j1 - j0a > (long long)U * TB;
        u64 thr = kNoKey;
        for (long long j0 = j0a + ts;; j0 += U * TB) {
            if (!first && j0 >= j1)
                break;  // (every thread of the team runs a first batch: it holds a barrier)
            float v[U][4];
            int sc[U][4];
            unsigned m4[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long j = j0 + (long long)u * TB;
                m4[u] = 0u;
                if (j < j1) {
                    const float4 a = LDCG(R4 + j);
                    const int4 b = LDCG(S4 + j);
                    v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
                    sc[u][0] = b.x; sc[u][1] = b.y; sc[u][2] = b.z; sc[u][3] = b.w;
                    const long long c = j << 2;
                    m4[u] = (bitmap[c >> 5] >> (c & 31)) & 15u;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (((m4[u] >> e) & 1u) && sc[u][e] > sr)
                        v[u][e] = LDCG(log + sc[u][e]);
            }
            if (first) {
                u64 mn = kNoKey;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long c = (j0 + (long long)u * TB) << 2;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const u64 k = make_key(v[u][e], (unsigned)(c + e));
                        if (((m4[u] >> e) & 1u) && k < mn)
                            mn = k;
                    }
                }
                u64 M4[K] = {mn, kNoKey, kNoKey, kNoKey};
                block_topk<NT, S, K, TB>(M4, sh);
                thr = sh.tko[K - 1];
                first = false;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long c = (j0 + (long long)u * TB) << 2;
                cnt += __popc(m4[u]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const u64 k = make_key(v[u][e], (unsigned)(c + e));
                    if (((m4[u] >> e) & 1u) && k <= thr && k < L[K - 1])
                        list_insert(L, k);
                }
            }
        }
    }
    live_cells += cnt;
    block_topk<NT, S, K, TB>(L, sh);
    if (tlog && ts == 0)
        tlog[1] += global_ns() - tm0;
}

// K smallest keys of row r over live columns, computed by one warp (the
// rows of a one-CTA job are refreshed this way, several warps side by side).
// Adds the live cells read to `live_cells`.  Result in out (all lanes).
__device__ __noinline__ void warp_row_refresh(const MergeParams &p, long long r, const unsigned *bitmap,
                                              u64 (&out)[K],
                                 long long &live_cells)
{
    const int lane = threadIdx.x & 31;
    const long long start = row_base(p, r) + r + 1;
    const long long end = start + (p.n - r - 1);
    const long long base_c = r + 1 - start;
    u64 L[K];
#pragma unroll
    for (int q = 0; q < K; ++q)
        L[q] = kNoKey;
    long long cnt = 0;
    auto take = [&](float v, long long q) {
        const long long c = q + base_c;
        if (live(bitmap, c)) {
            ++cnt;
            const u64 key = make_key(v, (unsigned)c);
            if (key < L[K - 1])  // the whole key: ties on the value stop here
                list_insert(L, key);
        }
    };
    long long a0 = p.aligned16 ? ((start + 3) & ~3LL) : end;
    if (a0 > end)
        a0 = end;
    const long long a1 = a0 + ((end - a0) & ~3LL);
    for (long long q = start + lane; q < a0; q += 32)
        take(LDCG(p.D + q), q);
    for (long long q = a1 + lane; q < end; q += 32)
        take(LDCG(p.D + q), q);
    const float4 *D4 = reinterpret_cast<const float4 *>(p.D);
    const long long j1 = a1 >> 2;
    for (long long j0 = (a0 >> 2) + lane; j0 < j1; j0 += 8 * 32) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long j = j0 + 32 * u;
            v[u] = j < j1 ? LDCG(D4 + j) : make_float4(-1.0f, -1.0f, -1.0f, -1.0f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (v[u].x >= 0.0f) {
                const long long q = (j0 + 32 * u) << 2;
                take(v[u].x, q);
                take(v[u].y, q + 1);
                take(v[u].z, q + 2);
                take(v[u].w, q + 3);
            }
        }
    }
    live_cells += cnt;
    warp_topk(L, out);
}

// All n - 1 merges of one job, run by CTA b of the job's G CTAs (every CTA
// of the job calls this with the same p).  smem_raw: merge_smem_bytes(n, G)
// bytes of dynamic shared memory.
template <int NT, int PUB>
__device__ void merge_job(const MergeParams &p, const int b, unsigned char *smem_raw,
                          Shared<NT, round_of(PUB)> &sh)
{
    constexpr int S = round_of(PUB);
    constexpr int W = NT / 32;
    const long long n = p.n;
    const int G = p.G;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const long long nb = (n + kRowBlock - 1) / kRowBlock;      // row blocks
    const long long my_blocks = b < nb ? (nb - b + G - 1) / G : 0;
    const int R = (int)(my_blocks * kRowBlock);                 // owned row slots
    const long long Rmax = ((nb + G - 1) / G) * kRowBlock;
    const long long nwords = (n + 31) / 32;

    // dynamic shared memory: liveness bitmap; the published entries of every
    // CTA (keys, column words); then per owned slot l: cache
    // keys (key q of slot l at ck[q * Rmax + l]: consecutive threads read
    // consecutive words), bound, size, key count, pending refill (round,
    // list position) and a flag for rows in this round's chain
    unsigned char *q0 = smem_raw;
    unsigned *bitmap = reinterpret_cast<unsigned *>(q0);
    q0 += (nwords * 4 + 15) & ~15LL;
    // row-log layout: merges whose survivor is live and has not merged again
    // (bit q), and a scratch bitmap of columns for the row scans
    unsigned *vpos = reinterpret_cast<unsigned *>(q0);
    unsigned *newer = vpos + nwords;
    q0 += G > 1 ? (2 * nwords * 4 + 15) & ~15LL : 0;
    u64 *wkey = reinterpret_cast<u64 *>(q0);
    q0 += (size_t)G * PUB * 8;
    u64 *ck = reinterpret_cast<u64 *>(q0);
    q0 += (size_t)Rmax * K * 8;
    u64 *cB = reinterpret_cast<u64 *>(q0);
    q0 += (size_t)Rmax * 8;
    unsigned *wcol = reinterpret_cast<unsigned *>(q0);
    q0 += (size_t)G * PUB * 4;
    // more than 16 pairs per round: pass-1 values of the rows of one chunk of
    // NT owned rows, kvs[q * KVP + a] for chunk row q and pair a (up to 16
    // pairs they stay in registers)
    constexpr int KVP = S + 1;
    float *kvs = reinterpret_cast<float *>(q0);
    q0 += S > 16 ? (size_t)(Rmax < NT ? Rmax : NT) * KVP * 4 : 0;
    int *rsize = reinterpret_cast<int *>(q0);
    int *ccnt = rsize + Rmax;
    int *pend_t = ccnt + Rmax;
    int *pend_s = pend_t + Rmax;
    int *rlist = pend_s + Rmax;
    int *rstamp = rlist + Rmax;  // row-log layout: each owned row's stamp
    unsigned char *mflag = reinterpret_cast<unsigned char *>(rstamp + Rmax);
    unsigned char *okf = mflag + Rmax;  // [NT]: chunk row q got pass-1 values

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
    // a refill request for slot l in round r (list par = r & 1)
    auto request = [&](int l, int r) {
        const int par = r & 1;
        const int q = atomicAdd(&sh.nmyreq[par], 1);
        if (q < kReqPerCta) {
            sh.myreq_l[par][q] = l;
            pend_t[l] = r;
        }
    };

    // per-phase wall-clock totals of this CTA (thread 0), when timing is on
    auto &ty = sh.ty;
    u64 &ph0 = ty.ph[0], &ph1 = ty.ph[1], &ph2 = ty.ph[2], &ph3 = ty.ph[3], &ph4 = ty.ph[4], &ph5 = ty.ph[5];
    // finer split: ph1 = xs0 (records) + xs1 (walk, installs) + xs2 (chain
    // sizes, stamps, member cells); ph4 = xs3 (cross-CTA minima) + xs4
    // (certification) + xs5 (bookkeeping, survivor caches); ph5 = xs6 (pass 2)
    // + xs7 (owner rescans) + the publish
    u64 &xs0 = ty.xs[0], &xs1 = ty.xs[1], &xs2 = ty.xs[2], &xs3 = ty.xs[3];
    u64 &xs4 = ty.xs[4], &xs5 = ty.xs[5], &xs6 = ty.xs[6], &xs7 = ty.xs[7];
    // ty.xscan: refill scans in the row-log layout (log part, matrix part);
    // ty.xwalk: the walk itself (warp 0); ty.xlast, ty.nlast: barriers this
    // CTA completed (arrived last at), its wait then being the barrier's own
    // latency, with counts of those at B (nlast_b) and of those while serving
    // a refill scan (at B, at A)
    if (tid == 0) {
        for (int q = 0; q < 6; ++q)
            ty.ph[q] = 0;
        for (int q = 0; q < 8; ++q)
            ty.xs[q] = 0;
        ty.xscan[0] = ty.xscan[1] = ty.xwalk = ty.xlast = ty.tmark = 0;
        ty.fills = ty.installs = ty.rounds = ty.idle = ty.walk = ty.rescans = 0;
        ty.nlast = ty.nlast_b = ty.nlast_b_scan = ty.nlast_a_scan = 0;
    }
    auto lap = [&](u64 &acc) {
        if (p.timing && threadIdx.x == 0) {
            const u64 now = global_ns();
            acc += now - ty.tmark;
            ty.tmark = now;
        }
    };

    long long st_updates = 0, st_fill_cells = 0, st_resc_cells = 0;

    // The records of round rr: this CTA's PUB smallest entries (cached keys
    // and bound marks of its rows) and its refill requests of round rr - 1.
    // Also lists the refills to install in round rr (served in round rr - 1).
    auto publish = [&](int rr) {
        u64 Lst[PUB];
#pragma unroll
        for (int q = 0; q < PUB; ++q)
            Lst[q] = kNoKey;
        for (int l = tid; l < R; l += NT) {
            const int c = ccnt[l];
            const u64 B = cB[l];
            if (c > 0 || B != kNoKey) {
                const u64 rowbits = (u64)row_of(l) << 3;
                // a row's entries ascend: skip the ones that cannot enter
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    if (q < c) {
                        const u64 e = (ck[(size_t)q * Rmax + l] & kHi) | rowbits | (u64)q;
                        if (e < Lst[PUB - 1])
                            list_insert_n(Lst, e);
                    }
                }
                if (B != kNoKey) {
                    const u64 e = (B & kHi) | rowbits | (u64)c;
                    if (e < Lst[PUB - 1])
                        list_insert_n(Lst, e);
                }
            }
            if (rr >= 2 && pend_t[l] == rr - 2) {
                const int s2 = atomicAdd(&sh.ninst, 1);
                sh.inst_slot[s2] = l;
            }
        }
        block_topk(Lst, sh);
        if (tid < PUB) {
            // entry tid: its column word
            const u64 key = sh.tko[tid];
            unsigned col = 0;
            if (key != kNoKey) {
                const unsigned lo = (unsigned)key;
                const int slot = slot_of((long long)(lo >> 3));
                const int rank = (int)(lo & 7u);
                col = rank < ccnt[slot] ? (unsigned)ck[(size_t)rank * Rmax + slot] : kRowStop;
                if (tid == PUB - 1)
                    col |= kHardStop;  // more entries may follow: none is published
            }
            STCG(&p.recA[b].key[tid], key);
            STCG(&p.recA[b].col[tid], col);
        }
        if (tid == 0) {
            const int par = (rr - 1) & 1;
            int nq = rr >= 1 ? sh.nmyreq[par] : 0;
            nq = nq < kReqPerCta ? nq : kReqPerCta;
            if (rr >= 1)
                sh.nmyreq[par] = nq;
            int rows[kReqPerCta];
#pragma unroll
            for (int q = 0; q < kReqPerCta; ++q)
                rows[q] = q < nq ? (int)row_of(sh.myreq_l[par][q]) : -1;
            uint4 *dst = reinterpret_cast<uint4 *>(&p.recA[b].nreq);
            STCG(dst + 0, make_uint4((unsigned)nq, (unsigned)rows[0], (unsigned)rows[1], (unsigned)rows[2]));
            STCG(dst + 1, make_uint4((unsigned)rows[3], (unsigned)rows[4], (unsigned)rows[5], (unsigned)rows[6]));
            STCG(dst + 2, make_uint4((unsigned)rows[7], 0u, 0u, 0u));
        }
    };

    // ---- setup
    for (long long w = tid; w < nwords; w += NT) {
        const long long live_n = n - w * 32;
        bitmap[w] = live_n >= 32 ? 0xffffffffu : ((1u << live_n) - 1u);
        if (G > 1)
            vpos[w] = 0u;
    }
    for (int l = tid; l < R; l += NT) {
        rsize[l] = 1;
        pend_t[l] = -1;
        rstamp[l] = -1;
        mflag[l] = 0;
    }
    for (long long r = (long long)b * NT + tid; r < n; r += (long long)G * NT) {
        STCG(p.size_g + r, 1);
        if (p.full)
            STCG(p.stamp + r, -1);
    }
    if (tid == 0) {
        sh.ninst = 0;
        sh.nexec = 0;
        sh.nmyreq[0] = 0;
        sh.nmyreq[1] = 0;
        sh.nprev = 0;
        sh.nresc = 0;
    }

    // ---- phase 0: validate the matrix and fill the caches of owned rows
    // (one warp per owned row; the rows of a CTA are spread over the whole
    // triangle, so every CTA reads about the same number of cells)
    {
        int bad = 0;
        for (int l = warp; l < R; l += W) {
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
    publish(0);

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
        ty.tmark = global_ns();

    long long t = 0;   // merges done
    const long long max_rounds = 2 * n + 64;
    for (int r = 0;; ++r) {
        const int par = r & 1;
        if (r > max_rounds) {
            // no progress: a stop mark that no refill lifts (every CTA sees the
            // same count and leaves here together)
            if (tid == 0)
                atomicCAS(p.status, 0, kErrInternal);
            return;
        }

        // ---- A: every CTA's published entries and refill requests
        {
            int rcnt = 0;
            int rq[kReqPerCta];
#pragma unroll
            for (int q = 0; q < kReqPerCta; ++q)
                rq[q] = -1;
            if (tid < G) {
                const RecA *rec = p.recA + tid;
                const ulonglong2 *ks = reinterpret_cast<const ulonglong2 *>(rec->key);
#pragma unroll
                for (int q = 0; q < PUB / 2; ++q) {
                    const ulonglong2 kk = LDCG(ks + q);
                    wkey[tid * PUB + 2 * q] = kk.x;
                    wkey[tid * PUB + 2 * q + 1] = kk.y;
                }
                const uint4 *cs = reinterpret_cast<const uint4 *>(rec->col);
#pragma unroll
                for (int q = 0; q < PUB / 4; ++q) {
                    const uint4 cc = LDCG(cs + q);
                    wcol[tid * PUB + 4 * q] = cc.x;
                    wcol[tid * PUB + 4 * q + 1] = cc.y;
                    wcol[tid * PUB + 4 * q + 2] = cc.z;
                    wcol[tid * PUB + 4 * q + 3] = cc.w;
                }
                const uint4 *src = reinterpret_cast<const uint4 *>(&rec->nreq);
                const uint4 w3 = LDCG(src), w4 = LDCG(src + 1), w5 = LDCG(src + 2);
                rcnt = (int)w3.x;
                rq[0] = (int)w3.y;
                rq[1] = (int)w3.z;
                rq[2] = (int)w3.w;
                rq[3] = (int)w4.x;
                rq[4] = (int)w4.y;
                rq[5] = (int)w4.z;
                rq[6] = (int)w4.w;
                rq[7] = (int)w5.x;
            }
            exchange_requests(rcnt, rq, b, sh, par ^ 1, pend_t, pend_s);
        }
        if (tid == 0)
            sh.nmyreq[par] = 0;
        lap(xs0);

        const u64 twalk0 = p.timing && tid == 0 ? global_ns() : 0;
        if (warp == 0) {
            // ---- the walk: merge the G published lists in key order.  Lane
            // l keeps the heads of the lists of CTAs l, l + 32, ... in registers.
            constexpr int UMAX = 8;  // G <= 256
            u64 hk[UMAX];
            int hp[UMAX];
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
                const int g = lane + 32 * u;
                hp[u] = 0;
                hk[u] = g < G ? wkey[g * PUB] : kNoKey;
            }
            auto local_min = [&](u64 &lm, int &lu) {
                lm = hk[0];
                lu = 0;
#pragma unroll
                for (int u = 1; u < UMAX; ++u) {
                    if (hk[u] < lm) {
                        lm = hk[u];
                        lu = u;
                    }
                }
            };
            u64 lm;
            int lu;
            local_min(lm, lu);
            int np = 0;
            // member 2a = i_a, 2a + 1 = j_a: lane l holds members l and l + 32
            int member0 = -1, member1 = -1;
            unsigned front = 0;  // value bits of the last entry visited
            // lane a fetches the sizes and stamps of pair a as soon as it is
            // accepted: they arrive while the walk goes on (asynchronous copies
            // of the aligned words around them, when the arrays allow it)
            const bool qa = ((reinterpret_cast<uintptr_t>(p.size_g) |
                              reinterpret_cast<uintptr_t>(p.stamp)) & 15u) == 0;
            int q_szi = 0, q_szj = 0, q_si = 0, q_sj = 0;
            int nwalk = 0;
            for (int guard = 0; guard <= G * PUB; ++guard) {
                const u64 m = warp_u64_min(lm);
                if (m == kNoKey)
                    break;
                ++nwalk;
                front = (unsigned)(m >> 32);
                const int src = __ffs(__ballot_sync(kFull, lm == m)) - 1;
                unsigned col = 0;
                if (lane == src) {
#pragma unroll
                    for (int u = 0; u < UMAX; ++u) {
                        if (u == lu) {
                            const int g = lane + 32 * u;
                            col = wcol[g * PUB + hp[u]];
                            hp[u] += 1;
                            hk[u] = hp[u] < PUB ? wkey[g * PUB + hp[u]] : kNoKey;
                        }
                    }
                    local_min(lm, lu);
                }
                col = __shfl_sync(kFull, col, src);
                const int row = (int)(((unsigned)m) >> 3);
                bool stop = (col & kHardStop) != 0;
                if (!__any_sync(kFull, member0 == row || member1 == row)) {
                    if (col & kRowStop) {
                        stop = true;  // the row's smallest untouched cell is unknown
                    } else {
                        const int c = (int)(col & kColMask);
                        if (!__any_sync(kFull, member0 == c || member1 == c)) {
                            if (2 * np < 32) {
                                if (lane == 2 * np)
                                    member0 = row;
                                if (lane == 2 * np + 1)
                                    member0 = c;
                            } else {
                                if (lane == 2 * np - 32)
                                    member1 = row;
                                if (lane == 2 * np - 31)
                                    member1 = c;
                            }
                            if (lane == 0) {
                                sh.pi[np] = row;
                                sh.pj[np] = c;
                                sh.ph[np] = __uint_as_float((unsigned)(m >> 32));
                            }
                            // (a pair out of range is caught before any other access)
                            if (lane == np && row >= 0 && row < c && c < n) {
                                if (qa) {
                                    // (the arrays are padded to whole 16-byte words)
                                    int *w = sh.qw[np];
                                    if (CHECKED_16(p.size_g + (row & ~3)) && CHECKED_16(p.size_g + (c & ~3))) {
                                        copy16_async(w, p.size_g + (row & ~3));
                                        copy16_async(w + 4, p.size_g + (c & ~3));
                                    }
                                    if (p.full && CHECKED_16(p.stamp + (row & ~3)) && CHECKED_16(p.stamp + (c & ~3))) {
                                        copy16_async(w + 8, p.stamp + (row & ~3));
                                        copy16_async(w + 12, p.stamp + (c & ~3));
                                    }
                                } else {
                                    q_szi = LDCG(p.size_g + row);
                                    q_szj = LDCG(p.size_g + c);
                                    if (p.full) {
                                        q_si = LDCG(p.stamp + row);
                                        q_sj = LDCG(p.stamp + c);
                                    }
                                }
                            }
                            ++np;
                            if (np == S)
                                stop = true;
                        }
                    }
                }
                if (stop)
                    break;
            }
            if (lane == 0) {
                sh.np = np;
                sh.front = front;
                ty.walk += nwalk;
            }
            copy_async_wait_all();
            __syncwarp();
            if (lane < np) {
                const int row = sh.pi[lane], c = sh.pj[lane];
                if (qa && row >= 0 && row < c && c < n) {
                    // lane a issued pair a's copies, so they are complete
                    const int *w = sh.qw[lane];
                    q_szi = w[row & 3];
                    q_szj = w[4 + (c & 3)];
                    if (p.full) {
                        q_si = w[8 + (row & 3)];
                        q_sj = w[12 + (c & 3)];
                    }
                }
                sh.szi[lane] = q_szi;
                sh.szj[lane] = q_szj;
                sh.si[lane] = q_si;
                sh.sj[lane] = q_sj;
                sh.bi[lane] = row_base(p, sh.pi[lane]);  // cell (i, c) at bi + c (packed: for c > i)
                sh.bj[lane] = row_base(p, sh.pj[lane]);
            }
            if (p.timing && tid == 0)
                ty.xwalk += global_ns() - twalk0;
        } else {
            // ---- refills served in the previous round: take the row's list,
            // then replay that round's merges (the scan ran before them, or
            // while they were being written)
            const int ninst = sh.ninst;
            const int ipar = par ^ 1;
            for (int s2 = warp - 1; s2 < ninst; s2 += W - 1) {
                const int l = sh.inst_slot[s2];
                const int pos = pend_s[l];
                const long long row = row_of(l);
                u64 M[K];
                {
                    const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(
                        p.parts + ((size_t)ipar * kMaxReq + pos) * K);
#pragma unroll
                    for (int q = 0; q < K / 2; ++q) {
                        const ulonglong2 v = LDCG(src + q);
                        M[2 * q] = v.x;
                        M[2 * q + 1] = v.y;
                    }
                }
                // the new cells (row, i_a) of the previous round's merges, one lane each
                const int np2 = sh.nprev;
                const long long base = row_base(p, row);  // cell (row, c) at base + c
                u64 xr = kNoKey;
                if (lane < np2) {
                    const long long ia = sh.ppi[lane];
                    if (ia > row)
                        xr = make_key(LDCG(p.full ? p.D + ia * p.pitch + row : p.D + base + ia), (unsigned)ia);
                }
                u64 xs[S];
#pragma unroll
                for (int a = 0; a < S; ++a)
                    xs[a] = __shfl_sync(kFull, xr, a);
                // keys whose column a merge of that round retired or rewrote
                const int c0 = list_count(M);
                const u64 B0 = c0 == K ? M[K - 1] : kNoKey;
                const int mi = lane < np2 ? sh.ppi[lane] : -1;
                const int mj = lane < np2 ? sh.ppj[lane] : -1;
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    const int col = (int)(unsigned)M[q];
                    if (__any_sync(kFull, M[q] != kNoKey && (col == mi || col == mj)))
                        M[q] = kNoKey;
                }
                if (lane == 0) {
                    u64 B = B0;
                    sort_list(M);
                    int c = list_count(M);
#pragma unroll
                    for (int a = 0; a < S; ++a) {
                        const u64 x = xs[a];
                        if (x != kNoKey && x <= B) {
                            list_insert(M, x);
                            if (c == K)
                                B = M[K - 1];
                            else
                                ++c;
                        }
                    }
                    cache_store(l, M);
                    ccnt[l] = c;
                    cB[l] = B;
                    pend_t[l] = -1;
                }
            }
            if (tid == 32)
                ty.installs += ninst;
            // ---- the refills asked for in the previous round, served now by
            // warps 1.. while warp 0 walks (row s of the list by CTA
            // G - 1 - s mod G: rows are owned in blocks of 32 from CTA 0 up,
            // so the last CTAs own a block fewer and take the scans first):
            // the K smallest keys of the row over live columns, as the
            // previous round left it; the owner installs the list at the start
            // of the next round and replays this round's merges on it
            constexpr int TB = NT - 32;
            const int nexec = sh.nexec;
            const bool cols_ok = ((reinterpret_cast<uintptr_t>(p.D) | reinterpret_cast<uintptr_t>(p.stamp)) & 15u) == 0;
            for (int s2 = G - 1 - b; s2 < nexec; s2 += G) {
                const long long rr = sh.exec_row[s2];
                if (rr < 0 || rr >= n - 1)
                    continue;  // the same for every thread of the team
                if (p.full && cols_ok)
                    block_row_topk_cols<NT, S, TB>(p, rr, bitmap, sh, st_fill_cells, p.timing ? ty.xscan : nullptr);
                else if (p.full)
                    block_row_topk_log<NT, S, TB>(p, rr, bitmap, vpos, newer, sh, t, 0, st_fill_cells,
                                                  p.timing ? ty.xscan : nullptr);
                else
                    block_row_topk<NT, S, TB>(p, rr, bitmap, sh, st_fill_cells);
                if (tid - 32 < K / 2) {
                    const int h = tid - 32;
                    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(p.parts + ((size_t)par * kMaxReq + s2) * K);
                    STCG(dst + h, make_ulonglong2(sh.tko[2 * h], sh.tko[2 * h + 1]));
                }
            }
            if (tid == 32)
                ty.fills += nexec;
        }
        __syncthreads();
        lap(xs1);
        const int s = sh.np;
        {
            // every CTA read the same records and walked them the same way, so
            // every CTA takes this exit together
            int bad = 0;
            if (tid < s) {
                const int i = sh.pi[tid], j = sh.pj[tid];
                bad = !(i >= 0 && i < j && j < n);
            }
            if (__syncthreads_or(bad)) {
                if (tid == 0)
                    atomicCAS(p.status, 0, kErrInternal);
                return;
            }
        }

        // ---- the chain's sizes, member flags and the cells between members
        for (int e = tid; e < W * S; e += NT) {
            sh.wam[e / S][e % S] = kNoKey;
            sh.whm[e / S][e % S] = kNoKey;
        }
        if (tid < 2 * s) {
            const long long m = (tid & 1) ? sh.pj[tid >> 1] : sh.pi[tid >> 1];
            if (owner_of(m) == b)
                mflag[slot_of(m)] = 1;
        }
        // the cells between members of different pairs: loaded now, landed in
        // shared memory after pass 1 (member u = 2a + (0 for i_a, 1 for j_a))
        // (more than eight per thread go to shared memory at once)
        constexpr int DMALL = (4 * S * S + NT - 1) / NT;
        constexpr bool DM_REG = DMALL <= 8;
        constexpr int DMR = DM_REG ? DMALL : 1;
        float dmv[DMR];
        if (DM_REG) {
#pragma unroll
            for (int q = 0; q < DMR; ++q) {
                const int e = tid + q * NT;
                const int u = e / (2 * S), v = e % (2 * S);
                dmv[q] = 0.0f;
                if (e < 4 * S * S && u < v && v < 2 * s && (u >> 1) != (v >> 1)) {
                    const long long mu = (u & 1) ? sh.pj[u >> 1] : sh.pi[u >> 1];
                    const long long mv = (v & 1) ? sh.pj[v >> 1] : sh.pi[v >> 1];
                    const int su = (u & 1) ? sh.sj[u >> 1] : sh.si[u >> 1];
                    const int sv = (v & 1) ? sh.sj[v >> 1] : sh.si[v >> 1];
                    dmv[q] = member_cell(p, mu, su, mv, sv);
                }
            }
        } else {
            for (int e = tid; e < 4 * S * S; e += NT) {
                const int u = e / (2 * S), v = e % (2 * S);
                if (u < v && v < 2 * s && (u >> 1) != (v >> 1)) {
                    const long long mu = (u & 1) ? sh.pj[u >> 1] : sh.pi[u >> 1];
                    const long long mv = (v & 1) ? sh.pj[v >> 1] : sh.pi[v >> 1];
                    const int su = (u & 1) ? sh.sj[u >> 1] : sh.si[u >> 1];
                    const int sv = (v & 1) ? sh.sj[v >> 1] : sh.si[v >> 1];
                    const float d = member_cell(p, mu, su, mv, sv);
                    sh.Dm[u][v] = d;
                    sh.Dm[v][u] = d;
                }
            }
        }
        __syncthreads();
        lap(xs2);

        // ---- pass 1: new cells of every live k outside the chain (reads only),
        // the pairs in groups of 16; the values of each thread's first row are
        // kept in shared memory for pass 2
        constexpr int PG = 16;
        // up to 16 pairs the values stay in registers; more go to shared memory
        constexpr bool KV_REG = S <= PG;
        float kv[KV_REG ? S : 1];
#pragma unroll
        for (int a = 0; a < (KV_REG ? S : 1); ++a)
            kv[a] = 0.0f;
        bool kok = false;
        constexpr int PC = 8;  // pairs whose cells one thread loads at once
        if constexpr (S > PG) {
            // every owned row's new cells, a chunk of NT rows at a time (the
            // last chunk first, so chunk 0 stays in kvs for pass 2); after each
            // chunk, NT / S threads per pair take its smallest new cell over
            // the chunk's rows (all k and k > i_a), then reduce across lanes
            constexpr int TPP = NT / S;
            const int ra = tid / TPP, rpart = tid % TPP;
            u64 ma = kNoKey, mh = kNoKey;
            if (s > 0) {
                for (int l0 = ((R - 1) / NT) * NT; l0 >= 0; l0 -= NT) {
                    const int l = l0 + tid;
                    bool ok = false;
                    long long k = 0;
                    if (l < R) {
                        k = row_of(l);
                        ok = k < n && live(bitmap, k) && !mflag[l];
                    }
                    okf[tid] = ok;
                    if (ok) {
                        const int nk = rsize[l];
                        const long long bk = row_base(p, k);
                        const bool full = p.full;
                        const int sk = full ? rstamp[l] : 0;
                        float *kr = kvs + (size_t)tid * KVP;
#pragma unroll 1
                        for (int a0 = 0; a0 < s; a0 += PC) {
                            float va[PC], vb[PC];
#pragma unroll
                            for (int u = 0; u < PC; ++u) {
                                const int a = a0 + u;
                                va[u] = 0.0f;
                                vb[u] = 0.0f;
                                if (a < s) {
                                    if (full) {
                                        va[u] = LDCG(sh.si[a] >= sk ? p.D + sh.bi[a] + k : p.TL + sh.bi[a] + sk);
                                        vb[u] = LDCG(sh.sj[a] >= sk ? p.D + sh.bj[a] + k : p.TL + sh.bj[a] + sk);
                                    } else {
                                        const long long i = sh.pi[a], j = sh.pj[a];
                                        va[u] = LDCG(p.D + (k > i ? sh.bi[a] + k : bk + i));
                                        vb[u] = LDCG(p.D + (k > j ? sh.bj[a] + k : bk + j));
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < PC; ++u) {
                                const int a = a0 + u;
                                if (a < s)
                                    kr[a] = lw_cell(p.linkage, va[u], vb[u], sh.ph[a], sh.szi[a], sh.szj[a], nk);
                            }
                        }
                    }
                    __syncthreads();
                    if (ra < s) {
                        const long long ia = sh.pi[ra];
                        for (int q = rpart; q < NT && l0 + q < R; q += TPP) {
                            if (!okf[q])
                                continue;
                            const long long kq = row_of(l0 + q);
                            const u64 key = make_key(kvs[(size_t)q * KVP + ra], (unsigned)kq);
                            ma = key < ma ? key : ma;
                            if (kq > ia && key < mh)
                                mh = key;
                        }
                    }
                    __syncthreads();
                }
            }
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                const u64 x = __shfl_xor_sync(kFull, ma, o);
                const u64 y = __shfl_xor_sync(kFull, mh, o);
                ma = x < ma ? x : ma;
                mh = y < mh ? y : mh;
            }
            if (rpart == 0) {
                STCG(p.recB + (size_t)b * 2 * kRound + ra, ma);
                STCG(p.recB + (size_t)b * 2 * kRound + kRound + ra, mh);
            }
        } else if (s > 0) {
            for (int l0 = 0; l0 < R; l0 += NT) {
                const int l = l0 + tid;
                bool ok = false;
                long long k = 0;
                int nk = 1;
                if (l < R) {
                    k = row_of(l);
                    ok = k < n && live(bitmap, k) && !mflag[l];
                    if (ok)
                        nk = rsize[l];
                }
                // cell (k, i): packed, row i for k > i (consecutive k of a warp
                // read consecutive words) and row k for k < i; row-log layout,
                // row i of M when i was stamped no earlier than k, else i's
                // log at k's stamp (words of one contiguous range)
                const long long bk = row_base(p, k);
                const bool full = p.full;
                const int sk = full && l < R ? rstamp[l] : 0;
#pragma unroll
                for (int a0 = 0; a0 < S; a0 += PG) {
                    if (a0 >= s)
                        break;
                    float va[PG], vb[PG];
#pragma unroll
                    for (int u = 0; u < PG; ++u) {
                        const int a = a0 + u;
                        va[u] = 0.0f;
                        vb[u] = 0.0f;
                        if (ok && a < s) {
                            const long long i = sh.pi[a], j = sh.pj[a];
                            if (full) {
                                va[u] = LDCG(sh.si[a] >= sk ? p.D + sh.bi[a] + k : p.TL + sh.bi[a] + sk);
                                vb[u] = LDCG(sh.sj[a] >= sk ? p.D + sh.bj[a] + k : p.TL + sh.bj[a] + sk);
                            } else {
                                va[u] = LDCG(p.D + (k > i ? sh.bi[a] + k : bk + i));
                                vb[u] = LDCG(p.D + (k > j ? sh.bj[a] + k : bk + j));
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < PG; ++u) {
                        const int a = a0 + u;
                        if (a >= s)
                            break;
                        u64 ka = kNoKey, kh = kNoKey;
                        if (ok) {
                            const float v = lw_cell(p.linkage, va[u], vb[u], sh.ph[a], sh.szi[a], sh.szj[a], nk);
                            if (l0 == 0) {
                                kv[KV_REG ? a : 0] = v;
                            }
                            ka = make_key(v, (unsigned)k);
                            if (k > sh.pi[a])
                                kh = ka;
                        }
                        // a warp's rows are one block of 32 consecutive k: unless the
                        // block holds i_a, "k > i_a" is all of it or none of it
                        const long long k0 = (long long)(b + (long long)G * (l >> 5)) * kRowBlock;
                        const u64 ma = warp_u64_min(ka);
                        u64 mh;
                        if (k0 > sh.pi[a])
                            mh = ma;
                        else if (k0 + kRowBlock <= sh.pi[a])
                            mh = kNoKey;
                        else
                            mh = warp_u64_min(kh);
                        // each warp keeps its own minima (no shared-memory atomics)
                        if (lane == 0) {
                            if (ma < sh.wam[warp][a])
                                sh.wam[warp][a] = ma;
                            if (mh < sh.whm[warp][a])
                                sh.whm[warp][a] = mh;
                        }
                    }
                }
                if (l0 == 0)
                    kok = ok;
            }
        }
        if (DM_REG) {
#pragma unroll
            for (int q = 0; q < DMR; ++q) {
                const int e = tid + q * NT;
                const int u = e / (2 * S), v = e % (2 * S);
                if (e < 4 * S * S && u < v && v < 2 * s && (u >> 1) != (v >> 1)) {
                    sh.Dm[u][v] = dmv[q];
                    sh.Dm[v][u] = dmv[q];
                }
            }
        }
        if constexpr (S <= PG) {
            __syncthreads();
            if (tid < 2 * S) {
                // this CTA's minima per pair: over its warps
                const int a = tid % S;
                u64 m = kNoKey;
                for (int w = 0; w < W; ++w) {
                    const u64 x = tid < S ? sh.wam[w][a] : sh.whm[w][a];
                    m = x < m ? x : m;
                }
                STCG(p.recB + (size_t)b * 2 * kRound + (tid < S ? tid : kRound + tid - S), m);
            }
        }
        lap(ph2);
        bool last_b = false;
        grid_arrive(p, epoch, p.timing ? &last_b : nullptr);

        // ---- window of barrier B: the cells (i_a, i_b) and (i_a, j_b) after
        // merge a alone, then (i_a, i_b) after merges a and b (read only after
        // barrier B)
        for (int e = tid; e < s * s; e += NT) {
            const int a = e / s, c = e % s;
            if (a != c) {
                sh.X[a][c] = lw_cell(p.linkage, sh.Dm[2 * c][2 * a], sh.Dm[2 * c][2 * a + 1], sh.ph[a],
                                     sh.szi[a], sh.szj[a], sh.szi[c]);
                sh.Y[a][c] = lw_cell(p.linkage, sh.Dm[2 * c + 1][2 * a], sh.Dm[2 * c + 1][2 * a + 1],
                                     sh.ph[a], sh.szi[a], sh.szj[a], sh.szj[c]);
            }
        }
        __syncthreads();
        for (int e = tid; e < s * s; e += NT) {
            const int a = e / s, c = e % s;
            if (a < c)
                sh.C[a][c] = lw_cell(p.linkage, sh.X[a][c], sh.Y[a][c], sh.ph[c], sh.szi[c], sh.szj[c],
                                     sh.szi[a] + sh.szj[a]);
        }
        lap(ph3);
        const u64 twb = p.timing && tid == 0 ? global_ns() : 0;
        if (!grid_wait(p, epoch, sh))
            return;
        if (p.timing && tid == 0 && last_b) {
            ty.xlast += global_ns() - twb;
            ++ty.nlast;
            ++ty.nlast_b;
            ty.nlast_b_scan += G - 1 - b < sh.nexec;
        }
        lap(ph0);

        // ---- B: the global per-pair minima, then the certified prefix
        if (s > 0) {
            const int a = tid % S;
            u64 ma = kNoKey, mh = kNoKey;
            if (a < s) {
                for (int g = tid / S; g < G; g += NT / S) {
                    const u64 x = LDCG(p.recB + (size_t)g * 2 * kRound + a);
                    const u64 y = LDCG(p.recB + (size_t)g * 2 * kRound + kRound + a);
                    ma = x < ma ? x : ma;
                    mh = y < mh ? y : mh;
                }
            }
#pragma unroll
            for (int o = S; o < 32; o <<= 1) {
                const u64 x = __shfl_xor_sync(kFull, ma, o);
                const u64 y = __shfl_xor_sync(kFull, mh, o);
                ma = x < ma ? x : ma;
                mh = y < mh ? y : mh;
            }
            // lanes below S of every warp hold the warp's minima per pair
            if (lane < S) {
                sh.wam[warp][lane] = ma;
                sh.whm[warp][lane] = mh;
            }
            __syncthreads();
            if (tid < 2 * S) {
                const int a2 = tid % S;
                u64 m = kNoKey;
                for (int w = 0; w < W; ++w) {
                    const u64 x = tid < S ? sh.wam[w][a2] : sh.whm[w][a2];
                    m = x < m ? x : m;
                }
                if (tid < S)
                    sh.gamin[a2] = m;
                else
                    sh.ghmin[a2] = m;
            }
        }
        __syncthreads();
        lap(xs3);
        // certification: P_p is accepted when it is smaller than every cell
        // that merges a < p rewrote, as seen after merge p - 1: for merge a,
        // its published minimum over the other rows, the cells (i_a, i_c) and
        // (i_a, j_c) after merge a alone for the pairs c >= p not merged yet,
        // and (i_a, i_c) after merges a and c for a < c < p.  Warp per row a,
        // lane c: the first term by a suffix minimum over the lanes, the second
        // by an exclusive prefix minimum, so candidate R(a, p) sits in lane p;
        // then warp per p, lane a: the minimum over a < p.  (R is kept in the
        // member-cell table, whose values the round no longer needs.)
        {
            static_assert(sizeof(float) * 2 * S * (2 * S + 1) >= 12 * S * S, "candidates fit the member-cell table");
            u64 *RA = reinterpret_cast<u64 *>(&sh.Dm[0][0]);
            unsigned *Rc = reinterpret_cast<unsigned *>(RA + S * S);
            const Cand none = {kNoKey, 0xffffffffu};
            for (int a = warp; a + 1 < s; a += W) {  // (row s - 1 rewrites nothing a later p sees)
                const int c = lane;
                const bool in = c > a && c < s;
                Cand xy = none, cc = none;
                if (in) {
                    const unsigned ia = (unsigned)sh.pi[a];
                    xy = cell_cand(__float_as_uint(sh.X[a][c]), ia, (unsigned)sh.pi[c]);
                    cand_min(xy, cell_cand(__float_as_uint(sh.Y[a][c]), ia, (unsigned)sh.pj[c]));
                    cc = cell_cand(__float_as_uint(sh.C[a][c]), ia, (unsigned)sh.pi[c]);
                }
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    Cand y, z;
                    y.A = __shfl_down_sync(kFull, xy.A, d);
                    y.c = __shfl_down_sync(kFull, xy.c, d);
                    z.A = __shfl_up_sync(kFull, cc.A, d);
                    z.c = __shfl_up_sync(kFull, cc.c, d);
                    if (lane + d < 32)
                        cand_min(xy, y);
                    if (lane >= d)
                        cand_min(cc, z);
                }
                Cand e;
                e.A = __shfl_up_sync(kFull, cc.A, 1);
                e.c = __shfl_up_sync(kFull, cc.c, 1);
                if (in) {
                    cand_min(xy, lane >= 1 ? e : none);
                    const u64 g = sh.gamin[a];
                    if (g != kNoKey)
                        cand_min(xy, cell_cand((unsigned)(g >> 32), (unsigned)sh.pi[a], (unsigned)g));
                    RA[a * S + c] = xy.A;
                    Rc[a * S + c] = xy.c;
                }
            }
            __syncthreads();
            for (int pp = 1 + warp; pp < s; pp += W) {
                Cand M = none;
                if (lane < pp) {
                    M.A = RA[lane * S + pp];
                    M.c = Rc[lane * S + pp];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    Cand y;
                    y.A = __shfl_xor_sync(kFull, M.A, o);
                    y.c = __shfl_xor_sync(kFull, M.c, o);
                    cand_min(M, y);
                }
                if (lane == 0) {
                    const u64 PA = ((u64)__float_as_uint(sh.ph[pp]) << 32) | (unsigned)sh.pi[pp];
                    const unsigned Pc = (unsigned)sh.pj[pp];
                    sh.okp[pp] = PA < M.A || (PA == M.A && Pc < M.c);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int L = s;
            for (int pp = 1; pp < s; ++pp) {
                if (!sh.okp[pp]) {
                    L = pp;
                    break;
                }
            }
            sh.nacc = L;
            sh.ninst = 0;
        }
        __syncthreads();
        const int L = sh.nacc;
        lap(xs4);

        // ---- bookkeeping of the L merges
        if (b == 0) {
            if (tid < L) {
                STCG(p.merges + 2 * (t + tid), (int32_t)sh.pi[tid]);
                STCG(p.merges + 2 * (t + tid) + 1, (int32_t)sh.pj[tid]);
                STCG(p.heights + t + tid, sh.ph[tid]);
                STCG(p.size_g + sh.pi[tid], sh.szi[tid] + sh.szj[tid]);
            }
            for (int e = tid; e < L * L; e += NT) {
                const int a = e / L, c = e % L;
                if (a < c) {
                    if (p.full) {
                        // merge c, the later one, rewrites row i_c; i_a's log at merge c
                        STCG(p.D + (long long)sh.pi[c] * p.pitch + sh.pi[a], sh.C[a][c]);
                        STCG(p.TL + (long long)sh.pi[a] * p.pitch + t + c, sh.C[a][c]);
                    } else {
                        STCG(p.D + pair_idx(sh.pi[a], sh.pi[c], n), sh.C[a][c]);
                    }
                }
            }
            // each pair a < c stands for three updates of the step-by-step
            // order: merge a rewrites (i_a, i_c) and (i_a, j_c), merge c (i_c, i_a)
            if (tid == 0)
                st_updates += 3LL * L * (L - 1) / 2;
        }
        if (tid < L) {
            const int j = sh.pj[tid];
            atomicAnd(&bitmap[j >> 5], ~(1u << (j & 31)));  // Section 4 step 2: slot j retires
            // row-log layout: merge t + tid rewrites row i (every CTA writes the
            // same value, so each one sees the new stamps in its own rescans)
            if (p.full) {
                STCG(p.stamp + sh.pi[tid], (int)(t + tid));
                // the members' earlier merges are no longer the latest; this one is
                const int si = sh.si[tid], sj = sh.sj[tid];
                if (si >= 0)
                    atomicAnd(&vpos[si >> 5], ~(1u << (si & 31)));
                if (sj >= 0)
                    atomicAnd(&vpos[sj >> 5], ~(1u << (sj & 31)));
                const long long q = t + tid;
                atomicOr(&vpos[q >> 5], 1u << (q & 31));
            }
        }
        if (tid >= 2 * L && tid < 2 * s) {
            const long long m = (tid & 1) ? sh.pj[tid >> 1] : sh.pi[tid >> 1];
            if (owner_of(m) == b)
                mflag[slot_of(m)] = 0;  // proposed but not merged this round
        }
        if (tid < L) {
            const int a = tid;
            const long long ja = sh.pj[a];
            if (owner_of(ja) == b) {
                const int l = slot_of(ja);
                ccnt[l] = 0;
                cB[l] = kNoKey;
                pend_t[l] = -1;
            }
            const long long ia = sh.pi[a];
            if (G == 1) {
                // a job's only CTA sees every write after pass 2: it rescans
                // the survivor row then
                const int l = slot_of(ia);
                ccnt[l] = 0;
                cB[l] = kNoKey;
                rsize[l] = sh.szi[a] + sh.szj[a];
                pend_t[l] = -1;
                rlist[atomicAdd(&sh.nresc, 1)] = l;
            } else if (owner_of(ia) == b) {
                // the survivor's cache: its smallest new cell outside the chain
                // and, below it, the new cells to chain members
                const int l = slot_of(ia);
                rstamp[l] = (int)(t + a);
                const u64 m = sh.ghmin[a];
                u64 M[K];
#pragma unroll
                for (int q = 0; q < K; ++q)
                    M[q] = kNoKey;
                int ncand = 0;
                for (int c = 0; c < s; ++c) {
                    if (c == a)
                        continue;
                    u64 x0 = kNoKey, x1 = kNoKey;
                    if (c < L) {
                        if (sh.pi[c] > ia)
                            x0 = make_key(a < c ? sh.C[a][c] : sh.C[c][a], (unsigned)sh.pi[c]);
                    } else {
                        if (sh.pi[c] > ia)
                            x0 = make_key(sh.X[a][c], (unsigned)sh.pi[c]);
                        if (sh.pj[c] > ia)
                            x1 = make_key(sh.Y[a][c], (unsigned)sh.pj[c]);
                    }
                    if (x0 != kNoKey && x0 < m) {
                        list_insert(M, x0);
                        ++ncand;
                    }
                    if (x1 != kNoKey && x1 < m) {
                        list_insert(M, x1);
                        ++ncand;
                    }
                }
                int c;
                u64 B;
                if (m != kNoKey) {
                    list_insert(M, m);
                    c = list_count(M);
                    B = M[c - 1];
                } else {
                    c = list_count(M);
                    B = ncand > K ? M[K - 1] : kNoKey;
                }
                cache_store(l, M);
                ccnt[l] = c;
                cB[l] = B;
                rsize[l] = sh.szi[a] + sh.szj[a];
                pend_t[l] = -1;
                // a survivor holds little more than its smallest cell: ask for
                // its row now (other rows wait until their cache empties)
                if (c <= kSurvivorRefillAt && B != kNoKey)
                    request(l, r);
            }
        }
        __syncthreads();
        lap(xs5);

        // ---- pass 2: apply the L merges to every live k outside them (in a
        // round without merges it only renews refill requests that the
        // per-round cap turned away: a row waiting for one may hold every
        // later round up)
        {
            for (int l0 = 0; l0 < R; l0 += NT) {
                const int l = l0 + tid;
                bool ok = false;
                long long k = 0;
                int nk = 1;
                if (l < R) {
                    k = row_of(l);
                    ok = k < n && live(bitmap, k) && !mflag[l];
                    if (ok)
                        nk = rsize[l];
                }
                if (!ok)
                    continue;
                // rows outside the chain kept their pass-1 values; rows of
                // pairs the round did not merge, and rows past the first
                // chunk, compute them now
                const long long bk = row_base(p, k);
                const bool full = p.full;
                const int sk = full ? rstamp[l] : 0;
                u64 Cc[K];
                cache_load(Cc, l);
                int c = ccnt[l];
                u64 B = cB[l];
                // merge a gave row k the new cell v = D(k, i_a + j_a): store it
                // and keep the cache
                auto apply = [&](int a, float v) {
                    const long long ia = sh.pi[a], ja = sh.pj[a];
                    if (full) {
                        // row i_a is rewritten whole; row k keeps its stale copy
                        // and the new value goes to k's log at this merge
                        STCG(p.D + sh.bi[a] + k, v);
                        STCG(p.TL + bk + t + a, v);
                    } else {
                        STCG(p.D + (k > ia ? sh.bi[a] + k : bk + ia), v);
                    }
                    ++st_updates;
                    if (k < ja) {
                        // row k loses column j; if k < i its cell (k, i) changed as well
                        bool drop = false;
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            const long long col = (long long)(unsigned)Cc[q];
                            if (Cc[q] != kNoKey && (col == ja || (k < ia && col == ia))) {
                                Cc[q] = kNoKey;
                                drop = true;
                            }
                        }
                        if (drop) {
                            close_holes(Cc);
                            c = list_count(Cc);
                        }
                        if (k < ia) {
                            const u64 x = make_key(v, (unsigned)ia);
                            if (x <= B) {
                                list_insert(Cc, x);
                                if (c == K)
                                    B = Cc[K - 1];
                                else
                                    ++c;
                            }
                        }
                    }
                };
                if constexpr (S > PG) {
                    if (l0 == 0 && okf[tid]) {
                        const float *kr = kvs + (size_t)tid * KVP;
#pragma unroll 1
                        for (int a = 0; a < L; ++a)
                            apply(a, kr[a]);
                    } else {
#pragma unroll 1
                        for (int a0 = 0; a0 < L; a0 += PC) {
                            float va[PC], vb[PC];
#pragma unroll
                            for (int u = 0; u < PC; ++u) {
                                const int a = a0 + u;
                                va[u] = 0.0f;
                                vb[u] = 0.0f;
                                if (a < L) {
                                    if (full) {
                                        va[u] = LDCG(sh.si[a] >= sk ? p.D + sh.bi[a] + k : p.TL + sh.bi[a] + sk);
                                        vb[u] = LDCG(sh.sj[a] >= sk ? p.D + sh.bj[a] + k : p.TL + sh.bj[a] + sk);
                                    } else {
                                        const long long i = sh.pi[a], j = sh.pj[a];
                                        va[u] = LDCG(p.D + (k > i ? sh.bi[a] + k : bk + i));
                                        vb[u] = LDCG(p.D + (k > j ? sh.bj[a] + k : bk + j));
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < PC; ++u) {
                                const int a = a0 + u;
                                if (a < L)
                                    apply(a, lw_cell(p.linkage, va[u], vb[u], sh.ph[a], sh.szi[a], sh.szj[a], nk));
                            }
                        }
                    }
                } else {
                    const bool have = l0 == 0 && kok;
#pragma unroll
                    for (int a0 = 0; a0 < S; a0 += PG) {
                        if (a0 >= L)
                            break;
                        float va[PG], vb[PG];
#pragma unroll
                        for (int u = 0; u < PG; ++u) {
                            const int a = a0 + u;
                            va[u] = 0.0f;
                            vb[u] = 0.0f;
                            if (!have && a < L) {
                                const long long i = sh.pi[a], j = sh.pj[a];
                                va[u] = LDCG(p.D + (k > i ? sh.bi[a] + k : bk + i));
                                vb[u] = LDCG(p.D + (k > j ? sh.bj[a] + k : bk + j));
                            }
                        }
#pragma unroll
                        for (int u = 0; u < PG; ++u) {
                            const int a = a0 + u;
                            if (a >= L)
                                break;
                            apply(a, have ? kv[KV_REG ? a : 0]
                                          : lw_cell(p.linkage, va[u], vb[u], sh.ph[a], sh.szi[a], sh.szj[a], nk));
                        }
                    }
                }
                cache_store(l, Cc);
                ccnt[l] = c;
                cB[l] = B;
                if (G == 1) {
                    // one CTA: no one else to ask, refill right after this pass
                    if (c <= kRefillAt && B != kNoKey)
                        rlist[atomicAdd(&sh.nresc, 1)] = l;
                } else if (c == 0 && B != kNoKey && (unsigned)(B >> 32) <= sh.front) {
                    // live cells remain, none is cached, and the bound sits at
                    // the front of the merges: its bare stop mark would hold
                    // the next rounds up until a refill lands, so rescan now
                    rlist[atomicAdd(&sh.nresc, 1)] = l;
                    pend_t[l] = -1;
                } else if (c <= kRefillAt && B != kNoKey && pend_t[l] < 0) {
                    // (a cache that holds every live cell of its row needs no refill)
                    request(l, r);
                }
            }
        }
        __syncthreads();
        lap(xs6);
        // ---- rows whose cache emptied (one-CTA job: also survivors and rows
        // running low, a warp each)
        if (G == 1) {
            const int nresc = sh.nresc;
            for (int q = warp; q < nresc; q += W) {
                const int l = rlist[q];
                u64 top[K];
                warp_row_refresh(p, row_of(l), bitmap, top, st_resc_cells);
                if (lane == 0) {
                    cache_store(l, top);
                    const int c = list_count(top);
                    ccnt[l] = c;
                    cB[l] = c == K ? top[K - 1] : kNoKey;
                }
            }
            if (tid == 0)
                ty.rescans += nresc;
            if (nresc > 0)
                __syncthreads();
        } else {
            const int nresc = sh.nresc;
            for (int q = 0; q < nresc; ++q) {
                const int l = rlist[q];
                if (p.full)
                    block_row_topk_log(p, row_of(l), bitmap, vpos, newer, sh, t, L, st_resc_cells);
                else
                    block_row_topk(p, row_of(l), bitmap, sh, st_resc_cells);
                if (tid == 0) {
                    cache_store(l, sh.tko);
                    const int c = list_count(sh.tko);
                    ccnt[l] = c;
                    cB[l] = c == K ? sh.tko[K - 1] : kNoKey;
                }
            }
            if (tid == 0)
                ty.rescans += nresc;
            if (nresc > 0)
                __syncthreads();  // the rescanned caches (written by thread 0) before anyone reads them
        }
        if (tid < 2 * L) {
            const long long m = (tid & 1) ? sh.pj[tid >> 1] : sh.pi[tid >> 1];
            if (owner_of(m) == b)
                mflag[slot_of(m)] = 0;
        }
        lap(xs7);
        if (tid < L) {
            sh.ppi[tid] = sh.pi[tid];
            sh.ppj[tid] = sh.pj[tid];
        }
        if (tid == 0) {
            sh.nprev = L;
            sh.nresc = 0;
            ++ty.rounds;
            ty.idle += L == 0;
        }
        t += L;
        if (t >= n - 1)
            break;  // that was the last merge
        publish(r + 1);
        lap(ph5);
        bool last_a = false;
        grid_arrive(p, epoch, p.timing ? &last_a : nullptr);
        const u64 twa = p.timing && tid == 0 ? global_ns() : 0;
        if (!grid_wait(p, epoch, sh))
            return;
        if (p.timing && tid == 0 && last_a) {
            ty.xlast += global_ns() - twa;
            ++ty.nlast;
            ty.nlast_a_scan += G - 1 - b < sh.nexec;
        }
        lap(ph0);
    }

    if (p.stats) {
        u64 *St = reinterpret_cast<u64 *>(p.stats);
        atomicAdd(St + 2, (u64)st_updates);
        atomicAdd(St + 5, (u64)st_fill_cells);
        atomicAdd(St + 15, (u64)st_resc_cells);
        if (tid == 32) {
            atomicAdd(St + 6, (u64)ty.installs);
            if (b == 0)
                St[4] = (u64)ty.fills;  // every CTA read the same request lists
            if (p.timing) {
                atomicAdd(St + 24, ty.xscan[0]);
                atomicAdd(St + 25, ty.xscan[1]);
            }
        }
        if (tid == 0) {
            atomicAdd(St + 14, (u64)ty.rescans);
            if (b == 0) {
                St[0] = (u64)ty.rounds;
                St[1] = (u64)ty.idle;
                St[7] = (u64)ty.walk;
                St[3] = (u64)G;
            }
            if (p.timing) {
                ph1 += xs0 + xs1 + xs2;
                ph4 += xs3 + xs4 + xs5;
                ph5 += xs6 + xs7;
                for (int q = 0; q < 6; ++q)
                    atomicAdd(St + 8 + q, ty.ph[q]);
                for (int q = 0; q < 8; ++q)
                    atomicAdd(St + 16 + q, ty.xs[q]);
                atomicAdd(St + 26, ty.xwalk);
                atomicAdd(St + 27, ty.xlast);
                atomicAdd(St + 28, (u64)ty.nlast);
                atomicAdd(St + 29, (u64)ty.nlast_b);
                atomicAdd(St + 30, (u64)ty.nlast_b_scan);
                atomicAdd(St + 31, (u64)ty.nlast_a_scan);
                if (b == 0)
                    St[32] = (u64)ty.nlast;
            }
        }
    }
}

template <int NT, int MINB, int PUB>
__global__ void __launch_bounds__(NT, MINB) merge_kernel(MergeParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<NT, round_of(PUB)> sh;
    merge_job<NT, PUB>(p, blockIdx.x, smem_raw, sh);
}

// Many independent jobs in one persistent launch: each CTA takes the next job
// from a queue (atomicAdd on a counter) and runs all its merges alone (a
// one-CTA job needs no grid barrier), then takes another, until the queue is
// empty.  CTA c keeps its scratch in workspace slot c.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) batch_kernel(BatchParams bp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<NT, kRoundOne> sh;
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
        p.TL = nullptr;
        p.stamp = nullptr;
        p.full = 0;
        p.n = J.n;
        p.pitch = J.n;
        p.linkage = J.linkage;
        p.G = 1;
        p.aligned16 = ((uintptr_t)J.D & 15u) == 0;
        p.merges = J.merges;
        p.heights = J.heights;
        bind_workspace(p, ws, L);
        check_range(p, J.D, (unsigned long long)J.n * (unsigned long long)(J.n - 1) / 2 * sizeof(float));
        check_range(p, J.merges, 8ull * (unsigned long long)(J.n > 1 ? J.n - 1 : 0));
        check_range(p, J.heights, 4ull * (unsigned long long)(J.n > 1 ? J.n - 1 : 0));
        p.stats = nullptr;
        p.timeout_ns = bp.timeout_ns;
        p.skip_arrive_cta = -1;
        p.timing = 0;
        // the slot keeps the previous job's words: clear the ones that must start at zero
        for (size_t q = threadIdx.x; q < (L.total - L.zero) / 4; q += NT)
            reinterpret_cast<int *>(ws + L.zero)[q] = 0;
        __syncthreads();
        if (J.n > 1)
            merge_job<NT, kPubOne>(p, 0, smem_raw, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            bp.job_status[jb] = J.n > 1 ? LDCG(p.status) : 0;
            merges_done += J.n > 1 ? J.n - 1 : 0;
        }
    }
    if (threadIdx.x == 0 && bp.merges_done)
        atomicAdd(reinterpret_cast<unsigned long long *>(bp.merges_done), (unsigned long long)merges_done);
}

// The symmetric matrix from the packed triangle, one 32 x 32 tile of the
// upper triangle per CTA (32 x 8 threads): the tile is read row by row and
// written both as it is and transposed through shared memory, so every
// global access of a warp is 32 consecutive words.
__global__ void __launch_bounds__(256) expand_kernel(const float *__restrict__ P, float *__restrict__ F,
                                                     long long n, long long pitch, int *status)
{
    __shared__ float tile[32][33];
    const long long tr = blockIdx.y, tc = blockIdx.x;
    if (tr > tc)
        return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    int bad = 0;
    for (int yy = ty; yy < 32; yy += 8) {
        const long long r = tr * 32 + yy, c = tc * 32 + tx;
        float v = 0.0f;
        if (c > r && c < n) {
            v = __ldg(P + tri_off(r, n) + (c - r - 1));
            const unsigned u = __float_as_uint(v);
            if (u == 0x80000000u)
                v = 0.0f;  // -0 reads as +0 from here on
            else if (u > 0x7f7fffffu)
                bad = 1;   // NaN, infinite or negative
            F[r * pitch + c] = v;
        }
        tile[yy][tx] = v;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const long long c = tc * 32 + yy, r = tr * 32 + tx;
        if (c > r && c < n)
            F[c * pitch + r] = tile[tx][yy];
    }
    if (bad)
        atomicCAS(status, 0, kErrInput);
}

}  // namespace

cudaError_t launch_expand(const float *packed, float *full, long long n, long long pitch, int *status,
                          cudaStream_t stream)
{
    const long long nb = (n + 31) / 32;
    if (nb > 65535)
        return cudaErrorInvalidValue;
    expand_kernel<<<dim3((unsigned)nb, (unsigned)nb), dim3(32, 8), 0, stream>>>(packed, full, n, pitch, status);
    return cudaGetLastError();
}

size_t merge_smem_bytes(long long n, int G, int nt)
{
    const long long nb = (n + kRowBlock - 1) / kRowBlock;
    const long long Rmax = ((nb + G - 1) / G) * kRowBlock;
    const long long nwords = (n + 31) / 32;
    // bitmap; published entries (keys, column words); per
    // slot: K keys, bound, size, count, refill round and position, rescan
    // list entry, stamp, chain flag; pass-1 values of one chunk of rows (one
    // float per pair) and their flags
    const long long pub = G == 1 ? kPubOne : kPub;
    const long long S = round_of((int)pub);
    const long long chunk = Rmax < nt ? Rmax : nt;
    const long long logbits = G > 1 ? (2 * nwords * 4 + 15) & ~15LL : 0;
    return (size_t)(((nwords * 4 + 15) & ~15LL) + logbits + (long long)G * pub * 12 +
                    (S > 16 ? chunk * (S + 1) * 4 : 0) +
                    ((Rmax * (8 * K + 8 + 4 * 6 + 1) + nt + 15) & ~15LL));
}

namespace {

// The kernel instantiations: CTA size nt and the CTAs per SM its registers allow.
// A one-CTA job publishes more entries per round (nothing else is read).
const void *merge_fn(int nt, int G)
{
    if (G == 1) {
        switch (nt) {
        case 128: return (const void *)merge_kernel<128, 4, kPubOne>;
        case 256: return (const void *)merge_kernel<256, 2, kPubOne>;
        default: return (const void *)merge_kernel<512, 1, kPubOne>;
        }
    }
    switch (nt) {
    case 128: return (const void *)merge_kernel<128, 4, kPub>;
    case 256: return (const void *)merge_kernel<256, 2, kPub>;
    default: return (const void *)merge_kernel<512, 1, kPub>;
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

size_t static_smem(int nt, int G)
{
    if (G == 1) {
        switch (nt) {
        case 128: return sizeof(Shared<128, kRoundOne>);
        case 256: return sizeof(Shared<256, kRoundOne>);
        default: return sizeof(Shared<512, kRoundOne>);
        }
    }
    switch (nt) {
    case 128: return sizeof(Shared<128, kRound>);
    case 256: return sizeof(Shared<256, kRound>);
    default: return sizeof(Shared<512, kRound>);
    }
}

int fit_per_sm(const void *fn, int nt, int G, size_t smem)
{
    int dev = 0, limit = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    if (smem + static_smem(nt, G) > (size_t)limit)
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
    return fit_per_sm(merge_fn(nt, G), nt, G, merge_smem_bytes(n, G, nt)) >= 1;
}

int batch_ctas_per_sm(long long n_max, int nt)
{
    return fit_per_sm(batch_fn(nt), nt, 1, merge_smem_bytes(n_max, 1, nt));
}

cudaError_t launch_batch(const BatchParams &bp, int grid, int nt, cudaStream_t stream)
{
    // batch_ctas_per_sm(bp.n_max, nt) has set the kernel's shared-memory limit
    // (this launch may be recorded into a graph, where no attribute is set)
    const size_t smem = merge_smem_bytes(bp.n_max, 1, nt);
    BatchParams q = bp;
    void *args[] = {&q};
    return cudaLaunchKernel(batch_fn(nt), dim3(grid), dim3(nt), args, smem, stream);
}

cudaError_t launch_merge(const MergeParams &p, int nt, cudaStream_t stream)
{
    const size_t smem = merge_smem_bytes(p.n, p.G, nt);
    const void *fn = merge_fn(nt, p.G);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    MergeParams q = p;
    void *args[] = {&q};
    return cudaLaunchCooperativeKernel(fn, dim3(p.G), dim3(nt), args, smem, stream);
}

}  // namespace lw
