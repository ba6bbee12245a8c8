// lw_merge.cu -- the persistent cooperative Lance-Williams merge kernel.
//
// One launch performs all n - 1 merges of one matrix (Section 4, "Lance-William
// Algorithm", steps 1-4) so that no merge pays a kernel launch.  The paper
// spreads the packed upper triangle over MPI processes and exchanges local
// minima and (i, j, distance) triples by messages (Section 5.3 steps 1-6b); on
// one GB300 the whole triangle sits in HBM, so the "processors" become CTAs,
// the broadcast of local minima becomes a 32-byte record per CTA read after
// one grid barrier, and the triple exchange disappears: every CTA addresses
// row and column i and j directly.
//
// Work split.  Rows are dealt to CTAs in blocks of 32 consecutive rows,
// round-robin (block q -> CTA q mod G).  The CTA that owns row k
//   - keeps row k's cached minimum key (smallest (value, column) over live
//     columns c > k) in shared memory,
//   - applies the update of Section 4 step 3 for k at every merge: reads
//     D(k,i), D(k,j), writes D(k,i+j) into D(k,i),
//   - repairs row k's cached minimum, rescanning row k when the cached
//     minimum pointed at i or j and the new value is larger.
// The survivor row i is rewritten by every CTA (one cell per owned k > i);
// each CTA folds its part of row i into the candidate it publishes, and the
// owner of i reassembles row i's minimum from all records after the barrier.
//
// One grid barrier per merge:
//   [barrier] read G records -> global minimum (value, i, j) -> emit step
//   -> update + repairs + rescans -> publish record -> [barrier]
//
// Exact arithmetic: every product and sum of the update uses __fmul_rn /
// __fadd_rn / __fsub_rn (never contracted into FMA), the coefficient
// divisions __fdiv_rn; the four terms are added left to right.  The minimum
// is the smallest (value, row, column); values are non-negative floats, so
// their bit patterns order like the values and a 64-bit integer compare of
// (bits << 32 | index) gives the lexicographic order.
//
// Memory model.  L1 is not coherent across SMs, so every load of data that
// another CTA may have written (matrix cells, keys, records, sizes) is an
// L2 load (ld.global.cg) and every store bypasses L1 (st.global.cg).  The
// barrier is the cooperative-groups pattern: __syncthreads, one thread
// fences, arrives with a release add and spins with acquire loads.  Each spin
// is bounded by a wall-clock limit after which the kernel records
// LW_ERR_TIMEOUT and returns.

#include "lw_internal.h"

#include <cstdint>

namespace lw {
namespace {

typedef unsigned long long u64;

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

// Candidate of the global minimum plus the survivor-row partial minimum.
struct Cand {
    u64 A;       // (bits(v) << 32) | row
    unsigned c;  // column
    u64 K;       // (bits(v) << 32) | column, survivor row partial
};

__device__ __forceinline__ void cand_min(Cand &x, const Cand &y)
{
    if (y.A < x.A || (y.A == x.A && y.c < x.c)) {
        x.A = y.A;
        x.c = y.c;
    }
    if (y.K < x.K)
        x.K = y.K;
}

__device__ __forceinline__ Cand warp_cand_min(Cand v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Cand o;
        o.A = __shfl_xor_sync(0xffffffffu, v.A, off);
        o.c = __shfl_xor_sync(0xffffffffu, v.c, off);
        o.K = __shfl_xor_sync(0xffffffffu, v.K, off);
        cand_min(v, o);
    }
    return v;
}

__device__ __forceinline__ u64 warp_u64_min(u64 v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        u64 o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    return v;
}

struct Shared {
    Cand red[kWarps + 1];
    u64 kred[kWarps + 1];
    int flag;
    int nresc;
};

__device__ Cand block_cand_min(Cand v, Shared &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_cand_min(v);
    if (lane == 0)
        sh.red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        Cand w = {kNoKey, 0xffffffffu, kNoKey};
        if (lane < kWarps)
            w = sh.red[lane];
        w = warp_cand_min(w);
        if (lane == 0)
            sh.red[kWarps] = w;
    }
    __syncthreads();
    return sh.red[kWarps];
}

__device__ u64 block_u64_min(u64 v, Shared &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_u64_min(v);
    if (lane == 0)
        sh.kred[warp] = v;
    __syncthreads();
    if (warp == 0) {
        u64 w = lane < kWarps ? sh.kred[lane] : kNoKey;
        w = warp_u64_min(w);
        if (lane == 0)
            sh.kred[kWarps] = w;
    }
    __syncthreads();
    return sh.kred[kWarps];
}

// Grid-wide barrier with a bounded wait.  Returns false when the run must
// stop (this CTA gave up waiting, or another CTA flagged an error).
__device__ bool grid_sync(const MergeParams &p, unsigned &epoch, Shared &sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        int st = 0;
        if (p.G > 1) {
            const unsigned target = epoch * (unsigned)p.G;
            __threadfence();
            red_release_add(p.bar, 1u);
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
            __threadfence();
        }
        sh.flag = st;
    }
    __syncthreads();
    return sh.flag == 0;
}

// Row r of the packed triangle that holds flat index q (0 <= q < n(n-1)/2).
__device__ long long row_of_flat(long long q, long long n)
{
    const double b = 2.0 * (double)n - 1.0;
    double disc = b * b - 8.0 * (double)q;
    if (disc < 0.0)
        disc = 0.0;
    long long r = (long long)((b - sqrt(disc)) * 0.5);
    if (r < 0)
        r = 0;
    if (r > n - 2)
        r = n - 2;
    while (r < n - 2 && tri_off(r + 1, n) <= q)
        ++r;
    while (r > 0 && tri_off(r, n) > q)
        --r;
    return r;
}

// Checks one input cell (finite and >= 0), canonicalises -0, returns its key.
__device__ __forceinline__ u64 init_cell(float v, long long q, unsigned c, const MergeParams &p,
                                         int &bad)
{
    const unsigned bits = __float_as_uint(v);
    if (!(v >= 0.0f) || bits == 0x7f800000u) {
        bad = 1;
        return kNoKey;
    }
    if (bits == 0x80000000u) {
        __stcg(p.D + q, 0.0f);
        return (u64)c;
    }
    return ((u64)bits << 32) | (u64)c;
}

// Phase 0: validate every cell and build the row-minimum keys.  The packed
// triangle is split into equal, 512-cell-aligned chunks, one per warp of the
// grid (the paper's even split of the non-blank cells, Section 5.2); a warp walks its
// chunk with 128-bit loads and flushes each row's minimum with atomicMin.
__device__ void initial_scan(const MergeParams &p)
{
    const long long n = p.n;
    const long long N = n * (n - 1) / 2;
    const int lane = threadIdx.x & 31;
    const long long W = (long long)p.G * kWarps;
    const long long w = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    long long S = (N + W - 1) / W;
    S = (S + 511) & ~511LL;
    const long long lo = w * S;
    const long long hi = lo + S < N ? lo + S : N;
    if (lo >= hi)
        return;
    long long r = row_of_flat(lo, n);
    long long rs = tri_off(r, n), re = tri_off(r + 1, n);
    u64 run = kNoKey;
    int bad = 0;
    for (long long s = lo; s < hi; s += 512) {
        float v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long q = s + 128 * u + 4 * lane;
            if (p.aligned16 && q + 4 <= hi) {
                const float4 x = __ldcg(reinterpret_cast<const float4 *>(p.D + q));
                v[u][0] = x.x; v[u][1] = x.y; v[u][2] = x.z; v[u][3] = x.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    v[u][e] = q + e < hi ? __ldcg(p.D + q + e) : 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long q0 = s + 128 * u;
            if (q0 >= hi)
                break;
            const long long span_end = q0 + 128 < hi ? q0 + 128 : hi;
            while (true) {
                const long long seg_end = re < span_end ? re : span_end;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long long q = q0 + 4 * lane + e;
                    if (q >= rs && q < seg_end) {
                        const u64 k = init_cell(v[u][e], q, (unsigned)(q - rs + r + 1), p, bad);
                        run = k < run ? k : run;
                    }
                }
                if (seg_end == re) {
                    const u64 m = warp_u64_min(run);
                    if (lane == 0 && m != kNoKey)
                        atomicMin(p.rowkey_g + r, m);
                    run = kNoKey;
                    ++r;
                    rs = re;
                    re = tri_off(r + 1, n);
                    if (rs >= span_end)
                        break;
                } else {
                    break;
                }
            }
        }
    }
    const u64 m = warp_u64_min(run);
    if (lane == 0 && m != kNoKey)
        atomicMin(p.rowkey_g + r, m);
    if (bad)
        atomicCAS(p.status, 0, kErrInput);
}

// Minimum key over the live columns c > k of row k, computed by the whole
// CTA; adds the number of live cells read to `live`.
__device__ u64 rescan_row(const MergeParams &p, long long k, const unsigned *bitmap, Shared &sh,
                          long long &live)
{
    const long long n = p.n;
    const long long start = tri_off(k, n);
    const long long end = start + (n - k - 1);
    const long long base_c = k + 1 - start;  // column of flat index q is q + base_c
    u64 best = kNoKey;
    long long cnt = 0;
    long long a0 = p.aligned16 ? ((start + 3) & ~3LL) : end;
    if (a0 > end)
        a0 = end;
    const long long a1 = a0 + ((end - a0) & ~3LL);
    // scalar head and tail
    for (long long q = start + threadIdx.x; q < a0; q += kThreads) {
        const unsigned c = (unsigned)(q + base_c);
        if ((bitmap[c >> 5] >> (c & 31)) & 1u) {
            const u64 key = make_key(__ldcg(p.D + q), c);
            best = key < best ? key : best;
            ++cnt;
        }
    }
    for (long long q = a1 + threadIdx.x; q < end; q += kThreads) {
        const unsigned c = (unsigned)(q + base_c);
        if ((bitmap[c >> 5] >> (c & 31)) & 1u) {
            const u64 key = make_key(__ldcg(p.D + q), c);
            best = key < best ? key : best;
            ++cnt;
        }
    }
    for (long long q = a0 + 4 * (long long)threadIdx.x; q < a1; q += 4 * kThreads) {
        const float4 x = __ldcg(reinterpret_cast<const float4 *>(p.D + q));
        const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned c = (unsigned)(q + e + base_c);
            if ((bitmap[c >> 5] >> (c & 31)) & 1u) {
                const u64 key = make_key(xv[e], c);
                best = key < best ? key : best;
                ++cnt;
            }
        }
    }
    live += cnt;
    return block_u64_min(best, sh);
}

__global__ void __launch_bounds__(kThreads, 1) merge_kernel(MergeParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared sh;

    const long long n = p.n;
    const int G = p.G;
    const int b = blockIdx.x;
    const int tid = threadIdx.x;
    const long long nb = (n + kRowBlock - 1) / kRowBlock;     // row blocks
    const long long my_blocks = b < nb ? (nb - b + G - 1) / G : 0;
    const int R = (int)(my_blocks * kRowBlock);                // owned row slots
    const long long Rmax = ((nb + G - 1) / G) * kRowBlock;
    const long long nwords = (n + 31) / 32;

    unsigned *bitmap = reinterpret_cast<unsigned *>(smem_raw);
    u64 *rkey = reinterpret_cast<u64 *>(smem_raw + ((nwords * 4 + 15) & ~15LL));
    int *rsize = reinterpret_cast<int *>(rkey + Rmax);
    int *rlist = rsize + Rmax;

    // global row of owned slot l, and (owner, slot) of a global row
    auto row_of = [&](int l) -> long long {
        return (long long)((long long)b + (long long)G * (l >> 5)) * kRowBlock + (l & 31);
    };
    auto owner_of = [&](long long r) -> int { return (int)((r / kRowBlock) % G); };
    auto slot_of = [&](long long r) -> int {
        return (int)(((r / kRowBlock) / G) * kRowBlock + (r & 31));
    };

    // ---- setup
    for (long long w = tid; w < nwords; w += kThreads) {
        const long long lo = w * 32;
        const long long live = n - lo;
        bitmap[w] = live >= 32 ? 0xffffffffu : ((1u << live) - 1u);
    }
    for (int l = tid; l < R; l += kThreads)
        rsize[l] = 1;
    for (long long r = (long long)b * kThreads + tid; r < n; r += (long long)G * kThreads)
        p.size_g[r] = 1;
    if (tid == 0)
        sh.nresc = 0;

    unsigned epoch = 0;
    initial_scan(p);
    if (b == p.skip_arrive_cta)
        return;
    if (!grid_sync(p, epoch, sh))
        return;
    if (tid == 0)
        sh.flag = ld_relaxed_s32(p.status);
    __syncthreads();
    if (sh.flag != 0)
        return;

    for (int l = tid; l < R; l += kThreads) {
        const long long r = row_of(l);
        rkey[l] = r < n ? __ldcg(p.rowkey_g + r) : kNoKey;
    }
    __syncthreads();

    long long st_updates = 0, st_rescan_live = 0, st_rescans = 0;

    // first records: each CTA's smallest row key
    {
        Cand c = {kNoKey, 0xffffffffu, kNoKey};
        for (int l = tid; l < R; l += kThreads) {
            const u64 k = rkey[l];
            if (k != kNoKey) {
                Cand o = {(k & 0xffffffff00000000ull) | (u64)row_of(l), (unsigned)k, kNoKey};
                cand_min(c, o);
            }
        }
        c = block_cand_min(c, sh);
        if (tid == 0) {
            ulonglong2 w0 = make_ulonglong2(c.A, c.K);
            ulonglong2 w1 = make_ulonglong2((u64)c.c, 0ull);
            __stcg(reinterpret_cast<ulonglong2 *>(p.recs + b), w0);
            __stcg(reinterpret_cast<ulonglong2 *>(p.recs + b) + 1, w1);
        }
    }
    if (!grid_sync(p, epoch, sh))
        return;

    int par = 0;
    long long prev_i = -1;
    int carried = 0;  // size of the cluster in slot prev_i after its merge

    for (long long t = 0; t < n - 1; ++t) {
        // ---- Section 4 step 1: global minimum from the G records
        Cand mine = {kNoKey, 0xffffffffu, kNoKey};
        if (tid < G) {
            const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(p.recs + par * G + tid);
            const ulonglong2 w0 = __ldcg(src);
            const ulonglong2 w1 = __ldcg(src + 1);
            mine.A = w0.x;
            mine.K = w0.y;
            mine.c = (unsigned)w1.x;
        }
        const Cand best = block_cand_min(mine, sh);
        const long long i = (long long)(best.A & 0xffffffffull);
        const long long j = (long long)best.c;
        const float h = __uint_as_float((unsigned)(best.A >> 32));
        // every CTA read the same records, so every CTA takes this exit together
        if (i >= n || j >= n || i >= j) {
            if (tid == 0)
                atomicCAS(p.status, 0, kErrInternal);
            return;
        }

        if (tid == 0) {
            if (prev_i >= 0 && owner_of(prev_i) == b) {
                rkey[slot_of(prev_i)] = best.K;        // survivor row reassembled
                __stcg(p.size_g + prev_i, carried);    // deferred size write
            }
            if (b == 0) {
                p.merges[2 * t] = (int32_t)i;
                p.merges[2 * t + 1] = (int32_t)j;
                p.heights[t] = h;
            }
            bitmap[j >> 5] &= ~(1u << (j & 31));       // step 2: slot j retires
            sh.nresc = 0;
        }
        int ni = 1, nj = 1;
        if (p.linkage >= 2) {
            ni = (i == prev_i) ? carried : __ldcg(p.size_g + i);
            nj = (j == prev_i) ? carried : __ldcg(p.size_g + j);
        }
        __syncthreads();

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
        u64 islice = kNoKey;
        for (int l = tid; l < R; l += kThreads) {
            const long long k = row_of(l);
            if (k >= n || k == i || k == j)
                continue;
            if (!((bitmap[k >> 5] >> (k & 31)) & 1u))
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
            if (k < i) {
                // row k: cell (k,i) changed, cell (k,j) left
                const u64 old = rkey[l];
                const unsigned arg = (unsigned)old;
                const u64 nkey = make_key(s, (unsigned)i);
                if (arg == (unsigned)i || arg == (unsigned)j) {
                    if (nkey <= old) {
                        rkey[l] = nkey;
                    } else {
                        rkey[l] = kNoKey;
                        rlist[atomicAdd(&sh.nresc, 1)] = l;
                    }
                } else if (nkey < old) {
                    rkey[l] = nkey;
                }
            } else {
                // cell (i,k) belongs to the survivor row i
                const u64 key = make_key(s, (unsigned)k);
                islice = key < islice ? key : islice;
                if (k < j && (unsigned)rkey[l] == (unsigned)j) {
                    rkey[l] = kNoKey;
                    rlist[atomicAdd(&sh.nresc, 1)] = l;
                }
            }
        }
        if (tid == 0) {
            if (owner_of(j) == b)
                rkey[slot_of(j)] = kNoKey;
            if (owner_of(i) == b) {
                rkey[slot_of(i)] = kNoKey;  // reassembled from the records next merge
                rsize[slot_of(i)] = ni + nj;
            }
        }
        __syncthreads();

        // ---- cache repair: rows that lost their minimum
        const int nresc = sh.nresc;
        for (int q = 0; q < nresc; ++q) {
            const int l = rlist[q];
            const u64 m = rescan_row(p, row_of(l), bitmap, sh, st_rescan_live);
            if (tid == 0)
                rkey[l] = m;
        }
        if (tid == 0)
            st_rescans += nresc;
        __syncthreads();

        // ---- publish this CTA's candidate and its part of the survivor row
        Cand c = {kNoKey, 0xffffffffu, islice};
        if (islice != kNoKey) {
            c.A = (islice & 0xffffffff00000000ull) | (u64)i;
            c.c = (unsigned)islice;
        }
        for (int l = tid; l < R; l += kThreads) {
            const u64 k = rkey[l];
            if (k != kNoKey) {
                Cand o = {(k & 0xffffffff00000000ull) | (u64)row_of(l), (unsigned)k, kNoKey};
                cand_min(c, o);
            }
        }
        c = block_cand_min(c, sh);
        par ^= 1;
        if (tid == 0) {
            ulonglong2 w0 = make_ulonglong2(c.A, c.K);
            ulonglong2 w1 = make_ulonglong2((u64)c.c, 0ull);
            __stcg(reinterpret_cast<ulonglong2 *>(p.recs + par * G + b), w0);
            __stcg(reinterpret_cast<ulonglong2 *>(p.recs + par * G + b) + 1, w1);
        }
        prev_i = i;
        carried = ni + nj;
        if (t + 2 < n && !grid_sync(p, epoch, sh))
            return;
    }

    if (p.stats) {
        atomicAdd(reinterpret_cast<u64 *>(p.stats + 1), (u64)st_rescan_live);
        atomicAdd(reinterpret_cast<u64 *>(p.stats + 2), (u64)st_updates);
        if (tid == 0)
            atomicAdd(reinterpret_cast<u64 *>(p.stats + 0), (u64)st_rescans);
        if (b == 0 && tid == 0)
            p.stats[3] = G;
    }
}

}  // namespace

size_t merge_smem_bytes(long long n, int G)
{
    const long long nb = (n + kRowBlock - 1) / kRowBlock;
    const long long Rmax = ((nb + G - 1) / G) * kRowBlock;
    const long long nwords = (n + 31) / 32;
    return (size_t)(((nwords * 4 + 15) & ~15LL) + Rmax * 8 + Rmax * 4 + Rmax * 4);
}

bool merge_config_ok(long long n, int G, int num_sms)
{
    if (G < 1 || G > num_sms)
        return false;
    int dev = 0, limit = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    const size_t smem = merge_smem_bytes(n, G);
    if (smem + sizeof(Shared) > (size_t)limit)
        return false;
    if (cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, merge_kernel, kThreads, smem) !=
        cudaSuccess)
        return false;
    return per_sm >= 1;
}

cudaError_t launch_merge(const MergeParams &p, cudaStream_t stream)
{
    const size_t smem = merge_smem_bytes(p.n, p.G);
    cudaError_t e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    MergeParams q = p;
    void *args[] = {&q};
    return cudaLaunchCooperativeKernel((const void *)merge_kernel, dim3(p.G), dim3(kThreads), args,
                                       smem, stream);
}

}  // namespace lw
