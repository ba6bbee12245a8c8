/*
 * lw_oracle.c -- CPU oracle of the Lance-Williams merge loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded input generators.
 *
 * What it computes (Yarmish, Listowsky, Dexter, "Distributed Lance-William
 * Clustering Algorithm"):
 *   - Section 4, "Lance-William Algorithm": starting from n singleton clusters, each
 *     iteration (1) takes the minimum distance of the matrix and its pair
 *     (i, j), (2) combines i and j into one cluster, (3) recomputes the
 *     distance from every other cluster k to the combined one with
 *         D(k, i+j) = a_i D(k,i) + a_j D(k,j) + b D(i,j) + g |D(k,i) - D(k,j)|,
 *     (4) outputs the current level of the tree.
 *   - Table 1: the coefficients (a_i, a_j, b, g) of its six rows: single,
 *     complete, group average (UPGMA), weighted average (WPGMA), centroid
 *     (UPGMC) and Ward linkage.  Section 5.3 step 6 gives the complete-linkage
 *     form .5 D(k,i) + .5 D(k,j) + .5 |D(k,i) - D(k,j)| the authors used.
 *   - Section 5.1 / Section 5.2: only the upper triangle of the symmetric matrix is
 *     stored; Section 5.3 step 6: the combined cluster keeps row/column i, row and
 *     column j are marked unused.
 *
 * Readings where the paper is silent (the kernel library takes the same ones):
 *   - storage and arithmetic are IEEE FP32, every operation rounded to nearest
 *     even, no fused multiply-add (build with -ffp-contract=off), the four
 *     terms added left to right in the order the formula prints them;
 *   - "For k = 1 to n" performs n - 1 merges (the n-th iteration has no pair);
 *   - ties in the minimum go to the lowest (i, j) in row-major order, i < j;
 *     the survivor keeps slot i and slot j retires;
 *   - group average (and centroid) a_i = fl(n_i / (n_i + n_j)),
 *     a_j = fl(n_j / (n_i + n_j)), each one correctly rounded FP32 division
 *     of exact integer-valued floats; Ward a_i = fl((n_i+n_k)/T),
 *     a_j = fl((n_j+n_k)/T), b = -fl(n_k/T), T = n_i + n_j + n_k;
 *   - centroid b = -fl(float(n_i n_j) / float((n_i + n_j)^2)): the two
 *     integers computed exactly, each converted to FP32 once, one correctly
 *     rounded division, then negated;
 *   - weighted average (0.5, 0.5, 0, 0) whatever the sizes;
 *   - NaN, infinite and negative distances are rejected; -0 becomes +0.
 *
 * Two loops:
 *   lwo_naive  -- the iteration exactly as Section 4 states it, searching the whole
 *                 active upper triangle for the minimum every time: O(n^3).
 *   lwo_cached -- the same iteration with a per-row minimum cache (a key per
 *                 row: the row's smallest (value, column) over active columns
 *                 to its right).  It must reproduce lwo_naive bit for bit;
 *                 OpenMP spreads each step over the host cores.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { LWO_SINGLE = 0, LWO_COMPLETE = 1, LWO_AVERAGE = 2, LWO_WARD = 3, LWO_WEIGHTED = 4, LWO_CENTROID = 5 };
enum { LWO_OK = 0, LWO_BAD_ARG = 1, LWO_BAD_INPUT = 2, LWO_NO_MEMORY = 3 };

/* Flat index of cell (r, c), r < c, of the packed row-major upper triangle. */
static int64_t cell_index(int64_t n, int64_t r, int64_t c)
{
    return r * n - r * (r + 1) / 2 + (c - r - 1);
}

/* Flat index of the unordered pair {a, b}, a != b. */
static int64_t pair_index(int64_t n, int64_t a, int64_t b)
{
    return a < b ? cell_index(n, a, b) : cell_index(n, b, a);
}

static double now_seconds(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

/* Table 1 coefficients for clusters of sizes ni, nj (merged) and nk (other). */
void lwo_coefficients(int linkage, int64_t ni, int64_t nj, int64_t nk, float out[4])
{
    float ai = 0.0f, aj = 0.0f, b = 0.0f, g = 0.0f;
    switch (linkage) {
    case LWO_SINGLE:
        ai = 0.5f; aj = 0.5f; b = 0.0f; g = -0.5f;
        break;
    case LWO_COMPLETE:
        ai = 0.5f; aj = 0.5f; b = 0.0f; g = 0.5f;
        break;
    case LWO_AVERAGE: {
        float sum = (float)(ni + nj);
        ai = (float)ni / sum;
        aj = (float)nj / sum;
        break;
    }
    case LWO_WARD: {
        float T = (float)(ni + nj + nk);
        ai = (float)(ni + nk) / T;
        aj = (float)(nj + nk) / T;
        b = -((float)nk / T);
        break;
    }
    case LWO_WEIGHTED:
        ai = 0.5f; aj = 0.5f;
        break;
    case LWO_CENTROID: {
        /* beta = -n_i n_j / (n_i + n_j)^2: numerator and denominator are exact
         * integers, each converted to float once, then one division */
        float sum = (float)(ni + nj);
        ai = (float)ni / sum;
        aj = (float)nj / sum;
        b = -((float)(ni * nj) / (float)((ni + nj) * (ni + nj)));
        break;
    }
    default:
        break;
    }
    out[0] = ai; out[1] = aj; out[2] = b; out[3] = g;
}

/* The update formula of Section 4 step 3, terms in printed order, left to right. */
static float lw_formula(const float co[4], float dki, float dkj, float dij)
{
    float s = co[0] * dki;
    s = s + co[1] * dkj;
    s = s + co[2] * dij;
    s = s + co[3] * fabsf(dki - dkj);
    return s;
}

float lwo_update(int linkage, float dki, float dkj, float dij, int64_t ni, int64_t nj, int64_t nk)
{
    float co[4];
    lwo_coefficients(linkage, ni, nj, nk, co);
    return lw_formula(co, dki, dkj, dij);
}

/* Rejects NaN, +-inf and negative cells; rewrites -0 as +0.  Returns 1 if bad. */
static int validate(float *D, int64_t cells)
{
    int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
    for (int64_t q = 0; q < cells; ++q) {
        float v = D[q];
        if (!(v >= 0.0f) || isinf(v))
            bad |= 1;
        else if (v == 0.0f)
            D[q] = 0.0f;
    }
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Section 4, literally: full search of the active upper triangle per iteration.  */
/* ------------------------------------------------------------------------- */
int lwo_naive(float *D, int64_t n, int linkage, int32_t *merges, float *heights,
              int64_t *scanned_per_iter)
{
    if (n < 1 || linkage < 0 || linkage > 5 || (n > 1 && (!D || !merges || !heights)))
        return LWO_BAD_ARG;
    if (n == 1)
        return LWO_OK;
    if (validate(D, n * (n - 1) / 2))
        return LWO_BAD_INPUT;

    unsigned char *active = malloc((size_t)n);
    int64_t *size = malloc(sizeof(int64_t) * (size_t)n);
    if (!active || !size) {
        free(active); free(size);
        return LWO_NO_MEMORY;
    }
    for (int64_t r = 0; r < n; ++r) {
        active[r] = 1;
        size[r] = 1;
    }

    for (int64_t t = 0; t + 1 < n; ++t) {
        /* 1. minimum distance over all active pairs; first (lowest (i,j)) wins ties */
        float h = 0.0f;
        int64_t i = -1, j = -1, scanned = 0;
        for (int64_t r = 0; r < n; ++r) {
            if (!active[r])
                continue;
            for (int64_t c = r + 1; c < n; ++c) {
                if (!active[c])
                    continue;
                float v = D[cell_index(n, r, c)];
                ++scanned;
                if (i < 0 || v < h) {
                    h = v; i = r; j = c;
                }
            }
        }
        if (scanned_per_iter)
            scanned_per_iter[t] = scanned;

        /* 3. new distances from every other cluster k to the combined i+j
         *    (coefficients from the sizes before combining) */
        int64_t ni = size[i], nj = size[j];
        for (int64_t k = 0; k < n; ++k) {
            if (!active[k] || k == i || k == j)
                continue;
            float co[4];
            lwo_coefficients(linkage, ni, nj, size[k], co);
            int64_t pi = pair_index(n, k, i);
            D[pi] = lw_formula(co, D[pi], D[pair_index(n, k, j)], h);
        }

        /* 2. combine: slot i holds i+j, slot j is never used again */
        size[i] = ni + nj;
        active[j] = 0;

        /* 4. output this level of the tree */
        merges[2 * t] = (int32_t)i;
        merges[2 * t + 1] = (int32_t)j;
        heights[t] = h;
    }
    free(active);
    free(size);
    return LWO_OK;
}

/* ------------------------------------------------------------------------- */
/* The same iteration with a per-row minimum cache.                           */
/* ------------------------------------------------------------------------- */

#define NO_KEY UINT64_MAX

/* Order key of cell value v in column c: for v >= +0 the unsigned order of
 * (bits(v), c) is the order of (v, c). */
static uint64_t cell_key(float v, int64_t c)
{
    uint32_t bits;
    memcpy(&bits, &v, sizeof bits);
    return ((uint64_t)bits << 32) | (uint64_t)(uint32_t)c;
}

/* Smallest key over the active columns c > r of row r; NO_KEY if none. */
static uint64_t row_minimum(const float *D, int64_t n, const unsigned char *active, int64_t r,
                            int64_t *active_cells)
{
    uint64_t best = NO_KEY;
    const float *row = D + cell_index(n, r, r + 1);
    int64_t cnt = 0;
    for (int64_t c = r + 1; c < n; ++c) {
        if (!active[c])
            continue;
        ++cnt;
        uint64_t k = cell_key(row[c - r - 1], c);
        if (k < best)
            best = k;
    }
    if (active_cells)
        *active_cells = cnt;
    return best;
}

/*
 * stats (nullable, 6 entries): [0] rows rescanned after losing their minimum,
 * [1] active cells read by those rescans, [2] cells updated by the formula,
 * [3] active cells of the rewritten rows i (recomputed minima), [4] merges done,
 * [5] sum over merges of the active cluster count m_t.
 * times (nullable, 2 entries): [0] seconds to validate and build the cache,
 * [1] seconds of the merge loop.
 * max_merges < 0 runs all n - 1 merges; otherwise it stops after that many.
 */
int lwo_cached(float *D, int64_t n, int linkage, int32_t *merges, float *heights,
               int64_t max_merges, int64_t *stats, double *times)
{
    if (n < 1 || linkage < 0 || linkage > 5 || (n > 1 && (!D || !merges || !heights)))
        return LWO_BAD_ARG;
    if (stats)
        memset(stats, 0, 6 * sizeof(int64_t));
    if (n == 1)
        return LWO_OK;
    double t0 = now_seconds();
    if (validate(D, n * (n - 1) / 2))
        return LWO_BAD_INPUT;

    unsigned char *active = malloc((size_t)n);
    unsigned char *rescan = malloc((size_t)n);
    int64_t *size = malloc(sizeof(int64_t) * (size_t)n);
    uint64_t *rowkey = malloc(sizeof(uint64_t) * (size_t)n);
    if (!active || !rescan || !size || !rowkey) {
        free(active); free(rescan); free(size); free(rowkey);
        return LWO_NO_MEMORY;
    }
    for (int64_t r = 0; r < n; ++r) {
        active[r] = 1;
        rescan[r] = 0;
        size[r] = 1;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n; ++r)
        rowkey[r] = row_minimum(D, n, active, r, NULL);
    double t1 = now_seconds();

    int64_t total = n - 1;
    if (max_merges >= 0 && max_merges < total)
        total = max_merges;
    int64_t n_rescans = 0, rescan_cells = 0, updated = 0, rowi_cells = 0, sum_m = 0;

    for (int64_t t = 0; t < total; ++t) {
        /* 1. global minimum: smallest (value, row, column) over the row keys */
        uint64_t best = NO_KEY;
#pragma omp parallel for reduction(min : best) schedule(static)
        for (int64_t r = 0; r < n; ++r) {
            if (active[r] && rowkey[r] != NO_KEY) {
                uint64_t cand = (rowkey[r] & 0xffffffff00000000ull) | (uint64_t)r;
                if (cand < best)
                    best = cand;
            }
        }
        int64_t i = (int64_t)(best & 0xffffffffu);
        int64_t j = (int64_t)(rowkey[i] & 0xffffffffu);
        uint32_t hb = (uint32_t)(best >> 32);
        float h;
        memcpy(&h, &hb, sizeof h);
        sum_m += n - t;

        /* 3. new distances to the combined cluster, and the cache repairs that
         *    each new value D(k, i) implies for row k */
        int64_t ni = size[i], nj = size[j];
        int64_t upd = 0;
#pragma omp parallel for reduction(+ : upd) schedule(static)
        for (int64_t k = 0; k < n; ++k) {
            if (!active[k] || k == i || k == j)
                continue;
            float co[4];
            lwo_coefficients(linkage, ni, nj, size[k], co);
            int64_t pi = pair_index(n, k, i);
            float v = lw_formula(co, D[pi], D[pair_index(n, k, j)], h);
            D[pi] = v;
            ++upd;
            if (k < i) {
                /* row k holds cells (k,i) and (k,j): (k,i) changed, (k,j) leaves */
                uint64_t old = rowkey[k];
                uint64_t arg = old & 0xffffffffu;
                uint64_t nk = cell_key(v, i);
                if (arg == (uint64_t)i || arg == (uint64_t)j) {
                    if (nk <= old)
                        rowkey[k] = nk;
                    else
                        rescan[k] = 1;
                } else if (nk < old) {
                    rowkey[k] = nk;
                }
            } else if (k < j) {
                /* row k holds cell (k,j) but not the pair (i,k) */
                if ((rowkey[k] & 0xffffffffu) == (uint64_t)j)
                    rescan[k] = 1;
            }
        }
        updated += upd;

        /* 2. combine i and j */
        size[i] = ni + nj;
        active[j] = 0;
        rowkey[j] = NO_KEY;

        /* cache repair: row i is new; rows that lost their minimum rescan */
        int64_t cnt = 0;
        rowkey[i] = row_minimum(D, n, active, i, &cnt);
        rowi_cells += cnt;
        int64_t rs = 0, rc = 0;
#pragma omp parallel for reduction(+ : rs, rc) schedule(dynamic, 1)
        for (int64_t k = 0; k < j; ++k) {
            if (rescan[k]) {
                int64_t c2 = 0;
                rowkey[k] = row_minimum(D, n, active, k, &c2);
                rescan[k] = 0;
                ++rs;
                rc += c2;
            }
        }
        n_rescans += rs;
        rescan_cells += rc;

        /* 4. output this level of the tree */
        merges[2 * t] = (int32_t)i;
        merges[2 * t + 1] = (int32_t)j;
        heights[t] = h;
    }
    double t2 = now_seconds();
    if (stats) {
        stats[0] = n_rescans;
        stats[1] = rescan_cells;
        stats[2] = updated;
        stats[3] = rowi_cells;
        stats[4] = total;
        stats[5] = sum_m;
    }
    if (times) {
        times[0] = t1 - t0;
        times[1] = t2 - t1;
    }
    free(active);
    free(rescan);
    free(size);
    free(rowkey);
    return LWO_OK;
}

int lwo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void lwo_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}
