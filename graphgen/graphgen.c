/*
 * graphgen.c -- seeded synthetic graph inputs (R-MAT/Kronecker and uniform
 * Erdos-Renyi edge tuples, vertex permutation, CSR assembly).
 *
 * This module only manufactures inputs.  It holds none of the BFS arithmetic:
 * both the oracle and the CUDA library consume the CSR it builds, and neither
 * depends on anything else here.
 *
 * Workload shape (paper Sec. 4.1 and Sec. 5.2): 2^SCALE vertices,
 * 2^SCALE * edgefactor generated tuples including self-loops and repeats,
 * initiator A/B/C/D = 0.57/0.19/0.19/0.05.  The paper used the Graph500
 * generator; that code is not used or reproduced here.  This is a plain R-MAT
 * quadrant descent with no per-level noise, driven by a counter-based
 * SplitMix64 stream (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so every tuple depends only on (seed, index) and
 * the output is identical for any thread count.
 *
 * Host code only; portable C11 + optional OpenMP; no architecture intrinsics.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- SplitMix64, indexed form: output_i = mix(base + (i+1)*gamma) -------- */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

static inline uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* stream base: distinct seeds and stream ids give unrelated sequences */
static inline uint64_t sm_base(uint64_t seed, uint64_t stream)
{
    return sm_mix(seed * SM_GAMMA + sm_mix(stream + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t sm_at(uint64_t base, uint64_t i)
{
    return sm_mix(base + (i + 1) * SM_GAMMA);
}

/* draw in [0, bound): Lemire multiply-shift of a 64-bit word (bias < bound/2^64) */
static inline uint64_t bounded(uint64_t r, uint64_t bound)
{
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

int gg_version(void) { return 1; }

int gg_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * R-MAT tuples.  Each tuple descends `scale` levels of the 2x2 initiator:
 * quadrant (0,0) with prob A, (0,1) with B, (1,0) with C, (1,1) otherwise.
 * Bits are assigned most-significant first.  Thresholds are compared as
 * 32-bit integers, two draws per 64-bit random word.
 */
void gg_rmat_tuples(int scale, int64_t nedges, double A, double B, double C,
                    uint64_t seed, int32_t *src, int32_t *dst)
{
    const uint64_t base = sm_base(seed, 1);
    const double two32 = 4294967296.0;
    const uint64_t tA = (uint64_t)(A * two32);
    const uint64_t tAB = (uint64_t)((A + B) * two32);
    const uint64_t tABC = (uint64_t)((A + B + C) * two32);
    const int words = (scale + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint32_t s = 0, d = 0;
        int bit = scale - 1;
        for (int w = 0; w < words; ++w) {
            uint64_t r = sm_at(base, (uint64_t)e * (uint64_t)words + (uint64_t)w);
            for (int h = 0; h < 2 && bit >= 0; ++h, --bit) {
                uint64_t x = (h == 0) ? (r & 0xFFFFFFFFULL) : (r >> 32);
                uint32_t sb, db;
                if (x < tA) { sb = 0; db = 0; }
                else if (x < tAB) { sb = 0; db = 1; }
                else if (x < tABC) { sb = 1; db = 0; }
                else { sb = 1; db = 1; }
                s |= sb << bit;
                d |= db << bit;
            }
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
}

/* Uniform random tuples over [0, n): both endpoints drawn from the seed. */
void gg_uniform_tuples(int64_t n, int64_t nedges, uint64_t seed,
                       int32_t *src, int32_t *dst)
{
    const uint64_t base = sm_base(seed, 2);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint64_t r0 = sm_at(base, 2 * (uint64_t)e);
        uint64_t r1 = sm_at(base, 2 * (uint64_t)e + 1);
        src[e] = (int32_t)bounded(r0, (uint64_t)n);
        dst[e] = (int32_t)bounded(r1, (uint64_t)n);
    }
}

/* Seeded Fisher-Yates permutation of [0, n). */
void gg_permutation(int64_t n, uint64_t seed, int32_t *perm)
{
    const uint64_t base = sm_base(seed, 3);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)bounded(sm_at(base, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* Relabel tuple endpoints through perm. */
void gg_apply_permutation(int64_t nedges, const int32_t *perm, int32_t *src, int32_t *dst)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        src[e] = perm[src[e]];
        dst[e] = perm[dst[e]];
    }
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_small(int32_t *a, int64_t len)
{
    if (len > 32) {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
        return;
    }
    for (int64_t i = 1; i < len; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

/*
 * Assemble a CSR from tuples.
 *   symmetrize : store both (u,v) and (v,u)
 *   drop_loops : skip u == v
 *   dedup      : sort each adjacency row and drop repeats
 * row_offsets must hold n+1 entries.  col must hold the upper bound
 * (symmetrize ? 2 : 1) * nedges entries; the final m entries are left at the
 * front of `col`.  Every row is sorted ascending.  Returns m, or
 * -1 if an endpoint is out of range, -2 if m would exceed INT32_MAX, -3 on
 * allocation failure.
 */
int64_t gg_build_csr(int64_t n, int64_t nedges, const int32_t *src, const int32_t *dst,
                     int symmetrize, int drop_loops, int dedup,
                     int32_t *row_offsets, int32_t *col)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -3;
    int bad = 0;
    /* 1. degree count */
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t e = 0; e < nedges; ++e) {
        int32_t u = src[e], v = dst[e];
        if (u < 0 || u >= n || v < 0 || v >= n) { bad = 1; continue; }
        if (drop_loops && u == v) continue;
#pragma omp atomic
        cnt[u + 1]++;
        if (symmetrize) {
#pragma omp atomic
            cnt[v + 1]++;
        }
    }
    if (bad) { free(cnt); return -1; }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    /* 2. scatter (order inside a row is fixed by the sort below) */
    int64_t *cur = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!cur) { free(cnt); return -3; }
    memcpy(cur, cnt, ((size_t)n + 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        int32_t u = src[e], v = dst[e];
        if (drop_loops && u == v) continue;
        int64_t p;
#pragma omp atomic capture
        p = cur[u]++;
        col[p] = v;
        if (symmetrize) {
#pragma omp atomic capture
            p = cur[v]++;
            col[p] = u;
        }
    }
    /* 3. per-row sort + dedup; cur[] reused as kept-length per row */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t u = 0; u < n; ++u) {
        int32_t *row = col + cnt[u];
        int64_t len = cnt[u + 1] - cnt[u];
        sort_small(row, len); /* makes the row order independent of threads */
        if (dedup) {
            int64_t k = 0;
            for (int64_t i = 0; i < len; ++i)
                if (k == 0 || row[i] != row[k - 1]) row[k++] = row[i];
            len = k;
        }
        cur[u] = len;
    }
    /* 4. compact to the front */
    int64_t m = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t len = cur[u];
        if (m + len > 2147483647LL) { free(cnt); free(cur); return -2; }
        row_offsets[u] = (int32_t)m;
        if (m != cnt[u]) memmove(col + m, col + cnt[u], (size_t)len * sizeof(int32_t));
        m += len;
    }
    row_offsets[n] = (int32_t)m;
    free(cnt);
    free(cur);
    return m;
}

/*
 * Seeded choice of k vertices with out-degree >= 1, by rejection over a
 * seeded stream.  With distinct != 0 no vertex is chosen twice (and k is cut
 * to the number of eligible vertices).  Returns the number chosen.
 */
int64_t gg_pick_roots(int64_t n, const int32_t *row_offsets, int64_t k, uint64_t seed,
                      int distinct, int32_t *roots)
{
    const uint64_t base = sm_base(seed, 4);
    int64_t have = 0, eligible = 0;
    for (int64_t v = 0; v < n; ++v) eligible += (row_offsets[v + 1] > row_offsets[v]);
    if (eligible == 0) return 0;
    if (distinct && k > eligible) k = eligible;
    uint8_t *taken = distinct ? (uint8_t *)calloc((size_t)n, 1) : NULL;
    if (distinct && !taken) return -3;
    uint64_t i = 0;
    while (have < k) {
        int64_t v = (int64_t)bounded(sm_at(base, i++), (uint64_t)n);
        if (row_offsets[v + 1] <= row_offsets[v]) continue;
        if (distinct) {
            if (taken[v]) continue;
            taken[v] = 1;
        }
        roots[have++] = (int32_t)v;
    }
    free(taken);
    return have;
}
