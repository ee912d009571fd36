/*
 * gen.c -- seeded synthetic input graphs (CSR, int32).
 *
 * Holds none of the coloring method's arithmetic: it only makes inputs.  The
 * random stream is counter based: draw(key, i) = fmix64(key + (i+1) * K) with
 * fmix64 the 64-bit MurmurHash3 finalizer (Appleby), so every value depends
 * only on (key, i) and the output is identical for any thread count and on
 * any host.  Multi-threaded with OpenMP when available.
 *
 * Families:
 *   - 3D stencils (7-point and 27-point), vertex id x + nx*(y + ny*z);
 *   - 2D 5-point grids with w = ceil(sqrt(n)) columns, last row partial;
 *   - R-MAT edge samples (Chakrabarti, Zhan, Faloutsos 2004), no noise, ids
 *     scrambled by v' = (v*0x9E3779B1 + 12345) mod 2^scale;
 *   - Erdos-Renyi G(n, m) edge samples;
 *   - random bipartite patterns with row length 1 + Poisson(lambda);
 *   - CSR assembly from an edge list: symmetrize, drop self-loops, sort and
 *     deduplicate each row.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

static inline uint64_t draw(uint64_t key, uint64_t i)
{
    return fmix64(key + (i + 1) * 0xD1B54A32D192ED03ULL);
}

/* uniform integer in [0, bound) from the top 32 bits (bound < 2^32) */
static inline uint32_t bounded(uint64_t r, uint32_t bound)
{
    return (uint32_t)(((r >> 32) * (uint64_t)bound) >> 32);
}

int gen_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* sorting one row (int32)                                                 */
/* ---------------------------------------------------------------------- */
static void isort(int32_t *a, int64_t n)
{
    for (int64_t i = 1; i < n; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

static void qsort_i32(int32_t *a, int64_t n)
{
    while (n > 24) {
        int32_t p = a[n / 2];
        int32_t x = a[0], y = a[n - 1];
        /* median of three */
        if ((x <= p && p <= y) || (y <= p && p <= x)) { }
        else if ((p <= x && x <= y) || (y <= x && x <= p)) p = x;
        else p = y;
        int64_t i = 0, j = n - 1;
        while (i <= j) {
            while (a[i] < p) ++i;
            while (a[j] > p) --j;
            if (i <= j) { int32_t t = a[i]; a[i] = a[j]; a[j] = t; ++i; --j; }
        }
        /* recurse into the smaller part */
        if (j + 1 < n - i) { qsort_i32(a, j + 1); a += i; n -= i; }
        else { qsort_i32(a + i, n - i); n = j + 1; }
    }
    isort(a, n);
}

/* ---------------------------------------------------------------------- */
/* CSR assembly                                                            */
/* ---------------------------------------------------------------------- */
/*
 * Builds a CSR over n vertices from m edges (src[i], dst[i]).  With
 * symmetrize, both directions are stored.  Self-loops are dropped when
 * drop_loops; each row is sorted and, with dedup, duplicates removed.
 * row_ptr: n+1 int64 (caller), col_idx: capacity entries (caller; m, or 2m
 * when symmetrizing).  Returns the final nnz, or -1 if capacity is short.
 */
int64_t gen_csr_from_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           int symmetrize, int drop_loops, int dedup,
                           int64_t *row_ptr, int32_t *col_idx, int64_t capacity)
{
    int64_t *cnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -2;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (drop_loops && s == d) continue;
        __atomic_fetch_add(&cnt[s], 1, __ATOMIC_RELAXED);
        if (symmetrize) __atomic_fetch_add(&cnt[d], 1, __ATOMIC_RELAXED);
    }
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) { int64_t c = cnt[v]; row_ptr[v] = total; total += c; }
    row_ptr[n] = total;
    if (total > capacity) { free(cnt); return -1; }
    /* cursors */
    for (int32_t v = 0; v < n; ++v) cnt[v] = row_ptr[v];
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (drop_loops && s == d) continue;
        col_idx[__atomic_fetch_add(&cnt[s], 1, __ATOMIC_RELAXED)] = d;
        if (symmetrize) col_idx[__atomic_fetch_add(&cnt[d], 1, __ATOMIC_RELAXED)] = s;
    }
    /* sort + dedup each row in place; cnt[v] = new length */
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int32_t v = 0; v < n; ++v) {
        int32_t *a = col_idx + row_ptr[v];
        int64_t len = row_ptr[v + 1] - row_ptr[v];
        qsort_i32(a, len);
        int64_t k = len;
        if (dedup && len > 1) {
            k = 1;
            for (int64_t j = 1; j < len; ++j)
                if (a[j] != a[k - 1]) a[k++] = a[j];
        }
        cnt[v] = k;
    }
    /* compact */
    int64_t out = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t start = row_ptr[v], k = cnt[v];
        if (out != start) memmove(col_idx + out, col_idx + start, (size_t)k * sizeof(int32_t));
        row_ptr[v] = out;
        out += k;
    }
    row_ptr[n] = out;
    free(cnt);
    return out;
}

/* ---------------------------------------------------------------------- */
/* stencils                                                                */
/* ---------------------------------------------------------------------- */
/* nnz of a 3D stencil; points = 7 or 27 */
int64_t gen_stencil3d_nnz(int32_t nx, int32_t ny, int32_t nz, int points)
{
    int64_t total = 0;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int nzero = (dx != 0) + (dy != 0) + (dz != 0);
                            if (nzero == 0) continue;
                            if (points == 7 && nzero != 1) continue;
                            int32_t X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                            total++;
                        }
            }
    return total;
}

/* sorted neighbors (ids increase with dz, then dy, then dx) */
void gen_stencil3d(int32_t nx, int32_t ny, int32_t nz, int points, int32_t *row_ptr, int32_t *col_idx)
{
    int64_t n = (int64_t)nx * ny * nz;
    /* pass 1: degrees */
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        int32_t x = (int32_t)(v % nx), y = (int32_t)((v / nx) % ny), z = (int32_t)(v / ((int64_t)nx * ny));
        int32_t d = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int nzero = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nzero == 0 || (points == 7 && nzero != 1)) continue;
                    int32_t X = x + dx, Y = y + dy, Z = z + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                    d++;
                }
        row_ptr[v + 1] = d;
    }
    row_ptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        int32_t x = (int32_t)(v % nx), y = (int32_t)((v / nx) % ny), z = (int32_t)(v / ((int64_t)nx * ny));
        int32_t k = row_ptr[v];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int nzero = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nzero == 0 || (points == 7 && nzero != 1)) continue;
                    int32_t X = x + dx, Y = y + dy, Z = z + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                    col_idx[k++] = (int32_t)(X + (int64_t)nx * (Y + (int64_t)ny * Z));
                }
    }
}

/* 2D 5-point grid over n vertices, w = ceil(sqrt(n)) columns, row-major,
 * last row partial.  Emits undirected edges (right and down neighbors);
 * returns the edge count.  src/dst need 2n capacity. */
int64_t gen_grid2d_edges(int32_t n, int32_t *src, int32_t *dst)
{
    int32_t w = 1;
    while ((int64_t)w * w < n) ++w;
    int64_t m = 0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t x = v % w;
        if (x + 1 < w && v + 1 < n) { src[m] = v; dst[m] = v + 1; ++m; }
        if ((int64_t)v + w < n) { src[m] = v; dst[m] = v + w; ++m; }
    }
    return m;
}

/* ---------------------------------------------------------------------- */
/* R-MAT and Erdos-Renyi samples                                           */
/* ---------------------------------------------------------------------- */
/*
 * m edge samples of an R-MAT graph with 2^scale vertices.  At each of the
 * scale levels the quadrant (a | b | c | d) is drawn from 32 random bits
 * against fixed-point thresholds.  Two levels per 64-bit draw.
 */
void gen_rmat_edges(int32_t scale, int64_t m, double a, double b, double c, uint64_t seed,
                    int scramble, int32_t *src, int32_t *dst)
{
    const uint64_t ta = (uint64_t)llround(a * 4294967296.0);
    const uint64_t tb = (uint64_t)llround((a + b) * 4294967296.0);
    const uint64_t tc = (uint64_t)llround((a + b + c) * 4294967296.0);
    const uint32_t nmask = (scale >= 32) ? 0xFFFFFFFFu : ((1u << scale) - 1u);
    const int levels_per_edge = (scale + 1) / 2;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u = 0, v = 0;
        int level = 0;
        for (int k = 0; k < levels_per_edge; ++k) {
            uint64_t r = draw(seed, (uint64_t)i * (uint64_t)levels_per_edge + (uint64_t)k);
            for (int half = 0; half < 2 && level < scale; ++half, ++level) {
                uint64_t x = half ? (r >> 32) : (r & 0xFFFFFFFFULL);
                uint32_t bu = 0, bv = 0;
                if (x < ta) { }
                else if (x < tb) { bv = 1; }
                else if (x < tc) { bu = 1; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
        }
        if (scramble) {
            u = (uint32_t)(((uint64_t)u * 0x9E3779B1ULL + 12345ULL) & nmask);
            v = (uint32_t)(((uint64_t)v * 0x9E3779B1ULL + 12345ULL) & nmask);
        }
        src[i] = (int32_t)u;
        dst[i] = (int32_t)v;
    }
}

/* m uniform vertex pairs over n vertices (loops and repeats possible; the
 * CSR assembly removes them). */
void gen_er_edges(int32_t n, int64_t m, uint64_t seed, int32_t *src, int32_t *dst)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint64_t r = draw(seed, (uint64_t)i);
        src[i] = (int32_t)bounded(r << 32, (uint32_t)n);
        dst[i] = (int32_t)bounded(r, (uint32_t)n);
    }
}

/* ---------------------------------------------------------------------- */
/* random bipartite pattern: row r has 1 + Poisson(lambda) column draws     */
/* ---------------------------------------------------------------------- */
/* Poisson CDF thresholds in 2^-64 units, built from pmf ratios with a given
 * p0 = exp(-lambda) (passed in so that every host builds the same table). */
static int poisson_table(double lambda, double p0, uint64_t *thr, int cap)
{
    double p = p0, F = p0;
    int k = 0;
    for (; k < cap - 1; ++k) {
        double t = F * 18446744073709551616.0;
        thr[k] = t >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)t;
        if (F >= 1.0 - 1e-17) break;
        p = p * lambda / (double)(k + 1);
        F = F + p;
    }
    thr[k] = UINT64_MAX;
    return k + 1;
}

/* Row lengths (before duplicate removal); returns the total. */
int64_t gen_bipartite_lengths(int32_t n_rows, double lambda, double p0, uint64_t seed, int32_t *len)
{
    uint64_t thr[256];
    int nthr = poisson_table(lambda, p0, thr, 256);
    int64_t total = 0;
    #pragma omp parallel for schedule(static) reduction(+:total)
    for (int32_t r = 0; r < n_rows; ++r) {
        uint64_t u = draw(seed, (uint64_t)r);
        int k = 0;
        while (k < nthr - 1 && u >= thr[k]) ++k;
        len[r] = 1 + k;
        total += 1 + k;
    }
    return total;
}

/* Column draws for each row: entries [off[r], off[r]+len[r]) of dst, src = r. */
void gen_bipartite_entries(int32_t n_rows, int32_t n_cols, uint64_t seed, const int32_t *len,
                           const int64_t *off, int32_t *src, int32_t *dst)
{
    const uint64_t key = fmix64(seed ^ 0x5851F42D4C957F2DULL);
    #pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < n_rows; ++r) {
        for (int32_t j = 0; j < len[r]; ++j) {
            int64_t e = off[r] + j;
            src[e] = r;
            dst[e] = (int32_t)bounded(draw(key, (uint64_t)e), (uint32_t)n_cols);
        }
    }
}
