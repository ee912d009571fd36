/*
 * pgc_cpu_omp.c -- CPU BASELINE, not product code and not the oracle.
 *
 * The distance-1 round loop of pgc_oracle.c run on all host cores with
 * OpenMP, so that the benchmark can report a multi-core CPU figure beside
 * the single-core oracle.  The method is the same deterministic
 * round-synchronous speculate-and-resolve coloring (Bogle et al., Sec. 3.2,
 * Alg. 1-4 with recolorDegrees of Sec. 3.3), so the colors are bit-identical
 * to the oracle's for any thread count: within a round, the first-fit step
 * reads only colors committed before the round and the detection step reads
 * a snapshot, so the vertices of the worklist are independent of each other
 * inside each step.  The tests check the equality on many graphs.
 *
 * Per round:
 *   assign  (parallel over the worklist): t = smallest color not committed
 *           in N(v) (Alg. 1), using a per-thread stamp array;
 *   detect  (parallel): v loses iff some u in N(v) holds the same current
 *           color and Alg. 4 recolors v against u;
 *   commit  (parallel count, prefix sum, parallel scatter): winners commit,
 *           losers form the next worklist in worklist order.
 *
 * Only the benchmark's CPU leg and the tests load this file.  Every array
 * is host memory owned by the caller.  Returns 0, -1 (bad arguments), -2
 * (allocation failure) or -3 (max_rounds reached).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static uint64_t mix64(uint64_t x)   /* splitmix64 output for state x */
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* 1 if v is recolored against u (the decision order of Alg. 4). */
static int recolor_v(int32_t dv, uint64_t rv, int32_t v, int32_t du, uint64_t ru, int32_t u,
                     int use_deg)
{
    if (use_deg && dv != du) return dv < du;
    if (rv != ru) return rv > ru;
    return v > u;
}

int cpu_omp_color_d1(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     uint64_t seed, int32_t recolor_degrees, int32_t max_rounds,
                     int32_t threads, int32_t *colors, int32_t *rounds_out,
                     int32_t *num_colors_out, int32_t *threads_used)
{
    if (n < 0 || !rounds_out || !num_colors_out || (n > 0 && (!row_ptr || !colors)))
        return -1;
    *rounds_out = 0;
    *num_colors_out = 0;
    if (threads > 0) omp_set_num_threads(threads);
    if (threads_used) *threads_used = omp_get_max_threads();
    if (n == 0) return 0;
    if (row_ptr[n] > 0 && !col_idx) return -1;
    if (max_rounds <= 0) max_rounds = n + 1;

    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t d = row_ptr[v + 1] - row_ptr[v];
        if (d < 0) return -1;
        if (d > maxdeg) maxdeg = d;
    }
    const int nt = omp_get_max_threads();
    int32_t *committed = calloc((size_t)n, sizeof(int32_t));
    int32_t *tent = calloc((size_t)n, sizeof(int32_t));
    uint64_t *rnd = malloc((size_t)n * sizeof(uint64_t));
    int32_t *work = malloc((size_t)n * sizeof(int32_t));
    int32_t *next = malloc((size_t)n * sizeof(int32_t));
    unsigned char *lose = calloc((size_t)n, 1);
    int64_t *counts = calloc((size_t)nt + 1, sizeof(int64_t));
    /* per-thread forbidden stamps: colors 1..maxdeg+1 */
    const size_t fw = (size_t)maxdeg + 2;
    int64_t *forbidden = calloc(fw * (size_t)nt, sizeof(int64_t));
    if (!committed || !tent || !rnd || !work || !next || !lose || !counts || !forbidden) {
        free(committed); free(tent); free(rnd); free(work); free(next); free(lose);
        free(counts); free(forbidden);
        return -2;
    }
    #pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; ++v) {
        rnd[v] = mix64(seed ^ (uint64_t)(uint32_t)v);
        work[v] = v;
    }
    int32_t wn = n, r = 0;
    int status = 0;
    int64_t stamp_base = 0;
    while (wn > 0) {
        if (r >= max_rounds) { status = -3; break; }
        r += 1;
        const int64_t stamp0 = stamp_base;
        #pragma omp parallel
        {
            const int tid = omp_get_thread_num();
            int64_t *fb = forbidden + (size_t)tid * fw;
            int64_t stamp = stamp0;
            #pragma omp for schedule(dynamic, 256)
            for (int32_t i = 0; i < wn; ++i) {
                const int32_t v = work[i];
                stamp += 1;
                for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                    const int32_t u = col_idx[e];
                    const int32_t c = committed[u];
                    if (u != v && c > 0 && c <= maxdeg + 1) fb[c] = stamp;
                }
                int32_t t = 1;
                while (fb[t] == stamp) t += 1;
                tent[v] = t;
            }
        }
        /* every thread's stamps stay below stamp0 + wn */
        stamp_base += wn + 1;
        #pragma omp parallel for schedule(dynamic, 256)
        for (int32_t i = 0; i < wn; ++i) {
            const int32_t v = work[i];
            const int32_t dv = row_ptr[v + 1] - row_ptr[v];
            unsigned char l = 0;
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1] && !l; ++e) {
                const int32_t u = col_idx[e];
                if (u == v) continue;
                const int32_t cu = committed[u] > 0 ? committed[u] : tent[u];
                if (cu == tent[v] &&
                    recolor_v(dv, rnd[v], v, row_ptr[u + 1] - row_ptr[u], rnd[u], u,
                              recolor_degrees))
                    l = 1;
            }
            lose[v] = l;
        }
        /* commit and compact, keeping worklist order */
        #pragma omp parallel
        {
            const int tid = omp_get_thread_num(), nth = omp_get_num_threads();
            const int64_t lo = (int64_t)wn * tid / nth, hi = (int64_t)wn * (tid + 1) / nth;
            int64_t c = 0;
            for (int64_t i = lo; i < hi; ++i) c += lose[work[i]];
            counts[tid + 1] = c;
            #pragma omp barrier
            #pragma omp single
            {
                counts[0] = 0;
                for (int k = 1; k <= nth; ++k) counts[k] += counts[k - 1];
            }
            int64_t o = counts[tid];
            for (int64_t i = lo; i < hi; ++i) {
                const int32_t v = work[i];
                if (lose[v]) { next[o++] = v; tent[v] = 0; }
                else committed[v] = tent[v];
            }
            #pragma omp barrier
            #pragma omp single
            wn = (int32_t)counts[nth];
        }
        int32_t *tmp = work; work = next; next = tmp;
    }
    int32_t maxc = 0;
    #pragma omp parallel for reduction(max : maxc)
    for (int32_t v = 0; v < n; ++v) {
        colors[v] = committed[v];
        if (committed[v] > maxc) maxc = committed[v];
    }
    *rounds_out = r;
    *num_colors_out = maxc;
    free(committed); free(tent); free(rnd); free(work); free(next); free(lose);
    free(counts); free(forbidden);
    return status;
}
