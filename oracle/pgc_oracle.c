/*
 * pgc_oracle.c -- TEST INFRASTRUCTURE, not product code.
 *
 * A plain, slow, single-threaded CPU restatement of the deterministic
 * round-synchronous speculate-and-resolve coloring used to check the CUDA
 * library bit for bit.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (Bogle et al., "Parallel Graph Coloring Algorithms for
 * Distributed GPU Environments"):
 *   - Problems: distance-1, distance-2 and partial distance-2 coloring
 *     (Sec. 2.1).  Colors are positive integers; 0 means "no color yet"
 *     (Alg. 1, Sec. 3.2).
 *   - Each round gives every vertex on the worklist the smallest color not
 *     used by an already-colored vertex of its neighborhood (the first-fit
 *     rule of Alg. 1), then detects conflicts (Alg. 3 for D1, Alg. 5 for D2
 *     and PD2) and keeps exactly one vertex of each conflicting pair by the
 *     rule of Alg. 4 with recolorDegrees on (Sec. 3.3): the lower-degree
 *     vertex is recolored; on equal degree the one with the higher random
 *     number; on equal random number the one with the higher id.  The outer
 *     loop is Alg. 2 without the ghost/MPI steps (one process owns every
 *     vertex).
 *   - Readings where the paper leaves a choice (they are the same on the GPU
 *     side, which is written separately):
 *       * speculation is round-synchronous (Jacobi): the first-fit step of a
 *         round sees only colors committed before the round; worklist
 *         vertices are uncolored to each other while they choose;
 *       * conflict detection reads a snapshot: every worklist vertex decides
 *         only its own fate, from the colors as they stood after the
 *         first-fit step (Alg. 4 uncolors in place, which would make the
 *         result depend on processing order);
 *       * rand(GID) is splitmix64(seed XOR id), compared as unsigned 64-bit;
 *         the id is the vertex index;
 *       * degree is the row length of the input (D1, D2) or the column length
 *         of the bipartite matrix (PD2), computed once (Sec. 3.3);
 *       * distance-2 neighborhoods exclude the vertex itself (the formula in
 *         Sec. 2.1 is garbled; Alg. 5 is read as skipping x == v);
 *       * PD2 colors only the column vertices; rows are the shared "nets"
 *         (oracle_color_pd2); the paper's own PD2 colors every vertex of the
 *         bipartite graph (Sec. 3.6), which oracle_color_pd2_bipartite
 *         computes with vertex ids columns first, then rows (the id is the
 *         GID of rand(GID));
 *       * self-loop entries are skipped as neighbors but counted in the
 *         degree; duplicate entries are harmless.
 *
 * Every array here is host memory owned by the caller.  Scratch is malloc'ed
 * and freed inside each call.  Return value: 0 on success, -1 on bad
 * arguments, -2 on allocation failure, -3 if the loop has not finished after
 * max_rounds rounds (never the case for valid input: each round commits at
 * least the worklist vertex with the largest key, so at most n rounds run).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* splitmix64 (Steele, Lea, Flood 2014), as a function of its state: the   */
/* output the generator gives after its state is advanced to x + gamma.    */
/* ---------------------------------------------------------------------- */
uint64_t oracle_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* rand(GID) of Alg. 4 under the reading above. */
static uint64_t rand_of(uint64_t seed, int32_t v)
{
    return oracle_splitmix64(seed ^ (uint64_t)(uint32_t)v);
}

/*
 * Alg. 4 (Check-Conflicts), the decision only: given that v and u hold the
 * same color, return 1 if v is the vertex to be recolored, 0 if u is.
 * The branches follow the algorithm's order.
 */
int oracle_v_is_recolored(int32_t deg_v, uint64_t rand_v, int32_t v,
                          int32_t deg_u, uint64_t rand_u, int32_t u,
                          int32_t recolor_degrees)
{
    if (recolor_degrees && deg_v < deg_u) return 1;
    if (recolor_degrees && deg_u < deg_v) return 0;
    if (rand_v > rand_u) return 1;
    if (rand_u > rand_v) return 0;
    if (v > u) return 1;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Neighborhoods S(v).  A neighborhood is visited through a callback-free  */
/* "cursor" so that the first-fit step and the detection step walk the     */
/* very same set.                                                           */
/* ---------------------------------------------------------------------- */
enum { KIND_D1 = 1, KIND_D2 = 2, KIND_PD2 = 3, KIND_PD2B = 4 };

typedef struct {
    int kind;
    int32_t n;                 /* vertices that get colors */
    const int32_t *row_ptr, *col_idx;   /* D1/D2: the graph; PD2: rows -> columns */
    const int32_t *col_ptr, *row_idx;   /* PD2 only: columns -> rows            */
    int32_t n_cols;            /* PD2 over all of B: vertices [0, n_cols) are the
                                  columns, n_cols + i is row i               */
} graph_t;

/*
 * Calls visit(x) for every x in S(v), possibly more than once.
 *   D1 : x in N(v), x != v                                    (Sec. 2.1)
 *   D2 : x in N(v) or x in N(u) for some u in N(v), x != v     (Sec. 2.1, Alg. 5)
 *   PD2: x a column sharing a row with column v, x != v        (Sec. 3.6)
 *   PD2 over all of B (Sec. 3.6: every vertex of the bipartite graph gets a
 *   color, two-hop conflicts only): a column as for PD2; row i (vertex
 *   n_cols + i) has the rows sharing a column with it, as vertices n_cols + r
 * Implemented as a macro-free loop that fills a caller buffer, to keep the
 * three cases side by side.  Returns the number of entries written.
 */
static int64_t neighborhood(const graph_t *g, int32_t v, int32_t *buf)
{
    int64_t k = 0;
    if (g->kind == KIND_D1) {
        for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            int32_t u = g->col_idx[e];
            if (u != v) buf[k++] = u;
        }
    } else if (g->kind == KIND_D2) {
        for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            int32_t u = g->col_idx[e];
            if (u != v) buf[k++] = u;                 /* one hop */
            for (int32_t f = g->row_ptr[u]; f < g->row_ptr[u + 1]; ++f) {
                int32_t x = g->col_idx[f];
                if (x != v) buf[k++] = x;             /* two hops via u */
            }
        }
    } else if (g->kind == KIND_PD2 || v < g->n_cols) { /* a column */
        for (int32_t e = g->col_ptr[v]; e < g->col_ptr[v + 1]; ++e) {
            int32_t row = g->row_idx[e];
            for (int32_t f = g->row_ptr[row]; f < g->row_ptr[row + 1]; ++f) {
                int32_t x = g->col_idx[f];
                if (x != v) buf[k++] = x;
            }
        }
    } else { /* KIND_PD2B, row i = v - n_cols */
        int32_t i = v - g->n_cols;
        for (int32_t e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) {
            int32_t col = g->col_idx[e];
            for (int32_t f = g->col_ptr[col]; f < g->col_ptr[col + 1]; ++f) {
                int32_t r = g->row_idx[f];
                if (r != i) buf[k++] = g->n_cols + r;
            }
        }
    }
    return k;
}

/* Upper bound on the entries neighborhood() writes for any v. */
static int64_t neighborhood_capacity(const graph_t *g)
{
    int64_t best = 0;
    for (int32_t v = 0; v < g->n; ++v) {
        int64_t k = 0;
        if (g->kind == KIND_D1) {
            k = g->row_ptr[v + 1] - g->row_ptr[v];
        } else if (g->kind == KIND_D2) {
            for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
                int32_t u = g->col_idx[e];
                k += 1 + (g->row_ptr[u + 1] - g->row_ptr[u]);
            }
        } else if (g->kind == KIND_PD2 || v < g->n_cols) {
            for (int32_t e = g->col_ptr[v]; e < g->col_ptr[v + 1]; ++e) {
                int32_t row = g->row_idx[e];
                k += g->row_ptr[row + 1] - g->row_ptr[row];
            }
        } else {
            int32_t i = v - g->n_cols;
            for (int32_t e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) {
                int32_t col = g->col_idx[e];
                k += g->col_ptr[col + 1] - g->col_ptr[col];
            }
        }
        if (k > best) best = k;
    }
    return best;
}

/* deg(v): row length (D1, D2); for PD2 the vertex's degree in B: a column's
 * CSC length, a row's CSR length (Sec. 3.3, computed once). */
static int32_t degree_of(const graph_t *g, int32_t v)
{
    if (g->kind == KIND_PD2 || (g->kind == KIND_PD2B && v < g->n_cols))
        return g->col_ptr[v + 1] - g->col_ptr[v];
    if (g->kind == KIND_PD2B)
        return g->row_ptr[v - g->n_cols + 1] - g->row_ptr[v - g->n_cols];
    return g->row_ptr[v + 1] - g->row_ptr[v];
}

/* ---------------------------------------------------------------------- */
/* Priorities that change from round to round (Sec. 3.3, closing paragraph: */
/* a "dynamic" degree based on how many neighbors have been colored, or the */
/* "saturation degree", how many colors the colored neighbors hold).  They   */
/* take the place of deg() in Alg. 4; the degree-first decision stays.      */
/* Readings (D1 only): both are taken at the start of each round;           */
/*   dynamic:    the adjacency entries of v whose vertex is still uncolored  */
/*               (the degree with colored neighbors removed; equal to deg(v)  */
/*               in round 1);                                                */
/*   saturation: the distinct colors held by colored neighbors of v, counting */
/*               only colors 1 .. deg(v)+1 (the colors v's first fit can      */
/*               meet; 0 in round 1).                                        */
/* ---------------------------------------------------------------------- */
enum { PRIO_STATIC = 0, PRIO_DYNAMIC = 1, PRIO_SATURATION = 2 };

static int32_t round_priority(const graph_t *g, int32_t v, const int32_t *committed,
                              const int32_t *deg, int32_t mode, int64_t *mark, int64_t *stamp)
{
    int32_t p = 0;
    if (mode == PRIO_DYNAMIC) {
        for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e)
            if (committed[g->col_idx[e]] == 0) p += 1;
        return p;
    }
    *stamp += 1;
    for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
        int32_t u = g->col_idx[e];
        int32_t c = committed[u];
        if (u != v && c > 0 && c <= deg[v] + 1 && mark[c] != *stamp) {
            mark[c] = *stamp;
            p += 1;
        }
    }
    return p;
}

/* ---------------------------------------------------------------------- */
/* The round loop (Alg. 2 on one process).                                  */
/* ---------------------------------------------------------------------- */
static int color_rounds(const graph_t *g, uint64_t seed, int32_t recolor_degrees,
                        int32_t prio_mode, int32_t max_rounds, int32_t *colors,
                        int32_t *rounds_out, int32_t *num_colors_out, int64_t *trace_w,
                        int64_t *trace_s, int32_t trace_cap)
{
    const int32_t n = g->n;
    *rounds_out = 0;
    *num_colors_out = 0;
    if (n == 0) return 0;
    if (max_rounds <= 0) max_rounds = n + 1;

    int64_t cap = neighborhood_capacity(g);
    int32_t *committed = calloc((size_t)n, sizeof(int32_t)); /* 0 = uncolored */
    int32_t *tent = calloc((size_t)n, sizeof(int32_t));
    int32_t *deg = malloc((size_t)n * sizeof(int32_t));
    int32_t *key = malloc((size_t)n * sizeof(int32_t));   /* the degree term of Alg. 4 */
    int64_t *pmark = calloc((size_t)n + 2, sizeof(int64_t));
    uint64_t *rnd = malloc((size_t)n * sizeof(uint64_t));
    int32_t *work = malloc((size_t)n * sizeof(int32_t));
    int32_t *next = malloc((size_t)n * sizeof(int32_t));
    unsigned char *lose = calloc((size_t)n, 1);
    int32_t *buf = malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    /* forbidden[c] == stamp marks color c as used in the current scan */
    int64_t *forbidden = calloc((size_t)n + 2, sizeof(int64_t));
    if (!committed || !tent || !deg || !key || !pmark || !rnd || !work || !next || !lose ||
        !buf || !forbidden) {
        free(committed); free(tent); free(deg); free(key); free(pmark); free(rnd); free(work);
        free(next); free(lose); free(buf); free(forbidden);
        return -2;
    }

    /* Degrees are computed once (Sec. 3.3). */
    for (int32_t v = 0; v < n; ++v) {
        deg[v] = degree_of(g, v);
        key[v] = deg[v];
        rnd[v] = rand_of(seed, v);
    }
    int64_t pstamp = 0;
    int32_t wn = n;
    for (int32_t v = 0; v < n; ++v) work[v] = v;   /* every vertex starts uncolored */

    int64_t stamp = 0;
    int32_t r = 0;
    int status = 0;
    while (wn > 0) {
        if (r >= max_rounds) { status = -3; break; }
        r += 1;
        if (trace_w && r <= trace_cap) {
            int64_t s = 0;
            for (int32_t i = 0; i < wn; ++i) s += deg[work[i]];
            trace_w[r - 1] = wn;
            trace_s[r - 1] = s;
        }
        if (prio_mode != PRIO_STATIC)
            for (int32_t i = 0; i < wn; ++i)
                key[work[i]] = round_priority(g, work[i], committed, deg, prio_mode, pmark,
                                              &pstamp);

        /* (1) Speculative coloring: first-fit over committed colors only
         *     (Alg. 1's rule, Jacobi reading). */
        for (int32_t i = 0; i < wn; ++i) {
            int32_t v = work[i];
            int64_t k = neighborhood(g, v, buf);
            stamp += 1;
            for (int64_t j = 0; j < k; ++j) {
                int32_t c = committed[buf[j]];
                if (c > 0 && c <= n + 1) forbidden[c] = stamp;
            }
            int32_t t = 1;
            while (forbidden[t] == stamp) t += 1;
            tent[v] = t;
        }

        /* (2) Conflict detection on the snapshot (Alg. 3 / Alg. 5 with the
         *     decision of Alg. 4).  The current color of a vertex is its
         *     committed color, else its tentative color of this round. */
        for (int32_t i = 0; i < wn; ++i) {
            int32_t v = work[i];
            int64_t k = neighborhood(g, v, buf);
            lose[v] = 0;
            for (int64_t j = 0; j < k; ++j) {
                int32_t u = buf[j];
                int32_t cu = committed[u] > 0 ? committed[u] : tent[u];
                if (cu == tent[v] &&
                    oracle_v_is_recolored(key[v], rnd[v], v, key[u], rnd[u], u,
                                          prio_mode != PRIO_STATIC || recolor_degrees)) {
                    lose[v] = 1;
                    break;
                }
            }
        }

        /* (3) Winners keep their color; losers are uncolored and form the
         *     next worklist (Sec. 3.2: recolored vertices get color zero). */
        int32_t nn = 0;
        for (int32_t i = 0; i < wn; ++i) {
            int32_t v = work[i];
            if (lose[v]) {
                next[nn++] = v;
                tent[v] = 0;
            } else {
                committed[v] = tent[v];
            }
        }
        int32_t *tmp = work; work = next; next = tmp;
        wn = nn;
    }

    int32_t maxc = 0;
    for (int32_t v = 0; v < n; ++v) {
        colors[v] = committed[v];
        if (committed[v] > maxc) maxc = committed[v];
    }
    *rounds_out = r;
    *num_colors_out = maxc;
    free(committed); free(tent); free(deg); free(key); free(pmark); free(rnd); free(work);
    free(next);
    free(lose); free(buf); free(forbidden);
    return status;
}

static int check_csr(int32_t n, const int32_t *ptr, const int32_t *idx, int32_t idx_bound)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!ptr || ptr[0] != 0) return -1;
    for (int32_t v = 0; v < n; ++v)
        if (ptr[v + 1] < ptr[v]) return -1;
    if (ptr[n] > 0 && !idx) return -1;
    for (int32_t e = 0; e < ptr[n]; ++e)
        if (idx[e] < 0 || idx[e] >= idx_bound) return -1;
    return 0;
}

/* D1 (Sec. 3.2).  trace_w/trace_s (nullable) receive |W_r| and the sum of
 * the degrees of W_r for the first trace_cap rounds. */
int oracle_color_d1(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                    uint64_t seed, int32_t recolor_degrees, int32_t max_rounds,
                    int32_t *colors, int32_t *rounds, int32_t *num_colors,
                    int64_t *trace_w, int64_t *trace_s, int32_t trace_cap)
{
    if (check_csr(n, row_ptr, col_idx, n) || (n > 0 && !colors) || !rounds || !num_colors)
        return -1;
    graph_t g = { KIND_D1, n, row_ptr, col_idx, NULL, NULL, 0 };
    return color_rounds(&g, seed, recolor_degrees, PRIO_STATIC, max_rounds, colors, rounds,
                        num_colors, trace_w, trace_s, trace_cap);
}

/* D1 with a priority that changes each round (Sec. 3.3, closing paragraph):
 * prio_mode 1 = dynamic degree, 2 = saturation degree (readings above); the
 * rest as oracle_color_d1 with recolorDegrees on. */
int oracle_color_d1_priority(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             uint64_t seed, int32_t prio_mode, int32_t max_rounds,
                             int32_t *colors, int32_t *rounds, int32_t *num_colors,
                             int64_t *trace_w, int64_t *trace_s, int32_t trace_cap)
{
    if (check_csr(n, row_ptr, col_idx, n) || (n > 0 && !colors) || !rounds || !num_colors ||
        (prio_mode != PRIO_DYNAMIC && prio_mode != PRIO_SATURATION))
        return -1;
    graph_t g = { KIND_D1, n, row_ptr, col_idx, NULL, NULL, 0 };
    return color_rounds(&g, seed, 1, prio_mode, max_rounds, colors, rounds, num_colors,
                        trace_w, trace_s, trace_cap);
}

/* D2 (Sec. 3.5, Alg. 5 with doPartialColoring false). */
int oracle_color_d2(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                    uint64_t seed, int32_t recolor_degrees, int32_t max_rounds,
                    int32_t *colors, int32_t *rounds, int32_t *num_colors,
                    int64_t *trace_w, int64_t *trace_s, int32_t trace_cap)
{
    if (check_csr(n, row_ptr, col_idx, n) || (n > 0 && !colors) || !rounds || !num_colors)
        return -1;
    graph_t g = { KIND_D2, n, row_ptr, col_idx, NULL, NULL, 0 };
    return color_rounds(&g, seed, recolor_degrees, PRIO_STATIC, max_rounds, colors, rounds,
                        num_colors, trace_w, trace_s, trace_cap);
}

/* PD2 (Sec. 3.6, Alg. 5 with doPartialColoring true): colors the n_cols
 * column vertices; row_ptr/col_idx is the CSR (rows -> columns) and
 * col_ptr/row_idx the CSC (columns -> rows) of the same pattern. */
int oracle_color_pd2(int32_t n_rows, int32_t n_cols,
                     const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *col_ptr, const int32_t *row_idx,
                     uint64_t seed, int32_t recolor_degrees, int32_t max_rounds,
                     int32_t *colors, int32_t *rounds, int32_t *num_colors,
                     int64_t *trace_w, int64_t *trace_s, int32_t trace_cap)
{
    if (check_csr(n_rows, row_ptr, col_idx, n_cols) ||
        check_csr(n_cols, col_ptr, row_idx, n_rows) ||
        (n_cols > 0 && !colors) || !rounds || !num_colors)
        return -1;
    if (n_rows > 0 && n_cols > 0 && row_ptr[n_rows] != col_ptr[n_cols]) return -1;
    graph_t g = { KIND_PD2, n_cols, row_ptr, col_idx, col_ptr, row_idx, 0 };
    return color_rounds(&g, seed, recolor_degrees, PRIO_STATIC, max_rounds, colors, rounds,
                        num_colors, trace_w, trace_s, trace_cap);
}

/* PD2 over all of B (Sec. 3.6: the method colors every vertex of the
 * bipartite graph B(V_s, V_t, E_B)): the n_cols columns are vertices
 * 0 .. n_cols-1 and row i is vertex n_cols + i (that vertex index is the GID
 * in rand(GID)); two vertices conflict when they share a neighbor in B.
 * colors: int32[n_cols + n_rows]. */
int oracle_color_pd2_bipartite(int32_t n_rows, int32_t n_cols,
                               const int32_t *row_ptr, const int32_t *col_idx,
                               const int32_t *col_ptr, const int32_t *row_idx,
                               uint64_t seed, int32_t recolor_degrees, int32_t max_rounds,
                               int32_t *colors, int32_t *rounds, int32_t *num_colors,
                               int64_t *trace_w, int64_t *trace_s, int32_t trace_cap)
{
    if (check_csr(n_rows, row_ptr, col_idx, n_cols) ||
        check_csr(n_cols, col_ptr, row_idx, n_rows) ||
        ((int64_t)n_cols + n_rows > INT32_MAX) ||
        (n_cols + n_rows > 0 && !colors) || !rounds || !num_colors)
        return -1;
    if (n_rows > 0 && n_cols > 0 && row_ptr[n_rows] != col_ptr[n_cols]) return -1;
    graph_t g = { KIND_PD2B, n_cols + n_rows, row_ptr, col_idx, col_ptr, row_idx, n_cols };
    return color_rounds(&g, seed, recolor_degrees, PRIO_STATIC, max_rounds, colors, rounds,
                        num_colors, trace_w, trace_s, trace_cap);
}

/* ---------------------------------------------------------------------- */
/* Checkers.  kind: 1 = D1, 2 = D2, 3 = PD2, 4 = PD2 over all of B (row/col  */
/* arrays as above; for D1/D2 pass n_rows = n_cols = n and NULL CSC).      */
/* ---------------------------------------------------------------------- */
static int make_graph(int32_t kind, int32_t n_rows, int32_t n_cols,
                      const int32_t *row_ptr, const int32_t *col_idx,
                      const int32_t *col_ptr, const int32_t *row_idx, graph_t *g)
{
    if (kind == KIND_D1 || kind == KIND_D2) {
        if (check_csr(n_rows, row_ptr, col_idx, n_rows)) return -1;
        *g = (graph_t){ kind, n_rows, row_ptr, col_idx, NULL, NULL, 0 };
        return 0;
    }
    if (kind == KIND_PD2 || kind == KIND_PD2B) {
        if (check_csr(n_rows, row_ptr, col_idx, n_cols) ||
            check_csr(n_cols, col_ptr, row_idx, n_rows)) return -1;
        *g = (graph_t){ kind, kind == KIND_PD2 ? n_cols : n_cols + n_rows, row_ptr, col_idx,
                        col_ptr, row_idx, n_cols };
        return 0;
    }
    return -1;
}

/*
 * Properness (Sec. 2.1): returns the number of pairs (v, x), x in S(v),
 * with equal colors, plus the number of vertices whose color is < 1.
 * -1 on bad arguments, -2 on allocation failure.
 */
int64_t oracle_count_improper(int32_t kind, int32_t n_rows, int32_t n_cols,
                              const int32_t *row_ptr, const int32_t *col_idx,
                              const int32_t *col_ptr, const int32_t *row_idx,
                              const int32_t *colors)
{
    graph_t g;
    if (make_graph(kind, n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, &g)) return -1;
    int64_t cap = neighborhood_capacity(&g);
    int32_t *buf = malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    if (!buf) return -2;
    int64_t bad = 0;
    for (int32_t v = 0; v < g.n; ++v) {
        if (colors[v] < 1) { bad += 1; continue; }
        int64_t k = neighborhood(&g, v, buf);
        for (int64_t j = 0; j < k; ++j)
            if (colors[buf[j]] == colors[v]) bad += 1;
    }
    free(buf);
    return bad;
}

/*
 * Grundy fixed point: the number of vertices v whose color differs from the
 * smallest positive integer not used in S(v).  Every coloring this method
 * produces has none: a committed color never changes, and when v committed
 * t, every color below t was already held by a committed vertex of S(v).
 */
int64_t oracle_count_non_grundy(int32_t kind, int32_t n_rows, int32_t n_cols,
                                const int32_t *row_ptr, const int32_t *col_idx,
                                const int32_t *col_ptr, const int32_t *row_idx,
                                const int32_t *colors)
{
    graph_t g;
    if (make_graph(kind, n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, &g)) return -1;
    int64_t cap = neighborhood_capacity(&g);
    int32_t *buf = malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    int64_t *seen = calloc((size_t)g.n + 2, sizeof(int64_t));
    if (!buf || !seen) { free(buf); free(seen); return -2; }
    int64_t bad = 0, stamp = 0;
    for (int32_t v = 0; v < g.n; ++v) {
        int64_t k = neighborhood(&g, v, buf);
        stamp += 1;
        for (int64_t j = 0; j < k; ++j) {
            int32_t c = colors[buf[j]];
            if (c > 0 && c <= g.n + 1) seen[c] = stamp;
        }
        int32_t m = 1;
        while (seen[m] == stamp) m += 1;
        if (colors[v] != m) bad += 1;
    }
    free(buf); free(seen);
    return bad;
}
