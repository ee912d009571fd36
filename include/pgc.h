/*
 * pgc.h -- C ABI of the GB300 speculative graph-coloring library.
 *
 * Computes distance-1 (D1), distance-2 (D2) and partial distance-2 (PD2)
 * colorings by the speculate-and-resolve method of Bogle, Slota, Boman,
 * Devine and Rajamanickam, "Parallel Graph Coloring Algorithms for
 * Distributed GPU Environments" (arXiv 2107.00075), on one GPU:
 *
 *   round r: every vertex v on the worklist W_r takes the smallest color not
 *   held by an already-colored vertex of its neighborhood S(v) (first fit,
 *   Alg. 1); then each v in W_r checks S(v) for a vertex u holding the same
 *   color with a higher priority, and if there is one v is uncolored and
 *   goes to W_{r+1} (conflict detection, Alg. 3 for D1 and Alg. 5 for
 *   D2/PD2; priority order of Alg. 4 with the recolorDegrees heuristic of
 *   Sec. 3.3); otherwise v keeps its color.  The loop of Alg. 2 repeats
 *   until the worklist is empty.
 *
 * Priority: key(v) = (deg(v), -h(v), -v) compared lexicographically, with
 * h(v) = splitmix64(seed XOR v) as an unsigned 64-bit number.  So the
 * lower-degree vertex of a conflict is recolored, on equal degree the one
 * with the larger h, on equal h the one with the larger id (Alg. 4).
 * deg(v) is the row length of the input (D1, D2) or the column length of
 * the pattern (PD2), computed once (Sec. 3.3).  PGC_NO_DEGREE_RULE drops
 * the degree term (the paper's "D1-baseline").
 *
 * The form is round-synchronous: within a round the first-fit step sees
 * only colors committed in earlier rounds, and detection reads the round's
 * colors as a snapshot.  The output is therefore a deterministic function
 * of (graph, seed, flags): any launch configuration, batch composition or
 * request mix gives the same colors.  Colors are 1..num_colors; every color
 * in that range is used, and each vertex holds the smallest color absent
 * from its neighborhood (a Grundy coloring).
 *
 * Memory: array arguments may be device memory (used in place) or host
 * memory (staged through library-owned device buffers; the call then also
 * copies the colors back).  The library never frees caller memory.  Scratch
 * (degrees, worklists, masks, counters) is library-owned, allocated on
 * first use per device and reused; pgc_release() frees it.
 *
 * Threads and streams: calls on one device are serialized by the library;
 * `stream` (a cudaStream_t, NULL = the legacy default stream) orders the
 * work after prior work on that stream.  Each call synchronizes `stream`
 * before returning, because it returns rounds and num_colors by value.
 *
 * Errors: every entry point returns a pgc_status; on error the colors
 * array is unspecified.  No C++ exception crosses this boundary.
 * pgc_last_error() gives a message for the last error on the calling thread.
 */
#ifndef PGC_H
#define PGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PGC_OK = 0,
    PGC_ERR_INVALID_ARG = 1,   /* bad sizes/pointers, malformed CSR (PGC_VALIDATE) */
    PGC_ERR_CUDA = 2,          /* a CUDA call failed; see pgc_last_error() */
    PGC_ERR_OOM = 3,           /* device allocation failed */
    PGC_ERR_NO_CONVERGE = 4,   /* max_rounds reached, or a round made no progress */
    PGC_ERR_TIMEOUT = 5,       /* the device round loop ran past timeout_ms */
    PGC_ERR_BUSY = 6,          /* server: admission refused (footprint over budget) */
    PGC_ERR_NOT_FOUND = 7      /* server: unknown request id */
} pgc_status;

/* option flags */
#define PGC_NO_DEGREE_RULE 0x1u  /* priority (-h(v), -v): Alg. 4 with recolorDegrees off */
#define PGC_VALIDATE       0x2u  /* check CSR shape and ids before coloring */
#define PGC_HOST_LOOP      0x4u  /* drive rounds from the host (one sync per round)
                                    instead of the device-side graph loop; enables
                                    per-kernel timing in pgc_profile */
#define PGC_AUTOTUNE       0x8u  /* pgc_color_d1_batch: time a few launch
                                    configurations on the first batch of a size
                                    class, reuse the fastest (in memory, and in
                                    the file named by $PGC_TUNE_FILE if set);
                                    colors never depend on the choice */
#define PGC_ASYNC          0x10u /* D1 (and its batched form): asynchronous
                                    speculation, as KokkosKernels' VB_BIT colors
                                    in place (Sec. 3.2): first fit also avoids the
                                    tentative colors neighbors have already
                                    written in the same round.  Conflicts are
                                    still resolved by Alg. 4 on a snapshot, so the
                                    result is a proper coloring with every color
                                    at most deg(v) + 1, but it depends on timing:
                                    NOT deterministic, and not a Grundy coloring.
                                    The last rounds do not use the core phase. */
#define PGC_PRIORITY_DYNAMIC    0x20u /* D1 (and batched): Alg. 4's degree term is
                                    the "dynamic" degree of Sec. 3.3's closing
                                    paragraph, taken at the start of each round:
                                    v's adjacency entries whose vertex is still
                                    uncolored.  Deterministic (an oracle mode
                                    matches it bit for bit); detection then scans
                                    every neighbor, and the last rounds do not use
                                    the core phase. */
#define PGC_PRIORITY_SATURATION 0x40u /* as PGC_PRIORITY_DYNAMIC, with the
                                    "saturation degree": the distinct colors
                                    1 .. deg(v)+1 held by v's colored neighbors.
                                    The two exclude each other, PGC_ASYNC and
                                    PGC_NO_DEGREE_RULE (PGC_ERR_INVALID_ARG). */

/* Per-kernel timing and per-round trace, filled when non-NULL in pgc_opts. */
#define PGC_MAX_KERNELS 8
typedef struct {
    /* per-round trace, entry r describes round r+1's worklist W_{r+1}:
       w[r] = |W_{r+1}|, s[r] = sum of deg(v), h[r] = sum of the lengths of
       the detection lists (D1: neighbors with higher priority) */
    int64_t *trace_w;          /* host array of trace_cap entries, or NULL */
    int64_t *trace_s;          /* host array of trace_cap entries, or NULL */
    int64_t *trace_h;          /* host array of trace_cap entries, or NULL */
    int32_t trace_cap;
    /* PGC_HOST_LOOP only: CUDA-event time per kernel (ms, summed over
       launches) and launch counts; names in kernel_names[]. */
    int32_t num_kernels;
    double kernel_ms[PGC_MAX_KERNELS];
    int64_t kernel_launches[PGC_MAX_KERNELS];
    const char *kernel_names[PGC_MAX_KERNELS];
    /* PGC_HOST_LOOP only, nullable: every timed launch in order, its kernel
       slot and its time (ms); at most launch_cap entries are written and
       num_launches counts them all. */
    int32_t *launch_slot;
    float *launch_ms;
    int32_t launch_cap;
    int32_t num_launches;
    /* D2/PD2 only, nullable host arrays of trace_cap entries: entry r-1
       describes round r's detection -- the nets it visited (every net, or
       those with a member on the worklist) and their total member count */
    int64_t *trace_nets;
    int64_t *trace_members;
} pgc_profile;

typedef struct {
    uint32_t flags;            /* PGC_* flags above */
    int32_t max_rounds;        /* 0 => n + 1 (an upper bound: each round commits
                                  the worklist vertex with the largest key) */
    int32_t mid_degree;        /* 0 => 64: a vertex whose per-round scan list
                                  (D1: neighbors with higher priority) is longer
                                  gets a warp instead of a thread */
    int32_t hub_degree;        /* 0 => 16384: longer lists get a thread block */
    int32_t block;             /* 0 => default threads per block (128..1024) */
    int32_t grid_per_sm;       /* 0 => occupancy-derived blocks per SM */
    int32_t timeout_ms;        /* 0 => 60000: device loop gives up after this */
    int32_t tail_vertices;     /* D1: once the worklist has at most this many
                                  vertices, the remaining rounds run on the
                                  subgraph the worklist induces, in one
                                  cooperative launch with grid barriers;
                                  0 => 4096, < 0 => never */
    pgc_profile *profile;      /* nullable */
} pgc_opts;

/* Initialise an options struct to defaults. */
void pgc_opts_init(pgc_opts *opts);

/*
 * Distance-1 coloring (Sec. 2.1; Sec. 3.2 with Alg. 3 and 4).
 *   n        number of vertices, >= 0
 *   row_ptr  int32[n+1], CSR offsets, row_ptr[0] = 0, non-decreasing
 *   col_idx  int32[row_ptr[n]], neighbor ids in [0, n); the graph must be
 *            symmetric (u in N(v) iff v in N(u)); self-loops are skipped as
 *            neighbors but count in the degree; duplicates count in the degree
 *   seed     priority seed for h(v)
 *   colors   int32[n], output, fully overwritten with 1..num_colors
 *   rounds   host int32*, output: number of rounds executed (0 when n == 0)
 *   num_colors host int32*, output: the largest color (0 when n == 0)
 *   opts     nullable
 *   stream   cudaStream_t or NULL
 */
pgc_status pgc_color_d1(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                        uint64_t seed, int32_t *colors, int32_t *rounds,
                        int32_t *num_colors, const pgc_opts *opts, void *stream);

/*
 * Distance-2 coloring (Sec. 2.1; Sec. 3.5 with Alg. 5, doPartialColoring
 * false): every two vertices joined by a path of one or two edges get
 * different colors.  Arguments, layout and ownership as pgc_color_d1; the
 * priority degree is the row length (1-hop degree).  Colors up to 4096 are
 * supported (PGC_ERR_NO_CONVERGE beyond).  Detection is net based: the
 * closed neighborhood N[u] of every vertex u is a net (Sec. 3.5, NB_BIT).
 */
pgc_status pgc_color_d2(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                        uint64_t seed, int32_t *colors, int32_t *rounds,
                        int32_t *num_colors, const pgc_opts *opts, void *stream);

/*
 * Partial distance-2 coloring of the columns of an n_rows x n_cols pattern
 * (Sec. 2.1, Sec. 3.6; Alg. 5 with doPartialColoring true): two columns that
 * have an entry in a common row get different colors; rows get no color.
 *   row_ptr int32[n_rows+1], col_idx int32[nnz]  CSR of the pattern
 *           (column ids in [0, n_cols))
 *   col_ptr int32[n_cols+1], row_idx int32[nnz]  CSC of the same pattern
 *           (row ids in [0, n_rows)); row_ptr[n_rows] must equal
 *           col_ptr[n_cols], else PGC_ERR_INVALID_ARG
 *   colors  int32[n_cols], output
 * The priority degree of a column is its CSC length.  Colors up to 4096.
 */
pgc_status pgc_color_pd2(int32_t n_rows, int32_t n_cols, const int32_t *row_ptr,
                         const int32_t *col_idx, const int32_t *col_ptr,
                         const int32_t *row_idx, uint64_t seed, int32_t *colors,
                         int32_t *rounds, int32_t *num_colors, const pgc_opts *opts,
                         void *stream);

/*
 * Partial distance-2 coloring of EVERY vertex of the bipartite graph
 * B(V_s, V_t, E_B) of the pattern, as the paper's PD2 does (Sec. 3.6: it
 * colors all of B; Alg. 5 with doPartialColoring true, two-hop conflicts
 * only): two columns sharing a row differ, and two rows sharing a column
 * differ; a row and a column never conflict.  Arrays as pgc_color_pd2.
 *   colors  int32[n_cols + n_rows], output: the columns' colors at [0, n_cols),
 *           row i's color at n_cols + i
 * Vertex index = GID in rand(GID) (Alg. 4): column j is j, row i is
 * n_cols + i; the priority degree is the vertex's degree in B (a column's CSC
 * length, a row's CSR length).  The columns therefore get exactly the colors
 * pgc_color_pd2 gives them; rounds and num_colors cover both sides.
 * Requires 2 * nnz < 2^31 and n_rows + n_cols < 2^31 - 1.  Colors up to 4096.
 */
pgc_status pgc_color_pd2_bipartite(int32_t n_rows, int32_t n_cols, const int32_t *row_ptr,
                                   const int32_t *col_idx, const int32_t *col_ptr,
                                   const int32_t *row_idx, uint64_t seed, int32_t *colors,
                                   int32_t *rounds, int32_t *num_colors, const pgc_opts *opts,
                                   void *stream);

/*
 * Batched distance-1 coloring of G independent graphs in one launch (the
 * batched form of Sec. 3.2; the paper has no batched API).  Graph g has
 * n_g = vtx_off[g+1] - vtx_off[g] vertices and m_g = nnz_off[g+1] - nnz_off[g]
 * adjacency entries; ids, degrees and the priority hash are graph-local, so
 * each graph's colors, rounds and color count equal those of pgc_color_d1 on
 * that graph alone with the same seed and flags.
 *   vtx_off, nnz_off int64[G+1], prefix offsets starting at 0
 *   row_ptr int32[N + G]: graph g's local row_ptr (n_g + 1 entries, from 0
 *           to m_g) at row_ptr[vtx_off[g] + g ...]   (N = vtx_off[G] < 2^31)
 *   col_idx int32[nnz_off[G]]: graph g's local ids in [0, n_g) at
 *           col_idx[nnz_off[g] ...]; each graph symmetric
 *   colors  int32[N] output (graph g at colors[vtx_off[g] ...])
 *   rounds_per_g, ncolors_per_g  int32[G] outputs (0 for empty graphs)
 *   rounds  host int32*, nullable: rounds of the whole launch (the maximum
 *           over the graphs)
 * Any array may be host or device memory.  PGC_AUTOTUNE applies here.
 */
pgc_status pgc_color_d1_batch(int32_t G, const int64_t *vtx_off, const int64_t *nnz_off,
                              const int32_t *row_ptr, const int32_t *col_idx, uint64_t seed,
                              int32_t *colors, int32_t *rounds_per_g, int32_t *ncolors_per_g,
                              int32_t *rounds, const pgc_opts *opts, void *stream);

/*
 * pgc_color_d1_noalloc -- pgc_color_d1 for callers that must not have the
 * library allocate device memory (the paper has no counterpart; this is a
 * deployment variant).  Callers whose device memory is owned by another
 * allocator, or who cannot accept the device-wide synchronisation of
 * cudaFree, get the same colors, rounds and color count as pgc_color_d1 with
 * no cudaMalloc, cudaFree or other allocating call.  All scratch is one
 * fixed array of about 6.5 MB in device memory that every GPU loading the
 * library keeps until the process exits.
 *   Limits: n <= 32768 and row_ptr[n] <= 524288; larger inputs are rejected
 *           with PGC_ERR_INVALID_ARG before any work is launched.
 *   row_ptr, col_idx, colors: DEVICE memory only (host pointers are rejected,
 *           since staging them would need an allocation); layout as
 *           pgc_color_d1.  rounds, num_colors: host outputs.
 *   flags:  PGC_NO_DEGREE_RULE or 0.  The other options take pgc_color_d1's
 *           defaults (the same detection tiers), except that the last rounds
 *           do not use the core phase: every round runs the per-round kernels,
 *           which give the same colors.
 *   The first call on a device looks up the array's device address (once per
 *           device and CUDA context, with that device current); make that
 *           first call before any stream capture.
 *   Every call reuses the same array and the array keeps the previous call's
 *           contents; the call clears what must start at zero.  Two calls
 *           whose GPU work overlapped would race on the array: calls take a
 *           process-wide lock and synchronize `stream` before returning (on
 *           error too, once work was enqueued), so calls made through this
 *           function never overlap.
 */
pgc_status pgc_color_d1_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                uint64_t seed, int32_t *colors, int32_t *rounds,
                                int32_t *num_colors, uint32_t flags, void *stream);

/*
 * Coloring server with continuous batching (the served form; the paper has
 * no serving API).  Any host thread submits distance-1 graphs or partial
 * distance-2 patterns; one engine thread admits them first come first
 * served, at round-loop boundaries, when an execution slot and room for the
 * request's device footprint (inputs + colors + scratch) in the server's
 * HBM arena are both free.  Each active request runs the device-side round
 * loop on its own stream, so requests overlap on the GPU; CSR and color
 * state stay on the device for all rounds.  Colors, rounds and color counts
 * equal those of pgc_color_d1 / pgc_color_pd2 on the request alone.
 *
 * Buffers passed to submit belong to the caller and must stay valid and
 * unchanged until the request is reported done (wait, or poll with done=1).
 * Inputs are read with cudaMemcpyDefault (host or device memory; pinned host
 * memory keeps the upload asynchronous); colors may be host or device memory.
 */
typedef struct pgc_server pgc_server;

typedef struct {
    int32_t status;            /* pgc_status of the request */
    int32_t rounds;
    int32_t num_colors;
    int32_t reserved;
    int64_t t_submit_ns;       /* steady-clock stamps: submit, admission, done */
    int64_t t_admit_ns;
    int64_t t_done_ns;
    int64_t footprint_bytes;   /* device bytes the request held while active */
} pgc_request_info;

typedef struct {
    int64_t submitted, completed, rejected;
    int32_t active, queued;
    int64_t bytes_in_use, peak_bytes, budget_bytes;
    int32_t max_active_seen;
    int32_t reserved;
} pgc_server_counters;

/* A server on the current device with an HBM arena of hbm_budget_bytes
   (allocated here) and at most max_active concurrent requests (1..256). */
pgc_status pgc_server_create(size_t hbm_budget_bytes, int32_t max_active, pgc_server **out);

/* Queue a distance-1 request (CSR as in pgc_color_d1; colors: int32[n]).
   PGC_ERR_BUSY if its footprint exceeds the whole budget. */
pgc_status pgc_server_submit_d1(pgc_server *srv, int32_t n, const int32_t *row_ptr,
                                const int32_t *col_idx, uint64_t seed, int32_t *colors,
                                int64_t *req_id);

/* Queue a partial distance-2 request (arrays as in pgc_color_pd2, host
   memory; colors: int32[n_cols]). */
pgc_status pgc_server_submit_pd2(pgc_server *srv, int32_t n_rows, int32_t n_cols,
                                 const int32_t *row_ptr, const int32_t *col_idx,
                                 const int32_t *col_ptr, const int32_t *row_idx, uint64_t seed,
                                 int32_t *colors, int64_t *req_id);

/* done = 1 once finished; the request's info is then returned and its id
   released (later calls with it give PGC_ERR_NOT_FOUND). */
pgc_status pgc_server_poll(pgc_server *srv, int64_t req_id, int32_t *done,
                           pgc_request_info *info);

/* Block until the request is done (timeout_ms < 0: no limit; otherwise
   PGC_ERR_TIMEOUT and the request stays pending).  Releases the id. */
pgc_status pgc_server_wait(pgc_server *srv, int64_t req_id, int32_t timeout_ms,
                           pgc_request_info *info);

pgc_status pgc_server_stats(pgc_server *srv, pgc_server_counters *out);

/* Finishes every queued and active request, then frees the server. */
pgc_status pgc_server_destroy(pgc_server *srv);

/* Message for the last error on this thread ("" if none). */
const char *pgc_last_error(void);

/* Name of a status code. */
const char *pgc_status_string(pgc_status s);

/* Free library-owned device scratch on the current device. */
pgc_status pgc_release(void);

/* Library version string. */
const char *pgc_version(void);

/*
 * Test hooks: fault injection for the failure-path tests (no production use;
 * the paper has no counterpart).  Both act process-wide on later calls.
 *
 * pgc_test_fail_alloc(after): the device allocation the library attempts
 *   after `after` further successful ones fails as if the device were out of
 *   memory, once; the call that meets it returns PGC_ERR_OOM having freed
 *   the scratch of that engine.  after < 0 disarms.
 * pgc_test_core_barrier(polls, slow_block, slow_us): the grid barrier of the
 *   D1 core loop gives up after `polls` polls (0: the default, about one
 *   second), and block `slow_block` of the core loop (-1: none) reaches its
 *   first barrier `slow_us` microseconds late (at most 2 s, else
 *   PGC_ERR_INVALID_ARG).  With a late block and a short poll limit the
 *   waiting blocks give up, and the coloring returns PGC_ERR_TIMEOUT ("a
 *   grid barrier of the core loop timed out") with the context intact; every
 *   wait stays bounded.
 */
pgc_status pgc_test_fail_alloc(int32_t after);
pgc_status pgc_test_core_barrier(uint32_t polls, int32_t slow_block, uint32_t slow_us);

#ifdef __cplusplus
}
#endif

#endif /* PGC_H */
