// d1_engine.cuh -- distance-1 coloring engine (kernels + host driver),
// templated on the graph view so that one engine colors a single graph
// (SingleView) or a flattened batch of independent graphs (BatchView).
//
// Method (Bogle et al., Sec. 3.2-3.3, Alg. 1-4), round-synchronous form:
//   round 1       every vertex holds tentative color 1; detection decides;
//   round r >= 2  assign: each worklist vertex takes the smallest color not
//                 committed in its neighborhood (first fit, Alg. 1);
//                 detect: a worklist vertex loses if a neighbor holds the
//                 same color and has priority (Alg. 3 + Alg. 4); winners
//                 commit, losers form the next worklist.
//
// How the GPU computes exactly that, with less work than re-reading every
// worklist vertex's adjacency each round:
//   * Detection only needs the neighbors that have priority over v (Alg. 4
//     recolors the lower-priority end of a conflict), so setup builds, per
//     vertex, the list H(v) = {u in N(v) : key(u) > key(v)}.  Every edge is
//     in exactly one list, and hubs -- which stay on the worklist for many
//     rounds -- have short lists.  A committed neighbor never holds v's
//     tentative color (first fit excluded it), so v loses iff some u in H(v)
//     currently holds v's tentative color.
//   * First fit reads a per-vertex set of forbidden colors: one 64-bit word
//     for colors 1..64 and, for vertices of degree >= 64, an overflow bitmap
//     up to color deg(v)+1 (a first-fit color never exceeds deg(v)+1).  When
//     a vertex commits color c it sets bit c in its neighbors' sets ("push");
//     each vertex pushes once, so the total push work is one pass over the
//     adjacency.
//
// Color encoding in col[]: > 0 committed; < 0 tentative (-t) for a vertex
// on the current worklist.  Every uncolored vertex is on the worklist, so
// |col[u]| is u's current color during detection; a winner flips its own
// sign in place without disturbing concurrent readers.
//
// Work decomposition (no result depends on it):
//   detect, by |H(v)| (defaults; options mid_degree / hub_degree): up to 64
//   entries one thread per vertex; up to 16384 one warp per vertex; longer
//   lists one thread block per vertex.  A loser stops at the step that finds
//   its conflict.  In round 1 every vertex holds color 1, so v loses exactly
//   when H(v) is not empty and no list is read.  Losers keep their worklist
//   entry: they are re-appended by source index (the list counters are the
//   hottest atomics of the kernel).  Setup cuts long rows into 512-entry
//   items and push into 128-entry items, one warp each.
// The round loop runs on the device: a CUDA graph with a conditional WHILE
// node around {assign, detect, push}; the last block of detect updates the
// round state and sets the loop condition.  Once the worklist has at most
// tail_w vertices the remaining rounds run in the core phase: on the
// subgraph the worklist induces, in one cooperative launch whose blocks
// meet at (bounded) grid barriers -- the only waits in the engine.
//
// Batches: graph g owns global vertices [vtx_off[g], vtx_off[g+1]); ids,
// the priority hash and degrees are graph-local, so every graph is colored
// exactly as it would be alone; the rounds of all graphs run together and a
// graph simply has no worklist vertices once it is done.
#pragma once
#include "runtime.h"
#include "device_common.cuh"

#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>
#include <type_traits>
#include <unordered_map>

namespace pgc {
std::vector<std::function<void()>>& release_hooks();

namespace d1 {

// ---------------------------------------------------------------------------
// graph views
// ---------------------------------------------------------------------------
// One graph: int32 CSR.
struct SingleView {
    const int* rp;
    const int* ci;
    __device__ __forceinline__ int graph(int) const { return 0; }
    __device__ __forceinline__ int base(int) const { return 0; }
    __device__ __forceinline__ void row(int v, int, long long& b, int& d) const {
        const int r0 = __ldg(rp + v);
        b = r0;
        d = __ldg(rp + v + 1) - r0;
    }
    __device__ __forceinline__ int nbr(long long e, int) const { return __ldg(ci + e); }
    // start of v's row relative to its graph, and the absolute start from it
    __device__ __forceinline__ void local_row(int v, int, int& r0, int& d) const {
        r0 = __ldg(rp + v);
        d = __ldg(rp + v + 1) - r0;
    }
    __device__ __forceinline__ long long begin(int, int r0) const { return r0; }
};

// A batch: graph-local row_ptr blocks (n_g + 1 entries each) and graph-local
// column ids; int64 offsets into the flattened arrays.
struct BatchView {
    const long long* vtx_off;
    const long long* nnz_off;
    const int* rp;
    const int* ci;
    const int* gid;   // graph of each global vertex
    __device__ __forceinline__ int graph(int v) const { return __ldg(gid + v); }
    __device__ __forceinline__ int base(int g) const { return (int)__ldg(vtx_off + g); }
    __device__ __forceinline__ void row(int v, int g, long long& b, int& d) const {
        const int r0 = __ldg(rp + v + g);
        b = __ldg(nnz_off + g) + r0;
        d = __ldg(rp + v + g + 1) - r0;
    }
    __device__ __forceinline__ int nbr(long long e, int base_g) const {
        return base_g + __ldg(ci + e);
    }
    __device__ __forceinline__ void local_row(int v, int g, int& r0, int& d) const {
        r0 = __ldg(rp + v + g);
        d = __ldg(rp + v + g + 1) - r0;
    }
    __device__ __forceinline__ long long begin(int g, int r0) const {
        return __ldg(nnz_off + g) + r0;
    }
};

constexpr int kBuildS = 32;     // setup: degree up to this: one thread
constexpr int kBuildM = 512;    // setup: degree up to this: one warp
constexpr int kBuildItem = 512; // setup: adjacency items of this length
constexpr int kPushItem = 128;  // push: adjacency items of this length
constexpr int kInlinePush = 32; // S-tier winners up to this degree push inline

enum : int { ST_OK = 0, ST_NO_PROGRESS = 1, ST_MAX_ROUNDS = 2, ST_TIMEOUT = 3, ST_BARRIER = 4 };

struct State {
    int round;        // round being executed (1-based)
    int done;         // 1 once the loop has ended
    int status;       // ST_*
    int max_color;
    int ns[2];        // S-tier worklist sizes per parity
    int nm[2];        // M-tier worklist sizes
    int nl[2];        // L-tier worklist sizes
    int bs, bm, bc;   // setup: vertices (S, M) and items (C) per degree class
    int push_cnt;     // push work items queued this round
    unsigned blocks_done;
    unsigned l_next;  // dynamic index into the L-tier worklist
    int tail;         // 1: the graph loop handed the remaining rounds to the core phase
    unsigned bar_count;         // core loop grid barrier: arrivals
    unsigned bar_gen;           // core loop grid barrier: generation
    int bar_timeout;            // core loop: a barrier wait gave up
    unsigned long long s_next;  // sum of degrees of the next worklist
    unsigned long long h_next;  // sum of |H(v)| over the next worklist
    unsigned long long h_first; // sum of |H(v)| over all vertices
    unsigned long long t0;      // globaltimer at start
    int core_k;       // core phase: vertices of the induced subgraph
    int core_par;     // core phase: parity whose worklist buffers hold its arrays
    int core_cur;     // core phase: size of the current local worklist
    int core_nxt;     // core phase: appends to the next local worklist
    int core_win;     // core phase: winners of the current round
};

template <class V>
struct Problem {
    V g;
    int* col;
    int* deg;
    int* hlen;
    int* hadj;                 // H(v) stored at hadj[row start of v ...]
    unsigned long long* bm0;   // forbidden colors 1..64, one word per vertex
    unsigned* bmx;             // forbidden colors 65..deg+1 (deg >= 64)
    unsigned* live;            // bit v set while v is uncolored
    // worklists per parity; an entry is {v, |H(v)|, deg(v), row start of v
    // within its graph}, so a scan needs no further lookup to begin
    int4* ws[2];               // S tier
    int4* wm[2];               // M tier
    int4* wl[2];               // L tier
    int2* items;               // setup: (vertex, item) list for long rows
    int2* push_q;              // (vertex, item) push work
    int* g_rounds;             // batch: rounds per graph (nullable)
    int* g_colors;             // batch: colors per graph (nullable)
    long long* trace_w;
    long long* trace_s;
    long long* trace_h;
    State* st;
    unsigned long long seed;
    unsigned long long timeout_ns;
    long long nnz;
    int trace_cap;
    int n;
    int use_deg;
    int async_mode;    // PGC_ASYNC: first fit also avoids tentative colors written this round
    int prio_mode;     // 0: static degree; 1: dynamic degree; 2: saturation degree
    int* prio;         // prio_mode != 0: each vertex's priority this round
    int max_rounds;
    int det_s;
    int det_m;
    int tail_w;        // hand over to the core phase once the worklist is this small (0: never)
    unsigned bar_polls;   // core loop: grid-barrier polls before giving up
    int slow_block;       // test hook: this core-loop block starts late (-1: none)
    unsigned slow_ns;     // ... by this much
};

// key(u) > key(v) for u, v of the same graph (hash of graph-local ids),
// hashing only when the degree term does not decide.
__device__ __forceinline__ bool higher(int du, int u, int dv, uint64_t hv, int v, int base,
                                       unsigned long long seed, bool use_deg) {
    if (use_deg && du != dv) return du > dv;
    const uint64_t hu = prio_hash(seed, (uint32_t)(u - base));
    if (hu != hv) return hu < hv;
    return u < v;
}

__device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }


__device__ __forceinline__ long long bm_offset(long long row_begin, int v) {
    return (row_begin >> 5) + v;
}

// Forbid color c for u (a vertex of graph g).  Setting bits of an already
// colored vertex is harmless (its set is never read again), so colors 1..64
// need no check and the update is a fire-and-forget reduction.
// VARYING (a priority that changes each round): also keep u's priority for
// the next round: the dynamic degree drops by one per adjacency entry of a
// newly colored neighbor; the saturation degree grows when c is a color u
// had not yet seen among its colored neighbors and c <= deg(u) + 1.
template <bool VARYING, class V>
__device__ __forceinline__ void push_color_live(const Problem<V>& P, int u, int g, int c) {
    if (VARYING && P.prio_mode == 1) atomicSub(P.prio + u, 1);
    if (c <= 64) {
        const unsigned long long bit = 1ull << (c - 1);
        if (VARYING && P.prio_mode == 2) {
            const unsigned long long old = atomicOr(P.bm0 + u, bit);
            if (!(old & bit) && c - 1 <= P.deg[u]) atomicAdd(P.prio + u, 1);
        } else {
            atomicOr(P.bm0 + u, bit);
        }
        return;
    }
    long long bu;
    int du;
    P.g.row(u, g, bu, du);
    if (c - 1 > du) return;   // u's own first fit never reaches c
    const int b = c - 65;
    if (VARYING && P.prio_mode == 2) {
        const unsigned old = atomicOr(P.bmx + bm_offset(bu, u) + (b >> 5), 1u << (b & 31));
        if (!(old & (1u << (b & 31)))) atomicAdd(P.prio + u, 1);
    } else {
        atomicOr(P.bmx + bm_offset(bu, u) + (b >> 5), 1u << (b & 31));
    }
}
template <class V>
__device__ __forceinline__ void push_color(const Problem<V>& P, int u, int g, int c) {
    // most neighbors of a late winner are colored already: skip them
    if ((P.live[u >> 5] >> (u & 31)) & 1u) {
        if (P.prio_mode) push_color_live<true>(P, u, g, c);
        else push_color_live<false>(P, u, g, c);
    }
}

// Batch bookkeeping: arr[g] = max(arr[g], val) over the lanes with pred,
// one atomic per (warp, graph).  All 32 lanes call.
__device__ __forceinline__ void graph_max(int* arr, bool pred, int g, int val) {
    const int key = pred ? g : -1 - (int)lane_id();
    const unsigned peers = __match_any_sync(kFullMask, key);
    const int m = __reduce_max_sync(peers, pred ? val : 0);
    if (pred && (int)lane_id() == __ffs(peers) - 1) atomicMax(arr + g, m);
}

// ---------------------------------------------------------------------------
// setup 1: degrees, tentative color 1, empty forbidden sets, degree classes
// ---------------------------------------------------------------------------
template <class V>
__global__ void d1_classify(const Problem<V>* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem<V>& P = *Pp;
    State* st = P.st;
    const int warp = threadIdx.x >> 5;
    int4* sm4 = reinterpret_cast<int4*>(smem);
    WarpAppend4 as = {sm4 + warp * 2 * kAppend4Slots, 0},
                am = {sm4 + warp * 2 * kAppend4Slots + kAppend4Slots, 0};
    const int n = P.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < n;
         wbase += stride) {
        const long long i = wbase + lane_id();
        const bool valid = i < n;
        int d = -1, r0 = 0;
        if (valid) {
            const int v = (int)i;
            const int g = P.g.graph(v);
            P.g.local_row(v, g, r0, d);
            const long long b = P.g.begin(g, r0);
            P.deg[v] = d;
            P.col[v] = P.async_mode ? 0 : -1;
            if (P.prio_mode) P.prio[v] = P.prio_mode == 1 ? d : 0;
            P.hlen[v] = 0;
            P.bm0[v] = 0ull;
            if (d >= 64) {
                unsigned* w = P.bmx + bm_offset(b, v);
                for (int k = 0; k <= (d >> 5); ++k) w[k] = 0u;
            }
            if (d > kBuildM) {
                const int nit = ceil_div(d, kBuildItem);
                const int base = atomicAdd(&st->bc, nit);
                for (int k = 0; k < nit; ++k) P.items[base + k] = make_int2(v, k);
            }
        }
        const unsigned vm = __ballot_sync(kFullMask, valid);
        if (lane_id() == 0) P.live[wbase >> 5] = vm;   // wbase is a multiple of 32
        const int4 ent = make_int4((int)i, 0, d, r0);
        wa4_push(as, valid && d <= kBuildS, ent, P.ws[0], &st->bs);
        wa4_push(am, valid && d > kBuildS && d <= kBuildM, ent, P.wm[0], &st->bm);
    }
    wa4_flush(as, P.ws[0], &st->bs);
    wa4_flush(am, P.wm[0], &st->bm);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->round = 1;
        st->t0 = global_ns();
        if (P.trace_cap > 0) {
            P.trace_w[0] = n;
            P.trace_s[0] = P.nnz;
        }
    }
}

// ---------------------------------------------------------------------------
// setup 2: H(v) = neighbors with higher priority, stored at v's row start.
// Only the vertices in [lo, hi) (one launch may cover a part of the graph,
// so the rest of the adjacency can still be on its way to the device).
// ---------------------------------------------------------------------------
template <class V>
__global__ void __maxnreg__(40) d1_build(const Problem<V>* __restrict__ Pp, int lo, int hi) {
    const Problem<V>& P = *Pp;
    State* st = P.st;
    const int* __restrict__ dg = P.deg;
    const unsigned long long seed = P.seed;
    const bool use_deg = P.use_deg != 0;
    const int lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + warp, nw = gridDim.x * wpb;
    const int nS = st->bs, nM = st->bm, nC = st->bc;
    // priorities that change each round: the lists hold every neighbor
    const bool all = P.prio_mode != 0;
    unsigned long long my_h = 0ull;

    // long rows: one warp per 512-entry item; positions by atomicAdd
    for (int q = gw; q < nC; q += nw) {
        const int2 it = P.items[q];
        const int v = it.x;
        if (v < lo || v >= hi) continue;
        const int g = P.g.graph(v), base = P.g.base(g);
        long long beg;
        int d;
        P.g.row(v, g, beg, d);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        const int e0 = it.y * kBuildItem, e1 = min(d, e0 + kBuildItem);
        for (int b0 = e0; b0 < e1; b0 += 32) {
            const int e = b0 + lane;
            int u = -1;
            bool keep = false;
            if (e < e1) {
                u = P.g.nbr(beg + e, base);
                keep = u != v && (all || higher(__ldg(dg + u), u, d, hv, v, base, seed, use_deg));
            }
            const unsigned m = __ballot_sync(kFullMask, keep);
            if (m == 0u) continue;
            int pos = 0;
            if (lane == 0) pos = atomicAdd(P.hlen + v, __popc(m));
            pos = __shfl_sync(kFullMask, pos, 0);
            if (keep) P.hadj[beg + pos + __popc(m & ((1u << lane) - 1u))] = u;
            if (lane == 0) my_h += (unsigned long long)__popc(m);
        }
    }

    // medium rows: one warp per vertex, ordered compaction by ballot
    for (int i = gw; i < nM; i += nw) {
        const int4 ent = P.wm[0][i];
        const int v = ent.x, d = ent.z;
        if (v < lo || v >= hi) continue;
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, ent.w);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        int pos = 0;
        for (int b0 = 0; b0 < d; b0 += 32) {
            const int e = b0 + lane;
            int u = -1;
            bool keep = false;
            if (e < d) {
                u = P.g.nbr(beg + e, base);
                keep = u != v && (all || higher(__ldg(dg + u), u, d, hv, v, base, seed, use_deg));
            }
            const unsigned m = __ballot_sync(kFullMask, keep);
            if (keep) P.hadj[beg + pos + __popc(m & ((1u << lane) - 1u))] = u;
            pos += __popc(m);
        }
        if (lane == 0) {
            P.hlen[v] = pos;
            my_h += (unsigned long long)pos;
        }
    }

    // short rows: one thread per vertex
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nS; i += stride) {
        const int4 ent = P.ws[0][i];
        const int v = ent.x, d = ent.z;
        if (v < lo || v >= hi) continue;
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, ent.w);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        int pos = 0;
        for (int e0 = 0; e0 < d; e0 += 4) {
            int u[4], du[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) u[j] = e0 + j < d ? P.g.nbr(beg + e0 + j, base) : v;
#pragma unroll
            for (int j = 0; j < 4; ++j) du[j] = u[j] != v ? __ldg(dg + u[j]) : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (u[j] != v && (all || higher(du[j], u[j], d, hv, v, base, seed, use_deg)))
                    P.hadj[beg + pos++] = u[j];
        }
        P.hlen[v] = pos;
        my_h += (unsigned long long)pos;
    }
    my_h = warp_sum(my_h);
    if (lane == 0 && my_h) atomicAdd(&st->h_first, my_h);
}

// Append v to the worklist of its H-list tier (all 32 lanes call).
struct TierAppend {
    WarpAppend4 s, m;
};

__device__ __forceinline__ TierAppend tier_appender(int* smem) {
    int4* sm4 = reinterpret_cast<int4*>(smem);
    const int warp = threadIdx.x >> 5;
    return TierAppend{{sm4 + warp * 2 * kAppend4Slots, 0},
                      {sm4 + warp * 2 * kAppend4Slots + kAppend4Slots, 0}};
}

// e = {v, |H(v)|, deg(v), local row start}
template <class V>
__device__ __forceinline__ void tier_push(const Problem<V>& P, TierAppend& a, bool pred, int4 e,
                                          int p) {
    State* st = P.st;
    const int hl = e.y;
    wa4_push(a.s, pred && hl <= P.det_s, e, P.ws[p], &st->ns[p]);
    wa4_push(a.m, pred && hl > P.det_s && hl <= P.det_m, e, P.wm[p], &st->nm[p]);
    if (pred && hl > P.det_m) P.wl[p][atomicAdd(&st->nl[p], 1)] = e;
}

// ---------------------------------------------------------------------------
// setup 3: round-1 worklists by |H(v)|
// ---------------------------------------------------------------------------
template <class V>
__global__ void d1_tier(const Problem<V>* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem<V>& P = *Pp;
    TierAppend a = tier_appender(smem);
    const int n = P.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < n;
         wbase += stride) {
        const long long i = wbase + lane_id();
        const bool valid = i < n;
        int4 e = make_int4((int)i, 0, 0, 0);
        if (valid) {
            int r0, d;
            P.g.local_row((int)i, P.g.graph((int)i), r0, d);
            e = make_int4((int)i, P.hlen[i], d, r0);
        }
        tier_push(P, a, valid, e, 1);
    }
    wa4_flush(a.s, P.ws[1], &P.st->ns[1]);
    wa4_flush(a.m, P.wm[1], &P.st->nm[1]);
}

// ---------------------------------------------------------------------------
// assign: first fit from the forbidden-color set
// ---------------------------------------------------------------------------
// First fit for worklist entry e = {v, |H(v)|, deg(v), local row start}.
// The forbidden set only grows from round to round (committed colors are
// final), so the first free color never decreases: the scan starts at the
// previous round's tentative color, -col[v].
template <class V>
__device__ __forceinline__ int first_fit(const Problem<V>& P, int4 e, int tp) {
    const int v = e.x;
    int t;
    unsigned long long w0 = ~0ull;
    if (tp <= 64) w0 = P.bm0[v];
    if (w0 != ~0ull) {
        t = __ffsll((long long)~w0);
    } else {   // colors 1..64 all taken: deg(v) >= 64, scan the overflow bitmap
        const int g = P.g.graph(v);
        const long long b = P.g.begin(g, e.w);
        const int words = (e.z >> 5) + 1;
        const unsigned* w = P.bmx + bm_offset(b, v);
        // four words per step, from the word that holds the previous color
        int k = tp > 64 ? (tp - 65) >> 5 : 0;
        for (;;) {
            unsigned x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = k + j < words ? w[k + j] : 0u;
            int j = 0;
            unsigned y = x[0];
            if (y == kFullMask) {
                j = 1;
                y = x[1];
                if (y == kFullMask) {
                    j = 2;
                    y = x[2];
                    if (y == kFullMask) {
                        j = 3;
                        y = x[3];
                    }
                }
            }
            if (y != kFullMask || k + 4 >= words) {
                t = 64 + (k + j) * 32 + __ffs(~y);
                break;
            }
            k += 4;
        }
    }
    return t;
}

template <class V>
__device__ __forceinline__ void assign_phase(const Problem<V>& P) {
    State* st = P.st;
    const int cp = *(volatile int*)&st->round & 1;
    const int n0 = st->ns[cp], n1 = st->nm[cp], n2 = st->nl[cp];
    const long long total = (long long)n0 + n1 + n2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int4 e = i < n0 ? P.ws[cp][i]
                     : (i < n0 + n1 ? P.wm[cp][i - n0] : P.wl[cp][i - n0 - n1]);
        P.col[e.x] = -first_fit(P, e, -P.col[e.x]);
    }
}

// Asynchronous speculation (PGC_ASYNC; the in-place coloring of VB_BIT in
// KokkosKernels, Sec. 3.2): first fit avoids the committed colors of N(v)
// and also every tentative color a neighbor has already written in this
// round (losers were reset to 0 at the end of the previous round, so a
// negative color is this round's).  One warp per worklist vertex scans its
// adjacency once per 64-color window.  Which tentative colors a vertex sees
// depends on timing, so the result is a proper coloring but not a
// deterministic one; detection is the same snapshot rule as always.
template <class V>
__device__ __forceinline__ void assign_async_phase(const Problem<V>& P) {
    State* st = P.st;
    const int cp = *(volatile int*)&st->round & 1;
    const int n0 = st->ns[cp], n1 = st->nm[cp], n2 = st->nl[cp];
    const long long total = (long long)n0 + n1 + n2;
    const int lane = lane_id(), wpb = blockDim.x >> 5;
    const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * wpb;
    for (long long i = gw; i < total; i += nw) {
        const int4 e = i < n0 ? P.ws[cp][i]
                     : (i < n0 + n1 ? P.wm[cp][i - n0] : P.wl[cp][i - n0 - n1]);
        const int v = e.x, d = e.z;
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, e.w);
        int t = 0;
        for (int w = 0; t == 0; ++w) {
            unsigned long long f = 0ull;
            if (w == 0) {
                f = P.bm0[v];
            } else {   // overflow bitmap words for colors 64w+1 .. 64w+64
                const unsigned* x = P.bmx + bm_offset(beg, v);
                const int k = 2 * (w - 1), words = (d >> 5) + 1;
                const unsigned lo = k < words ? x[k] : 0u;
                const unsigned hi = k + 1 < words ? x[k + 1] : 0u;
                f = ((unsigned long long)hi << 32) | lo;
            }
            unsigned long long tb = 0ull;
            for (int j = lane; j < d; j += 32) {
                const int u = P.g.nbr(beg + j, base);
                const int c = u != v ? *(volatile const int*)(P.col + u) : 0;
                if (c < 0) {
                    const int b = -c - 1 - 64 * w;
                    if (b >= 0 && b < 64) tb |= 1ull << b;
                }
            }
            const unsigned tlo = __reduce_or_sync(kFullMask, (unsigned)tb);
            const unsigned thi = __reduce_or_sync(kFullMask, (unsigned)(tb >> 32));
            f |= ((unsigned long long)thi << 32) | tlo;
            if (f != ~0ull) t = 64 * w + __ffsll((long long)~f);
        }
        if (lane == 0) *(volatile int*)(P.col + v) = -t;
    }
}

template <class V>
__global__ void d1_assign(const Problem<V>* __restrict__ Pp, cudaGraphConditionalHandle h,
                          int use_cond) {
    const Problem<V>& P = *Pp;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // The loop continues only if this round's detect says so: should its
        // round control ever not run, the device loop ends instead of spinning.
        if (use_cond) cudaGraphSetConditional(h, 0u);
        P.st->push_cnt = 0;   // the previous round's push kernel has finished
    }
    if (P.async_mode) assign_async_phase(P);
    else assign_phase(P);
}

// ---------------------------------------------------------------------------
// detect + commit + compact + inline push (+ round control in the last block)
// ---------------------------------------------------------------------------
// End of round r: record the trace, decide whether to go on, set up round
// r+1.  Returns 1 when the coloring is finished (or has failed).
template <class V>
__device__ int round_decide(const Problem<V>& P) {
    State* st = P.st;
    const int r = st->round;
    const int cp = r & 1, np = cp ^ 1;
    const long long cur = (long long)st->ns[cp] + st->nm[cp] + st->nl[cp];
    const long long nxt = (long long)*(volatile int*)&st->ns[np] + *(volatile int*)&st->nm[np] +
                          *(volatile int*)&st->nl[np];
    if (r < P.trace_cap) {
        P.trace_w[r] = nxt;
        P.trace_s[r] = (long long)*(volatile unsigned long long*)&st->s_next;
        P.trace_h[r] = (long long)*(volatile unsigned long long*)&st->h_next;
    }
    if (r == 1 && P.trace_cap > 0) P.trace_h[0] = (long long)st->h_first;
    int done = 0, status = ST_OK;
    if (nxt == 0) {
        done = 1;
    } else if (nxt >= cur) {
        done = 1;
        status = ST_NO_PROGRESS;
    } else if (r >= P.max_rounds) {
        done = 1;
        status = ST_MAX_ROUNDS;
    } else if (global_ns() - st->t0 > P.timeout_ns) {
        done = 1;
        status = ST_TIMEOUT;
    }
    if (!done) {
        st->ns[cp] = st->nm[cp] = st->nl[cp] = 0;
        st->round = r + 1;
        st->s_next = 0ull;
        st->h_next = 0ull;
    }
    st->status = status;
    st->done = done;
    st->blocks_done = 0u;
    st->l_next = 0u;
    st->tail = (!done && nxt <= P.tail_w) ? 1 : 0;
    __threadfence();
    return done;
}

// Round control of the launch-per-round loop: the WHILE node repeats while
// the coloring is unfinished and the worklist is larger than tail_w; the
// remaining rounds go to the core phase.
template <class V>
__device__ void round_control(const Problem<V>& P, cudaGraphConditionalHandle h, int use_cond) {
    const int done = round_decide(P);
    if (use_cond) cudaGraphSetConditional(h, (done || P.st->tail) ? 0u : 1u);
}

// Queue the push of v's color: ceil(deg / kPushItem) work items.
template <class V>
__device__ __forceinline__ void queue_push(const Problem<V>& P, int v, int d) {
    const int nit = ceil_div(d, kPushItem);
    const int base = atomicAdd(&P.st->push_cnt, nit);
    for (int k = 0; k < nit; ++k) P.push_q[base + k] = make_int2(v, k);
}

// The vertex v whose list is being checked, with what a priority that
// changes each round needs: its priority this round and its hash.
struct Me {
    int v, p, base;
    uint64_t h;
};
struct NoMe {};   // the static order needs nothing about v
template <bool DYN>
using MeOf = typename std::conditional<DYN, Me, NoMe>::type;

template <class V>
__device__ __forceinline__ Me round_me(const Problem<V>& P, int v, int g) {
    const int base = P.g.base(g);
    return Me{v, P.prio[v], base, prio_hash(P.seed, (uint32_t)(v - base))};
}

// Priorities that change each round (Sec. 3.3, closing paragraph): u beats v
// when its priority this round is larger; ties go to the smaller hash, then
// the smaller id (Alg. 4 with the priority in place of the degree).
template <class V>
__device__ __forceinline__ bool beats(const Problem<V>& P, int u, const Me& me) {
    const int pu = P.prio[u];
    if (pu != me.p) return pu > me.p;
    const uint64_t hu = prio_hash(P.seed, (uint32_t)(u - me.base));
    if (hu != me.h) return hu < me.h;
    return u < me.v;
}

// u (an entry of v's list, < 0: none) holds v's tentative color t and, with
// DYN, beats v this round.  Without DYN the list holds only neighbors with
// priority over v (a static order), so the color alone decides.
template <bool DYN, class V>
__device__ __forceinline__ bool conflict(const Problem<V>& P, int u, int t, MeOf<DYN> me) {
    if constexpr (DYN) return u >= 0 && abs(P.col[u]) == t && beats(P, u, me);
    else return u >= 0 && abs(P.col[u]) == t;
}

// Warp-wide: does any of the list entries [b0, min(b0 + 32K, hl)) of v
// (starting at h) conflict with v's color t?  K ids per lane are loaded,
// then their K colors, so a step costs two dependent loads whatever K is.
template <int K, bool DYN, class V>
__device__ __forceinline__ bool warp_step(const Problem<V>& P, const int* h, int b0, int hl,
                                          int t, MeOf<DYN> me) {
    const int lane = lane_id();
    int u[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int e = b0 + 32 * j + lane;
        u[j] = e < hl ? __ldg(h + e) : -1;
    }
    bool hit = false;
#pragma unroll
    for (int j = 0; j < K; ++j) hit |= conflict<DYN>(P, u[j], t, me);
    return __any_sync(kFullMask, hit);
}

// Warp-wide: does any of the H-list entries [from, hl) of v (starting at
// hadj[beg]) currently hold color t?  The steps grow 64, 128, 256, 256, ...
// entries: most losers meet their conflict in the first step, while a
// winner, which must read its whole list, needs few dependent steps.
template <bool DYN, class V>
__device__ __forceinline__ bool warp_conflict(const Problem<V>& P, long long beg, int hl, int t,
                                              int from, MeOf<DYN> me) {
    const int* h = P.hadj + beg;
    int b0 = from;
    if (b0 < hl) {
        if (warp_step<2, DYN>(P, h, b0, hl, t, me)) return true;
        b0 += 64;
    }
    if (b0 < hl) {
        if (warp_step<4, DYN>(P, h, b0, hl, t, me)) return true;
        b0 += 128;
    }
    for (; b0 < hl; b0 += 256)
        if (warp_step<8, DYN>(P, h, b0, hl, t, me)) return true;
    return false;
}

// Detection, commit, compaction and inline push for one round (every block
// of the grid takes part).  DYN: priorities that change each round -- the
// lists then hold every neighbor, a neighbor holding v's color must also
// beat v this round, and every winner's push is queued (an inline push would
// change neighbors' priorities while others still compare them).
template <class V, bool DYN>
__device__ __forceinline__ void detect_phase(const Problem<V>& P, int* smem) {
    State* st = P.st;
    const int r = *(volatile int*)&st->round;
    const int cp = r & 1, np = cp ^ 1;
    const int nS = st->ns[cp], nM = st->nm[cp], nL = st->nl[cp];
    const int* __restrict__ ha = P.hadj;
    int* col = P.col;
    const bool batch = P.g_rounds != nullptr;
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + warp, nw = gridDim.x * wpb;
    int my_max = 0;
    unsigned long long my_s = 0ull, my_h = 0ull;
    // losers keep their entry and tier: appended by source index
    IdxAppend app_s = {smem + warp * 2 * kIdxSlots, 0};
    IdxAppend app_m = {smem + warp * 2 * kIdxSlots + kIdxSlots, 0};
    // Round 1: every vertex holds tentative color 1, so v loses exactly when
    // H(v) is not empty -- no list needs to be read.
    const bool first = r == 1 && !P.async_mode && !DYN;

    // --- L tier: one block per vertex (static assignment) ---
    for (int i = blockIdx.x; i < nL; i += gridDim.x) {
        const int4 ent = P.wl[cp][i];
        const int v = ent.x, hl = ent.y, d = ent.z;
        const int g = P.g.graph(v);
        const long long beg = P.g.begin(g, ent.w);
        const int t = -col[v];
        MeOf<DYN> me{};
        if constexpr (DYN) me = round_me(P, v, g);
        bool lose = first && hl > 0;
        int nxt = !first && (int)threadIdx.x < hl ? __ldg(ha + beg + threadIdx.x) : -1;
        for (int b0 = 0; !first && b0 < hl; b0 += blockDim.x) {
            const int u = nxt;
            const int e = b0 + blockDim.x + threadIdx.x;
            nxt = e < hl ? __ldg(ha + beg + e) : -1;
            if (__syncthreads_or(conflict<DYN>(P, u, t, me))) {
                lose = true;
                break;
            }
        }
        if (threadIdx.x == 0) {
            if (lose) {
                P.wl[np][atomicAdd(&st->nl[np], 1)] = ent;
                my_s += (unsigned long long)d;
                my_h += (unsigned long long)hl;
                if (batch) atomicMax(P.g_rounds + g, r + 1);
            } else {
                col[v] = t;
                atomicAnd(P.live + (v >> 5), ~(1u << (v & 31)));
                my_max = max(my_max, t);
                if (batch) atomicMax(P.g_colors + g, t);
                queue_push(P, v, d);
            }
        }
        __syncthreads();
    }

    // --- M tier: one warp per vertex.  The next vertex's entry is loaded
    // while this one's first 32 list colors are gathered, and its own color
    // and first 32 list ids while this one is committed or appended. ---
    int4 ent = make_int4(-1, 0, 0, 0);
    long long beg = 0;
    int g = 0, t = 0, u0 = -1;
    if (gw < nM) {
        ent = P.wm[cp][gw];
        g = P.g.graph(ent.x);
        beg = P.g.begin(g, ent.w);
        t = -col[ent.x];
        u0 = !first && lane < ent.y ? __ldg(ha + beg + lane) : -1;
    }
    for (int i = gw; i < nM; i += nw) {
        const int v = ent.x, hl = ent.y, d = ent.z;
        const int in = i + nw;
        int4 en = make_int4(-1, 0, 0, 0);
        if (in < nM) en = P.wm[cp][in];
        MeOf<DYN> me{};
        if constexpr (DYN) me = round_me(P, v, g);
        bool lose = first ? hl > 0 : __any_sync(kFullMask, conflict<DYN>(P, u0, t, me));
        if (!first && !lose && hl > 32) lose = warp_conflict<DYN>(P, beg, hl, t, 32, me);
        int gn = 0, tn = 0, un = -1;
        long long bn = 0;
        if (in < nM) {
            gn = P.g.graph(en.x);
            bn = P.g.begin(gn, en.w);
            tn = -col[en.x];
            un = !first && lane < en.y ? __ldg(ha + bn + lane) : -1;
        }
        if (lane == 0) {
            if (lose) {
                my_s += (unsigned long long)d;
                my_h += (unsigned long long)hl;
                if (batch) atomicMax(P.g_rounds + g, r + 1);
            } else {
                col[v] = t;
                atomicAnd(P.live + (v >> 5), ~(1u << (v & 31)));
                my_max = max(my_max, t);
                if (batch) atomicMax(P.g_colors + g, t);
                queue_push(P, v, d);
            }
        }
        ia_push(app_m, lose && lane == 0, i, P.wm[cp], P.wm[np], &st->nm[np]);
        ent = en;
        beg = bn;
        g = gn;
        t = tn;
        u0 = un;
    }

    // --- S tier: one thread per vertex ---
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < nS;
         wbase += stride) {
        const long long i = wbase + lane;
        bool lose = false, win = false;
        int g = 0, t = 0;
        int4 ent = make_int4(-1, 0, 0, 0);
        if (i < nS) {
            ent = P.ws[cp][i];
            const int v = ent.x, hl = ent.y, d = ent.z;
            g = P.g.graph(v);
            const long long beg = P.g.begin(g, ent.w);
            t = -col[v];
            MeOf<DYN> me{};
            if constexpr (DYN) me = round_me(P, v, g);
            lose = first && hl > 0;
            // four list entries, then eight at a time (ids, then their colors)
            if (!first && hl > 0) {
                int u[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] = j < hl ? __ldg(ha + beg + j) : -1;
#pragma unroll
                for (int j = 0; j < 4; ++j) lose |= conflict<DYN>(P, u[j], t, me);
            }
            for (int e = 4; !first && e < hl && !lose; e += 8) {
                int u[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) u[j] = e + j < hl ? __ldg(ha + beg + e + j) : -1;
#pragma unroll
                for (int j = 0; j < 8; ++j) lose |= conflict<DYN>(P, u[j], t, me);
            }
            if (lose) {
                my_s += (unsigned long long)d;
                my_h += (unsigned long long)hl;
            } else {
                win = true;
                col[v] = t;
                atomicAnd(P.live + (v >> 5), ~(1u << (v & 31)));
                my_max = max(my_max, t);
                if (d <= kInlinePush && !DYN) {
                    // four neighbors at a time: ids, then their uncolored
                    // bits, then the updates
                    const int base = P.g.base(g);
                    for (int e0 = 0; e0 < d; e0 += 4) {
                        int u[4];
                        unsigned lw[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            u[j] = e0 + j < d ? P.g.nbr(beg + e0 + j, base) : v;
#pragma unroll
                        for (int j = 0; j < 4; ++j) lw[j] = u[j] != v ? P.live[u[j] >> 5] : 0u;
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if ((lw[j] >> (u[j] & 31)) & 1u) push_color_live<false>(P, u[j], g, t);
                    }
                } else {
                    queue_push(P, v, d);
                }
            }
        }
        if (batch) {
            graph_max(P.g_rounds, lose, g, r + 1);
            graph_max(P.g_colors, win, g, t);
        }
        ia_push(app_s, lose, (int)i, P.ws[cp], P.ws[np], &st->ns[np]);
    }
    ia_flush(app_s, P.ws[cp], P.ws[np], &st->ns[np]);
    ia_flush(app_m, P.wm[cp], P.wm[np], &st->nm[np]);

    // --- per-warp totals ---
    my_max = warp_max(my_max);
    my_s = warp_sum(my_s);
    my_h = warp_sum(my_h);
    if (lane == 0) {
        if (my_max > 0) atomicMax(&st->max_color, my_max);
        if (my_s > 0) atomicAdd(&st->s_next, my_s);
        if (my_h > 0) atomicAdd(&st->h_next, my_h);
    }

}

template <class V, bool DYN = false>
__global__ void __maxnreg__(48) d1_detect(const Problem<V>* __restrict__ Pp,
                                          cudaGraphConditionalHandle h, int use_cond) {
    extern __shared__ int smem[];
    const Problem<V>& P = *Pp;
    State* st = P.st;
    detect_phase<V, DYN>(P, smem);

    // --- last block runs the round control ---
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(&st->blocks_done, 1u);
        s_last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        round_control(P, h, use_cond);
    }
}

// ---------------------------------------------------------------------------
// push: winners' colors into the forbidden sets of their neighbors
// ---------------------------------------------------------------------------
template <class V>
__device__ __forceinline__ void push_phase(const Problem<V>& P) {
    const int nq = *(volatile int*)&P.st->push_cnt;
    const int lane = lane_id(), wpb = blockDim.x >> 5;
    for (int q = blockIdx.x * wpb + (threadIdx.x >> 5); q < nq; q += gridDim.x * wpb) {
        const int2 item = P.push_q[q];
        const int v = item.x;
        const int c = P.col[v];
        const int g = P.g.graph(v), base = P.g.base(g);
        long long beg;
        int d;
        P.g.row(v, g, beg, d);
        const int e0 = item.y * kPushItem, e1 = min(e0 + kPushItem, d);
        for (int b0 = e0; b0 < e1; b0 += 128) {
            int u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = b0 + j * 32 + lane;
                u[j] = e < e1 ? P.g.nbr(beg + e, base) : -1;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (u[j] >= 0 && u[j] != v) push_color(P, u[j], g, c);
        }
    }
}

// PGC_ASYNC: the next round's worklist vertices start uncolored (0), so that
// a negative color seen during its first fit is one written in that round.
template <class V>
__device__ __forceinline__ void reset_next_worklist(const Problem<V>& P) {
    const State* st = P.st;
    if (*(volatile const int*)&st->done) return;
    const int p = *(volatile const int*)&st->round & 1;
    const int n0 = st->ns[p], n1 = st->nm[p], n2 = st->nl[p];
    const long long total = (long long)n0 + n1 + n2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int v = i < n0 ? P.ws[p][i].x
                    : (i < n0 + n1 ? P.wm[p][i - n0].x : P.wl[p][i - n0 - n1].x);
        P.col[v] = 0;
    }
}

template <class V>
__global__ void d1_push(const Problem<V>* __restrict__ Pp) {
    push_phase(*Pp);
    if (Pp->async_mode) reset_next_worklist(*Pp);
}

// ---------------------------------------------------------------------------
// grid barrier of the core loop
// ---------------------------------------------------------------------------
// Grid-wide barrier for a cooperative launch (all blocks co-resident).  A
// wait that exceeds ~2^22 polls (about a second) gives up, records the
// failure and lets the kernel return with an error instead of hanging.
__device__ __forceinline__ bool grid_barrier(State* st, unsigned max_polls) {
    __threadfence();
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = *(volatile unsigned*)&st->bar_gen;
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
            st->bar_count = 0u;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            unsigned polls = 0;
            while (*(volatile unsigned*)&st->bar_gen == gen) {
                __nanosleep(128);
                if (++polls > max_polls || *(volatile int*)&st->bar_timeout) {
                    atomicExch(&st->bar_timeout, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// core: the last rounds on the subgraph induced by the worklist
// ---------------------------------------------------------------------------
// Once the worklist W is small (at most tail_w vertices), the remaining
// rounds only ever involve W: a vertex outside W is committed, so it can no
// longer conflict (first fit avoids committed colors) and its forbidden set
// is never read again.  The core phase therefore
//   1. gives the vertices of W local ids and extracts, for each, its
//      neighbors inside W -- the higher-priority ones first (the only ones
//      Alg. 4 can make it lose to), then the others (which only receive its
//      color when it commits);
//   2. runs the rounds (assign, detect, push, round control) in one
//      cooperative launch of a few 1024-thread blocks over these short
//      local lists, with grid barriers between the phases;
//   3. writes the colors back.
// The rounds are the same rounds the per-round kernels would run (same
// first fit on the same forbidden sets, same loser rule, same snapshot), so
// colors, round count and trace are unchanged.
//
// Scratch: local id of v in hlen[v] (the list lengths are dead after
// setup), induced lists in hadj (dead once the global lists are no longer
// scanned; the induced lists are a subset of W's adjacency, so they fit),
// per-vertex arrays in the other parity's worklist buffers (3 x 16n bytes).

#ifndef PGC_CORE_BLOCKS
#define PGC_CORE_BLOCKS 32
#endif
constexpr int kCoreBlocks = PGC_CORE_BLOCKS;
constexpr int kUploadChunks = 8;    // host adjacency uploaded in this many row ranges

// Adjacency still in (pinned) host memory when a coloring starts: it is
// copied in kUploadChunks row ranges on a second stream, and the list build
// of each range starts as soon as its rows have arrived, so the transfer
// overlaps the build.
struct Upload {
    const int* h_ci;   // host adjacency
    const int* h_rp;   // host row offsets (chunk boundaries)
    int* d_ci;         // device copy (the view's adjacency)
};     // blocks of the core loop (1024 threads each)
constexpr int kCoreWarpDeg = 4096;  // rows up to this length: one warp; longer: one block

struct CoreArrays {
    int4* lent;   // [k] worklist entry {v, |H(v)|, deg, local row start}
    int* vid;     // [k] global id
    int* lhn;     // [k] number of higher-priority induced neighbors
    int* lcol;    // [k] color (> 0 committed, -t tentative)
    int* qwin;    // [k] winners of the round
    int* loff;    // [k + 1] induced list offsets (higher ones first)
    int* lw0;     // [k] local worklists (two sides)
    int* lw1;
};

template <class V>
__device__ __forceinline__ CoreArrays core_arrays(const Problem<V>& P, int par, int k) {
    CoreArrays a;
    a.lent = P.ws[par];
    int* m = reinterpret_cast<int*>(P.wm[par]);
    a.vid = m;
    a.lhn = m + k;
    a.lcol = m + 2 * k;
    a.qwin = m + 3 * k;
    int* l = reinterpret_cast<int*>(P.wl[par]);
    a.loff = l;
    a.lw0 = l + k + 1;
    a.lw1 = l + 2 * k + 1;
    return a;
}

template <class V>
__device__ __forceinline__ int4 core_entry(const Problem<V>& P, int cp, int nS, int nM, int i) {
    return i < nS ? P.ws[cp][i] : (i < nS + nM ? P.wm[cp][i - nS] : P.wl[cp][i - nS - nM]);
}

__device__ __forceinline__ bool is_live(const unsigned* live, int u) {
    return (live[u >> 5] >> (u & 31)) & 1u;
}

// Phase 1a: local ids and induced degrees (total and higher-priority part).
// Rows up to kCoreWarpDeg: one warp each; longer rows: one block each.
template <class V>
__global__ void d1_core_map(const Problem<V>* __restrict__ Pp) {
    const Problem<V>& P = *Pp;
    State* st = P.st;
    if (*(volatile int*)&st->done || !*(volatile int*)&st->tail) return;
    const int cp = st->round & 1, np = cp ^ 1;
    const int nS = st->ns[cp], nM = st->nm[cp], nL = st->nl[cp], k = nS + nM + nL;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->core_k = k;
        st->core_par = np;
    }
    const CoreArrays A = core_arrays(P, np, k);
    const unsigned long long seed = P.seed;
    const bool use_deg = P.use_deg != 0;
    const int lane = lane_id(), wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    for (int i = gw; i < k; i += nw) {
        const int4 e = core_entry(P, cp, nS, nM, i);
        const int v = e.x, d = e.z;
        if (lane == 0) {
            A.vid[i] = v;
            A.lent[i] = e;
            A.lcol[i] = P.col[v];
            P.hlen[v] = i;
        }
        if (d > kCoreWarpDeg) continue;
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, e.w);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        int cnt = 0, hcnt = 0;
        for (int b0 = 0; b0 < d; b0 += 32) {
            const int j = b0 + lane;
            if (j < d) {
                const int u = P.g.nbr(beg + j, base);
                if (u != v && is_live(P.live, u)) {
                    ++cnt;
                    hcnt += higher(__ldg(P.deg + u), u, d, hv, v, base, seed, use_deg);
                }
            }
        }
        cnt = warp_sum(cnt);
        hcnt = warp_sum(hcnt);
        if (lane == 0) {
            A.loff[i + 1] = cnt;
            A.lhn[i] = hcnt;
        }
    }
    __shared__ int s_cnt, s_hcnt;
    for (int i = blockIdx.x; i < k; i += gridDim.x) {
        const int4 e = core_entry(P, cp, nS, nM, i);
        const int v = e.x, d = e.z;
        if (d <= kCoreWarpDeg) continue;   // block-uniform
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, e.w);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        if (threadIdx.x == 0) s_cnt = s_hcnt = 0;
        __syncthreads();
        int cnt = 0, hcnt = 0;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const int u = P.g.nbr(beg + j, base);
            if (u != v && is_live(P.live, u)) {
                ++cnt;
                hcnt += higher(__ldg(P.deg + u), u, d, hv, v, base, seed, use_deg);
            }
        }
        cnt = warp_sum(cnt);
        hcnt = warp_sum(hcnt);
        if (lane == 0) {
            atomicAdd(&s_cnt, cnt);
            atomicAdd(&s_hcnt, hcnt);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            A.loff[i + 1] = s_cnt;
            A.lhn[i] = s_hcnt;
        }
        __syncthreads();
    }
}

// Phase 1b (one block): offsets = exclusive scan of the induced degrees;
// the first local worklist holds every local vertex.
template <class V>
__global__ void d1_core_scan(const Problem<V>* __restrict__ Pp) {
    const Problem<V>& P = *Pp;
    State* st = P.st;
    if (*(volatile int*)&st->done || !*(volatile int*)&st->tail) return;
    const int k = st->core_k;
    const CoreArrays A = core_arrays(P, st->core_par, k);
    __shared__ int s_part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (k + T - 1) / T;
    const int lo = min(k, t * per), hi = min(k, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += A.loff[i + 1];
    s_part[t] = sum;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {   // inclusive scan of the per-thread sums
        const int x = t >= o ? s_part[t - o] : 0;
        __syncthreads();
        s_part[t] += x;
        __syncthreads();
    }
    int run = s_part[t] - sum;
    for (int i = lo; i < hi; ++i) {
        run += A.loff[i + 1];
        A.loff[i + 1] = run;
    }
    if (t == 0) A.loff[0] = 0;
    for (int i = t; i < k; i += T) A.lw0[i] = i;
    if (t == 0) {
        st->core_cur = k;
        st->core_nxt = 0;
        st->core_win = 0;
    }
}

// Phase 1c: the induced lists, as local ids: higher-priority neighbors at
// [loff[i], loff[i] + lhn[i]), the others after them.
template <class V>
__global__ void d1_core_fill(const Problem<V>* __restrict__ Pp) {
    const Problem<V>& P = *Pp;
    State* st = P.st;
    if (*(volatile int*)&st->done || !*(volatile int*)&st->tail) return;
    const int k = st->core_k;
    const CoreArrays A = core_arrays(P, st->core_par, k);
    int* adj = P.hadj;
    const unsigned long long seed = P.seed;
    const bool use_deg = P.use_deg != 0;
    const int lane = lane_id(), wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = gw; i < k; i += nw) {
        const int4 e = A.lent[i];
        const int v = e.x, d = e.z;
        if (d > kCoreWarpDeg) continue;
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, e.w);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        int* hi_out = adj + A.loff[i];
        int* lo_out = hi_out + A.lhn[i];
        int hp = 0, op = 0;
        for (int b0 = 0; b0 < d; b0 += 32) {
            const int j = b0 + lane;
            int u = -1;
            bool keep = false, hi = false;
            if (j < d) {
                u = P.g.nbr(beg + j, base);
                keep = u != v && is_live(P.live, u);
                hi = keep && higher(__ldg(P.deg + u), u, d, hv, v, base, seed, use_deg);
            }
            const unsigned bh = __ballot_sync(kFullMask, hi);
            const unsigned bo = __ballot_sync(kFullMask, keep && !hi);
            if (hi) hi_out[hp + __popc(bh & lt)] = P.hlen[u];
            else if (keep) lo_out[op + __popc(bo & lt)] = P.hlen[u];
            hp += __popc(bh);
            op += __popc(bo);
        }
    }
    __shared__ int s_hp, s_op;
    for (int i = blockIdx.x; i < k; i += gridDim.x) {
        const int4 e = A.lent[i];
        const int v = e.x, d = e.z;
        if (d <= kCoreWarpDeg) continue;   // block-uniform
        const int g = P.g.graph(v), base = P.g.base(g);
        const long long beg = P.g.begin(g, e.w);
        const uint64_t hv = prio_hash(seed, (uint32_t)(v - base));
        int* hi_out = adj + A.loff[i];
        int* lo_out = hi_out + A.lhn[i];
        if (threadIdx.x == 0) s_hp = s_op = 0;
        __syncthreads();
        for (int b0 = 0; b0 < d; b0 += blockDim.x) {
            const int j = b0 + threadIdx.x;
            int u = -1;
            bool keep = false, hi = false;
            if (j < d) {
                u = P.g.nbr(beg + j, base);
                keep = u != v && is_live(P.live, u);
                hi = keep && higher(__ldg(P.deg + u), u, d, hv, v, base, seed, use_deg);
            }
            const unsigned bh = __ballot_sync(kFullMask, hi);
            const unsigned bo = __ballot_sync(kFullMask, keep && !hi);
            int ph = 0, po = 0;
            if (lane == 0) {
                if (bh) ph = atomicAdd(&s_hp, __popc(bh));
                if (bo) po = atomicAdd(&s_op, __popc(bo));
            }
            ph = __shfl_sync(kFullMask, ph, 0);
            po = __shfl_sync(kFullMask, po, 0);
            if (hi) hi_out[ph + __popc(bh & lt)] = P.hlen[u];
            else if (keep) lo_out[po + __popc(bo & lt)] = P.hlen[u];
        }
        __syncthreads();
    }
}

// End of a core round: trace, termination, next round's counts (one thread).
template <class V>
__device__ void core_decide(const Problem<V>& P) {
    State* st = P.st;
    const int r = st->round;
    const long long cur = st->core_cur;
    const long long nxt = *(volatile int*)&st->core_nxt;
    if (r < P.trace_cap) {
        P.trace_w[r] = nxt;
        P.trace_s[r] = (long long)*(volatile unsigned long long*)&st->s_next;
        P.trace_h[r] = (long long)*(volatile unsigned long long*)&st->h_next;
    }
    int done = 0, status = ST_OK;
    if (nxt == 0) {
        done = 1;
    } else if (nxt >= cur) {
        done = 1;
        status = ST_NO_PROGRESS;
    } else if (r >= P.max_rounds) {
        done = 1;
        status = ST_MAX_ROUNDS;
    } else if (global_ns() - st->t0 > P.timeout_ns) {
        done = 1;
        status = ST_TIMEOUT;
    }
    if (!done) {
        st->round = r + 1;
        st->core_cur = (int)nxt;
        st->core_nxt = 0;
        st->s_next = 0ull;
        st->h_next = 0ull;
    }
    st->status = status;
    st->done = done;
    __threadfence();
}

// Phase 2 (cooperative, kCoreBlocks x 1024 threads): the rounds.
template <class V>
__global__ void __launch_bounds__(1024, 1) d1_core_loop(const Problem<V>* __restrict__ Pp) {
    const Problem<V>& P = *Pp;
    State* st = P.st;
    if (*(volatile int*)&st->done || !*(volatile int*)&st->tail) return;
    const int k = st->core_k;
    const CoreArrays A = core_arrays(P, st->core_par, k);
    const int* adj = P.hadj;
    int* lcol = A.lcol;
    const bool batch = P.g_rounds != nullptr;
    const int lane = lane_id(), wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    if ((int)blockIdx.x == P.slow_block && threadIdx.x == 0) {
        // test hook: this block reaches its first barrier late (bounded)
        const unsigned long long t_end = global_ns() + P.slow_ns;
        while (global_ns() < t_end) __nanosleep(1000);
    }
    int side = 0;
    for (;;) {
        const int r = *(volatile int*)&st->round;
        const int cur = *(volatile int*)&st->core_cur;
        const int* lw = side ? A.lw1 : A.lw0;
        int* lwn = side ? A.lw0 : A.lw1;
        if (gt == 0) st->core_win = 0;   // read last in the previous round's push
        // assign: first fit from the forbidden sets, from the previous color
        for (int x = gt; x < cur; x += nt) {
            const int i = lw[x];
            lcol[i] = -first_fit(P, A.lent[i], -lcol[i]);
        }
        if (!grid_barrier(st, P.bar_polls)) break;
        // detect: one warp per vertex over its higher-priority induced list
        int my_max = 0;
        unsigned long long my_s = 0ull, my_h = 0ull;
        for (int x = gw; x < cur; x += nw) {
            const int i = lw[x];
            const int t = -lcol[i];
            const int* h = adj + A.loff[i];
            const int hn = A.lhn[i];
            bool lose = false;
            for (int b0 = 0; b0 < hn && !lose; b0 += 128) {
                int c[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int e = b0 + 32 * j + lane;
                    c[j] = e < hn ? lcol[h[e]] : 0;
                }
                bool hit = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) hit |= abs(c[j]) == t;
                lose = __any_sync(kFullMask, hit);
            }
            if (lane == 0) {
                const int4 e = A.lent[i];
                const int g = batch ? P.g.graph(e.x) : 0;
                if (lose) {
                    lwn[atomicAdd(&st->core_nxt, 1)] = i;
                    my_s += (unsigned long long)e.z;
                    my_h += (unsigned long long)e.y;
                    if (batch) atomicMax(P.g_rounds + g, r + 1);
                } else {
                    lcol[i] = t;
                    A.qwin[atomicAdd(&st->core_win, 1)] = i;
                    my_max = max(my_max, t);
                    if (batch) atomicMax(P.g_colors + g, t);
                }
            }
        }
        my_max = warp_max(my_max);
        my_s = warp_sum(my_s);
        my_h = warp_sum(my_h);
        if (lane == 0) {
            if (my_max > 0) atomicMax(&st->max_color, my_max);
            if (my_s > 0) atomicAdd(&st->s_next, my_s);
            if (my_h > 0) atomicAdd(&st->h_next, my_h);
        }
        if (!grid_barrier(st, P.bar_polls)) break;
        // push the winners' colors to their uncolored induced neighbors,
        // while one thread closes the round.  The warps share the winners
        // (several warps per winner when winners are few); a warp takes four
        // list entries per lane at a time, and a neighbor's row start and
        // degree come from its local entry, not from row_ptr.
        if (gt == 0) core_decide(P);
        const int nwin = *(volatile int*)&st->core_win;
        if (nwin > 0) {
            const int wpw = max(1, nw / nwin);   // warps per winner
            const int slots = nw / wpw;
            const int sub = gw % wpw;
            for (int q = gw / wpw; q < nwin && gw < slots * wpw; q += slots) {
                const int i = A.qwin[q];
                const int c = lcol[i];
                const int g = batch ? P.g.graph(A.vid[i]) : 0;
                const int e1 = A.loff[i + 1];
                const int step = wpw * 32;
                for (int e0 = A.loff[i] + sub * 32 + lane; e0 < e1; e0 += 4 * step) {
                    int j[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + u * step;
                        j[u] = e < e1 ? adj[e] : -1;
                    }
                    int cj[4];
                    int4 ej[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        cj[u] = j[u] >= 0 ? lcol[j[u]] : 1;
                        ej[u] = j[u] >= 0 ? A.lent[j[u]] : make_int4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (cj[u] >= 0) continue;   // colored (or no entry)
                        const int v = ej[u].x;
                        if (c <= 64) {
                            atomicOr(P.bm0 + v, 1ull << (c - 1));
                        } else if (c - 1 <= ej[u].z) {
                            const int b = c - 65;
                            const long long bu = P.g.begin(g, ej[u].w);
                            atomicOr(P.bmx + bm_offset(bu, v) + (b >> 5), 1u << (b & 31));
                        }
                    }
                }
            }
        }
        if (!grid_barrier(st, P.bar_polls)) break;
        if (*(volatile int*)&st->done) break;
        side ^= 1;
    }
    if (*(volatile int*)&st->bar_timeout) {
        if (gt == 0) {
            st->status = ST_BARRIER;
            st->done = 1;
        }
        return;
    }
    // write the colors back
    for (int i = gt; i < k; i += nt) P.col[A.vid[i]] = lcol[i];
}

// ---------------------------------------------------------------------------
// host side: scratch layout and one engine instance per (device, view type)
// ---------------------------------------------------------------------------
// Device scratch of one coloring (n vertices, nnz adjacency entries).
struct Scratch {
    int* deg;
    int* hlen;
    int* hadj;
    unsigned long long* bm0;
    unsigned* bmx;
    unsigned* live;
    int4* ws;    // 2n entries: both parities
    int4* wm;
    int4* wl;
    int2* items;
    int2* pushq;
    int* prio = nullptr;   // n ints, only for priorities that change each round
};

struct ScratchSizes {
    size_t deg, hlen, hadj, bm0, bmx, live, list, items, pushq;
    size_t total() const {   // with 256-byte alignment of every buffer
        auto a = [](size_t x) { return (x + 255) / 256 * 256; };
        return a(deg) + a(hlen) + a(hadj) + a(bm0) + a(bmx) + a(live) + 3 * a(list) + a(items) +
               a(pushq);
    }
};

inline ScratchSizes scratch_sizes(long long n, long long nnz) {
    ScratchSizes z;
    z.deg = z.hlen = (size_t)n * 4;
    z.hadj = (size_t)std::max<long long>(nnz, 1) * 4;
    z.bm0 = (size_t)n * 8;
    z.bmx = ((size_t)(nnz >> 5) + (size_t)n + 1) * 4;
    z.live = ((size_t)n / 32 + 2) * 4;
    z.list = (size_t)n * sizeof(int4) * 2;
    z.items = ((size_t)n + (size_t)(nnz / kBuildItem) + 1) * sizeof(int2);
    z.pushq = ((size_t)n + (size_t)(nnz / kPushItem) + 1) * sizeof(int2);
    return z;
}

// Carves a scratch of scratch_sizes(n, nnz).total() bytes at base.
inline Scratch carve_scratch(void* base, long long n, long long nnz) {
    const ScratchSizes z = scratch_sizes(n, nnz);
    char* p = static_cast<char*>(base);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    Scratch sc;
    sc.deg = reinterpret_cast<int*>(take(z.deg));
    sc.hlen = reinterpret_cast<int*>(take(z.hlen));
    sc.hadj = reinterpret_cast<int*>(take(z.hadj));
    sc.bm0 = reinterpret_cast<unsigned long long*>(take(z.bm0));
    sc.bmx = reinterpret_cast<unsigned*>(take(z.bmx));
    sc.live = reinterpret_cast<unsigned*>(take(z.live));
    sc.ws = reinterpret_cast<int4*>(take(z.list));
    sc.wm = reinterpret_cast<int4*>(take(z.list));
    sc.wl = reinterpret_cast<int4*>(take(z.list));
    sc.items = reinterpret_cast<int2*>(take(z.items));
    sc.pushq = reinterpret_cast<int2*>(take(z.pushq));
    return sc;
}
template <class V>
struct Engine {
    std::mutex mu;
    DeviceInfo dev;
    DevBuf deg, hlen, hadj, bm0, bmx, live, ws, wm, wl, items, pushq, prio, state, problem, trace;
    HostBuf h_problem, h_state, h_misc;
    int trace_cap = 0;
    int last_want_trace = 0, last_tcap = 1;
    // [0]: setup + rounds; [1]: rounds only (setup enqueued by the host
    // while the adjacency is still being uploaded)
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int g_grid = 0, g_block = 0, g_det = 0, g_async = 0, g_dyn = 0;
    cudaStream_t up_stream = nullptr;             // adjacency upload
    cudaEvent_t up_fork = nullptr, up_done[kUploadChunks] = {};

    void destroy_graph() {
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
            exec[k] = nullptr;
            graph[k] = nullptr;
        }
        g_grid = 0;
    }

    void destroy_upload() {
        if (up_stream) cudaStreamDestroy(up_stream);
        if (up_fork) cudaEventDestroy(up_fork);
        for (cudaEvent_t& e : up_done)
            if (e) cudaEventDestroy(e);
        up_stream = nullptr;
        up_fork = nullptr;
        for (cudaEvent_t& e : up_done) e = nullptr;
    }
    void release() {
        destroy_graph();
        destroy_upload();
        for (DevBuf* b : {&deg, &hlen, &hadj, &bm0, &bmx, &live, &ws, &wm, &wl, &items, &pushq,
                          &prio, &state, &problem, &trace})
            b->release();
        for (HostBuf* b : {&h_problem, &h_state, &h_misc}) b->release();
        trace_cap = 0;
    }

    struct Geometry {
        int grid, block;
        size_t smem;   // two warp appenders per warp
        int core_grid; // co-resident 1024-thread blocks of the cooperative core loop
        int det_grid;  // detect: its own occupancy
    };

    pgc_status geometry(const Opts& o, Geometry* g) {
        g->block = o.block;
        g->smem = (size_t)(o.block / 32) * 2 * kAppend4Slots * sizeof(int4);
        if (g->smem > 48 * 1024) {   // 1024-thread blocks: 64 KB of append buffers
            for (const void* f : {(const void*)d1_classify<V>, (const void*)d1_tier<V>,
                                  (const void*)d1_detect<V>, (const void*)d1_detect<V, true>})
                PGC_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)g->smem));
        }
        int per_sm = o.grid_per_sm;
        g->det_grid = dev.num_sms * per_sm;
        if (per_sm == 0) {
            int a = 0, b = 0;
            PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, d1_detect<V>, o.block, g->smem));
            PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, d1_build<V>, o.block, 0));
            per_sm = std::max(1, std::min(a, b));
            g->det_grid = dev.num_sms * std::max(1, a);
        }
        g->grid = dev.num_sms * per_sm;
        int t = 0;
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t, d1_core_loop<V>, 1024, 0));
        g->core_grid = std::max(1, std::min(kCoreBlocks, dev.num_sms * std::max(t, 1)));
        return PGC_OK;
    }

    static cudaKernelNodeParams knode(void* func, const Geometry& g, size_t smem, void** args) {
        cudaKernelNodeParams k = {};
        k.func = func;
        k.gridDim = dim3(g.grid);
        k.blockDim = dim3(g.block);
        k.sharedMemBytes = (unsigned)smem;
        k.kernelParams = args;
        return k;
    }

    pgc_status build_graph(const Geometry& g, int async, int dyn) {
        destroy_graph();
        for (int k = 0; k < 2; ++k)
            if (pgc_status s = build_one_graph(g, k == 0, async, dyn, &graph[k], &exec[k]))
                return s;
        g_dyn = dyn;
        g_grid = g.grid;
        g_det = g.det_grid;
        g_block = g.block;
        g_async = async;
        return PGC_OK;
    }

    // Setup (optional), round 1 (assign first under PGC_ASYNC), then the
    // WHILE node of the later rounds and the core phase.
    pgc_status build_one_graph(const Geometry& g, bool setup, int async, int dyn,
                               cudaGraph_t* graph_out, cudaGraphExec_t* exec_out) {
        Problem<V>* dP = problem.as<Problem<V>>();
        PGC_CUDA(cudaGraphCreate(graph_out, 0));
        cudaGraph_t graph = *graph_out;
        cudaGraphConditionalHandle handle = 0;
        PGC_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 0u, cudaGraphCondAssignDefault));
        int use_cond = 1;
        cudaGraphConditionalHandle hnd = handle;
        int lo = 0, hi = INT32_MAX;
        void* p_args[] = {&dP};
        void* b_args[] = {&dP, &lo, &hi};
        void* c_args[] = {&dP, &hnd, &use_cond};
        cudaMemsetParams ms = {};
        ms.dst = state.ptr;
        ms.value = 0;
        ms.elementSize = 4;
        ms.width = sizeof(State) / 4;
        ms.height = 1;
        cudaGraphNode_t n_ms, n_cls, n_build, n_tier, n_asg1, n_det, n_push, n_loop;
        if (setup) PGC_CUDA(cudaGraphAddMemsetNode(&n_ms, graph, nullptr, 0, &ms));
        cudaKernelNodeParams k_cls = knode((void*)d1_classify<V>, g, g.smem, p_args);
        cudaKernelNodeParams k_build = knode((void*)d1_build<V>, g, 0, b_args);
        cudaKernelNodeParams k_tier = knode((void*)d1_tier<V>, g, g.smem, p_args);
        cudaKernelNodeParams k_det =
            knode(dyn ? (void*)d1_detect<V, true> : (void*)d1_detect<V>, g, g.smem, c_args);
        k_det.gridDim = dim3(g.det_grid);
        cudaKernelNodeParams k_push = knode((void*)d1_push<V>, g, 0, p_args);
        cudaKernelNodeParams k_asg = knode((void*)d1_assign<V>, g, 0, c_args);
        if (setup) {
            PGC_CUDA(cudaGraphAddKernelNode(&n_cls, graph, &n_ms, 1, &k_cls));
            PGC_CUDA(cudaGraphAddKernelNode(&n_build, graph, &n_cls, 1, &k_build));
            PGC_CUDA(cudaGraphAddKernelNode(&n_tier, graph, &n_build, 1, &k_tier));
        }
        if (async) {
            PGC_CUDA(cudaGraphAddKernelNode(&n_asg1, graph, setup ? &n_tier : nullptr,
                                            setup ? 1 : 0, &k_asg));
            PGC_CUDA(cudaGraphAddKernelNode(&n_det, graph, &n_asg1, 1, &k_det));
        } else {
            PGC_CUDA(cudaGraphAddKernelNode(&n_det, graph, setup ? &n_tier : nullptr,
                                            setup ? 1 : 0, &k_det));
        }
        PGC_CUDA(cudaGraphAddKernelNode(&n_push, graph, &n_det, 1, &k_push));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        PGC_CUDA(cudaGraphAddNode(&n_loop, graph, &n_push, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t b_asg, b_det, b_push;
        PGC_CUDA(cudaGraphAddKernelNode(&b_asg, body, nullptr, 0, &k_asg));
        PGC_CUDA(cudaGraphAddKernelNode(&b_det, body, &b_asg, 1, &k_det));
        PGC_CUDA(cudaGraphAddKernelNode(&b_push, body, &b_det, 1, &k_push));
        // the remaining small rounds: the core phase (no-ops unless the loop
        // stopped with st->tail set)
        cudaKernelNodeParams k_cmap = knode((void*)d1_core_map<V>, g, 0, p_args);
        cudaKernelNodeParams k_cscan = knode((void*)d1_core_scan<V>, g, 0, p_args);
        k_cscan.gridDim = dim3(1);
        k_cscan.blockDim = dim3(1024);
        cudaKernelNodeParams k_cfill = knode((void*)d1_core_fill<V>, g, 0, p_args);
        cudaKernelNodeParams k_cloop = knode((void*)d1_core_loop<V>, g, 0, p_args);
        k_cloop.gridDim = dim3(g.core_grid);
        k_cloop.blockDim = dim3(1024);
        cudaGraphNode_t n_cmap, n_cscan, n_cfill, n_cloop;
        PGC_CUDA(cudaGraphAddKernelNode(&n_cmap, graph, &n_loop, 1, &k_cmap));
        PGC_CUDA(cudaGraphAddKernelNode(&n_cscan, graph, &n_cmap, 1, &k_cscan));
        PGC_CUDA(cudaGraphAddKernelNode(&n_cfill, graph, &n_cscan, 1, &k_cfill));
        PGC_CUDA(cudaGraphAddKernelNode(&n_cloop, graph, &n_cfill, 1, &k_cloop));
        cudaLaunchAttributeValue coop = {};
        coop.cooperative = 1;
        PGC_CUDA(cudaGraphKernelNodeSetAttribute(n_cloop, cudaLaunchAttributeCooperative, &coop));
        PGC_CUDA(cudaGraphInstantiate(exec_out, graph, 0));
        return PGC_OK;
    }

    // Colors n vertices (nnz adjacency entries in total) described by view,
    // with scratch owned by this engine; waits for the result.
    pgc_status run(const V& view, int n, long long nnz, int* d_col, int* g_rounds,
                   int* g_colors, uint64_t seed, const Opts& o, cudaStream_t stream,
                   int* rounds, int* num_colors, const Upload* up = nullptr) {
        pgc_status s = run_scratch(view, n, nnz, d_col, g_rounds, g_colors, seed, o, stream,
                                   rounds, num_colors, up);
        // out of device memory: keep no half-grown scratch (the next call
        // allocates again)
        if (s == PGC_ERR_OOM) release();
        return s;
    }

    pgc_status run_scratch(const V& view, int n, long long nnz, int* d_col, int* g_rounds,
                           int* g_colors, uint64_t seed, const Opts& o, cudaStream_t stream,
                           int* rounds, int* num_colors, const Upload* up) {
        // scratch grows, never shrinks; pointers travel in the Problem struct,
        // so the captured graph stays valid across calls
        const ScratchSizes z = scratch_sizes(n, nnz);
        if (pgc_status s = deg.ensure(z.deg)) return s;
        if (pgc_status s = hlen.ensure(z.hlen)) return s;
        if (pgc_status s = hadj.ensure(z.hadj)) return s;
        if (pgc_status s = bm0.ensure(z.bm0)) return s;
        if (pgc_status s = bmx.ensure(z.bmx)) return s;
        if (pgc_status s = live.ensure(z.live)) return s;
        if (pgc_status s = ws.ensure(z.list)) return s;
        if (pgc_status s = wm.ensure(z.list)) return s;
        if (pgc_status s = wl.ensure(z.list)) return s;
        if (pgc_status s = items.ensure(z.items)) return s;
        if (pgc_status s = pushq.ensure(z.pushq)) return s;
        const bool varying = (o.flags & (PGC_PRIORITY_DYNAMIC | PGC_PRIORITY_SATURATION)) != 0;
        if (varying)
            if (pgc_status s = prio.ensure((size_t)std::max(n, 1) * 4)) return s;
        Scratch sc;
        sc.deg = deg.as<int>();
        sc.hlen = hlen.as<int>();
        sc.hadj = hadj.as<int>();
        sc.bm0 = bm0.as<unsigned long long>();
        sc.bmx = bmx.as<unsigned>();
        sc.live = live.as<unsigned>();
        sc.ws = ws.as<int4>();
        sc.wm = wm.as<int4>();
        sc.wl = wl.as<int4>();
        sc.items = items.as<int2>();
        sc.pushq = pushq.as<int2>();
        sc.prio = varying ? prio.as<int>() : nullptr;
        if (pgc_status s = launch(sc, view, n, nnz, d_col, g_rounds, g_colors, seed, o, stream,
                                  up))
            return s;
        PGC_CUDA(cudaStreamSynchronize(stream));
        return finish(o, rounds, num_colors);
    }

    // Enqueues one coloring on `stream` with caller-provided scratch (the
    // device loop in graph mode; host-loop mode drives the rounds and
    // therefore blocks).  The round state and trace are copied to pinned
    // host memory on the same stream; call finish() once the stream is done.
    pgc_status launch(const Scratch& sc, const V& view, int n, long long nnz, int* d_col,
                      int* g_rounds, int* g_colors, uint64_t seed, const Opts& o,
                      cudaStream_t stream, const Upload* up = nullptr) {
        const uint32_t pflags = o.flags & (PGC_PRIORITY_DYNAMIC | PGC_PRIORITY_SATURATION);
        if (pflags == (PGC_PRIORITY_DYNAMIC | PGC_PRIORITY_SATURATION))
            return fail(PGC_ERR_INVALID_ARG, "PGC_PRIORITY_DYNAMIC and PGC_PRIORITY_SATURATION "
                                             "exclude each other");
        if (pflags && (o.flags & (PGC_NO_DEGREE_RULE | PGC_ASYNC)))
            return fail(PGC_ERR_INVALID_ARG, "a round-varying priority excludes "
                                             "PGC_NO_DEGREE_RULE and PGC_ASYNC");
        if (pflags && !sc.prio)
            return fail(PGC_ERR_INVALID_ARG, "round-varying priorities need their scratch");
        if (pgc_status s = state.ensure(sizeof(State))) return s;
        if (pgc_status s = problem.ensure(sizeof(Problem<V>))) return s;
        if (pgc_status s = h_problem.ensure(sizeof(Problem<V>))) return s;
        if (pgc_status s = h_state.ensure(sizeof(State))) return s;
        const int want_trace = o.profile && o.profile->trace_cap > 0 ? o.profile->trace_cap : 0;
        const int tcap = std::max(want_trace, 1);
        if (trace_cap < tcap) {
            if (pgc_status s = trace.ensure((size_t)tcap * 3 * sizeof(long long))) return s;
            if (pgc_status s = h_misc.ensure((size_t)tcap * 3 * sizeof(long long))) return s;
            trace_cap = tcap;
        }
        last_want_trace = want_trace;
        last_tcap = tcap;

        Geometry g;
        if (pgc_status s = geometry(o, &g)) return s;

        Problem<V>* hp = h_problem.as<Problem<V>>();
        std::memset(hp, 0, sizeof(Problem<V>));
        hp->g = view;
        hp->col = d_col;
        hp->deg = sc.deg;
        hp->hlen = sc.hlen;
        hp->hadj = sc.hadj;
        hp->bm0 = sc.bm0;
        hp->bmx = sc.bmx;
        hp->live = sc.live;
        for (int p = 0; p < 2; ++p) {
            hp->ws[p] = sc.ws + (size_t)p * n;
            hp->wm[p] = sc.wm + (size_t)p * n;
            hp->wl[p] = sc.wl + (size_t)p * n;
        }
        hp->items = sc.items;
        hp->push_q = sc.pushq;
        hp->g_rounds = g_rounds;
        hp->g_colors = g_colors;
        hp->trace_w = trace.as<long long>();
        hp->trace_s = hp->trace_w + tcap;
        hp->trace_h = hp->trace_s + tcap;
        hp->trace_cap = want_trace;
        hp->st = state.as<State>();
        hp->seed = seed;
        hp->timeout_ns = (unsigned long long)o.timeout_ms * 1000000ull;
        hp->nnz = nnz;
        hp->n = n;
        hp->use_deg = (o.flags & PGC_NO_DEGREE_RULE) ? 0 : 1;
        hp->async_mode = (o.flags & PGC_ASYNC) ? 1 : 0;
        hp->prio_mode = (pflags & PGC_PRIORITY_DYNAMIC) ? 1 : (pflags ? 2 : 0);
        hp->prio = sc.prio;
        hp->max_rounds = o.max_rounds > 0 ? o.max_rounds : (n < INT32_MAX ? n + 1 : n);
        hp->det_s = o.mid_degree;
        hp->det_m = o.hub_degree;
        hp->tail_w = (o.flags & PGC_ASYNC) || pflags ? 0 : o.tail_vertices;
        const TestHooks th = test_hooks();
        hp->bar_polls = th.barrier_polls;
        hp->slow_block = th.slow_block;
        hp->slow_ns = th.slow_us * 1000u;
        PGC_CUDA(cudaMemcpyAsync(problem.ptr, hp, sizeof(Problem<V>), cudaMemcpyHostToDevice,
                                 stream));
        Problem<V>* dP = problem.as<Problem<V>>();

        State* hs = h_state.as<State>();
        if (!(o.flags & PGC_HOST_LOOP)) {
            const int dyn = hp->prio_mode != 0;
            if (!exec[0] || g_grid != g.grid || g_block != g.block || g_det != g.det_grid ||
                g_async != hp->async_mode || g_dyn != dyn) {
                if (pgc_status s = build_graph(g, hp->async_mode, dyn)) return s;
            }
            if (!up) {
                PGC_CUDA(cudaGraphLaunch(exec[0], stream));
            } else {
                // setup by hand: classify needs only the row offsets; the
                // build of row range k waits for that range's copy
                if (!up_stream) {
                    PGC_CUDA(cudaStreamCreateWithFlags(&up_stream, cudaStreamNonBlocking));
                    PGC_CUDA(cudaEventCreateWithFlags(&up_fork, cudaEventDisableTiming));
                    for (cudaEvent_t& e : up_done)
                        PGC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                }
                int cut[kUploadChunks + 1];
                cut[0] = 0;
                cut[kUploadChunks] = n;
                for (int k = 1; k < kUploadChunks; ++k) {   // first row past k/K of the entries
                    const long long want = nnz * k / kUploadChunks;
                    cut[k] = (int)(std::lower_bound(up->h_rp, up->h_rp + n, (int)want) - up->h_rp);
                    cut[k] = std::max(cut[k], cut[k - 1]);
                }
                PGC_CUDA(cudaEventRecord(up_fork, stream));
                PGC_CUDA(cudaStreamWaitEvent(up_stream, up_fork, 0));
                for (int k = 0; k < kUploadChunks; ++k) {
                    const size_t e0 = (size_t)up->h_rp[cut[k]], e1 = (size_t)up->h_rp[cut[k + 1]];
                    if (e1 > e0)
                        PGC_CUDA(cudaMemcpyAsync(up->d_ci + e0, up->h_ci + e0, (e1 - e0) * 4,
                                                 cudaMemcpyHostToDevice, up_stream));
                    PGC_CUDA(cudaEventRecord(up_done[k], up_stream));
                }
                PGC_CUDA(cudaMemsetAsync(state.ptr, 0, sizeof(State), stream));
                d1_classify<V><<<g.grid, g.block, g.smem, stream>>>(dP);
                for (int k = 0; k < kUploadChunks; ++k) {
                    PGC_CUDA(cudaStreamWaitEvent(stream, up_done[k], 0));
                    d1_build<V><<<g.grid, g.block, 0, stream>>>(dP, cut[k], cut[k + 1]);
                }
                d1_tier<V><<<g.grid, g.block, g.smem, stream>>>(dP);
                PGC_CUDA(cudaGetLastError());
                PGC_CUDA(cudaGraphLaunch(exec[1], stream));
            }
        } else {
            KernelTimer kt;
            kt.prof = o.profile;
            kt.stream = stream;
            const cudaGraphConditionalHandle none = 0;
            PGC_CUDA(cudaMemsetAsync(state.ptr, 0, sizeof(State), stream));
#define PGC_TIMED(slot, name, launch_)                        \
    do {                                                      \
        if (pgc_status s_ = kt.begin(slot, name)) return s_;  \
        launch_;                                              \
        PGC_CUDA(cudaGetLastError());                         \
        if (pgc_status s_ = kt.end()) return s_;              \
    } while (0)
            PGC_TIMED(0, "d1_classify", (d1_classify<V><<<g.grid, g.block, g.smem, stream>>>(dP)));
            PGC_TIMED(1, "d1_build",
                      (d1_build<V><<<g.grid, g.block, 0, stream>>>(dP, 0, INT32_MAX)));
            PGC_TIMED(2, "d1_tier", (d1_tier<V><<<g.grid, g.block, g.smem, stream>>>(dP)));
            for (int round = 1;; ++round) {
                if (round > 1 || hp->async_mode)
                    PGC_TIMED(3, "d1_assign",
                              (d1_assign<V><<<g.grid, g.block, 0, stream>>>(dP, none, 0)));
                PGC_TIMED(4, "d1_detect",
                          (hp->prio_mode
                               ? d1_detect<V, true><<<g.det_grid, g.block, g.smem, stream>>>(
                                     dP, none, 0)
                               : d1_detect<V><<<g.det_grid, g.block, g.smem, stream>>>(dP, none,
                                                                                      0)));
                PGC_TIMED(5, "d1_push", (d1_push<V><<<g.grid, g.block, 0, stream>>>(dP)));
                PGC_CUDA(cudaMemcpyAsync(hs, state.ptr, sizeof(State), cudaMemcpyDeviceToHost,
                                         stream));
                PGC_CUDA(cudaStreamSynchronize(stream));
                if (hs->done) break;
                if (hs->tail) {   // the remaining rounds: the core phase
                    if (pgc_status s_ = kt.begin(6, "d1_core")) return s_;
                    d1_core_map<V><<<g.grid, g.block, 0, stream>>>(dP);
                    d1_core_scan<V><<<1, 1024, 0, stream>>>(dP);
                    d1_core_fill<V><<<g.grid, g.block, 0, stream>>>(dP);
                    PGC_CUDA(cudaGetLastError());
                    void* args[] = {&dP};
                    PGC_CUDA(cudaLaunchCooperativeKernel((void*)d1_core_loop<V>, dim3(g.core_grid),
                                                         dim3(1024), args, 0, stream));
                    if (pgc_status s_ = kt.end()) return s_;
                    break;
                }
                if (round > hp->max_rounds + 1)
                    return fail(PGC_ERR_CUDA, "device round control did not finish the loop");
            }
#undef PGC_TIMED
            kt.destroy();
        }
        PGC_CUDA(cudaMemcpyAsync(hs, state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
        if (want_trace) {
            PGC_CUDA(cudaMemcpyAsync(h_misc.ptr, trace.ptr, (size_t)tcap * 3 * sizeof(long long),
                                     cudaMemcpyDeviceToHost, stream));
        }
        return PGC_OK;
    }

    // Reads the result of the last launch() (its stream must be complete).
    pgc_status finish(const Opts& o, int* rounds, int* num_colors) {
        State* hs = h_state.as<State>();
        const int want_trace = last_want_trace, tcap = last_tcap;
        if (want_trace && o.profile) {
            const long long* tw = h_misc.as<long long>();
            const long long* ts = tw + tcap;
            const long long* th = ts + tcap;
            const int nr = std::min(hs->round, want_trace);
            for (int i = 0; i < want_trace; ++i) {
                if (o.profile->trace_w) o.profile->trace_w[i] = i < nr ? tw[i] : 0;
                if (o.profile->trace_s) o.profile->trace_s[i] = i < nr ? ts[i] : 0;
                if (o.profile->trace_h) o.profile->trace_h[i] = i < nr ? th[i] : 0;
            }
        }
        *rounds = hs->round;
        *num_colors = hs->max_color;
        switch (hs->status) {
            case ST_OK: return PGC_OK;
            case ST_NO_PROGRESS:
                return fail(PGC_ERR_NO_CONVERGE, "a round committed no vertex (input not symmetric?)");
            case ST_MAX_ROUNDS: return fail(PGC_ERR_NO_CONVERGE, "max_rounds reached");
            case ST_TIMEOUT: return fail(PGC_ERR_TIMEOUT, "device round loop exceeded timeout_ms");
            case ST_BARRIER:
                return fail(PGC_ERR_TIMEOUT, "a grid barrier of the core loop timed out");
            default: return fail(PGC_ERR_CUDA, "unexpected device status");
        }
    }
};

// One engine per device and view type, created on first use.
template <class V>
Engine<V>* engine_for(int device) {
    static std::mutex mu;
    static std::unordered_map<int, std::unique_ptr<Engine<V>>> m;
    std::lock_guard<std::mutex> lk(mu);
    auto it = m.find(device);
    if (it != m.end()) return it->second.get();
    if (m.empty()) {
        release_hooks().push_back([] {
            std::lock_guard<std::mutex> lk2(mu);
            int cur = 0;
            cudaGetDevice(&cur);
            auto f = m.find(cur);
            if (f != m.end()) {
                std::lock_guard<std::mutex> lk3(f->second->mu);
                f->second->release();
            }
        });
    }
    auto e = std::make_unique<Engine<V>>();
    Engine<V>* p = e.get();
    m.emplace(device, std::move(e));
    return p;
}

}  // namespace d1
}  // namespace pgc
