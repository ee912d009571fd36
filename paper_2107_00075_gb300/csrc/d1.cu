// d1.cu -- distance-1 coloring: kernels and the pgc_color_d1 entry point.
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
//   * First fit reads a per-vertex bitmap of forbidden colors (deg(v)+1
//     bits).  When a vertex commits color c it sets bit c in the bitmaps of
//     its still-uncolored neighbors ("push"); each edge is pushed at most
//     once, so the total push work is one pass over the adjacency.
//
// Color encoding in col[]: > 0 committed; < 0 tentative (-t) for a vertex
// on the current worklist.  Every uncolored vertex is on the worklist, so
// |col[u]| is u's current color during detection; a winner flips its own
// sign in place without disturbing concurrent readers.
//
// Worklists are split by |H(v)| into tiers: S (one thread per vertex),
// M (one warp), L (one thread block).  The round loop runs on the device: a
// CUDA graph with a conditional WHILE node around {assign, detect, push};
// the last block of detect updates the round state and sets the condition.
#include "runtime.h"
#include "device_common.cuh"

#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>
#include <unordered_map>

namespace pgc {
std::vector<std::function<void()>>& release_hooks();

namespace d1 {

enum { TIER_S = 0, TIER_M = 1, TIER_L = 2, NTIER = 3 };
constexpr int kPushChunk = 512;      // adjacency entries per push work item
constexpr int kInlinePush = 32;      // S-tier winners up to this degree push inline

enum : int { ST_OK = 0, ST_NO_PROGRESS = 1, ST_MAX_ROUNDS = 2, ST_TIMEOUT = 3 };

struct State {
    int round;        // round being executed (1-based)
    int done;         // 1 once the loop has ended
    int status;       // ST_*
    int max_color;
    int cnt[2][NTIER];          // detect worklist sizes, [parity][tier]
    int cls_cnt[NTIER];         // setup: vertices per degree class
    int push_cnt;               // push work items queued this round
    unsigned blocks_done;       // last-block detection in detect
    unsigned hub_next_build;    // dynamic indices for block-per-vertex work
    unsigned hub_next_detect;
    int pad;
    unsigned long long s_next;  // sum of degrees of the next worklist
    unsigned long long h_next;  // sum of |H(v)| over the next worklist
    unsigned long long h_first; // sum of |H(v)| over all vertices
    unsigned long long t0;      // globaltimer at start
};

struct Problem {
    const int* row_ptr;
    const int* col_idx;
    int* col;
    int* deg;
    int* hlen;
    int* hadj;          // H(v) stored at hadj[row_ptr[v] ...]
    unsigned* bm;       // forbidden-color bitmaps
    int* wl[2][NTIER];  // worklists by parity and tier; wl[0] doubles as the
                        // degree classes during setup
    int2* push_q;       // (vertex, chunk) push work items
    long long* trace_w;
    long long* trace_s;
    long long* trace_h;
    State* st;
    unsigned long long seed;
    unsigned long long timeout_ns;
    int trace_cap;
    int n;
    int use_deg;
    int mid;            // tier thresholds on list length (detect) / degree (setup)
    int hub;
    int max_rounds;
};

__device__ __forceinline__ int tier_of(int d, int mid, int hub) {
    return d <= mid ? TIER_S : (d <= hub ? TIER_M : TIER_L);
}

// key(u) > key(v), hashing only when the degree term does not decide.
__device__ __forceinline__ bool higher(int du, int u, int dv, uint64_t hv, int v,
                                       unsigned long long seed, bool use_deg) {
    if (use_deg && du != dv) return du > dv;
    const uint64_t hu = prio_hash(seed, (uint32_t)u);
    if (hu != hv) return hu < hv;
    return u < v;
}

// Set bit (c-1) in u's bitmap if u is still uncolored and c <= deg(u)+1.
__device__ __forceinline__ void push_color(const Problem& P, int u, int c) {
    if (P.col[u] >= 0) return;
    const int ru = __ldg(P.row_ptr + u), du = __ldg(P.row_ptr + u + 1) - ru;
    if (c - 1 > du) return;
    atomicOr(P.bm + bitmap_offset(ru, u) + ((c - 1) >> 5), 1u << ((c - 1) & 31));
}

// ---------------------------------------------------------------------------
// setup 1: degrees, tentative color 1, empty bitmaps, degree classes
// ---------------------------------------------------------------------------
__global__ void d1_classify(const Problem* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int warp = threadIdx.x >> 5;
    WarpAppend app[NTIER];
    for (int t = 0; t < NTIER; ++t) app[t] = {smem + (warp * NTIER + t) * 64, 0};
    const int n = P.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < n;
         wbase += stride) {
        const long long i = wbase + lane_id();
        const bool valid = i < n;
        int t = -1;
        if (valid) {
            const int r0 = __ldg(P.row_ptr + i), d = __ldg(P.row_ptr + i + 1) - r0;
            P.deg[i] = d;
            P.col[i] = -1;
            unsigned* b = P.bm + bitmap_offset(r0, (int)i);
            for (int w = 0; w <= (d >> 5); ++w) b[w] = 0u;
            t = tier_of(d, P.mid, P.hub);
        }
        for (int k = 0; k < NTIER; ++k)
            wa_push(app[k], valid && t == k, (int)i, P.wl[0][k], &st->cls_cnt[k]);
    }
    for (int k = 0; k < NTIER; ++k) wa_flush(app[k], P.wl[0][k], &st->cls_cnt[k]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->round = 1;
        st->t0 = global_ns();
        if (P.trace_cap > 0) {
            P.trace_w[0] = n;
            P.trace_s[0] = __ldg(P.row_ptr + n);
        }
    }
}

// ---------------------------------------------------------------------------
// setup 2: H(v) lists and the round-1 worklists (tiered by |H(v)|)
// ---------------------------------------------------------------------------
__global__ void d1_build(const Problem* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int* __restrict__ rp = P.row_ptr;
    const int* __restrict__ ci = P.col_idx;
    const int* __restrict__ dg = P.deg;
    const unsigned long long seed = P.seed;
    const bool use_deg = P.use_deg != 0;
    const int lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int nS = st->cls_cnt[TIER_S], nM = st->cls_cnt[TIER_M], nL = st->cls_cnt[TIER_L];
    unsigned long long my_h = 0ull;
    __shared__ int s_idx, s_pos;

    // large degree: one block per vertex
    for (;;) {
        if (threadIdx.x == 0) {
            s_idx = nL > 0 ? (int)atomicAdd(&st->hub_next_build, 1u) : nL;
            s_pos = 0;
        }
        __syncthreads();
        const int i = s_idx;
        if (i >= nL) break;
        const int v = P.wl[0][TIER_L][i];
        const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
        const uint64_t hv = prio_hash(seed, (uint32_t)v);
        for (int e = threadIdx.x; e < d; e += blockDim.x) {
            const int u = __ldg(ci + beg + e);
            if (u != v && higher(__ldg(dg + u), u, d, hv, v, seed, use_deg))
                P.hadj[beg + atomicAdd(&s_pos, 1)] = u;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int hl = s_pos;
            P.hlen[v] = hl;
            const int k = tier_of(hl, P.mid, P.hub);
            P.wl[1][k][atomicAdd(&st->cnt[1][k], 1)] = v;
            my_h += (unsigned long long)hl;
        }
        __syncthreads();
    }

    WarpAppend app[NTIER];
    for (int t = 0; t < NTIER; ++t) app[t] = {smem + (warp * NTIER + t) * 64, 0};

    // medium degree: one warp per vertex, ordered compaction by ballot
    for (int i = blockIdx.x * wpb + warp; i < nM; i += gridDim.x * wpb) {
        const int v = P.wl[0][TIER_M][i];
        const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
        const uint64_t hv = prio_hash(seed, (uint32_t)v);
        int pos = 0;
        for (int base = 0; base < d; base += 32) {
            const int e = base + lane;
            int u = -1;
            bool keep = false;
            if (e < d) {
                u = __ldg(ci + beg + e);
                keep = u != v && higher(__ldg(dg + u), u, d, hv, v, seed, use_deg);
            }
            const unsigned m = __ballot_sync(kFullMask, keep);
            if (keep) P.hadj[beg + pos + __popc(m & ((1u << lane) - 1u))] = u;
            pos += __popc(m);
        }
        if (lane == 0) {
            P.hlen[v] = pos;
            my_h += (unsigned long long)pos;
        }
        const int k = tier_of(pos, P.mid, P.hub);
        for (int t = 0; t < NTIER; ++t)
            wa_push(app[t], lane == 0 && k == t, v, P.wl[1][t], &st->cnt[1][t]);
    }

    // small degree: one thread per vertex
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < nS;
         wbase += stride) {
        const long long i = wbase + lane;
        int k = -1, v = -1;
        if (i < nS) {
            v = P.wl[0][TIER_S][i];
            const int beg = __ldg(rp + v), end = __ldg(rp + v + 1), d = end - beg;
            const uint64_t hv = prio_hash(seed, (uint32_t)v);
            int pos = beg;
            for (int e = beg; e < end; ++e) {
                const int u = __ldg(ci + e);
                if (u != v && higher(__ldg(dg + u), u, d, hv, v, seed, use_deg)) P.hadj[pos++] = u;
            }
            const int hl = pos - beg;
            P.hlen[v] = hl;
            my_h += (unsigned long long)hl;
            k = tier_of(hl, P.mid, P.hub);
        }
        for (int t = 0; t < NTIER; ++t)
            wa_push(app[t], k == t, v, P.wl[1][t], &st->cnt[1][t]);
    }
    for (int t = 0; t < NTIER; ++t) wa_flush(app[t], P.wl[1][t], &st->cnt[1][t]);
    my_h = warp_sum(my_h);
    if (lane == 0 && my_h) atomicAdd(&st->h_first, my_h);
}

// ---------------------------------------------------------------------------
// assign: first fit from the forbidden-color bitmap
// ---------------------------------------------------------------------------
__global__ void d1_assign(const Problem* __restrict__ Pp, cudaGraphConditionalHandle h,
                          int use_cond) {
    const Problem& P = *Pp;
    State* st = P.st;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // The loop continues only if this round's detect says so: should its
        // round control ever not run, the device loop ends instead of spinning.
        if (use_cond) cudaGraphSetConditional(h, 0u);
        st->push_cnt = 0;   // the previous round's push kernel has finished
    }
    const int cp = *(volatile int*)&st->round & 1;
    const int n0 = st->cnt[cp][TIER_S], n1 = st->cnt[cp][TIER_M], n2 = st->cnt[cp][TIER_L];
    const int total = n0 + n1 + n2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int v = i < n0 ? P.wl[cp][TIER_S][i]
                    : (i < n0 + n1 ? P.wl[cp][TIER_M][i - n0] : P.wl[cp][TIER_L][i - n0 - n1]);
        const int r0 = __ldg(P.row_ptr + v);
        const int words = (__ldg(P.deg + v) >> 5) + 1;
        const unsigned* b = P.bm + bitmap_offset(r0, v);
        int w = 0;
        unsigned word = b[0];
        while (word == kFullMask && w + 1 < words) word = b[++w];
        P.col[v] = -(w * 32 + __ffs(~word));
    }
}

// ---------------------------------------------------------------------------
// detect + commit + compact + inline push (+ round control in the last block)
// ---------------------------------------------------------------------------
__device__ void round_control(const Problem& P, cudaGraphConditionalHandle h, int use_cond) {
    State* st = P.st;
    const int r = st->round;
    const int cp = r & 1, np = cp ^ 1;
    long long cur = 0, nxt = 0;
    for (int k = 0; k < NTIER; ++k) {
        cur += *(volatile int*)&st->cnt[cp][k];
        nxt += *(volatile int*)&st->cnt[np][k];
    }
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
        for (int k = 0; k < NTIER; ++k) st->cnt[cp][k] = 0;
        st->round = r + 1;
        st->s_next = 0ull;
        st->h_next = 0ull;
    }
    st->status = status;
    st->done = done;
    st->hub_next_detect = 0u;
    st->blocks_done = 0u;
    __threadfence();
    if (use_cond) cudaGraphSetConditional(h, done ? 0u : 1u);
}

// Queue the push of v's color: ceil(deg/kPushChunk) work items.
__device__ __forceinline__ void queue_push(const Problem& P, int v, int d) {
    const int nch = (d + kPushChunk - 1) / kPushChunk;
    const int base = atomicAdd(&P.st->push_cnt, nch);
    for (int k = 0; k < nch; ++k) P.push_q[base + k] = make_int2(v, k);
}

__global__ void d1_detect(const Problem* __restrict__ Pp, cudaGraphConditionalHandle h,
                          int use_cond) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int r = *(volatile int*)&st->round;
    const int cp = r & 1, np = cp ^ 1;
    const int nS = st->cnt[cp][TIER_S], nM = st->cnt[cp][TIER_M], nL = st->cnt[cp][TIER_L];
    const int* __restrict__ rp = P.row_ptr;
    const int* __restrict__ ci = P.col_idx;
    const int* __restrict__ ha = P.hadj;
    int* col = P.col;
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    int my_max = 0;
    unsigned long long my_s = 0ull, my_h = 0ull;
    __shared__ int s_idx;

    // --- L tier: block per vertex (long H lists) ---
    if (nL > 0) {
        for (;;) {
            if (threadIdx.x == 0) s_idx = (int)atomicAdd(&st->hub_next_detect, 1u);
            __syncthreads();
            const int i = s_idx;
            if (i >= nL) break;
            const int v = P.wl[cp][TIER_L][i];
            const int beg = __ldg(rp + v);
            const int hl = P.hlen[v];
            const int t = -col[v];
            bool lose = false;
            for (int base = 0; base < hl; base += blockDim.x) {
                const int e = base + threadIdx.x;
                const bool l = e < hl && abs(col[__ldg(ha + beg + e)]) == t;
                if (__syncthreads_or(l)) {
                    lose = true;
                    break;
                }
            }
            if (threadIdx.x == 0) {
                const int d = __ldg(rp + v + 1) - beg;
                if (lose) {
                    P.wl[np][TIER_L][atomicAdd(&st->cnt[np][TIER_L], 1)] = v;
                    my_s += (unsigned long long)d;
                    my_h += (unsigned long long)hl;
                } else {
                    col[v] = t;
                    my_max = max(my_max, t);
                    queue_push(P, v, d);
                }
            }
            __syncthreads();
        }
    }

    // --- M tier: warp per vertex ---
    WarpAppend app = {smem + warp * 64, 0};
    for (int i = blockIdx.x * wpb + warp; i < nM; i += gridDim.x * wpb) {
        const int v = P.wl[cp][TIER_M][i];
        const int beg = __ldg(rp + v);
        const int hl = P.hlen[v];
        const int t = -col[v];
        bool lose = false;
        for (int base = 0; base < hl; base += 32) {
            const int e = base + lane;
            const bool l = e < hl && abs(col[__ldg(ha + beg + e)]) == t;
            if (__any_sync(kFullMask, l)) {
                lose = true;
                break;
            }
        }
        if (lane == 0) {
            const int d = __ldg(rp + v + 1) - beg;
            if (lose) {
                my_s += (unsigned long long)d;
                my_h += (unsigned long long)hl;
            } else {
                col[v] = t;
                my_max = max(my_max, t);
                queue_push(P, v, d);
            }
        }
        wa_push(app, lose && lane == 0, v, P.wl[np][TIER_M], &st->cnt[np][TIER_M]);
    }
    wa_flush(app, P.wl[np][TIER_M], &st->cnt[np][TIER_M]);

    // --- S tier: thread per vertex ---
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < nS;
         wbase += stride) {
        const long long i = wbase + lane;
        bool lose = false;
        int v = -1;
        if (i < nS) {
            v = P.wl[cp][TIER_S][i];
            const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
            const int hl = P.hlen[v];
            const int t = -col[v];
            for (int e = 0; e < hl; ++e)
                if (abs(col[__ldg(ha + beg + e)]) == t) {
                    lose = true;
                    break;
                }
            if (lose) {
                my_s += (unsigned long long)d;
                my_h += (unsigned long long)hl;
            } else {
                col[v] = t;
                my_max = max(my_max, t);
                if (d <= kInlinePush) {
                    for (int e = beg; e < beg + d; ++e) {
                        const int u = __ldg(ci + e);
                        if (u != v) push_color(P, u, t);
                    }
                } else {
                    queue_push(P, v, d);
                }
            }
        }
        wa_push(app, lose, v, P.wl[np][TIER_S], &st->cnt[np][TIER_S]);
    }
    wa_flush(app, P.wl[np][TIER_S], &st->cnt[np][TIER_S]);

    // --- per-warp totals ---
    my_max = warp_max(my_max);
    my_s = warp_sum(my_s);
    my_h = warp_sum(my_h);
    if (lane == 0) {
        if (my_max > 0) atomicMax(&st->max_color, my_max);
        if (my_s > 0) atomicAdd(&st->s_next, my_s);
        if (my_h > 0) atomicAdd(&st->h_next, my_h);
    }

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
// push: winners' colors into the bitmaps of uncolored neighbors
// ---------------------------------------------------------------------------
__global__ void d1_push(const Problem* __restrict__ Pp) {
    const Problem& P = *Pp;
    const int nq = *(volatile int*)&P.st->push_cnt;
    const int lane = lane_id(), wpb = blockDim.x >> 5;
    for (int q = blockIdx.x * wpb + (threadIdx.x >> 5); q < nq; q += gridDim.x * wpb) {
        const int2 item = P.push_q[q];
        const int v = item.x;
        const int c = P.col[v];
        const int r0 = __ldg(P.row_ptr + v), r1 = __ldg(P.row_ptr + v + 1);
        const int beg = r0 + item.y * kPushChunk, end = min(beg + kPushChunk, r1);
        for (int e = beg + lane; e < end; e += 32) {
            const int u = __ldg(P.col_idx + e);
            if (u != v) push_color(P, u, c);
        }
    }
}

// ---------------------------------------------------------------------------
// optional input validation (PGC_VALIDATE): shape and id range
// ---------------------------------------------------------------------------
__global__ void d1_validate_offsets(const int* __restrict__ rp, int n, int* bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (rp[v + 1] < rp[v]) atomicOr(bad, 1);
    if (blockIdx.x == 0 && threadIdx.x == 0 && rp[0] != 0) atomicOr(bad, 1);
}

// Runs only after the offsets passed, so every e < rp[n] is inside col_idx.
__global__ void d1_validate_ids(const int* __restrict__ rp, const int* __restrict__ ci, int n,
                                int* bad) {
    const long long nnz = rp[n];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        if ((unsigned)ci[e] >= (unsigned)n) atomicOr(bad, 2);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Context {
    std::mutex mu;
    DeviceInfo dev;
    DevBuf deg, hlen, hadj, bm, wl, pushq, state, problem, trace, stage_rp, stage_ci, stage_col,
        flag;
    HostBuf h_problem, h_state, h_misc;
    int trace_cap = 0;
    // graph (valid for the launch geometry below)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int g_grid = 0, g_block = 0;

    void destroy_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        g_grid = 0;
    }
    void release() {
        destroy_graph();
        for (DevBuf* b : {&deg, &hlen, &hadj, &bm, &wl, &pushq, &state, &problem, &trace,
                          &stage_rp, &stage_ci, &stage_col, &flag})
            b->release();
        for (HostBuf* b : {&h_problem, &h_state, &h_misc}) b->release();
        trace_cap = 0;
    }
};

static std::mutex g_ctx_mu;
static std::unordered_map<int, std::unique_ptr<Context>>& contexts() {
    static std::unordered_map<int, std::unique_ptr<Context>> m;
    return m;
}

static Context* get_context(int device) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    auto& m = contexts();
    auto it = m.find(device);
    if (it != m.end()) return it->second.get();
    static bool hooked = false;
    if (!hooked) {
        hooked = true;
        release_hooks().push_back([] {
            std::lock_guard<std::mutex> lk2(g_ctx_mu);
            int cur = 0;
            cudaGetDevice(&cur);
            auto f = contexts().find(cur);
            if (f != contexts().end()) {
                std::lock_guard<std::mutex> lk3(f->second->mu);
                f->second->release();
            }
        });
    }
    auto c = std::make_unique<Context>();
    Context* p = c.get();
    m.emplace(device, std::move(c));
    return p;
}

struct Geometry {
    int grid, block;
    size_t smem_setup, smem_detect;
};

static pgc_status geometry(const Context& cx, const Opts& o, Geometry* g) {
    const int block = o.block;
    const int wpb = block / 32;
    g->block = block;
    g->smem_setup = (size_t)wpb * NTIER * 64 * sizeof(int);
    g->smem_detect = (size_t)wpb * 64 * sizeof(int);
    int per_sm = o.grid_per_sm;
    if (per_sm == 0) {
        int a = 0, b = 0;
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, d1_detect, block, g->smem_detect));
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, d1_build, block, g->smem_setup));
        per_sm = std::max(1, std::min(a, b));
    }
    g->grid = cx.dev.num_sms * per_sm;
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

static pgc_status build_graph(Context& cx, const Geometry& g) {
    cx.destroy_graph();
    Problem* dP = cx.problem.as<Problem>();
    PGC_CUDA(cudaGraphCreate(&cx.graph, 0));
    PGC_CUDA(cudaGraphConditionalHandleCreate(&cx.handle, cx.graph, 0u, cudaGraphCondAssignDefault));
    int use_cond = 1;
    cudaGraphConditionalHandle hnd = cx.handle;
    void* p_args[] = {&dP};
    void* c_args[] = {&dP, &hnd, &use_cond};

    cudaGraphNode_t n_memset, n_cls, n_build, n_det1, n_push1, n_loop;
    cudaMemsetParams ms = {};
    ms.dst = cx.state.ptr;
    ms.value = 0;
    ms.elementSize = 4;
    ms.width = sizeof(State) / 4;
    ms.height = 1;
    PGC_CUDA(cudaGraphAddMemsetNode(&n_memset, cx.graph, nullptr, 0, &ms));
    cudaKernelNodeParams k_cls = knode((void*)d1_classify, g, g.smem_setup, p_args);
    cudaKernelNodeParams k_build = knode((void*)d1_build, g, g.smem_setup, p_args);
    cudaKernelNodeParams k_det = knode((void*)d1_detect, g, g.smem_detect, c_args);
    cudaKernelNodeParams k_push = knode((void*)d1_push, g, 0, p_args);
    cudaKernelNodeParams k_asg = knode((void*)d1_assign, g, 0, c_args);
    PGC_CUDA(cudaGraphAddKernelNode(&n_cls, cx.graph, &n_memset, 1, &k_cls));
    PGC_CUDA(cudaGraphAddKernelNode(&n_build, cx.graph, &n_cls, 1, &k_build));
    PGC_CUDA(cudaGraphAddKernelNode(&n_det1, cx.graph, &n_build, 1, &k_det));
    PGC_CUDA(cudaGraphAddKernelNode(&n_push1, cx.graph, &n_det1, 1, &k_push));

    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cx.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    PGC_CUDA(cudaGraphAddNode(&n_loop, cx.graph, &n_push1, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t b_asg, b_det, b_push;
    PGC_CUDA(cudaGraphAddKernelNode(&b_asg, body, nullptr, 0, &k_asg));
    PGC_CUDA(cudaGraphAddKernelNode(&b_det, body, &b_asg, 1, &k_det));
    PGC_CUDA(cudaGraphAddKernelNode(&b_push, body, &b_det, 1, &k_push));

    PGC_CUDA(cudaGraphInstantiate(&cx.exec, cx.graph, 0));
    cx.g_grid = g.grid;
    cx.g_block = g.block;
    return PGC_OK;
}

static pgc_status run(Context& cx, int n, long long nnz, const int* d_rp, const int* d_ci,
                      int* d_col, uint64_t seed, const Opts& o, cudaStream_t stream, int* rounds,
                      int* num_colors) {
    // --- scratch (grows, never shrinks; pointers live in the Problem struct,
    //     so the captured graph stays valid across calls) ---
    const size_t bm_words = (size_t)(nnz >> 5) + (size_t)n + 1;
    const size_t q_items = (size_t)n + (size_t)(nnz / kPushChunk) + 1;
    if (pgc_status s = cx.deg.ensure((size_t)n * 4)) return s;
    if (pgc_status s = cx.hlen.ensure((size_t)n * 4)) return s;
    if (pgc_status s = cx.hadj.ensure((size_t)std::max<long long>(nnz, 1) * 4)) return s;
    if (pgc_status s = cx.bm.ensure(bm_words * 4)) return s;
    if (pgc_status s = cx.wl.ensure((size_t)n * 4 * 2 * NTIER)) return s;
    if (pgc_status s = cx.pushq.ensure(q_items * sizeof(int2))) return s;
    if (pgc_status s = cx.state.ensure(sizeof(State))) return s;
    if (pgc_status s = cx.problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_state.ensure(sizeof(State))) return s;
    const int want_trace = o.profile && o.profile->trace_cap > 0 ? o.profile->trace_cap : 0;
    const int tcap = std::max(want_trace, 1);
    if (cx.trace_cap < tcap) {
        if (pgc_status s = cx.trace.ensure((size_t)tcap * 3 * sizeof(long long))) return s;
        if (pgc_status s = cx.h_misc.ensure((size_t)tcap * 3 * sizeof(long long))) return s;
        cx.trace_cap = tcap;
    }

    Geometry g;
    if (pgc_status s = geometry(cx, o, &g)) return s;

    Problem* hp = cx.h_problem.as<Problem>();
    std::memset(hp, 0, sizeof(Problem));
    hp->row_ptr = d_rp;
    hp->col_idx = d_ci;
    hp->col = d_col;
    hp->deg = cx.deg.as<int>();
    hp->hlen = cx.hlen.as<int>();
    hp->hadj = cx.hadj.as<int>();
    hp->bm = cx.bm.as<unsigned>();
    int* wl = cx.wl.as<int>();
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < NTIER; ++k) hp->wl[p][k] = wl + (size_t)(p * NTIER + k) * n;
    hp->push_q = cx.pushq.as<int2>();
    hp->trace_w = cx.trace.as<long long>();
    hp->trace_s = hp->trace_w + tcap;
    hp->trace_h = hp->trace_s + tcap;
    hp->trace_cap = want_trace;
    hp->st = cx.state.as<State>();
    hp->seed = seed;
    hp->timeout_ns = (unsigned long long)o.timeout_ms * 1000000ull;
    hp->n = n;
    hp->use_deg = (o.flags & PGC_NO_DEGREE_RULE) ? 0 : 1;
    hp->mid = o.mid_degree;
    hp->hub = o.hub_degree;
    hp->max_rounds = o.max_rounds > 0 ? o.max_rounds : (n < INT32_MAX ? n + 1 : n);
    PGC_CUDA(cudaMemcpyAsync(cx.problem.ptr, hp, sizeof(Problem), cudaMemcpyHostToDevice, stream));
    Problem* dP = cx.problem.as<Problem>();

    State* hs = cx.h_state.as<State>();
    if (!(o.flags & PGC_HOST_LOOP)) {
        if (!cx.exec || cx.g_grid != g.grid || cx.g_block != g.block) {
            if (pgc_status s = build_graph(cx, g)) return s;
        }
        PGC_CUDA(cudaGraphLaunch(cx.exec, stream));
    } else {
        KernelTimer kt;
        kt.prof = o.profile;
        kt.stream = stream;
        const cudaGraphConditionalHandle none = 0;
        PGC_CUDA(cudaMemsetAsync(cx.state.ptr, 0, sizeof(State), stream));
        if (pgc_status s = kt.begin(0, "d1_classify")) return s;
        d1_classify<<<g.grid, g.block, g.smem_setup, stream>>>(dP);
        PGC_CUDA(cudaGetLastError());
        if (pgc_status s = kt.end()) return s;
        if (pgc_status s = kt.begin(1, "d1_build")) return s;
        d1_build<<<g.grid, g.block, g.smem_setup, stream>>>(dP);
        PGC_CUDA(cudaGetLastError());
        if (pgc_status s = kt.end()) return s;
        for (int round = 1;; ++round) {
            if (round > 1) {
                if (pgc_status s = kt.begin(2, "d1_assign")) return s;
                d1_assign<<<g.grid, g.block, 0, stream>>>(dP, none, 0);
                PGC_CUDA(cudaGetLastError());
                if (pgc_status s = kt.end()) return s;
            }
            if (pgc_status s = kt.begin(3, "d1_detect")) return s;
            d1_detect<<<g.grid, g.block, g.smem_detect, stream>>>(dP, none, 0);
            PGC_CUDA(cudaGetLastError());
            if (pgc_status s = kt.end()) return s;
            if (pgc_status s = kt.begin(4, "d1_push")) return s;
            d1_push<<<g.grid, g.block, 0, stream>>>(dP);
            PGC_CUDA(cudaGetLastError());
            if (pgc_status s = kt.end()) return s;
            PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
            PGC_CUDA(cudaStreamSynchronize(stream));
            if (hs->done) break;
            if (round > hp->max_rounds + 1)
                return fail(PGC_ERR_CUDA, "device round control did not finish the loop");
        }
        kt.destroy();
    }
    PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
    if (want_trace) {
        PGC_CUDA(cudaMemcpyAsync(cx.h_misc.ptr, cx.trace.ptr, (size_t)tcap * 3 * sizeof(long long),
                                 cudaMemcpyDeviceToHost, stream));
    }
    PGC_CUDA(cudaStreamSynchronize(stream));
    if (want_trace) {
        const long long* tw = cx.h_misc.as<long long>();
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
        default: return fail(PGC_ERR_CUDA, "unexpected device status");
    }
}

static pgc_status color(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, uint64_t seed,
                        int32_t* colors, int32_t* rounds, int32_t* num_colors,
                        const pgc_opts* opts, void* stream_v) {
    if (!rounds || !num_colors) return fail(PGC_ERR_INVALID_ARG, "rounds/num_colors must be non-NULL");
    if (n < 0) return fail(PGC_ERR_INVALID_ARG, "n < 0");
    Opts o;
    if (pgc_status s = read_opts(opts, &o)) return s;
    *rounds = 0;
    *num_colors = 0;
    if (n == 0) return PGC_OK;
    if (!row_ptr || !colors) return fail(PGC_ERR_INVALID_ARG, "NULL array");
    cudaStream_t stream = (cudaStream_t)stream_v;
    DeviceInfo dev;
    if (pgc_status s = current_device(&dev)) return s;
    Context* cx = get_context(dev.device);
    std::lock_guard<std::mutex> lk(cx->mu);
    cx->dev = dev;

    const bool host_rp = is_host_pointer(row_ptr);
    const bool host_ci = col_idx ? is_host_pointer(col_idx) : host_rp;
    const bool host_col = is_host_pointer(colors);
    const int* d_rp = row_ptr;
    const int* d_ci = col_idx;
    int* d_col = colors;
    int nnz = 0;
    if (host_rp) {
        nnz = row_ptr[n];
    } else {
        if (pgc_status s = cx->h_state.ensure(sizeof(State))) return s;
        int* hb = cx->h_state.as<int>();
        PGC_CUDA(cudaMemcpyAsync(hb, row_ptr + n, 4, cudaMemcpyDeviceToHost, stream));
        PGC_CUDA(cudaStreamSynchronize(stream));
        nnz = *hb;
    }
    if (nnz < 0) return fail(PGC_ERR_INVALID_ARG, "row_ptr[n] < 0");
    if (nnz > 0 && !col_idx) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx");
    if (host_rp || host_ci) {
        if (host_rp) {
            if (pgc_status s = cx->stage_rp.ensure((size_t)(n + 1) * 4)) return s;
            PGC_CUDA(cudaMemcpyAsync(cx->stage_rp.ptr, row_ptr, (size_t)(n + 1) * 4,
                                     cudaMemcpyHostToDevice, stream));
            d_rp = cx->stage_rp.as<int>();
        }
        if (host_ci && nnz > 0) {
            if (pgc_status s = cx->stage_ci.ensure((size_t)nnz * 4)) return s;
            PGC_CUDA(cudaMemcpyAsync(cx->stage_ci.ptr, col_idx, (size_t)nnz * 4,
                                     cudaMemcpyHostToDevice, stream));
            d_ci = cx->stage_ci.as<int>();
        }
    }
    if (host_col) {
        if (pgc_status s = cx->stage_col.ensure((size_t)n * 4)) return s;
        d_col = cx->stage_col.as<int>();
    }
    if (o.flags & PGC_VALIDATE) {
        if (pgc_status s = cx->flag.ensure(4)) return s;
        if (pgc_status s = cx->h_state.ensure(sizeof(State))) return s;
        int* hb = cx->h_state.as<int>();
        PGC_CUDA(cudaMemsetAsync(cx->flag.ptr, 0, 4, stream));
        d1_validate_offsets<<<cx->dev.num_sms * 4, 256, 0, stream>>>(d_rp, n, cx->flag.as<int>());
        PGC_CUDA(cudaGetLastError());
        PGC_CUDA(cudaMemcpyAsync(hb, cx->flag.ptr, 4, cudaMemcpyDeviceToHost, stream));
        PGC_CUDA(cudaStreamSynchronize(stream));
        if (*hb) return fail(PGC_ERR_INVALID_ARG, "row_ptr is not a valid offset array");
        if (!d_ci) {
            PGC_CUDA(cudaMemcpyAsync(hb, d_rp + n, 4, cudaMemcpyDeviceToHost, stream));
            PGC_CUDA(cudaStreamSynchronize(stream));
            if (*hb != 0) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx with row_ptr[n] > 0");
        } else {
            d1_validate_ids<<<cx->dev.num_sms * 4, 256, 0, stream>>>(d_rp, d_ci, n,
                                                                     cx->flag.as<int>());
            PGC_CUDA(cudaGetLastError());
            PGC_CUDA(cudaMemcpyAsync(hb, cx->flag.ptr, 4, cudaMemcpyDeviceToHost, stream));
            PGC_CUDA(cudaStreamSynchronize(stream));
            if (*hb) return fail(PGC_ERR_INVALID_ARG, "col_idx entry out of [0, n)");
        }
    }
    pgc_status s = run(*cx, n, nnz, d_rp, d_ci, d_col, seed, o, stream, rounds, num_colors);
    if (s != PGC_OK) return s;
    if (host_col) {
        PGC_CUDA(cudaMemcpyAsync(colors, d_col, (size_t)n * 4, cudaMemcpyDeviceToHost, stream));
        PGC_CUDA(cudaStreamSynchronize(stream));
    }
    return PGC_OK;
}

}  // namespace d1
}  // namespace pgc

extern "C" pgc_status pgc_color_d1(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                   uint64_t seed, int32_t* colors, int32_t* rounds,
                                   int32_t* num_colors, const pgc_opts* opts, void* stream) {
    try {
        return pgc::d1::color(n, row_ptr, col_idx, seed, colors, rounds, num_colors, opts, stream);
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    } catch (...) {
        return pgc::fail(PGC_ERR_CUDA, "unknown exception");
    }
}
