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
// Color encoding in col[]: > 0 committed; < 0 tentative (-t) for a vertex
// on the current worklist.  Every uncolored vertex is on the worklist, so
// |col[u]| is u's current color during detection; a winner flips its own
// sign in place without disturbing concurrent readers.  The first-fit step
// only looks at col[u] > 0 and so never sees this round's tentative colors.
//
// Work is split by degree into three worklists (tiers):
//   S: deg <= mid_degree  -- one thread per vertex, one 64-bit window
//   M: deg <= hub_degree  -- one warp per vertex, shared-memory bitmap
//   L: larger             -- one thread block per vertex, windowed bitmap
// The round loop runs on the device: a CUDA graph with a conditional WHILE
// node around {assign, detect}; the last block of detect updates the round
// state and sets the loop condition.
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
constexpr int kHubWords = 256;  // hub bitmap window: 8192 colors
constexpr unsigned kFull = 0xffffffffu;

enum : int { ST_OK = 0, ST_NO_PROGRESS = 1, ST_MAX_ROUNDS = 2, ST_TIMEOUT = 3, ST_BAD_INPUT = 4 };

struct State {
    int round;        // round being executed (1-based)
    int done;         // 1 once the loop has ended
    int status;       // ST_*
    int max_color;
    int cnt[2][NTIER];          // worklist sizes, [parity][tier]
    unsigned blocks_done;       // last-block detection in detect
    unsigned hub_next_assign;   // dynamic index into the hub worklist
    unsigned hub_next_detect;
    int pad;
    unsigned long long s_next;  // sum of degrees of the next worklist
    unsigned long long t0;      // globaltimer at start
};

struct Problem {
    const int* row_ptr;
    const int* col_idx;
    int* col;
    int* deg;
    int* wl[2][NTIER];
    long long* trace_w;
    long long* trace_s;
    State* st;
    unsigned long long seed;
    unsigned long long timeout_ns;
    int trace_cap;
    int n;
    int use_deg;
    int mid_deg;
    int hub_deg;
    int max_rounds;
};

// ---------------------------------------------------------------------------
// warp-aggregated worklist append: lanes push (pred, v); a per-warp shared
// buffer of 64 slots is flushed 32 at a time with one atomic.
// ---------------------------------------------------------------------------
struct WarpAppend {
    int* buf;    // 64 ints of shared memory owned by this warp
    int count;   // warp-uniform
};

__device__ __forceinline__ void wa_push(WarpAppend& a, bool pred, int v, int* out, int* out_cnt) {
    const unsigned lane = lane_id();
    unsigned m = __ballot_sync(kFull, pred);
    if (pred) a.buf[a.count + __popc(m & ((1u << lane) - 1u))] = v;
    a.count += __popc(m);
    __syncwarp();
    if (a.count >= 32) {
        int base = 0;
        if (lane == 0) base = atomicAdd(out_cnt, 32);
        base = __shfl_sync(kFull, base, 0);
        out[base + lane] = a.buf[lane];
        int rem = a.count - 32;
        int tmp = (int)lane < rem ? a.buf[32 + lane] : 0;
        __syncwarp();
        if ((int)lane < rem) a.buf[lane] = tmp;
        a.count = rem;
        __syncwarp();
    }
}

__device__ __forceinline__ void wa_flush(WarpAppend& a, int* out, int* out_cnt) {
    if (a.count == 0) return;
    const unsigned lane = lane_id();
    int base = 0;
    if (lane == 0) base = atomicAdd(out_cnt, a.count);
    base = __shfl_sync(kFull, base, 0);
    if ((int)lane < a.count) out[base + lane] = a.buf[lane];
    a.count = 0;
    __syncwarp();
}

__device__ __forceinline__ int tier_of(int d, int mid, int hub) {
    return d <= mid ? TIER_S : (d <= hub ? TIER_M : TIER_L);
}

__device__ __forceinline__ int warp_max(int x) {
    for (int o = 16; o; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
    return x;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// init: degrees, tentative color 1 for all, tier worklists for round 1
// ---------------------------------------------------------------------------
__global__ void d1_init(const Problem* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int warp = threadIdx.x >> 5;
    WarpAppend app[NTIER];
    for (int t = 0; t < NTIER; ++t) app[t] = {smem + (warp * NTIER + t) * 64, 0};
    const int n = P.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform trip count: the append below needs all 32 lanes
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < n;
         wbase += stride) {
        const long long i = wbase + lane_id();
        const bool valid = i < n;
        int d = 0, t = -1;
        if (valid) {
            d = __ldg(P.row_ptr + i + 1) - __ldg(P.row_ptr + i);
            P.deg[i] = d;
            P.col[i] = -1;
            t = tier_of(d, P.mid_deg, P.hub_deg);
        }
        for (int k = 0; k < NTIER; ++k)
            wa_push(app[k], valid && t == k, (int)i, P.wl[1][k], &st->cnt[1][k]);
    }
    for (int k = 0; k < NTIER; ++k) wa_flush(app[k], P.wl[1][k], &st->cnt[1][k]);
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
// assign: first fit over committed neighbor colors
// ---------------------------------------------------------------------------
__global__ void d1_assign(const Problem* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int r = *(volatile int*)&st->round;
    const int cp = r & 1;
    const int nS = st->cnt[cp][TIER_S], nM = st->cnt[cp][TIER_M], nL = st->cnt[cp][TIER_L];
    const int* __restrict__ rp = P.row_ptr;
    const int* __restrict__ ci = P.col_idx;
    int* col = P.col;
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int mid_words = (P.hub_deg + 1 + 31) / 32;

    // --- L tier: one block per hub vertex, 8192-color windows ---
    unsigned* hub_bm = reinterpret_cast<unsigned*>(smem);             // kHubWords
    __shared__ int s_idx, s_first;
    if (nL > 0) {
        for (;;) {
            if (threadIdx.x == 0) s_idx = (int)atomicAdd(&st->hub_next_assign, 1u);
            __syncthreads();
            const int i = s_idx;
            if (i >= nL) break;
            const int v = P.wl[cp][TIER_L][i];
            const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
            int t = 0;
            for (int base = 0; t == 0; base += kHubWords * 32) {
                for (int w = threadIdx.x; w < kHubWords; w += blockDim.x) hub_bm[w] = 0u;
                if (threadIdx.x == 0) s_first = kHubWords;
                __syncthreads();
                for (int e = threadIdx.x; e < d; e += blockDim.x) {
                    const int c = col[__ldg(ci + beg + e)] - 1 - base;
                    if (c >= 0 && c < kHubWords * 32) atomicOr(&hub_bm[c >> 5], 1u << (c & 31));
                }
                __syncthreads();
                for (int w = threadIdx.x; w < kHubWords; w += blockDim.x)
                    if (hub_bm[w] != kFull) atomicMin(&s_first, w);
                __syncthreads();
                if (s_first < kHubWords) t = base + s_first * 32 + __ffs(~hub_bm[s_first]);
                __syncthreads();
            }
            if (threadIdx.x == 0) col[v] = -t;
        }
    }

    // --- M tier: one warp per vertex, bitmap of deg+1 colors ---
    unsigned* bm = reinterpret_cast<unsigned*>(smem) + kHubWords + warp * mid_words;
    const int gw = blockIdx.x * wpb + warp, nw = gridDim.x * wpb;
    for (int i = gw; i < nM; i += nw) {
        const int v = P.wl[cp][TIER_M][i];
        const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
        const int words = (d + 1 + 31) >> 5;
        for (int w = lane; w < words; w += 32) bm[w] = 0u;
        __syncwarp();
        for (int e = lane; e < d; e += 32) {
            const int c = col[__ldg(ci + beg + e)] - 1;
            if (c >= 0 && c <= d) atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        int t = 0;
        for (int w0 = 0; w0 < words; w0 += 32) {
            const int w = w0 + lane;
            const unsigned word = w < words ? bm[w] : kFull;
            const unsigned m = __ballot_sync(kFull, word != kFull);
            if (m) {
                const int src = __ffs(m) - 1;
                const unsigned fw = __shfl_sync(kFull, word, src);
                t = (w0 + src) * 32 + __ffs(~fw);
                break;
            }
        }
        if (lane == 0) col[v] = -t;
        __syncwarp();
    }

    // --- S tier: one thread per vertex, colors 1..64 ---
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int i = gt; i < nS; i += nt) {
        const int v = P.wl[cp][TIER_S][i];
        const int beg = __ldg(rp + v), end = __ldg(rp + v + 1);
        unsigned long long mask = 0ull;
        for (int e = beg; e < end; ++e) {
            const int c = col[__ldg(ci + e)];
            if (c > 0 && c <= 64) mask |= 1ull << (c - 1);
        }
        col[v] = -__ffsll((long long)~mask);
    }
}

// ---------------------------------------------------------------------------
// detect + commit + compact (+ round control in the last block)
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
    const unsigned long long s_next = *(volatile unsigned long long*)&st->s_next;
    if (r < P.trace_cap) {
        P.trace_w[r] = nxt;
        P.trace_s[r] = (long long)s_next;
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
        for (int k = 0; k < NTIER; ++k) st->cnt[cp][k] = 0;
        st->round = r + 1;
        st->s_next = 0ull;
    }
    st->status = status;
    st->done = done;
    st->hub_next_assign = 0u;
    st->hub_next_detect = 0u;
    st->blocks_done = 0u;
    __threadfence();
    if (use_cond) cudaGraphSetConditional(h, done ? 0u : 1u);
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
    const int* __restrict__ dg = P.deg;
    int* col = P.col;
    const unsigned long long seed = P.seed;
    const bool use_deg = P.use_deg != 0;
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    int my_max = 0;
    unsigned long long my_s = 0ull;
    __shared__ int s_idx;

    // --- L tier: block per vertex ---
    if (nL > 0) {
        for (;;) {
            if (threadIdx.x == 0) s_idx = (int)atomicAdd(&st->hub_next_detect, 1u);
            __syncthreads();
            const int i = s_idx;
            if (i >= nL) break;
            const int v = P.wl[cp][TIER_L][i];
            const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
            const int t = -col[v];
            const uint64_t hv = prio_hash(seed, (uint32_t)v);
            bool lose = false;
            for (int base = 0; base < d; base += blockDim.x) {
                bool l = false;
                const int e = base + threadIdx.x;
                if (e < d) {
                    const int u = __ldg(ci + beg + e);
                    if (u != v && abs(col[u]) == t)
                        l = has_priority(__ldg(dg + u), prio_hash(seed, (uint32_t)u), u, d, hv, v,
                                         use_deg);
                }
                if (__syncthreads_or(l)) {
                    lose = true;
                    break;
                }
            }
            if (threadIdx.x == 0) {
                if (lose) {
                    const int pos = atomicAdd(&st->cnt[np][TIER_L], 1);
                    P.wl[np][TIER_L][pos] = v;
                    my_s += (unsigned long long)d;
                } else {
                    col[v] = t;
                    my_max = max(my_max, t);
                }
            }
            __syncthreads();
        }
    }

    // --- M tier: warp per vertex ---
    WarpAppend app = {smem + warp * 64, 0};
    const int gw = blockIdx.x * wpb + warp, nw = gridDim.x * wpb;
    for (int i = gw; i < nM; i += nw) {
        const int v = P.wl[cp][TIER_M][i];
        const int beg = __ldg(rp + v), d = __ldg(rp + v + 1) - beg;
        const int t = -col[v];
        const uint64_t hv = prio_hash(seed, (uint32_t)v);
        bool lose = false;
        for (int base = 0; base < d; base += 32) {
            bool l = false;
            const int e = base + lane;
            if (e < d) {
                const int u = __ldg(ci + beg + e);
                if (u != v && abs(col[u]) == t)
                    l = has_priority(__ldg(dg + u), prio_hash(seed, (uint32_t)u), u, d, hv, v,
                                     use_deg);
            }
            if (__any_sync(kFull, l)) {
                lose = true;
                break;
            }
        }
        if (lane == 0) {
            if (lose) my_s += (unsigned long long)d;
            else {
                col[v] = t;
                my_max = max(my_max, t);
            }
        }
        wa_push(app, lose && lane == 0, v, P.wl[np][TIER_M], &st->cnt[np][TIER_M]);
    }
    wa_flush(app, P.wl[np][TIER_M], &st->cnt[np][TIER_M]);

    // --- S tier: thread per vertex (warp-uniform trip count for the append) ---
    const long long nt = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < nS;
         wbase += nt) {
        const long long i = wbase + lane;
        bool lose = false;
        int v = -1;
        if (i < nS) {
            v = P.wl[cp][TIER_S][i];
            const int beg = __ldg(rp + v), end = __ldg(rp + v + 1);
            const int d = end - beg;
            const int t = -col[v];
            const uint64_t hv = prio_hash(seed, (uint32_t)v);
            for (int e = beg; e < end; ++e) {
                const int u = __ldg(ci + e);
                if (u != v && abs(col[u]) == t &&
                    has_priority(__ldg(dg + u), prio_hash(seed, (uint32_t)u), u, d, hv, v,
                                 use_deg)) {
                    lose = true;
                    break;
                }
            }
            if (lose) my_s += (unsigned long long)d;
            else {
                col[v] = t;
                my_max = max(my_max, t);
            }
        }
        wa_push(app, lose, v, P.wl[np][TIER_S], &st->cnt[np][TIER_S]);
    }
    wa_flush(app, P.wl[np][TIER_S], &st->cnt[np][TIER_S]);

    // --- per-warp totals ---
    my_max = warp_max(my_max);
    my_s = warp_sum(my_s);
    if (lane == 0) {
        if (my_max > 0) atomicMax(&st->max_color, my_max);
        if (my_s > 0) atomicAdd(&st->s_next, my_s);
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
    DevBuf deg, wl, state, problem, trace, stage_rp, stage_ci, stage_col, flag;
    HostBuf h_problem, h_state, h_misc;
    int wl_cap = 0;        // vertices per worklist array
    int trace_cap = 0;
    // graph (valid for the launch geometry below)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int g_grid = 0, g_block = 0, g_hub = 0;
    size_t g_smem_assign = 0, g_smem_detect = 0, g_smem_init = 0;

    void destroy_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        g_grid = 0;
    }
    void release() {
        destroy_graph();
        for (DevBuf* b : {&deg, &wl, &state, &problem, &trace, &stage_rp, &stage_ci, &stage_col, &flag})
            b->release();
        for (HostBuf* b : {&h_problem, &h_state, &h_misc}) b->release();
        wl_cap = 0;
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
    size_t smem_init, smem_assign, smem_detect;
};

static pgc_status geometry(const Context& cx, const Opts& o, Geometry* g) {
    const int block = o.block;
    const int wpb = block / 32;
    const int mid_words = (o.hub_degree + 1 + 31) / 32;
    g->block = block;
    g->smem_init = (size_t)wpb * NTIER * 64 * sizeof(int);
    g->smem_assign = (size_t)(kHubWords + wpb * mid_words) * sizeof(int);
    g->smem_detect = (size_t)wpb * 64 * sizeof(int);
    int per_sm = o.grid_per_sm;
    if (per_sm == 0) {
        int a = 0, b = 0;
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, d1_assign, block, g->smem_assign));
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, d1_detect, block, g->smem_detect));
        per_sm = std::max(1, std::min(a, b));
    }
    g->grid = cx.dev.num_sms * per_sm;
    return PGC_OK;
}

static pgc_status build_graph(Context& cx, const Geometry& g) {
    cx.destroy_graph();
    Problem* dP = cx.problem.as<Problem>();
    PGC_CUDA(cudaGraphCreate(&cx.graph, 0));
    PGC_CUDA(cudaGraphConditionalHandleCreate(&cx.handle, cx.graph, 0u, cudaGraphCondAssignDefault));

    cudaGraphNode_t n_memset, n_init, n_first, n_loop;
    cudaMemsetParams ms = {};
    ms.dst = cx.state.ptr;
    ms.value = 0;
    ms.elementSize = 4;
    ms.width = sizeof(State) / 4;
    ms.height = 1;
    ms.pitch = 0;
    PGC_CUDA(cudaGraphAddMemsetNode(&n_memset, cx.graph, nullptr, 0, &ms));

    void* init_args[] = {&dP};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)d1_init;
    kp.gridDim = dim3(g.grid);
    kp.blockDim = dim3(g.block);
    kp.sharedMemBytes = (unsigned)g.smem_init;
    kp.kernelParams = init_args;
    PGC_CUDA(cudaGraphAddKernelNode(&n_init, cx.graph, &n_memset, 1, &kp));

    int use_cond = 1;
    cudaGraphConditionalHandle hnd = cx.handle;
    void* det_args[] = {&dP, &hnd, &use_cond};
    cudaKernelNodeParams kd = {};
    kd.func = (void*)d1_detect;
    kd.gridDim = dim3(g.grid);
    kd.blockDim = dim3(g.block);
    kd.sharedMemBytes = (unsigned)g.smem_detect;
    kd.kernelParams = det_args;
    PGC_CUDA(cudaGraphAddKernelNode(&n_first, cx.graph, &n_init, 1, &kd));

    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cx.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    PGC_CUDA(cudaGraphAddNode(&n_loop, cx.graph, &n_first, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    cudaGraphNode_t b_assign, b_detect;
    void* asg_args[] = {&dP};
    cudaKernelNodeParams ka = {};
    ka.func = (void*)d1_assign;
    ka.gridDim = dim3(g.grid);
    ka.blockDim = dim3(g.block);
    ka.sharedMemBytes = (unsigned)g.smem_assign;
    ka.kernelParams = asg_args;
    PGC_CUDA(cudaGraphAddKernelNode(&b_assign, body, nullptr, 0, &ka));
    PGC_CUDA(cudaGraphAddKernelNode(&b_detect, body, &b_assign, 1, &kd));

    PGC_CUDA(cudaGraphInstantiate(&cx.exec, cx.graph, 0));
    cx.g_grid = g.grid;
    cx.g_block = g.block;
    cx.g_smem_assign = g.smem_assign;
    cx.g_smem_detect = g.smem_detect;
    cx.g_smem_init = g.smem_init;
    return PGC_OK;
}

static pgc_status run(Context& cx, int n, const int* d_rp, const int* d_ci, int* d_col,
                      uint64_t seed, const Opts& o, cudaStream_t stream, int* rounds,
                      int* num_colors) {
    // --- scratch ---
    if (cx.wl_cap < n) {
        cx.destroy_graph();
        if (pgc_status s = cx.deg.ensure((size_t)n * 4)) return s;
        if (pgc_status s = cx.wl.ensure((size_t)n * 4 * 2 * NTIER)) return s;
        cx.wl_cap = n;
    }
    if (pgc_status s = cx.state.ensure(sizeof(State))) return s;
    if (pgc_status s = cx.problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_state.ensure(sizeof(State))) return s;
    const int want_trace = o.profile && o.profile->trace_cap > 0 ? o.profile->trace_cap : 0;
    const int tcap = std::max(want_trace, 1);
    if (cx.trace_cap < tcap) {
        if (pgc_status s = cx.trace.ensure((size_t)tcap * 2 * sizeof(long long))) return s;
        if (pgc_status s = cx.h_misc.ensure((size_t)tcap * 2 * sizeof(long long))) return s;
        cx.trace_cap = tcap;
    }

    Geometry g;
    if (pgc_status s = geometry(cx, o, &g)) return s;
    if (g.smem_assign > 48 * 1024) {
        PGC_CUDA(cudaFuncSetAttribute(d1_assign, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)g.smem_assign));
    }

    // --- problem description (read by every kernel through one pointer) ---
    Problem* hp = cx.h_problem.as<Problem>();
    std::memset(hp, 0, sizeof(Problem));
    hp->row_ptr = d_rp;
    hp->col_idx = d_ci;
    hp->col = d_col;
    hp->deg = cx.deg.as<int>();
    int* wl = cx.wl.as<int>();
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < NTIER; ++k) hp->wl[p][k] = wl + (size_t)(p * NTIER + k) * n;
    hp->trace_w = cx.trace.as<long long>();
    hp->trace_s = cx.trace.as<long long>() + tcap;
    hp->trace_cap = want_trace;
    hp->st = cx.state.as<State>();
    hp->seed = seed;
    hp->timeout_ns = (unsigned long long)o.timeout_ms * 1000000ull;
    hp->n = n;
    hp->use_deg = (o.flags & PGC_NO_DEGREE_RULE) ? 0 : 1;
    hp->mid_deg = o.mid_degree;
    hp->hub_deg = o.hub_degree;
    hp->max_rounds = o.max_rounds > 0 ? o.max_rounds : (n < INT32_MAX ? n + 1 : n);
    PGC_CUDA(cudaMemcpyAsync(cx.problem.ptr, hp, sizeof(Problem), cudaMemcpyHostToDevice, stream));
    Problem* dP = cx.problem.as<Problem>();

    if (!(o.flags & PGC_HOST_LOOP)) {
        if (!cx.exec || cx.g_grid != g.grid || cx.g_block != g.block ||
            cx.g_smem_assign != g.smem_assign) {
            if (pgc_status s = build_graph(cx, g)) return s;
        }
        PGC_CUDA(cudaGraphLaunch(cx.exec, stream));
    } else {
        KernelTimer kt;
        kt.prof = o.profile;
        kt.stream = stream;
        PGC_CUDA(cudaMemsetAsync(cx.state.ptr, 0, sizeof(State), stream));
        d1_init<<<g.grid, g.block, g.smem_init, stream>>>(dP);
        PGC_CUDA(cudaGetLastError());
        State* hs = cx.h_state.as<State>();
        for (int round = 1;; ++round) {
            if (round > 1) {
                if (pgc_status s = kt.begin(0, "d1_assign")) return s;
                d1_assign<<<g.grid, g.block, g.smem_assign, stream>>>(dP);
                PGC_CUDA(cudaGetLastError());
                if (pgc_status s = kt.end()) return s;
            }
            if (pgc_status s = kt.begin(1, "d1_detect")) return s;
            d1_detect<<<g.grid, g.block, g.smem_detect, stream>>>(dP, 0, 0);
            PGC_CUDA(cudaGetLastError());
            if (pgc_status s = kt.end()) return s;
            PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
            PGC_CUDA(cudaStreamSynchronize(stream));
            if (hs->done) break;
        }
        kt.destroy();
    }
    State* hs = cx.h_state.as<State>();
    PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
    if (want_trace) {
        PGC_CUDA(cudaMemcpyAsync(cx.h_misc.ptr, cx.trace.ptr, (size_t)tcap * 2 * sizeof(long long),
                                 cudaMemcpyDeviceToHost, stream));
    }
    PGC_CUDA(cudaStreamSynchronize(stream));
    if (want_trace) {
        const long long* tw = cx.h_misc.as<long long>();
        const long long* ts = tw + tcap;
        const int nr = std::min(hs->round, want_trace);
        for (int i = 0; i < want_trace; ++i) {
            if (o.profile->trace_w) o.profile->trace_w[i] = i < nr ? tw[i] : 0;
            if (o.profile->trace_s) o.profile->trace_s[i] = i < nr ? ts[i] : 0;
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
    if (host_rp || host_ci) {
        int nnz = 0;
        if (host_rp) nnz = row_ptr[n];
        else {
            PGC_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, 4, cudaMemcpyDeviceToHost, stream));
            PGC_CUDA(cudaStreamSynchronize(stream));
        }
        if (nnz < 0) return fail(PGC_ERR_INVALID_ARG, "row_ptr[n] < 0");
        if (nnz > 0 && !col_idx) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx");
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
    pgc_status s = run(*cx, n, d_rp, d_ci, d_col, seed, o, stream, rounds, num_colors);
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
