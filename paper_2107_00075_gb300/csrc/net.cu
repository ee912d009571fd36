// net.cu -- distance-2 (D2) and partial distance-2 (PD2) coloring.
//
// Method (Bogle et al., Sec. 3.5-3.6, Alg. 5; first fit of Alg. 1, loser
// order of Alg. 4), round-synchronous form as for D1.  Both problems are
// written over "nets" (the net-based view of NB_BIT, Sec. 3.5): two vertices
// must differ iff they are members of a common net.
//   D2 : one net per vertex u, members N[u] = {u} + N(u); the nets of v are
//        N[v]'s indices {v} + N(v).  Two vertices share a net iff they are
//        within two hops (Sec. 2.1).
//   PD2: the nets are the rows of the pattern, members are the row's
//        columns (CSR); the nets of column v are its rows (CSC) (Sec. 3.6).
// Only the vertices (D2) or columns (PD2) are colored.
//
// Per round:
//   assign  v in W: forbidden(v) = OR of the color masks of v's nets;
//           t = first free color (Alg. 1); col[v] = -t.  Marks v's nets
//           active for this round (skipped while W's nets cover them all).
//   detect  per active net: each uncolored member v whose color is also
//           held by a member with priority loses (Alg. 5 + Alg. 4); small
//           nets are packed into 32-lane rows and each (net, color) group
//           keeps only its highest-priority member (warp reductions).  A
//           loser is marked by bit 0 of its packed word, written only if the
//           word the lane loaded does not show it yet.
//   commit  v in W: losers form W_{r+1}; a winner commits and sets bit t in
//           the masks of its nets (so a mask is always the OR of its
//           committed members' colors, kept incrementally: each vertex
//           updates its nets once).
// The loop runs on the device (CUDA graph, conditional WHILE node).
#include "runtime.h"
#include "device_common.cuh"

#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>
#include <unordered_map>

namespace pgc {
std::vector<std::function<void()>>& release_hooks();

namespace net {

constexpr int kThreadNets = 64;   // vertices with up to this many nets: one thread
constexpr int kMaxWindows = 64;   // masks hold colors 1..64*windows (<= 4096)

enum : int { ST_OK = 0, ST_NO_PROGRESS = 1, ST_MAX_ROUNDS = 2, ST_TIMEOUT = 3, ST_OVERFLOW = 4 };

struct State {
    int round;
    int done;
    int status;
    int max_color;
    int nt[2];        // thread-tier worklist sizes per parity
    int nw[2];        // warp-tier worklist sizes
    int all_active;   // this round every net is treated as active (no marking)
    unsigned blocks_done;
    int bound;        // max over v of sum over its nets of (|net| - 1)
    int pad;
    unsigned long long s_next;
    unsigned long long h_next;
    unsigned long long h_first;
    unsigned long long t0;
    unsigned long long nets_seen;      // traced: nets detection visited this round
    unsigned long long members_seen;   // traced: their members
    int max_deg;      // largest degree term of a key (sizes the 32-bit key of ck)
    int pad2;
};

struct Problem {
    const int* m_ptr;     // net -> members
    const int* m_idx;
    const int* r_ptr;     // vertex -> nets
    const int* r_idx;
    int* col;                   // output colors (written at commit)
    int2* ck;                   // per vertex {color: 0 / -tentative / committed, 32-bit key
                                // whose bit 0 marks a vertex that lost in some net this round}
    unsigned long long* key;    // priority key (see net_init)
    int* net_flag;              // = round number while the net is active
    unsigned long long* mask;   // [window][net]
    int* wt[2];
    int* ww[2];
    long long* trace_w;
    long long* trace_s;
    long long* trace_h;
    long long* trace_nets;
    long long* trace_members;
    State* st;
    unsigned long long seed;
    unsigned long long timeout_ns;
    int trace_cap;
    int n;            // colored vertices
    int n_nets;
    int self;         // 1: D2 (net u contains u; v's nets include v's own)
    int windows;
    int use_deg;
    int max_rounds;
};

// member j of net q (j < net_size)
__device__ __forceinline__ int net_member(const Problem& P, int q, int j) {
    if (P.self) return j == 0 ? q : __ldg(P.m_idx + __ldg(P.m_ptr + q) + j - 1);
    return __ldg(P.m_idx + __ldg(P.m_ptr + q) + j);
}
__device__ __forceinline__ int net_size(const Problem& P, int q) {
    return __ldg(P.m_ptr + q + 1) - __ldg(P.m_ptr + q) + P.self;
}
// k-th net of vertex v (k < nets_of_size)
__device__ __forceinline__ int vertex_net(const Problem& P, int v, int beg, int k) {
    if (P.self) return k == 0 ? v : __ldg(P.r_idx + beg + k - 1);
    return __ldg(P.r_idx + beg + k);
}

// ---------------------------------------------------------------------------
// init: priority keys, empty colors, worklists by number of nets, the bound
//
// key(v) = deg(v) << 32 | ~(h(v) >> 32) (deg term 0 without the degree
// rule): a larger key is a higher priority (Alg. 4: larger degree first,
// then the smaller hash), except between two keys that are equal -- same
// degree and same top 32 hash bits -- which the low hash bits and then the
// id decide.
// ---------------------------------------------------------------------------
__global__ void net_init(const Problem* __restrict__ Pp) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int warp = threadIdx.x >> 5;
    WarpAppend at = {smem + warp * 2 * kAppendSlots, 0},
               aw = {smem + warp * 2 * kAppendSlots + kAppendSlots, 0};
    int my_bound = 0, my_deg = 0;
    unsigned long long my_h = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         wbase < P.n; wbase += stride) {
        const long long i = wbase + lane_id();
        const bool valid = i < P.n;
        int k = 0;
        if (valid) {
            const int v = (int)i;
            const int beg = __ldg(P.r_ptr + v);
            const int d = __ldg(P.r_ptr + v + 1) - beg;
            const unsigned hi = (unsigned)(prio_hash(P.seed, (uint32_t)v) >> 32);
            P.key[v] = (P.use_deg ? (unsigned long long)d << 32 : 0ull) | (unsigned long long)~hi;
            P.col[v] = 0;
            my_deg = max(my_deg, d);
            k = d + P.self;
            long long b = 0;
            for (int j = 0; j < k; ++j) b += net_size(P, vertex_net(P, v, beg, j)) - 1;
            my_bound = max(my_bound, (int)min(b, (long long)INT32_MAX - 1));
            my_h += (unsigned long long)k;
        }
        wa_push(at, valid && k <= kThreadNets, (int)i, P.wt[1], &st->nt[1]);
        wa_push(aw, valid && k > kThreadNets, (int)i, P.ww[1], &st->nw[1]);
    }
    wa_flush(at, P.wt[1], &st->nt[1]);
    wa_flush(aw, P.ww[1], &st->nw[1]);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < P.n_nets; q += stride)
        P.net_flag[q] = 0;
    my_bound = warp_max(my_bound);
    my_deg = warp_max(my_deg);
    my_h = warp_sum(my_h);
    if (lane_id() == 0) {
        atomicMax(&st->bound, my_bound);
        if (P.use_deg) atomicMax(&st->max_deg, my_deg);
        if (my_h) atomicAdd(&st->h_first, my_h);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->round = 1;
        st->all_active = 1;
        st->t0 = global_ns();
        if (P.trace_cap > 0) {
            P.trace_w[0] = P.n;
            P.trace_s[0] = __ldg(P.r_ptr + P.n);
        }
    }
}

// ---------------------------------------------------------------------------
// assign: OR the nets' masks window by window, take the first free color
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mark_net(const Problem& P, int q, int r) {
    if (P.net_flag[q] != r) P.net_flag[q] = r;
}

// The 32-bit key stored beside the color: key >> b, where b is the bit
// width of the largest degree term, so the degree still dominates and the
// top 32 - b hash bits follow, with bit 0 cleared: detection sets it on a
// vertex that loses in some net, and compares keys without it.  It orders
// like the full key except that two different keys may share it; detection
// resolves such ties from the full key.
__device__ __forceinline__ unsigned key32(const Problem& P, int v, int b) {
    return (unsigned)(__ldg(P.key + v) >> b) & ~1u;
}

// OR of a 64-bit word over the warp
__device__ __forceinline__ unsigned long long warp_or64(unsigned long long f) {
    const unsigned lo = __reduce_or_sync(kFullMask, (unsigned)f);
    const unsigned hi = __reduce_or_sync(kFullMask, (unsigned)(f >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ int key_shift(const State* st) {
    const int d = *(volatile const int*)&st->max_deg;
    return d > 0 ? 32 - __clz(d) : 0;
}

__global__ void net_assign(const Problem* __restrict__ Pp, cudaGraphConditionalHandle h,
                           int use_cond) {
    const Problem& P = *Pp;
    State* st = P.st;
    // The loop continues only if this round's commit says so.
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    const int r = *(volatile int*)&st->round;
    const int cp = r & 1;
    const int nT = st->nt[cp], nW = st->nw[cp];
    const bool mark = *(volatile int*)&st->all_active == 0;
    const unsigned long long* mk = P.mask;
    const long long nn = P.n_nets;
    const int kb = key_shift(st);
    // thread tier (at most 64 nets per vertex), a warp's 32 worklist vertices
    // at a time.  While none has more than 32 nets, each lane walks its own
    // vertex's nets, eight at a time.  Otherwise (the lanes would idle while
    // the longest walk finishes) the warp takes the vertices as rows: lane j
    // reads nets j and j + 32 of the row's vertex (coalesced ids) and an OR
    // over the lanes gives the forbidden set, four vertices at a time.
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = lane_id();
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < nT;
         wbase += stride) {
        const long long i = wbase + lane;
        int v = -1, beg = 0, k = 0;
        if (i < nT) {
            v = P.wt[cp][i];
            beg = __ldg(P.r_ptr + v);
            k = __ldg(P.r_ptr + v + 1) - beg + P.self;
        }
        int t = 0;
        if (__reduce_max_sync(kFullMask, (unsigned)k) <= 32u) {
            if (i < nT) {
                for (int w = 0; w < P.windows && t == 0; ++w) {
                    // eight nets at a time: their ids, then their mask words
                    const unsigned long long* mw = mk + w * nn;
                    unsigned long long f = 0ull;
                    for (int j = 0; j < k; j += 8) {
                        int q[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            q[u] = j + u < k ? vertex_net(P, v, beg, j + u) : -1;
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (q[u] >= 0) f |= mw[q[u]];
                    }
                    if (f != ~0ull) t = 64 * w + __ffsll((long long)~f);
                }
                if (t == 0) {
                    atomicExch(&st->status, ST_OVERFLOW);
                    t = 64 * P.windows;
                }
                if (mark)
                    for (int j = 0; j < k; ++j) mark_net(P, vertex_net(P, v, beg, j), r);
            }
        } else {
            const int rows = (int)min(32LL, (long long)nT - wbase);
            for (int r0 = 0; r0 < rows; r0 += 4) {
                int q[4][2];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int vv = __shfl_sync(kFullMask, v, r0 + h);
                    const int bb = __shfl_sync(kFullMask, beg, r0 + h);
                    const int kk = __shfl_sync(kFullMask, k, r0 + h);
                    q[h][0] = lane < kk ? vertex_net(P, vv, bb, lane) : -1;
                    q[h][1] = lane + 32 < kk ? vertex_net(P, vv, bb, lane + 32) : -1;
                }
                unsigned long long f[4];
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    f[h] = (q[h][0] >= 0 ? mk[q[h][0]] : 0ull) | (q[h][1] >= 0 ? mk[q[h][1]] : 0ull);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    unsigned long long F = warp_or64(f[h]);
                    int th = F != ~0ull ? __ffsll((long long)~F) : 0;
                    for (int w = 1; w < P.windows && th == 0; ++w) {   // warp-uniform, rare
                        const unsigned long long* mw = mk + w * nn;
                        F = warp_or64((q[h][0] >= 0 ? mw[q[h][0]] : 0ull) |
                                      (q[h][1] >= 0 ? mw[q[h][1]] : 0ull));
                        if (F != ~0ull) th = 64 * w + __ffsll((long long)~F);
                    }
                    if (th == 0) {
                        if (lane == 0 && r0 + h < rows) atomicExch(&st->status, ST_OVERFLOW);
                        th = 64 * P.windows;
                    }
                    if (lane == r0 + h) t = th;
                    if (mark) {
                        if (q[h][0] >= 0) mark_net(P, q[h][0], r);
                        if (q[h][1] >= 0) mark_net(P, q[h][1], r);
                    }
                }
            }
        }
        if (i < nT) P.ck[v] = make_int2(-t, (int)key32(P, v, kb));
    }
    // warp tier
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nW; i += gridDim.x * wpb) {
        const int v = P.ww[cp][i];
        const int beg = __ldg(P.r_ptr + v);
        const int k = __ldg(P.r_ptr + v + 1) - beg + P.self;
        int t = 0;
        for (int w = 0; w < P.windows && t == 0; ++w) {
            unsigned long long f = 0ull;
            for (int j = lane; j < k; j += 32) f |= mk[w * nn + vertex_net(P, v, beg, j)];
            const unsigned lo = __reduce_or_sync(kFullMask, (unsigned)f);
            const unsigned hi = __reduce_or_sync(kFullMask, (unsigned)(f >> 32));
            f = ((unsigned long long)hi << 32) | lo;
            if (f != ~0ull) t = 64 * w + __ffsll((long long)~f);
        }
        if (t == 0) {
            if (lane == 0) atomicExch(&st->status, ST_OVERFLOW);
            t = 64 * P.windows;
        }
        if (lane == 0) P.ck[v] = make_int2(-t, (int)key32(P, v, kb));
        if (mark)
            for (int j = lane; j < k; j += 32) mark_net(P, vertex_net(P, v, beg, j), r);
    }
}

// ---------------------------------------------------------------------------
// detect: per active net, flag members that share a color with a member of
// higher priority.  Members holding a committed (positive) color never
// match: first fit excluded every committed color of v's nets.
//
// Within one net, the members holding tentative color c form a group; every
// member of the group except its highest-priority one is recolored (Alg. 4
// applied to each pair of the group).  So a group needs no pairwise loop: its
// winner is the member with the largest key.  Nets of 17..32 members take one
// 32-lane row each; smaller ones are packed whole into rows, several nets per
// row.  A warp loads four one-net rows or two packed rows at once, so it keeps
// many independent gathers in flight.  Within a row, match.any finds each
// lane's group.  In one-net rows, two warp-wide max reductions per contested
// group find its winner; in packed rows, which hold many groups, the group's
// lowest lane names a shared-memory slot that every member raises to its
// 32-bit key with one atomic max.  Larger nets compare every member against
// every other member, 32 x 32 at a time.
// ---------------------------------------------------------------------------
constexpr int kDenseRows = 4;      // rows loaded together: one net per row
constexpr int kPackedRows = 2;     // rows loaded together: packed small nets
constexpr int kDetSmemInts = 97;   // per warp: 32 net ids, 32 m_ptr, 33 packed starts
constexpr int kDetSlots = kPackedRows * 32;   // per warp: one max slot per lane of each packed row
constexpr size_t kDetWarpBytes = kDetSlots * sizeof(unsigned) + kDetSmemInts * sizeof(int);

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned lanemask_le() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

// g: the lanes (this one included) holding this lane's tentative color in
// the same net.  True if one of them has priority over this lane's x.
__device__ __forceinline__ bool group_loses(unsigned g, int x, unsigned long long k,
                                            unsigned long long seed) {
    const unsigned khi = (unsigned)(k >> 32), klo = (unsigned)k;
    const unsigned m1 = __reduce_max_sync(g, khi);
    const unsigned g1 = __ballot_sync(g, khi == m1) & g;
    if (khi != m1) return true;
    if (__popc(g1) == 1) return false;
    const unsigned m2 = __reduce_max_sync(g1, klo);
    const unsigned g2 = __ballot_sync(g1, klo == m2) & g1;
    if (klo != m2) return true;
    if (__popc(g2) == 1) return false;
    // equal keys: the low hash bits, then the id (equal ids: the same
    // vertex listed twice)
    const unsigned lo = (unsigned)prio_hash(seed, (uint32_t)x);
    const unsigned m3 = __reduce_min_sync(g2, lo);
    const unsigned g3 = __ballot_sync(g2, lo == m3) & g2;
    if (lo != m3) return true;
    if (__popc(g3) == 1) return false;
    return (unsigned)x != __reduce_min_sync(g3, (unsigned)x);
}

// True if u has priority over v, from their keys (ties: full hash, then id).
__device__ __forceinline__ bool key_priority(unsigned long long ku, int u, unsigned long long kv,
                                             int v, unsigned long long seed) {
    if (ku != kv) return ku > kv;
    const uint64_t hu = prio_hash(seed, (uint32_t)u), hv = prio_hash(seed, (uint32_t)v);
    if (hu != hv) return hu < hv;
    return u < v;
}

__device__ void big_net_detect(const Problem& P, int q, int m, int lane, int r) {
    const unsigned long long seed = P.seed;
    for (int i0 = 0; i0 < m; i0 += 32) {
        int x = -1, c = 0;
        unsigned kf = 0u;
        unsigned long long kx = 0ull;
        if (i0 + lane < m) {
            x = net_member(P, q, i0 + lane);
            const int2 px = P.ck[x];
            const int cx = px.x;
            c = cx < 0 ? -cx : 0;
            kf = (unsigned)px.y;
            if (c) kx = __ldg(P.key + x);
        }
        bool lose = false;
        for (int j0 = 0; j0 < m; j0 += 32) {
            // members of chunk j0 broadcast (id, color, key)
            int y = -1, cy = 0;
            unsigned long long ky = 0ull;
            if (j0 + lane < m) {
                y = net_member(P, q, j0 + lane);
                const int c2 = P.ck[y].x;
                cy = c2 < 0 ? -c2 : 0;
                if (cy) ky = __ldg(P.key + y);
            }
            unsigned cand = __ballot_sync(kFullMask, cy != 0);
            while (cand) {
                const int src = __ffs(cand) - 1;
                cand &= cand - 1;
                const int ys = __shfl_sync(kFullMask, y, src);
                const int cs = __shfl_sync(kFullMask, cy, src);
                const unsigned long long ks = __shfl_sync(kFullMask, ky, src);
                if (c && cs == c && ys != x && key_priority(ks, ys, kx, x, seed)) lose = true;
            }
        }
        if (lose && !(kf & 1u)) reinterpret_cast<int*>(P.ck + x)[1] = (int)(kf | 1u);
    }
}

// The exact decision for one lane of a group g (two or more lanes): the
// largest 32-bit key wins; members sharing it are decided by the full key,
// then the hash and the id.
__device__ __noinline__ bool group_exact(unsigned g, unsigned k32, int x,
                                         const unsigned long long* key, unsigned long long seed) {
    const unsigned m1 = __reduce_max_sync(g, k32);
    const unsigned ties = __ballot_sync(g, k32 == m1) & g;
    if (k32 != m1) return true;
    if (__popc(ties) == 1) return false;
    return group_loses(ties, x, __ldg(key + x), seed);
}

// What detection reads: the problem (in global memory, read through the
// read-only path; the compiler keeps in registers what fits).
using DetView = Problem;

// The rows' tentative colors and keys.  t: the group tag (color, net in the
// row), 0 for a lane that holds no tentative member; g: the lanes sharing it.
template <int R>
struct RowState {
    unsigned t[R], g[R], k32[R];
};

template <int R>
__device__ __forceinline__ void load_rows(const DetView& D, const int (&x)[R],
                                          const int (&id)[R], RowState<R>& S) {
    int2 p[R];
#pragma unroll
    for (int k = 0; k < R; ++k) p[k] = x[k] >= 0 ? D.ck[x[k]] : make_int2(0, 0);
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int c = p[k].x < 0 ? -p[k].x : 0;
        S.t[k] = c ? ((unsigned)c << 5) | (unsigned)(id[k] - 1) : 0u;
        S.g[k] = __match_any_sync(kFullMask, S.t[k]);
        S.k32[k] = (unsigned)p[k].y;   // bit 0: lost in some net this round
    }
}

// Rows where two members of one group both hold the group's largest 32-bit
// key (each row's winners outnumber its contested groups): those groups are
// decided again from the full keys.  Rare: the 32-bit key holds the degree
// and the top hash bits.
template <int R>
__device__ __forceinline__ void settle_ties(const DetView& D, const int (&x)[R],
                                            const RowState<R>& S, unsigned need,
                                            bool (&lose)[R]) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
        if (!(need >> k & 1u)) continue;   // warp-uniform
        const bool contested = S.t[k] != 0u && (S.g[k] & (S.g[k] - 1u)) != 0u;
        if (contested) lose[k] = group_exact(S.g[k], (S.k32[k] & ~1u), x[k], D.key, D.seed);
    }
}

// Group winners, one warp-wide max per contested group: the largest
// remaining tag names the next group, a max over its members' keys its
// winner.  A row with one contested group (every round-1 net) costs two
// reductions.
template <int R>
__device__ __forceinline__ void resolve_rows_iter(const DetView& D, const int (&x)[R],
                                                  const int (&id)[R], int r) {
    RowState<R> S;
    load_rows(D, x, id, S);
    bool lose[R];
    unsigned need = 0u;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const bool contested = S.t[k] != 0u && (S.g[k] & (S.g[k] - 1u)) != 0u;
        unsigned rem = contested ? S.t[k] : 0u, mx = 0u;
        int groups = 0;
        while (__any_sync(kFullMask, rem != 0u)) {   // warp-uniform
            const unsigned tc = __reduce_max_sync(kFullMask, rem);
            const bool in = rem == tc;
            const unsigned m = __reduce_max_sync(kFullMask, in ? (S.k32[k] & ~1u) : 0u);
            if (in) {
                mx = m;
                rem = 0u;
            }
            ++groups;
        }
        lose[k] = contested && (S.k32[k] & ~1u) < mx;
        const int winners = __popc(__ballot_sync(kFullMask, contested && (S.k32[k] & ~1u) == mx));
        if (winners > groups) need |= 1u << k;
    }
    if (need) settle_ties(D, x, S, need, lose);
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (lose[k] && !(S.k32[k] & 1u)) reinterpret_cast<int*>(D.ck + x[k])[1] = (int)(S.k32[k] | 1u);
}

// Group winners through shared memory: the group's lowest lane names a slot
// that every member raises to its key with one atomic max.  The cost does
// not grow with the number of groups in the row.  slot: this warp's
// kDetSlots words.
template <int R>
__device__ __forceinline__ void resolve_rows_slots(const DetView& D, const int (&x)[R],
                                                   const int (&id)[R], int r,
                                                   unsigned* slot) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 0; k < R; ++k) slot[k * 32 + lane] = 0u;
    RowState<R> S;
    load_rows(D, x, id, S);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (S.t[k] && (S.g[k] & (S.g[k] - 1u)))
            atomicMax(slot + k * 32 + (__ffs(S.g[k]) - 1), (S.k32[k] & ~1u));
    __syncwarp();
    bool lose[R];
    unsigned need = 0u;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const bool contested = S.t[k] != 0u && (S.g[k] & (S.g[k] - 1u)) != 0u;
        const int leader = __ffs(S.g[k]) - 1;
        const unsigned mx = contested ? slot[k * 32 + leader] : 0u;
        lose[k] = contested && (S.k32[k] & ~1u) < mx;
        const int winners = __popc(__ballot_sync(kFullMask, contested && (S.k32[k] & ~1u) == mx));
        const int groups = __popc(__ballot_sync(kFullMask, contested && leader == lane));
        if (winners > groups) need |= 1u << k;
    }
    __syncwarp();
    if (need) settle_ties(D, x, S, need, lose);
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (lose[k] && !(S.k32[k] & 1u)) reinterpret_cast<int*>(D.ck + x[k])[1] = (int)(S.k32[k] | 1u);
}

#ifndef PGC_PACKED_SLOTS
#define PGC_PACKED_SLOTS 1
#endif

__global__ void __maxnreg__(48) net_detect(const Problem* __restrict__ Pp) {
    // per warp: the tile's small active nets, compacted (net id, m_ptr,
    // start of the net in the packed tile)
    extern __shared__ unsigned det_smem[];
    const Problem& P = *Pp;
    const int r = *(volatile int*)&P.st->round;
    const bool all = *(volatile int*)&P.st->all_active != 0;
    const int lane = lane_id(), wpb = blockDim.x >> 5, w = threadIdx.x >> 5;
    const int self = P.self;
    const int nn = P.n_nets;
    unsigned* slot = det_smem + w * kDetSlots;
    int* sq = reinterpret_cast<int*>(det_smem + wpb * kDetSlots) + w * kDetSmemInts;
    int* sb = sq + 32;
    int* sp = sb + 32;
    const bool traced = P.trace_cap > 0;
    // per lane: nets visited and their members (fewer than 2^31 members in all)
    unsigned seen = 0u, seen_m = 0u;
    const DetView& D = P;
    // Tiles of 32 nets; each warp takes a contiguous run of tiles, so while
    // it works on one tile the next tile's member ids (which follow this
    // tile's in m_idx) can be prefetched into L2.
    const unsigned tiles = ((unsigned)nn + 31u) >> 5;
    const unsigned nwarps = gridDim.x * wpb;
    const unsigned per = (tiles + nwarps - 1u) / nwarps;
    const unsigned t0 = (blockIdx.x * wpb + w) * per;
    const unsigned t1 = min(tiles, t0 + per);
    const int m_end = __ldg(P.m_ptr + nn);
    for (unsigned t = t0; t < t1; ++t) {
        const unsigned b0 = t << 5;
        const int q = (int)b0 + lane;
        int beg = 0, m = 0;
        if (q < nn && (all || P.net_flag[q] == r)) {
            beg = __ldg(P.m_ptr + q);
            m = __ldg(P.m_ptr + q + 1) - beg + self;
        }
        if (all && t + 1u < t1) {
            // the next tile's ids: as many 128-byte lines as this tile spans
            const int e0 = __ldg(P.m_ptr + b0);
            const int e1 = __ldg(P.m_ptr + b0 + 32u);   // b0 + 32 < nn: a next tile exists
            const int at = e1 + lane * 32;
            if (lane * 32 < e1 - e0 && at < m_end) prefetch_l2(P.m_idx + at);
            if (lane == 0 && b0 + 64u < (unsigned)nn) prefetch_l2(P.m_ptr + b0 + 64u);
        }
        if (traced && q < nn && (all || P.net_flag[q] == r)) {   // profiling only
            seen += 1u;
            seen_m += (unsigned)m;
        }
        const bool small = m >= 2 && m <= 32;
        const unsigned sm = __ballot_sync(kFullMask, small);
        const unsigned big = __ballot_sync(kFullMask, m > 32);
        const int min_small = __reduce_min_sync(kFullMask, small ? m : 64);
        if (sm == kFullMask && min_small > 16) {
            // every net of the tile active with 17..32 members: net i is row
            // i, and its start and size come from lane i
#pragma unroll 1
            for (int i0 = 0; i0 < 32; i0 += kDenseRows) {
                int x[kDenseRows], id[kDenseRows];
#pragma unroll
                for (int k = 0; k < kDenseRows; ++k) {
                    const int bg = __shfl_sync(kFullMask, beg, i0 + k);
                    const int mm = __shfl_sync(kFullMask, m, i0 + k);
                    id[k] = 1;
                    x[k] = lane >= mm ? -1
                           : lane < self ? (int)b0 + i0 + k
                                         : __ldg(D.m_idx + bg + lane - self);
                }
                resolve_rows_iter(D, x, id, r);
            }
        } else if (sm && min_small > 16) {
            // every row holds exactly one net
            unsigned rest = sm;
            while (rest) {
                int x[kDenseRows], id[kDenseRows];
#pragma unroll
                for (int k = 0; k < kDenseRows; ++k) {
                    x[k] = -1;
                    id[k] = 0;
                    if (!rest) continue;   // warp-uniform
                    const int src = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const int qq = __shfl_sync(kFullMask, q, src);
                    const int bg = __shfl_sync(kFullMask, beg, src);
                    const int mm = __shfl_sync(kFullMask, m, src);
                    if (lane < mm) {
                        id[k] = 1;
                        x[k] = self ? (lane == 0 ? qq : __ldg(D.m_idx + bg + lane - 1))
                                    : __ldg(D.m_idx + bg + lane);
                    }
                }
                resolve_rows_iter(D, x, id, r);
            }
        } else if (sm) {
            // exclusive scan of the small nets' sizes = their packed starts
            const int sz = small ? m : 0;
            int e = sz;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFullMask, e, o);
                if (lane >= o) e += t;
            }
            const int rank = __popc(sm & ((1u << lane) - 1u));
            const int cnt = __popc(sm);
            if (small) {
                sq[rank] = q;
                sb[rank] = beg;
                sp[rank] = e - sz;
            }
            if (lane == 31) sp[cnt] = e;
            __syncwarp();
            // compacted net `lane`: its packed start and end
            const int cS = lane < cnt ? sp[lane] : 0x7fffffff;
            const int cE = lane < cnt ? sp[lane + 1] : 0x7fffffff;
            int r0 = 0;
            while (r0 < cnt) {
                int x[kPackedRows], id[kPackedRows];
#pragma unroll
                for (int k = 0; k < kPackedRows; ++k) {
                    x[k] = -1;
                    id[k] = 0;
                    if (r0 >= cnt) continue;   // warp-uniform
                    // the row: nets r0..r1-1, all that end within 32 lanes
                    const int base = __shfl_sync(kFullMask, cS, r0);
                    const unsigned fits = __ballot_sync(kFullMask, lane >= r0 && cE <= base + 32);
                    const int r1 = 32 - __clz(fits);
                    const unsigned starts = __reduce_or_sync(
                        kFullMask, (lane >= r0 && lane < r1) ? 1u << (cS - base) : 0u);
                    const int len = __shfl_sync(kFullMask, cE, r1 - 1) - base;
                    if (lane < len) {
                        const int i = r0 + __popc(starts & lanemask_le()) - 1;
                        const int off = base + lane - sp[i];
                        const int qq = sq[i], bg = sb[i];
                        id[k] = i - r0 + 1;
                        x[k] = self ? (off == 0 ? qq : __ldg(D.m_idx + bg + off - 1))
                                    : __ldg(D.m_idx + bg + off);
                    }
                    r0 = r1;
                }
                if (PGC_PACKED_SLOTS)
                    resolve_rows_slots(D, x, id, r, slot);
                else
                    resolve_rows_iter(D, x, id, r);
            }
        }
        // nets of more than 32 members, one at a time
        unsigned bg = big;
        while (bg) {
            const int src = __ffs(bg) - 1;
            bg &= bg - 1;
            const int qb = __shfl_sync(kFullMask, q, src);
            const int mb = __shfl_sync(kFullMask, m, src);
            big_net_detect(P, qb, mb, lane, r);
        }
        __syncwarp();
    }
    if (traced) {
        const unsigned long long a = warp_sum((unsigned long long)seen);
        const unsigned long long b = warp_sum((unsigned long long)seen_m);
        if (lane_id() == 0 && a) {
            atomicAdd(&P.st->nets_seen, a);
            atomicAdd(&P.st->members_seen, b);
        }
    }
}

// ---------------------------------------------------------------------------
// commit + compact + mask update (+ round control in the last block)
// ---------------------------------------------------------------------------
__device__ void round_control(const Problem& P, cudaGraphConditionalHandle h, int use_cond) {
    State* st = P.st;
    const int r = st->round;
    const int cp = r & 1, np = cp ^ 1;
    const long long cur = (long long)st->nt[cp] + st->nw[cp];
    const long long nxt = (long long)*(volatile int*)&st->nt[np] + *(volatile int*)&st->nw[np];
    if (r < P.trace_cap) {
        P.trace_w[r] = nxt;
        P.trace_s[r] = (long long)*(volatile unsigned long long*)&st->s_next;
        P.trace_h[r] = (long long)*(volatile unsigned long long*)&st->h_next;
    }
    if (r == 1 && P.trace_cap > 0) P.trace_h[0] = (long long)st->h_first;
    if (r - 1 < P.trace_cap) {
        P.trace_nets[r - 1] = (long long)*(volatile unsigned long long*)&st->nets_seen;
        P.trace_members[r - 1] = (long long)*(volatile unsigned long long*)&st->members_seen;
    }
    st->nets_seen = 0ull;
    st->members_seen = 0ull;
    int done = 0;
    int status = *(volatile int*)&st->status;
    if (status != ST_OK) {
        done = 1;
    } else if (nxt == 0) {
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
        // when the next worklist touches about every net (its vertices' net
        // memberships, estimated from the average, reach twice the nets),
        // skip the marking
        st->all_active = (unsigned long long)nxt * st->h_first >=
                         2ull * (unsigned long long)P.n_nets * (unsigned long long)P.n;
        st->nt[cp] = st->nw[cp] = 0;
        st->round = r + 1;
        st->s_next = 0ull;
        st->h_next = 0ull;
    }
    st->status = status;
    st->done = done;
    st->blocks_done = 0u;
    __threadfence();
    if (use_cond) cudaGraphSetConditional(h, done ? 0u : 1u);
}

__global__ void net_commit(const Problem* __restrict__ Pp, cudaGraphConditionalHandle h,
                           int use_cond) {
    extern __shared__ int smem[];
    const Problem& P = *Pp;
    State* st = P.st;
    const int r = *(volatile int*)&st->round;
    const int cp = r & 1, np = cp ^ 1;
    const int nT = st->nt[cp], nW = st->nw[cp];
    const long long total = (long long)nT + nW;
    const long long nn = P.n_nets;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    WarpAppend at = {smem + warp * 2 * kAppendSlots, 0},
               aw = {smem + warp * 2 * kAppendSlots + kAppendSlots, 0};
    int my_max = 0;
    unsigned long long my_s = 0ull, my_h = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wbase = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wbase < total;
         wbase += stride) {
        const long long i = wbase + lane;
        bool lost = false, thread_tier = false, won = false;
        int v = -1, beg = 0, k = 0, t = 0;
        if (i < total) {
            thread_tier = i < nT;
            v = thread_tier ? P.wt[cp][i] : P.ww[cp][i - nT];
            if (P.ck[v].y & 1) {   // lost this round: only the trace needs its degree
                lost = true;
                if (P.trace_cap > 0) {
                    const int d = __ldg(P.r_ptr + v + 1) - __ldg(P.r_ptr + v);
                    my_s += (unsigned long long)d;
                    my_h += (unsigned long long)(d + P.self);
                }
            } else {
                won = true;
                beg = __ldg(P.r_ptr + v);
                k = __ldg(P.r_ptr + v + 1) - beg + P.self;
                t = -P.ck[v].x;
                P.col[v] = t;
                reinterpret_cast<int*>(P.ck + v)[0] = t;
                my_max = max(my_max, t);
            }
        }
        // each winner sets bit t in the masks of its nets, the warp's lanes
        // taking its nets together (one winner at a time)
        unsigned wins = __ballot_sync(kFullMask, won);
        while (wins) {
            const int src = __ffs(wins) - 1;
            wins &= wins - 1;
            const int wv = __shfl_sync(kFullMask, v, src);
            const int wb = __shfl_sync(kFullMask, beg, src);
            const int wk = __shfl_sync(kFullMask, k, src);
            const int wt = __shfl_sync(kFullMask, t, src);
            unsigned long long* mw = P.mask + (long long)((wt - 1) >> 6) * nn;
            const unsigned long long bit = 1ull << ((wt - 1) & 63);
            for (int j = lane; j < wk; j += 32) atomicOr(mw + vertex_net(P, wv, wb, j), bit);
        }
        wa_push(at, lost && thread_tier, v, P.wt[np], &st->nt[np]);
        wa_push(aw, lost && !thread_tier, v, P.ww[np], &st->nw[np]);
    }
    wa_flush(at, P.wt[np], &st->nt[np]);
    wa_flush(aw, P.ww[np], &st->nw[np]);
    my_max = warp_max(my_max);
    my_s = warp_sum(my_s);
    my_h = warp_sum(my_h);
    if (lane == 0) {
        if (my_max > 0) atomicMax(&st->max_color, my_max);
        if (my_s > 0) atomicAdd(&st->s_next, my_s);
        if (my_h > 0) atomicAdd(&st->h_next, my_h);
    }
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        round_control(P, h, use_cond);
    }
}


// ---------------------------------------------------------------------------
// PD2 over every vertex of B (Sec. 3.6): one net problem with both sides.
// Vertices: the n_cols columns (ids 0..n_cols-1), then the rows (n_cols + i).
// Nets: the rows (net i, members = its columns), then the columns (net
// n_rows + c, members = its rows as vertices n_cols + r).  A column's nets
// are its rows, a row's nets are its columns.  Two vertices share a net iff
// they are on the same side and share a neighbor in B, so each side is
// colored exactly as partial distance-2 asks, with GIDs spanning B.
// ---------------------------------------------------------------------------
__global__ void pd2b_combine(const int* __restrict__ rp, const int* __restrict__ ci, int n_rows,
                             const int* __restrict__ cp, const int* __restrict__ ri, int n_cols,
                             int* __restrict__ mp, int* __restrict__ mi, int* __restrict__ vp,
                             int* __restrict__ vi) {
    const long long nnz = rp[n_rows];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // offsets: nets (rows, then columns) and vertices (columns, then rows)
    for (long long q = t0; q <= (long long)n_rows + n_cols; q += stride) {
        mp[q] = q <= n_rows ? rp[q] : (int)(nnz + cp[q - n_rows]);
        vp[q] = q <= n_cols ? cp[q] : (int)(nnz + rp[q - n_cols]);
    }
    // members and nets, 2 nnz entries each
    for (long long e = t0; e < 2 * nnz; e += stride) {
        if (e < nnz) {
            mi[e] = ci[e];
            vi[e] = ri[e];
        } else {
            mi[e] = n_cols + ri[e - nnz];
            vi[e] = n_rows + ci[e - nnz];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Context {
    std::mutex mu;
    DeviceInfo dev;
    DevBuf key, ck, flag, mask, wt, ww, state, problem, trace, stage[4], stage_col, both[4];
    HostBuf h_problem, h_state, h_misc;
    int trace_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int g_grid = 0, g_block = 0, g_det = 0;

    void destroy_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        g_grid = 0;
    }
    void release() {
        destroy_graph();
        for (DevBuf* b : {&key, &ck, &flag, &mask, &wt, &ww, &state, &problem, &trace,
                          &stage_col, &stage[0], &stage[1], &stage[2], &stage[3], &both[0],
                          &both[1], &both[2], &both[3]})
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
    int det_grid;      // detect (its own occupancy)
    size_t smem;       // init and commit
    size_t det_smem;   // detect
};

static pgc_status geometry(const Context& cx, const Opts& o, Geometry* g) {
    g->block = o.block;
    g->smem = (size_t)(o.block / 32) * 2 * kAppendSlots * sizeof(int);
    g->det_smem = (size_t)(o.block / 32) * kDetWarpBytes;
    if (g->smem > 48 * 1024) {   // 1024-thread blocks: 64 KB of append buffers
        for (const void* f : {(const void*)net_init, (const void*)net_commit})
            PGC_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)g->smem));
    }
    if (g->det_smem > 48 * 1024)
        PGC_CUDA(cudaFuncSetAttribute((const void*)net_detect,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)g->det_smem));
    int per_sm = o.grid_per_sm;
    if (per_sm == 0) {
        int a = 0, b = 0;
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, net_detect, o.block, g->det_smem));
        PGC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, net_commit, o.block, g->smem));
        per_sm = std::max(1, std::min(a, b));
        g->det_grid = cx.dev.num_sms * std::max(1, a);
    } else {
        g->det_grid = cx.dev.num_sms * per_sm;
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

// {assign, detect, commit} inside a WHILE node that starts with condition 1.
static pgc_status build_graph(Context& cx, const Geometry& g) {
    cx.destroy_graph();
    Problem* dP = cx.problem.as<Problem>();
    PGC_CUDA(cudaGraphCreate(&cx.graph, 0));
    PGC_CUDA(cudaGraphConditionalHandleCreate(&cx.handle, cx.graph, 1u, cudaGraphCondAssignDefault));
    int use_cond = 1;
    cudaGraphConditionalHandle hnd = cx.handle;
    void* p_args[] = {&dP};
    void* c_args[] = {&dP, &hnd, &use_cond};
    cudaGraphNode_t n_loop;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cx.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    PGC_CUDA(cudaGraphAddNode(&n_loop, cx.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaKernelNodeParams k_asg = knode((void*)net_assign, g, 0, c_args);
    cudaKernelNodeParams k_det = knode((void*)net_detect, g, g.det_smem, p_args);
    k_det.gridDim = dim3(g.det_grid);
    cudaKernelNodeParams k_com = knode((void*)net_commit, g, g.smem, c_args);
    cudaGraphNode_t b_asg, b_det, b_com;
    PGC_CUDA(cudaGraphAddKernelNode(&b_asg, body, nullptr, 0, &k_asg));
    PGC_CUDA(cudaGraphAddKernelNode(&b_det, body, &b_asg, 1, &k_det));
    PGC_CUDA(cudaGraphAddKernelNode(&b_com, body, &b_det, 1, &k_com));
    PGC_CUDA(cudaGraphInstantiate(&cx.exec, cx.graph, 0));
    cx.g_grid = g.grid;
    cx.g_det = g.det_grid;
    cx.g_block = g.block;
    return PGC_OK;
}

struct Input {
    int n, n_nets, self;
    const int *m_ptr, *m_idx, *r_ptr, *r_idx;
    int* col;
};

static pgc_status run_scratch(Context& cx, const Input& in, uint64_t seed, const Opts& o,
                              cudaStream_t stream, int* rounds, int* num_colors);

// Out of device memory: keep no half-grown scratch (the next call allocates
// again).
static pgc_status run(Context& cx, const Input& in, uint64_t seed, const Opts& o,
                      cudaStream_t stream, int* rounds, int* num_colors) {
    pgc_status s = run_scratch(cx, in, seed, o, stream, rounds, num_colors);
    if (s == PGC_ERR_OOM) cx.release();
    return s;
}

static pgc_status run_scratch(Context& cx, const Input& in, uint64_t seed, const Opts& o,
                              cudaStream_t stream, int* rounds, int* num_colors) {
    const int n = in.n;
    if (pgc_status s = cx.key.ensure((size_t)n * 8)) return s;
    if (pgc_status s = cx.ck.ensure((size_t)n * 8)) return s;
    if (pgc_status s = cx.flag.ensure((size_t)std::max(in.n_nets, 1) * 4)) return s;
    if (pgc_status s = cx.wt.ensure((size_t)n * 4 * 2)) return s;
    if (pgc_status s = cx.ww.ensure((size_t)n * 4 * 2)) return s;
    if (pgc_status s = cx.state.ensure(sizeof(State))) return s;
    if (pgc_status s = cx.problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_state.ensure(sizeof(State))) return s;
    const int want_trace = o.profile && o.profile->trace_cap > 0 ? o.profile->trace_cap : 0;
    const int tcap = std::max(want_trace, 1);
    if (cx.trace_cap < tcap) {
        if (pgc_status s = cx.trace.ensure((size_t)tcap * 5 * sizeof(long long))) return s;
        if (pgc_status s = cx.h_misc.ensure((size_t)tcap * 5 * sizeof(long long))) return s;
        cx.trace_cap = tcap;
    }
    Geometry g;
    if (pgc_status s = geometry(cx, o, &g)) return s;

    Problem* hp = cx.h_problem.as<Problem>();
    std::memset(hp, 0, sizeof(Problem));
    hp->m_ptr = in.m_ptr;
    hp->m_idx = in.m_idx;
    hp->r_ptr = in.r_ptr;
    hp->r_idx = in.r_idx;
    hp->col = in.col;
    hp->key = cx.key.as<unsigned long long>();
    hp->ck = cx.ck.as<int2>();
    hp->net_flag = cx.flag.as<int>();
    for (int p = 0; p < 2; ++p) {
        hp->wt[p] = cx.wt.as<int>() + (size_t)p * n;
        hp->ww[p] = cx.ww.as<int>() + (size_t)p * n;
    }
    hp->trace_w = cx.trace.as<long long>();
    hp->trace_s = hp->trace_w + tcap;
    hp->trace_h = hp->trace_s + tcap;
    hp->trace_nets = hp->trace_h + tcap;
    hp->trace_members = hp->trace_nets + tcap;
    hp->trace_cap = want_trace;
    hp->st = cx.state.as<State>();
    hp->seed = seed;
    hp->timeout_ns = (unsigned long long)o.timeout_ms * 1000000ull;
    hp->n = n;
    hp->n_nets = in.n_nets;
    hp->self = in.self;
    hp->use_deg = (o.flags & PGC_NO_DEGREE_RULE) ? 0 : 1;
    hp->max_rounds = o.max_rounds > 0 ? o.max_rounds : (n < INT32_MAX ? n + 1 : n);
    hp->windows = 1;
    Problem* dP = cx.problem.as<Problem>();
    State* hs = cx.h_state.as<State>();

    // setup, then the color bound decides how many 64-color mask windows
    PGC_CUDA(cudaMemcpyAsync(dP, hp, sizeof(Problem), cudaMemcpyHostToDevice, stream));
    PGC_CUDA(cudaMemsetAsync(cx.state.ptr, 0, sizeof(State), stream));
    KernelTimer kt;
    kt.prof = (o.flags & PGC_HOST_LOOP) ? o.profile : nullptr;
    kt.stream = stream;
    if (pgc_status s = kt.begin(0, "net_init")) return s;
    net_init<<<g.grid, g.block, g.smem, stream>>>(dP);
    PGC_CUDA(cudaGetLastError());
    if (pgc_status s = kt.end()) return s;
    PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    const long long need = (long long)hs->bound + 1;   // a first-fit color is <= |S(v)| + 1
    const int windows = (int)std::min<long long>(kMaxWindows, (need + 63) / 64);
    hp->windows = std::max(1, windows);
    const size_t mask_bytes = (size_t)hp->windows * (size_t)std::max(in.n_nets, 1) * 8;
    if (pgc_status s = cx.mask.ensure(mask_bytes)) return s;
    hp->mask = cx.mask.as<unsigned long long>();
    PGC_CUDA(cudaMemcpyAsync(dP, hp, sizeof(Problem), cudaMemcpyHostToDevice, stream));
    PGC_CUDA(cudaMemsetAsync(cx.mask.ptr, 0, mask_bytes, stream));

    if (!(o.flags & PGC_HOST_LOOP)) {
        if (!cx.exec || cx.g_grid != g.grid || cx.g_block != g.block || cx.g_det != g.det_grid) {
            if (pgc_status s = build_graph(cx, g)) return s;
        }
        PGC_CUDA(cudaGraphLaunch(cx.exec, stream));
    } else {
        const cudaGraphConditionalHandle none = 0;
        for (int round = 1;; ++round) {
            if (pgc_status s = kt.begin(1, "net_assign")) return s;
            net_assign<<<g.grid, g.block, 0, stream>>>(dP, none, 0);
            PGC_CUDA(cudaGetLastError());
            if (pgc_status s = kt.end()) return s;
            if (pgc_status s = kt.begin(2, "net_detect")) return s;
            net_detect<<<g.det_grid, g.block, g.det_smem, stream>>>(dP);
            PGC_CUDA(cudaGetLastError());
            if (pgc_status s = kt.end()) return s;
            if (pgc_status s = kt.begin(3, "net_commit")) return s;
            net_commit<<<g.grid, g.block, g.smem, stream>>>(dP, none, 0);
            PGC_CUDA(cudaGetLastError());
            if (pgc_status s = kt.end()) return s;
            PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
            PGC_CUDA(cudaStreamSynchronize(stream));
            if (hs->done) break;
            if (round > hp->max_rounds + 1)
                return fail(PGC_ERR_CUDA, "device round control did not finish the loop");
        }
    }
    kt.destroy();
    PGC_CUDA(cudaMemcpyAsync(hs, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost, stream));
    if (want_trace) {
        PGC_CUDA(cudaMemcpyAsync(cx.h_misc.ptr, cx.trace.ptr, (size_t)tcap * 5 * sizeof(long long),
                                 cudaMemcpyDeviceToHost, stream));
    }
    PGC_CUDA(cudaStreamSynchronize(stream));
    if (want_trace) {
        const long long* tw = cx.h_misc.as<long long>();
        const long long* ts = tw + tcap;
        const long long* th = ts + tcap;
        const long long* tn = th + tcap;
        const long long* tm = tn + tcap;
        const int nr = std::min(hs->round, want_trace);
        for (int i = 0; i < want_trace; ++i) {
            if (o.profile->trace_w) o.profile->trace_w[i] = i < nr ? tw[i] : 0;
            if (o.profile->trace_s) o.profile->trace_s[i] = i < nr ? ts[i] : 0;
            if (o.profile->trace_h) o.profile->trace_h[i] = i < nr ? th[i] : 0;
            if (o.profile->trace_nets) o.profile->trace_nets[i] = i < nr ? tn[i] : 0;
            if (o.profile->trace_members) o.profile->trace_members[i] = i < nr ? tm[i] : 0;
        }
    }
    *rounds = hs->round;
    *num_colors = hs->max_color;
    switch (hs->status) {
        case ST_OK: return PGC_OK;
        case ST_NO_PROGRESS:
            return fail(PGC_ERR_NO_CONVERGE, "a round committed no vertex (inconsistent input?)");
        case ST_MAX_ROUNDS: return fail(PGC_ERR_NO_CONVERGE, "max_rounds reached");
        case ST_TIMEOUT: return fail(PGC_ERR_TIMEOUT, "device round loop exceeded timeout_ms");
        case ST_OVERFLOW:
            return fail(PGC_ERR_NO_CONVERGE, "a color above 4096 was needed (mask capacity)");
        default: return fail(PGC_ERR_CUDA, "unexpected device status");
    }
}

// ---------------------------------------------------------------------------
// asynchronous launch with caller-provided scratch (used by the server): the
// number of mask windows is given, so nothing waits on the device
// ---------------------------------------------------------------------------
size_t scratch_bytes(int n, int n_nets, int windows) {
    auto a = [](size_t x) { return (x + 255) / 256 * 256; };
    return a((size_t)n * 8) + a((size_t)n * 8) + a((size_t)std::max(n_nets, 1) * 4) +
           a((size_t)windows * (size_t)std::max(n_nets, 1) * 8) + a((size_t)n * 8) * 2;
}

static pgc_status launch_known(Context& cx, void* scratch, const Input& in, int windows,
                               uint64_t seed, const Opts& o, cudaStream_t stream) {
    const int n = in.n;
    auto a = [](size_t x) { return (x + 255) / 256 * 256; };
    char* p = static_cast<char*>(scratch);
    unsigned long long* key = reinterpret_cast<unsigned long long*>(p);
    p += a((size_t)n * 8);
    int2* ck = reinterpret_cast<int2*>(p);
    p += a((size_t)n * 8);
    int* flag = reinterpret_cast<int*>(p);
    p += a((size_t)std::max(in.n_nets, 1) * 4);
    unsigned long long* mask = reinterpret_cast<unsigned long long*>(p);
    const size_t mask_bytes = (size_t)windows * (size_t)std::max(in.n_nets, 1) * 8;
    p += a(mask_bytes);
    int* wt = reinterpret_cast<int*>(p);
    p += a((size_t)n * 8);
    int* ww = reinterpret_cast<int*>(p);
    if (pgc_status s = cx.state.ensure(sizeof(State))) return s;
    if (pgc_status s = cx.problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_problem.ensure(sizeof(Problem))) return s;
    if (pgc_status s = cx.h_state.ensure(sizeof(State))) return s;
    if (pgc_status s = cx.trace.ensure(3 * sizeof(long long))) return s;
    Geometry g;
    if (pgc_status s = geometry(cx, o, &g)) return s;
    Problem* hp = cx.h_problem.as<Problem>();
    std::memset(hp, 0, sizeof(Problem));
    hp->m_ptr = in.m_ptr;
    hp->m_idx = in.m_idx;
    hp->r_ptr = in.r_ptr;
    hp->r_idx = in.r_idx;
    hp->col = in.col;
    hp->key = key;
    hp->ck = ck;
    hp->net_flag = flag;
    hp->mask = mask;
    for (int q = 0; q < 2; ++q) {
        hp->wt[q] = wt + (size_t)q * n;
        hp->ww[q] = ww + (size_t)q * n;
    }
    hp->trace_w = hp->trace_s = hp->trace_h = cx.trace.as<long long>();
    hp->trace_nets = hp->trace_members = cx.trace.as<long long>();
    hp->trace_cap = 0;
    hp->st = cx.state.as<State>();
    hp->seed = seed;
    hp->timeout_ns = (unsigned long long)o.timeout_ms * 1000000ull;
    hp->n = n;
    hp->n_nets = in.n_nets;
    hp->self = in.self;
    hp->use_deg = (o.flags & PGC_NO_DEGREE_RULE) ? 0 : 1;
    hp->max_rounds = o.max_rounds > 0 ? o.max_rounds : (n < INT32_MAX ? n + 1 : n);
    hp->windows = windows;
    Problem* dP = cx.problem.as<Problem>();
    PGC_CUDA(cudaMemcpyAsync(dP, hp, sizeof(Problem), cudaMemcpyHostToDevice, stream));
    PGC_CUDA(cudaMemsetAsync(cx.state.ptr, 0, sizeof(State), stream));
    PGC_CUDA(cudaMemsetAsync(mask, 0, mask_bytes, stream));
    net_init<<<g.grid, g.block, g.smem, stream>>>(dP);
    PGC_CUDA(cudaGetLastError());
    if (!cx.exec || cx.g_grid != g.grid || cx.g_block != g.block || cx.g_det != g.det_grid) {
        if (pgc_status s = build_graph(cx, g)) return s;
    }
    PGC_CUDA(cudaGraphLaunch(cx.exec, stream));
    PGC_CUDA(cudaMemcpyAsync(cx.h_state.ptr, cx.state.ptr, sizeof(State), cudaMemcpyDeviceToHost,
                             stream));
    return PGC_OK;
}

static pgc_status finish_known(Context& cx, int* rounds, int* num_colors) {
    const State* hs = cx.h_state.as<State>();
    *rounds = hs->round;
    *num_colors = hs->max_color;
    switch (hs->status) {
        case ST_OK: return PGC_OK;
        case ST_NO_PROGRESS:
            return fail(PGC_ERR_NO_CONVERGE, "a round committed no vertex (inconsistent input?)");
        case ST_MAX_ROUNDS: return fail(PGC_ERR_NO_CONVERGE, "max_rounds reached");
        case ST_TIMEOUT: return fail(PGC_ERR_TIMEOUT, "device round loop exceeded timeout_ms");
        case ST_OVERFLOW:
            return fail(PGC_ERR_NO_CONVERGE, "a color above 4096 was needed (mask capacity)");
        default: return fail(PGC_ERR_CUDA, "unexpected device status");
    }
}

// Reads a[idx] whether a is host or device memory.
static pgc_status read_int(const int* a, bool host, long long idx, int* out, Context& cx,
                           cudaStream_t stream) {
    if (host) {
        *out = a[idx];
        return PGC_OK;
    }
    if (pgc_status s = cx.h_state.ensure(sizeof(State))) return s;
    int* hb = cx.h_state.as<int>();
    PGC_CUDA(cudaMemcpyAsync(hb, a + idx, 4, cudaMemcpyDeviceToHost, stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    *out = *hb;
    return PGC_OK;
}

// Stages a host array of count ints into slot; returns the device pointer.
static pgc_status stage(Context& cx, int slot, const int* a, long long count, cudaStream_t stream,
                        const int** out) {
    if (!is_host_pointer(a)) {
        *out = a;
        return PGC_OK;
    }
    if (pgc_status s = cx.stage[slot].ensure((size_t)std::max<long long>(count, 1) * 4)) return s;
    if (count > 0)
        PGC_CUDA(cudaMemcpyAsync(cx.stage[slot].ptr, a, (size_t)count * 4, cudaMemcpyHostToDevice,
                                 stream));
    *out = cx.stage[slot].as<int>();
    return PGC_OK;
}

static pgc_status color(int kind, int32_t n_rows, int32_t n_cols, const int32_t* row_ptr,
                        const int32_t* col_idx, const int32_t* col_ptr, const int32_t* row_idx,
                        uint64_t seed, int32_t* colors, int32_t* rounds, int32_t* num_colors,
                        const pgc_opts* opts, void* stream_v) {
    if (!rounds || !num_colors) return fail(PGC_ERR_INVALID_ARG, "rounds/num_colors must be non-NULL");
    if (n_rows < 0 || n_cols < 0) return fail(PGC_ERR_INVALID_ARG, "negative size");
    Opts o;
    if (pgc_status s = read_opts(opts, &o)) return s;
    *rounds = 0;
    *num_colors = 0;
    if (o.flags & (PGC_ASYNC | PGC_PRIORITY_DYNAMIC | PGC_PRIORITY_SATURATION))
        return fail(PGC_ERR_INVALID_ARG, "PGC_ASYNC and the round-varying priorities are D1 "
                                         "options");
    const long long n_ll = kind == 2 ? n_rows : kind == 4 ? (long long)n_cols + n_rows : n_cols;
    if (n_ll > INT32_MAX - 1) return fail(PGC_ERR_INVALID_ARG, "n_rows + n_cols too large");
    const int n = (int)n_ll;
    if (n == 0) return PGC_OK;
    if (!row_ptr || !colors || (kind >= 3 && !col_ptr))
        return fail(PGC_ERR_INVALID_ARG, "NULL array");
    cudaStream_t stream = (cudaStream_t)stream_v;
    DeviceInfo dev;
    if (pgc_status s = current_device(&dev)) return s;
    Context* cx = get_context(dev.device);
    std::lock_guard<std::mutex> lk(cx->mu);
    cx->dev = dev;

    int nnz = 0, nnz_c = 0;
    if (pgc_status s = read_int(row_ptr, is_host_pointer(row_ptr), n_rows, &nnz, *cx, stream))
        return s;
    if (nnz < 0) return fail(PGC_ERR_INVALID_ARG, "row_ptr[n] < 0");
    if (nnz > 0 && !col_idx) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx");
    if (kind >= 3) {
        if (pgc_status s = read_int(col_ptr, is_host_pointer(col_ptr), n_cols, &nnz_c, *cx, stream))
            return s;
        if (nnz_c != nnz) return fail(PGC_ERR_INVALID_ARG, "CSR and CSC have different nnz");
        if (nnz > 0 && !row_idx) return fail(PGC_ERR_INVALID_ARG, "NULL row_idx");
    }
    if (kind == 4 && 2ll * nnz > (long long)INT32_MAX)
        return fail(PGC_ERR_INVALID_ARG, "PD2 over all of B needs 2 * nnz < 2^31");
    Input in;
    in.self = kind == 2 ? 1 : 0;
    in.n = n;
    in.n_nets = kind == 4 ? n_rows + n_cols : n_rows;
    if (pgc_status s = stage(*cx, 0, row_ptr, (long long)n_rows + 1, stream, &in.m_ptr)) return s;
    if (nnz > 0) {
        if (pgc_status s = stage(*cx, 1, col_idx, nnz, stream, &in.m_idx)) return s;
    } else {
        in.m_idx = col_idx;
    }
    if (kind == 2) {
        in.r_ptr = in.m_ptr;
        in.r_idx = in.m_idx;
    } else {
        if (pgc_status s = stage(*cx, 2, col_ptr, (long long)n_cols + 1, stream, &in.r_ptr))
            return s;
        if (nnz > 0) {
            if (pgc_status s = stage(*cx, 3, row_idx, nnz, stream, &in.r_idx)) return s;
        } else {
            in.r_idx = row_idx;
        }
    }
    if (kind == 4) {
        // the validation below reads the caller's CSR/CSC, still in in.m_*/in.r_*
        if (o.flags & PGC_VALIDATE) {
            if (pgc_status s = validate::csr_csc_pair(in.m_ptr, in.m_idx, n_rows, in.r_ptr,
                                                      in.r_idx, n_cols, dev, stream))
                return s;
        }
        const size_t offs = ((size_t)n_rows + n_cols + 1) * 4, ents = (size_t)std::max(nnz, 1) * 8;
        for (int k = 0; k < 4; ++k)
            if (pgc_status s = cx->both[k].ensure(k % 2 == 0 ? offs : ents)) return s;
        const long long work = std::max<long long>(2ll * nnz, (long long)n_rows + n_cols + 1);
        const int grid = (int)std::min<long long>((work + 255) / 256, (long long)dev.num_sms * 8);
        pd2b_combine<<<grid, 256, 0, stream>>>(in.m_ptr, in.m_idx, n_rows, in.r_ptr, in.r_idx,
                                               n_cols, cx->both[0].as<int>(),
                                               cx->both[1].as<int>(), cx->both[2].as<int>(),
                                               cx->both[3].as<int>());
        PGC_CUDA(cudaGetLastError());
        in.m_ptr = cx->both[0].as<int>();
        in.m_idx = cx->both[1].as<int>();
        in.r_ptr = cx->both[2].as<int>();
        in.r_idx = cx->both[3].as<int>();
    } else if (o.flags & PGC_VALIDATE) {
        if (kind == 2) {
            if (pgc_status s = validate::symmetric_csr(in.m_ptr, in.m_idx, n_rows, dev, stream))
                return s;
        } else if (pgc_status s = validate::csr_csc_pair(in.m_ptr, in.m_idx, n_rows, in.r_ptr,
                                                         in.r_idx, n_cols, dev, stream)) {
            return s;
        }
    }
    const bool host_col = is_host_pointer(colors);
    in.col = colors;
    if (host_col) {
        if (pgc_status s = cx->stage_col.ensure((size_t)n * 4)) return s;
        in.col = cx->stage_col.as<int>();
    }
    pgc_status s = run(*cx, in, seed, o, stream, rounds, num_colors);
    if (s != PGC_OK) return s;
    if (host_col) {
        PGC_CUDA(cudaMemcpyAsync(colors, in.col, (size_t)n * 4, cudaMemcpyDeviceToHost, stream));
        PGC_CUDA(cudaStreamSynchronize(stream));
    }
    return PGC_OK;
}

}  // namespace net
}  // namespace pgc

extern "C" pgc_status pgc_color_d2(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                   uint64_t seed, int32_t* colors, int32_t* rounds,
                                   int32_t* num_colors, const pgc_opts* opts, void* stream) {
    try {
        return pgc::net::color(2, n, n, row_ptr, col_idx, nullptr, nullptr, seed, colors, rounds,
                               num_colors, opts, stream);
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    } catch (...) {
        return pgc::fail(PGC_ERR_CUDA, "unknown exception");
    }
}

extern "C" pgc_status pgc_color_pd2(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr,
                                    const int32_t* col_idx, const int32_t* col_ptr,
                                    const int32_t* row_idx, uint64_t seed, int32_t* colors,
                                    int32_t* rounds, int32_t* num_colors, const pgc_opts* opts,
                                    void* stream) {
    try {
        return pgc::net::color(3, n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, seed, colors,
                               rounds, num_colors, opts, stream);
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    } catch (...) {
        return pgc::fail(PGC_ERR_CUDA, "unknown exception");
    }
}

extern "C" pgc_status pgc_color_pd2_bipartite(int32_t n_rows, int32_t n_cols,
                                               const int32_t* row_ptr, const int32_t* col_idx,
                                               const int32_t* col_ptr, const int32_t* row_idx,
                                               uint64_t seed, int32_t* colors, int32_t* rounds,
                                               int32_t* num_colors, const pgc_opts* opts,
                                               void* stream) {
    try {
        return pgc::net::color(4, n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, seed, colors,
                               rounds, num_colors, opts, stream);
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    } catch (...) {
        return pgc::fail(PGC_ERR_CUDA, "unknown exception");
    }
}

namespace pgc {
namespace net {

// Slot API for the server (declared in runtime.h).
void* slot_create() { return new Context(); }

void slot_destroy(void* c) {
    auto* cx = static_cast<Context*>(c);
    cx->release();
    delete cx;
}

pgc_status slot_launch_pd2(void* c, void* scratch, int n_rows, int n_cols, const int* row_ptr,
                           const int* col_idx, const int* col_ptr, const int* row_idx, int* colors,
                           int windows, uint64_t seed, cudaStream_t stream) {
    auto* cx = static_cast<Context*>(c);
    if (pgc_status s = current_device(&cx->dev)) return s;
    Input in;
    in.n = n_cols;
    in.n_nets = n_rows;
    in.self = 0;
    in.m_ptr = row_ptr;
    in.m_idx = col_idx;
    in.r_ptr = col_ptr;
    in.r_idx = row_idx;
    in.col = colors;
    Opts o;
    return launch_known(*cx, scratch, in, windows, seed, o, stream);
}

bool slot_overflowed(void* c) {
    return static_cast<Context*>(c)->h_state.as<State>()->status == ST_OVERFLOW;
}

pgc_status slot_finish(void* c, int* rounds, int* num_colors) {
    return finish_known(*static_cast<Context*>(c), rounds, num_colors);
}

}  // namespace net
}  // namespace pgc
