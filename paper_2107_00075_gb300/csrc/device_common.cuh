// device_common.cuh -- device helpers shared by the coloring kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pgc {

constexpr int kWarp = 32;

// h(v) = splitmix64(seed XOR v): the priority hash standing in for rand(GID)
// of Alg. 4.  splitmix64 (Steele, Lea, Flood 2014) maps state x to
// mix(x + 0x9E3779B97F4A7C15) with the two xor-shift-multiply rounds below.
__device__ __forceinline__ uint64_t prio_hash(uint64_t seed, uint32_t v) {
    uint64_t z = (seed ^ (uint64_t)v) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// True if u has priority over v: key(u) > key(v) with key = (deg, -h, -id).
// This is Alg. 4 read as one comparison: of two equal-colored vertices the
// one that does NOT have priority is recolored.
__device__ __forceinline__ bool has_priority(int du, uint64_t hu, int u,
                                             int dv, uint64_t hv, int v, bool use_deg) {
    if (use_deg && du != dv) return du > dv;
    if (hu != hv) return hu < hv;
    return u < v;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & (kWarp - 1); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Streaming (read-once) 32-bit load for adjacency data.
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }

}  // namespace pgc

namespace pgc {

constexpr unsigned kFullMask = 0xffffffffu;

// Warp-aggregated worklist append: lanes push (pred, v); a per-warp shared
// buffer of kAppendSlots entries is flushed kAppendFlush entries at a time
// with one atomicAdd, so list writes are coalesced and the list counter --
// one address that every warp of the grid hits -- takes kAppendFlush times
// fewer atomics.  All 32 lanes must call wa_push / wa_flush together.
constexpr int kAppendFlush = 224;               // a multiple of 32
constexpr int kAppendSlots = kAppendFlush + 32; // per appender

struct WarpAppend {
    int* buf;    // kAppendSlots ints of shared memory owned by this warp
    int count;   // warp-uniform, < kAppendFlush between calls
};

__device__ __forceinline__ void wa_push(WarpAppend& a, bool pred, int v, int* out, int* out_cnt) {
    const unsigned lane = lane_id();
    const unsigned m = __ballot_sync(kFullMask, pred);
    if (pred) a.buf[a.count + __popc(m & ((1u << lane) - 1u))] = v;
    a.count += __popc(m);
    __syncwarp();
    if (a.count >= kAppendFlush) {
        int base = 0;
        if (lane == 0) base = atomicAdd(out_cnt, kAppendFlush);
        base = __shfl_sync(kFullMask, base, 0);
#pragma unroll
        for (int k = 0; k < kAppendFlush; k += 32) out[base + k + lane] = a.buf[k + lane];
        const int rem = a.count - kAppendFlush;
        const int tmp = (int)lane < rem ? a.buf[kAppendFlush + lane] : 0;
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
    base = __shfl_sync(kFullMask, base, 0);
    for (int k = lane; k < a.count; k += 32) out[base + k] = a.buf[k];
    a.count = 0;
    __syncwarp();
}

__device__ __forceinline__ int warp_max(int x) {
    for (int o = 16; o; o >>= 1) x = max(x, __shfl_xor_sync(kFullMask, x, o));
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
    return x;
}

// Index of the first word of v's forbidden-color bitmap.  Vertex v owns
// floor(deg(v)/32) + 1 words (bits for colors 1..deg(v)+1, enough because a
// first-fit color never exceeds deg(v)+1); with offset floor(rp[v]/32) + v
// consecutive vertices never overlap and the total is nnz/32 + n + 1 words.
__device__ __forceinline__ long long bitmap_offset(int rp_v, int v) {
    return (long long)(rp_v >> 5) + v;
}

}  // namespace pgc

namespace pgc {

// WarpAppend for 16-byte entries (kAppend4Slots int4 per appender).  Its
// buffer is kept at 32 + 32 entries: the distance-1 detection kernel that
// uses it relies on L1, and a larger shared buffer costs more L1 than the
// saved counter atomics are worth (measured: round 2 of R-MAT-24 took 50%
// longer with 96-entry flushes).
constexpr int kAppend4Flush = 32;
constexpr int kAppend4Slots = kAppend4Flush + 32;

struct WarpAppend4 {
    int4* buf;
    int count;
};

__device__ __forceinline__ void wa4_push(WarpAppend4& a, bool pred, int4 e, int4* out,
                                         int* out_cnt) {
    const unsigned lane = lane_id();
    const unsigned m = __ballot_sync(kFullMask, pred);
    if (pred) a.buf[a.count + __popc(m & ((1u << lane) - 1u))] = e;
    a.count += __popc(m);
    __syncwarp();
    if (a.count >= kAppend4Flush) {
        int base = 0;
        if (lane == 0) base = atomicAdd(out_cnt, kAppend4Flush);
        base = __shfl_sync(kFullMask, base, 0);
#pragma unroll
        for (int k = 0; k < kAppend4Flush; k += 32) out[base + k + lane] = a.buf[k + lane];
        const int rem = a.count - kAppend4Flush;
        int4 tmp = make_int4(0, 0, 0, 0);
        if ((int)lane < rem) tmp = a.buf[kAppend4Flush + lane];
        __syncwarp();
        if ((int)lane < rem) a.buf[lane] = tmp;
        a.count = rem;
        __syncwarp();
    }
}

// Re-append of entries that already sit in a source list (a loser keeps
// its entry for the next round): the shared buffer holds 4-byte source
// indices instead of 16-byte entries, so the same shared memory takes
// kIdxFlush entries per counter atomic; the flush copies the entries from
// the source list (just read, so mostly cache hits).
constexpr int kIdxFlush = 224;
constexpr int kIdxSlots = kIdxFlush + 32;

struct IdxAppend {
    int* buf;    // kIdxSlots ints of shared memory owned by this warp
    int count;   // warp-uniform, < kIdxFlush between calls
};

__device__ __forceinline__ void ia_push(IdxAppend& a, bool pred, int idx, const int4* src,
                                        int4* out, int* out_cnt) {
    const unsigned lane = lane_id();
    const unsigned m = __ballot_sync(kFullMask, pred);
    if (pred) a.buf[a.count + __popc(m & ((1u << lane) - 1u))] = idx;
    a.count += __popc(m);
    __syncwarp();
    if (a.count >= kIdxFlush) {
        int base = 0;
        if (lane == 0) base = atomicAdd(out_cnt, kIdxFlush);
        base = __shfl_sync(kFullMask, base, 0);
#pragma unroll
        for (int k = 0; k < kIdxFlush; k += 32) out[base + k + lane] = src[a.buf[k + lane]];
        const int rem = a.count - kIdxFlush;
        const int tmp = (int)lane < rem ? a.buf[kIdxFlush + lane] : 0;
        __syncwarp();
        if ((int)lane < rem) a.buf[lane] = tmp;
        a.count = rem;
        __syncwarp();
    }
}

__device__ __forceinline__ void ia_flush(IdxAppend& a, const int4* src, int4* out, int* out_cnt) {
    if (a.count == 0) return;
    const unsigned lane = lane_id();
    int base = 0;
    if (lane == 0) base = atomicAdd(out_cnt, a.count);
    base = __shfl_sync(kFullMask, base, 0);
    for (int k = lane; k < a.count; k += 32) out[base + k] = src[a.buf[k]];
    a.count = 0;
    __syncwarp();
}

__device__ __forceinline__ void wa4_flush(WarpAppend4& a, int4* out, int* out_cnt) {
    if (a.count == 0) return;
    const unsigned lane = lane_id();
    int base = 0;
    if (lane == 0) base = atomicAdd(out_cnt, a.count);
    base = __shfl_sync(kFullMask, base, 0);
    for (int k = lane; k < a.count; k += 32) out[base + k] = a.buf[k];
    a.count = 0;
    __syncwarp();
}

}  // namespace pgc
