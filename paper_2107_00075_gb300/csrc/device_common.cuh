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
// buffer of 64 slots is flushed 32 entries at a time with one atomicAdd, so
// list writes are coalesced and counter atomics are 32x fewer.  All 32
// lanes must call wa_push / wa_flush together.
struct WarpAppend {
    int* buf;    // 64 ints of shared memory owned by this warp
    int count;   // warp-uniform, < 32 between calls
};

__device__ __forceinline__ void wa_push(WarpAppend& a, bool pred, int v, int* out, int* out_cnt) {
    const unsigned lane = lane_id();
    const unsigned m = __ballot_sync(kFullMask, pred);
    if (pred) a.buf[a.count + __popc(m & ((1u << lane) - 1u))] = v;
    a.count += __popc(m);
    __syncwarp();
    if (a.count >= 32) {
        int base = 0;
        if (lane == 0) base = atomicAdd(out_cnt, 32);
        base = __shfl_sync(kFullMask, base, 0);
        out[base + lane] = a.buf[lane];
        const int rem = a.count - 32;
        const int tmp = (int)lane < rem ? a.buf[32 + lane] : 0;
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
    if ((int)lane < a.count) out[base + lane] = a.buf[lane];
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

// WarpAppend for 16-byte entries (a 64-entry int4 buffer per warp).
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
    if (a.count >= 32) {
        int base = 0;
        if (lane == 0) base = atomicAdd(out_cnt, 32);
        base = __shfl_sync(kFullMask, base, 0);
        out[base + lane] = a.buf[lane];
        const int rem = a.count - 32;
        int4 tmp = make_int4(0, 0, 0, 0);
        if ((int)lane < rem) tmp = a.buf[32 + lane];
        __syncwarp();
        if ((int)lane < rem) a.buf[lane] = tmp;
        a.count = rem;
        __syncwarp();
    }
}

__device__ __forceinline__ void wa4_flush(WarpAppend4& a, int4* out, int* out_cnt) {
    if (a.count == 0) return;
    const unsigned lane = lane_id();
    int base = 0;
    if (lane == 0) base = atomicAdd(out_cnt, a.count);
    base = __shfl_sync(kFullMask, base, 0);
    if ((int)lane < a.count) out[base + lane] = a.buf[lane];
    a.count = 0;
    __syncwarp();
}

}  // namespace pgc
