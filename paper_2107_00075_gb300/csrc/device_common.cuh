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
