// runtime.h -- host-side internals of the coloring library (not installed).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pgc.h"

namespace pgc {

// Records msg as the calling thread's last error and returns s.
pgc_status fail(pgc_status s, const std::string& msg);
pgc_status cuda_fail(cudaError_t e, const char* what);

#define PGC_CUDA(call)                                           \
    do {                                                         \
        cudaError_t e__ = (call);                                \
        if (e__ != cudaSuccess) return ::pgc::cuda_fail(e__, #call); \
    } while (0)

// A device allocation that grows on demand and is reused across calls.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    pgc_status ensure(size_t need);   // grows (never shrinks); contents lost on growth
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Pinned host staging buffer.
struct HostBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    pgc_status ensure(size_t need);
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// true if p is host memory the GPU must not dereference (pageable or pinned
// host allocation); false for device or managed memory.
bool is_host_pointer(const void* p);

// Fault-injection settings of the test hooks (pgc_test_* in pgc.h).
struct TestHooks {
    int fail_alloc_after = -1;          // allocations left before one fails (-1: off)
    unsigned barrier_polls = 1u << 22;  // core-loop grid barrier: polls before giving up
    int slow_block = -1;                // core loop: this block arrives late (-1: none)
    unsigned slow_us = 0;               // ... by this many microseconds
};
TestHooks test_hooks();                 // a snapshot
bool test_take_alloc_failure();         // true if this allocation must fail

// Effective options (defaults filled in).
struct Opts {
    uint32_t flags = 0;
    int32_t max_rounds = 0;
    int32_t mid_degree = 64;
    int32_t hub_degree = 16384;
    int32_t block = 256;
    int32_t grid_per_sm = 0;
    int32_t timeout_ms = 60000;
    int32_t tail_vertices = 4096;
    pgc_profile* profile = nullptr;
};
pgc_status read_opts(const pgc_opts* in, Opts* out);

// Device properties cached per device.
struct DeviceInfo {
    int device = 0;
    int num_sms = 0;
};
pgc_status current_device(DeviceInfo* out);

// Times kernels with CUDA events in host-loop mode.
struct KernelTimer {
    pgc_profile* prof = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int slot = -1;
    pgc_status begin(int slot, const char* name);
    pgc_status end();
    void destroy();
};

// PGC_VALIDATE checks (validate.cu): offsets and id ranges, and
// symmetric_csr: the graph is symmetric (as a multiset of entries);
// csr_csc_pair: the CSR and the CSC hold the same (row, column) pairs.
// PGC_ERR_INVALID_ARG with a message on the first failed check.
namespace validate {
pgc_status symmetric_csr(const int* rp, const int* ci, int n, const DeviceInfo& dev,
                         cudaStream_t stream);
pgc_status csr_csc_pair(const int* rp, const int* ci, int n_rows, const int* cp, const int* ri,
                        int n_cols, const DeviceInfo& dev, cudaStream_t stream);
}  // namespace validate

// Partial distance-2 engine slots for the server (net.cu).
namespace net {
size_t scratch_bytes(int n, int n_nets, int windows);
void* slot_create();
void slot_destroy(void* slot);
pgc_status slot_launch_pd2(void* slot, void* scratch, int n_rows, int n_cols, const int* row_ptr,
                           const int* col_idx, const int* col_ptr, const int* row_idx, int* colors,
                           int windows, uint64_t seed, cudaStream_t stream);
pgc_status slot_finish(void* slot, int* rounds, int* num_colors);
bool slot_overflowed(void* slot);   // the last launch needed more mask windows
}  // namespace net

}  // namespace pgc
