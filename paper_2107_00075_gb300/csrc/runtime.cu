// runtime.cu -- error state, buffers, options and the general C ABI calls.
#include "runtime.h"

#include <cstdio>
#include <cstring>
#include <functional>

namespace pgc {

static thread_local std::string t_last_error;

pgc_status fail(pgc_status s, const std::string& msg) {
    t_last_error = msg;
    return s;
}

pgc_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return fail(PGC_ERR_OOM, m);
    }
    return fail(PGC_ERR_CUDA, m);
}

static std::mutex g_hooks_mu;
static TestHooks g_hooks;

TestHooks test_hooks() {
    std::lock_guard<std::mutex> lk(g_hooks_mu);
    return g_hooks;
}

bool test_take_alloc_failure() {
    std::lock_guard<std::mutex> lk(g_hooks_mu);
    if (g_hooks.fail_alloc_after < 0) return false;
    if (g_hooks.fail_alloc_after == 0) {
        g_hooks.fail_alloc_after = -1;
        return true;
    }
    g_hooks.fail_alloc_after -= 1;
    return false;
}

pgc_status DevBuf::ensure(size_t need) {
    if (need <= bytes && ptr) return PGC_OK;
    release();
    size_t sz = need < 256 ? 256 : need;
    if (test_take_alloc_failure())
        return fail(PGC_ERR_OOM, "cudaMalloc: injected allocation failure (pgc_test_fail_alloc)");
    cudaError_t e = cudaMalloc(&ptr, sz);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return cuda_fail(e, "cudaMalloc");
    }
    bytes = sz;
    return PGC_OK;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

pgc_status HostBuf::ensure(size_t need) {
    if (need <= bytes && ptr) return PGC_OK;
    release();
    size_t sz = need < 256 ? 256 : need;
    cudaError_t e = cudaMallocHost(&ptr, sz);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return cuda_fail(e, "cudaMallocHost");
    }
    bytes = sz;
    return PGC_OK;
}

void HostBuf::release() {
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
}

bool is_host_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown to CUDA: plain pageable host memory
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

pgc_status read_opts(const pgc_opts* in, Opts* out) {
    Opts o;
    if (in) {
        o.flags = in->flags;
        if (in->max_rounds < 0) return fail(PGC_ERR_INVALID_ARG, "max_rounds < 0");
        o.max_rounds = in->max_rounds;
        if (in->mid_degree < 0 || in->hub_degree < 0)
            return fail(PGC_ERR_INVALID_ARG, "negative degree threshold");
        if (in->mid_degree > 0) o.mid_degree = in->mid_degree;
        if (in->hub_degree > 0) o.hub_degree = in->hub_degree;
        if (in->block != 0) {
            if (in->block < 128 || in->block > 1024 || in->block % 32)
                return fail(PGC_ERR_INVALID_ARG, "block must be a multiple of 32 in [128, 1024]");
            o.block = in->block;
        }
        if (in->grid_per_sm < 0) return fail(PGC_ERR_INVALID_ARG, "grid_per_sm < 0");
        o.grid_per_sm = in->grid_per_sm;
        if (in->timeout_ms < 0) return fail(PGC_ERR_INVALID_ARG, "timeout_ms < 0");
        if (in->timeout_ms > 0) o.timeout_ms = in->timeout_ms;
        if (in->tail_vertices > 0) o.tail_vertices = in->tail_vertices;
        if (in->tail_vertices < 0) o.tail_vertices = 0;
        o.profile = in->profile;
    }
    if (o.hub_degree < o.mid_degree) o.hub_degree = o.mid_degree;
    *out = o;
    return PGC_OK;
}

pgc_status current_device(DeviceInfo* out) {
    int dev = 0;
    PGC_CUDA(cudaGetDevice(&dev));
    int sms = 0;
    PGC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    out->device = dev;
    out->num_sms = sms;
    return PGC_OK;
}

pgc_status KernelTimer::begin(int s, const char* name) {
    if (!prof) return PGC_OK;
    if (s < 0 || s >= PGC_MAX_KERNELS) return PGC_OK;
    if (!a) {
        PGC_CUDA(cudaEventCreate(&a));
        PGC_CUDA(cudaEventCreate(&b));
    }
    slot = s;
    if (prof->num_kernels < s + 1) prof->num_kernels = s + 1;
    prof->kernel_names[s] = name;
    PGC_CUDA(cudaEventRecord(a, stream));
    return PGC_OK;
}

pgc_status KernelTimer::end() {
    if (!prof || slot < 0) return PGC_OK;
    PGC_CUDA(cudaEventRecord(b, stream));
    PGC_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    PGC_CUDA(cudaEventElapsedTime(&ms, a, b));
    prof->kernel_ms[slot] += ms;
    prof->kernel_launches[slot] += 1;
    const int k = prof->num_launches++;
    if (k < prof->launch_cap) {
        if (prof->launch_slot) prof->launch_slot[k] = slot;
        if (prof->launch_ms) prof->launch_ms[k] = ms;
    }
    slot = -1;
    return PGC_OK;
}

void KernelTimer::destroy() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    a = b = nullptr;
}

// Release hooks registered by the problem-specific translation units.
std::vector<std::function<void()>>& release_hooks() {
    static std::vector<std::function<void()>> h;
    return h;
}

}  // namespace pgc

extern "C" {

void pgc_opts_init(pgc_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
}

const char* pgc_last_error(void) { return pgc::t_last_error.c_str(); }

const char* pgc_status_string(pgc_status s) {
    switch (s) {
        case PGC_OK: return "PGC_OK";
        case PGC_ERR_INVALID_ARG: return "PGC_ERR_INVALID_ARG";
        case PGC_ERR_CUDA: return "PGC_ERR_CUDA";
        case PGC_ERR_OOM: return "PGC_ERR_OOM";
        case PGC_ERR_NO_CONVERGE: return "PGC_ERR_NO_CONVERGE";
        case PGC_ERR_TIMEOUT: return "PGC_ERR_TIMEOUT";
        case PGC_ERR_BUSY: return "PGC_ERR_BUSY";
        case PGC_ERR_NOT_FOUND: return "PGC_ERR_NOT_FOUND";
    }
    return "PGC_ERR_UNKNOWN";
}

const char* pgc_version(void) { return "pgc 0.1.0 (sm_103a)"; }

pgc_status pgc_release(void) {
    for (auto& f : pgc::release_hooks()) f();
    return PGC_OK;
}

pgc_status pgc_test_fail_alloc(int32_t after) {
    std::lock_guard<std::mutex> lk(pgc::g_hooks_mu);
    pgc::g_hooks.fail_alloc_after = after < 0 ? -1 : after;
    return PGC_OK;
}

pgc_status pgc_test_core_barrier(uint32_t polls, int32_t slow_block, uint32_t slow_us) {
    if (slow_us > 2000000u)
        return pgc::fail(PGC_ERR_INVALID_ARG, "pgc_test_core_barrier: slow_us above 2 s");
    std::lock_guard<std::mutex> lk(pgc::g_hooks_mu);
    pgc::g_hooks.barrier_polls = polls == 0 ? (1u << 22) : polls;
    pgc::g_hooks.slow_block = slow_block;
    pgc::g_hooks.slow_us = slow_block < 0 ? 0u : slow_us;
    return PGC_OK;
}

}  // extern "C"
