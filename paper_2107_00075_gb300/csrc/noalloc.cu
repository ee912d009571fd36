// noalloc.cu -- pgc_color_d1_noalloc: distance-1 coloring that allocates
// no memory at all.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: code that
// runs while a framework's caching allocator owns the whole device (an
// out-of-band allocation can fail or fragment its pool), latency-critical
// loops where cudaFree's implicit device synchronisation is not acceptable,
// and plug-ins that are forbidden to allocate by their host application.
// This entry point serves them for small graphs: every scratch buffer of the
// distance-1 engine (degrees, priority lists, forbidden-color sets,
// worklists, round state) lives in one file-scope __device__ array of fixed
// size, which every GPU that loads the library keeps until the process
// exits.  The caller still passes the graph and the output in device memory.
// The kernels are the same as pgc_color_d1's, with its default detection
// tiers; the rounds are driven from the host (one small device-to-host read
// per round), so no CUDA graph is built, and the core phase (a cooperative
// launch for the last rounds) is not used: every round runs the per-round
// kernels, which give the same colors.
#include "d1_engine.cuh"

#include <cuda.h>

namespace pgc {
namespace d1 {

constexpr int kNoAllocMaxN = 32768;             // vertices
constexpr long long kNoAllocMaxNnz = 524288;    // adjacency entries

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of every buffer inside the scratch array (sized for the
// maximum problem; a smaller problem uses a prefix of each buffer).
struct NoAllocLayout {
    static constexpr size_t n = kNoAllocMaxN, nnz = kNoAllocMaxNnz;
    static constexpr size_t state = 0;
    static constexpr size_t problem = align256(state + sizeof(State));
    static constexpr size_t deg = align256(problem + sizeof(Problem<SingleView>));
    static constexpr size_t hlen = align256(deg + 4 * n);
    static constexpr size_t hadj = align256(hlen + 4 * n);
    static constexpr size_t bm0 = align256(hadj + 4 * nnz);
    static constexpr size_t bmx = align256(bm0 + 8 * n);
    static constexpr size_t live = align256(bmx + 4 * ((nnz >> 5) + n + 1));
    static constexpr size_t lists = align256(live + 4 * (n / 32 + 2));
    static constexpr size_t items = align256(lists + 16 * n * 6);
    static constexpr size_t pushq = align256(items + 8 * (n + nnz / kBuildItem + 1));
    static constexpr size_t trace = align256(pushq + 8 * (n + nnz / kPushItem + 1));
    static constexpr size_t total = align256(trace + 3 * sizeof(long long));
};

// The scratch itself (about 6.5 MB).  In host code this name is only a
// stand-in for the device object; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NoAllocLayout::total];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_ptr[kMaxDevices];
static CUcontext g_noalloc_ctx[kMaxDevices];

// Once per device (and context), with that device current: resolve the
// array's address.  The address is cached with the context it belongs to,
// so a new context on the device (after cudaDeviceReset, or a context the
// caller made current) resolves it again.
// The current driver context, through the runtime's driver entry point (the
// library does not link the driver library itself); nullptr if unavailable.
static CUcontext current_context() {
    using GetCurrent = CUresult (*)(CUcontext*);
    static GetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetCurrent>(f);
    }();
    CUcontext ctx = nullptr;
    if (!fn || fn(&ctx) != CUDA_SUCCESS) return nullptr;
    return ctx;
}

static pgc_status noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices)
        return fail(PGC_ERR_INVALID_ARG, "device ordinal out of range for the no-alloc scratch");
    CUcontext ctx = current_context();
    if (!g_noalloc_ptr[device] || !ctx || ctx != g_noalloc_ctx[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[device] = static_cast<unsigned char*>(p);
        g_noalloc_ctx[device] = ctx ? ctx : current_context();
    }
    *out = g_noalloc_ptr[device];
    return PGC_OK;
}

// Once work is enqueued on the shared array, every exit waits for it, so that
// the next call (which may use another stream) never overlaps it.
struct DrainOnExit {
    cudaStream_t stream;
    bool armed = false;
    ~DrainOnExit() {
        if (armed) cudaStreamSynchronize(stream);
    }
};

static pgc_status color_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                uint64_t seed, int32_t* colors, int32_t* rounds,
                                int32_t* num_colors, uint32_t flags, void* stream_v) {
    if (!rounds || !num_colors) return fail(PGC_ERR_INVALID_ARG, "rounds/num_colors must be non-NULL");
    if (n < 0) return fail(PGC_ERR_INVALID_ARG, "n < 0");
    *rounds = 0;
    *num_colors = 0;
    if (n > kNoAllocMaxN)
        return fail(PGC_ERR_INVALID_ARG, "pgc_color_d1_noalloc: n exceeds the maximum of 32768 "
                                         "vertices; use pgc_color_d1");
    if (n == 0) return PGC_OK;
    if (!row_ptr || !colors) return fail(PGC_ERR_INVALID_ARG, "NULL array");
    if (is_host_pointer(row_ptr) || is_host_pointer(colors) ||
        (col_idx && is_host_pointer(col_idx)))
        return fail(PGC_ERR_INVALID_ARG, "pgc_color_d1_noalloc takes device memory only");
    cudaStream_t stream = (cudaStream_t)stream_v;
    int device = 0;
    PGC_CUDA(cudaGetDevice(&device));
    int sms = 0;
    PGC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned char* base = nullptr;
    if (pgc_status s = noalloc_scratch(device, &base)) return s;

    int nnz = 0;   // pageable read: no pinned staging buffer is allocated
    PGC_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, 4, cudaMemcpyDeviceToHost, stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    if (nnz < 0) return fail(PGC_ERR_INVALID_ARG, "row_ptr[n] < 0");
    if (nnz > kNoAllocMaxNnz)
        return fail(PGC_ERR_INVALID_ARG, "pgc_color_d1_noalloc: more than 524288 adjacency "
                                         "entries; use pgc_color_d1");
    if (nnz > 0 && !col_idx) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx");

    using L = NoAllocLayout;
    const size_t nn = (size_t)n;
    Problem<SingleView> hp;
    std::memset(&hp, 0, sizeof hp);
    hp.g = SingleView{row_ptr, col_idx};
    hp.col = colors;
    hp.deg = reinterpret_cast<int*>(base + L::deg);
    hp.hlen = reinterpret_cast<int*>(base + L::hlen);
    hp.hadj = reinterpret_cast<int*>(base + L::hadj);
    hp.bm0 = reinterpret_cast<unsigned long long*>(base + L::bm0);
    hp.bmx = reinterpret_cast<unsigned*>(base + L::bmx);
    hp.live = reinterpret_cast<unsigned*>(base + L::live);
    int4* lists = reinterpret_cast<int4*>(base + L::lists);
    for (int p = 0; p < 2; ++p) {
        hp.ws[p] = lists + (size_t)(0 + p) * nn;
        hp.wm[p] = lists + (size_t)(2 + p) * nn;
        hp.wl[p] = lists + (size_t)(4 + p) * nn;
    }
    hp.items = reinterpret_cast<int2*>(base + L::items);
    hp.push_q = reinterpret_cast<int2*>(base + L::pushq);
    hp.trace_w = hp.trace_s = hp.trace_h = reinterpret_cast<long long*>(base + L::trace);
    hp.trace_cap = 0;
    hp.st = reinterpret_cast<State*>(base + L::state);
    hp.seed = seed;
    hp.timeout_ns = 60000ull * 1000000ull;
    hp.nnz = nnz;
    hp.n = n;
    hp.use_deg = (flags & PGC_NO_DEGREE_RULE) ? 0 : 1;
    hp.max_rounds = n + 1;
    const Opts defaults;
    hp.det_s = defaults.mid_degree;
    hp.det_m = defaults.hub_degree;
    hp.tail_w = 0;
    hp.bar_polls = 1u << 22;
    hp.slow_block = -1;
    auto* dP = reinterpret_cast<Problem<SingleView>*>(base + L::problem);
    DrainOnExit drain{stream};
    drain.armed = true;
    PGC_CUDA(cudaMemcpyAsync(dP, &hp, sizeof hp, cudaMemcpyHostToDevice, stream));
    // The array keeps the previous call's contents: the round state must
    // start at zero; every other buffer is written before it is read.
    PGC_CUDA(cudaMemsetAsync(hp.st, 0, sizeof(State), stream));

    const int block = 256;
    const int grid = sms * 4;
    const size_t smem = (size_t)(block / 32) * 2 * kAppend4Slots * sizeof(int4);
    const cudaGraphConditionalHandle none = 0;
    d1_classify<SingleView><<<grid, block, smem, stream>>>(dP);
    d1_build<SingleView><<<grid, block, 0, stream>>>(dP, 0, INT32_MAX);
    d1_tier<SingleView><<<grid, block, smem, stream>>>(dP);
    PGC_CUDA(cudaGetLastError());
    State hs;
    for (int round = 1;; ++round) {
        if (round > 1) d1_assign<SingleView><<<grid, block, 0, stream>>>(dP, none, 0);
        d1_detect<SingleView><<<grid, block, smem, stream>>>(dP, none, 0);
        d1_push<SingleView><<<grid, block, 0, stream>>>(dP);
        PGC_CUDA(cudaGetLastError());
        PGC_CUDA(cudaMemcpyAsync(&hs, hp.st, sizeof hs, cudaMemcpyDeviceToHost, stream));
        PGC_CUDA(cudaStreamSynchronize(stream));
        if (hs.done) break;
        if (round > n + 2) return fail(PGC_ERR_CUDA, "device round control did not finish the loop");
    }
    *rounds = hs.round;
    *num_colors = hs.max_color;
    switch (hs.status) {
        case ST_OK: return PGC_OK;
        case ST_NO_PROGRESS:
            return fail(PGC_ERR_NO_CONVERGE, "a round committed no vertex (input not symmetric?)");
        case ST_MAX_ROUNDS: return fail(PGC_ERR_NO_CONVERGE, "max_rounds reached");
        case ST_TIMEOUT: return fail(PGC_ERR_TIMEOUT, "device round loop exceeded 60 s");
        default: return fail(PGC_ERR_CUDA, "unexpected device status");
    }
}

}  // namespace d1
}  // namespace pgc

extern "C" pgc_status pgc_color_d1_noalloc(int32_t n, const int32_t* row_ptr,
                                           const int32_t* col_idx, uint64_t seed,
                                           int32_t* colors, int32_t* rounds, int32_t* num_colors,
                                           uint32_t flags, void* stream) {
    try {
        return pgc::d1::color_noalloc(n, row_ptr, col_idx, seed, colors, rounds, num_colors,
                                      flags, stream);
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    } catch (...) {
        return pgc::fail(PGC_ERR_CUDA, "unknown exception");
    }
}
