// d1.cu -- pgc_color_d1: distance-1 coloring of one graph (Sec. 3.2-3.3).
// The engine (kernels and device-side round loop) is in d1_engine.cuh; this
// file adds argument checks, host-buffer staging and optional validation
// (validate.cu).
#include "d1_engine.cuh"

namespace pgc {
namespace d1 {

// Staging buffers for host-memory arguments (per device).
struct Staging {
    DevBuf rp, ci, col, flag;
    void release() {
        for (DevBuf* b : {&rp, &ci, &col, &flag}) b->release();
    }
};

static Staging& staging_for(int device) {
    static std::mutex mu;
    static std::unordered_map<int, std::unique_ptr<Staging>> m;
    std::lock_guard<std::mutex> lk(mu);
    auto it = m.find(device);
    if (it != m.end()) return *it->second;
    if (m.empty()) {
        release_hooks().push_back([] {
            std::lock_guard<std::mutex> lk2(mu);
            int cur = 0;
            cudaGetDevice(&cur);
            auto f = m.find(cur);
            if (f != m.end()) f->second->release();
        });
    }
    auto e = std::make_unique<Staging>();
    Staging* p = e.get();
    m.emplace(device, std::move(e));
    return *p;
}

constexpr int kOverlapMinEntries = 1 << 24;   // smaller host adjacencies are copied whole

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
    Engine<SingleView>* cx = engine_for<SingleView>(dev.device);
    std::lock_guard<std::mutex> lk(cx->mu);
    cx->dev = dev;
    Staging& stg = staging_for(dev.device);

    const bool host_rp = is_host_pointer(row_ptr);
    const bool host_ci = col_idx ? is_host_pointer(col_idx) : host_rp;
    const bool host_col = is_host_pointer(colors);
    const int* d_rp = row_ptr;
    const int* d_ci = col_idx;
    int* d_col = colors;
    int nnz = 0;
    bool overlap = false;
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
            if (pgc_status s = stg.rp.ensure((size_t)(n + 1) * 4)) return s;
            PGC_CUDA(cudaMemcpyAsync(stg.rp.ptr, row_ptr, (size_t)(n + 1) * 4,
                                     cudaMemcpyHostToDevice, stream));
            d_rp = stg.rp.as<int>();
        }
        if (host_ci && nnz > 0) {
            if (pgc_status s = stg.ci.ensure((size_t)nnz * 4)) return s;
            // a large host adjacency is uploaded by the engine in row ranges
            // that overlap the list build (device-side round loop only);
            // otherwise it is copied before the coloring starts
            overlap = host_rp && nnz >= kOverlapMinEntries &&
                      !(o.flags & (PGC_VALIDATE | PGC_HOST_LOOP));
            if (!overlap)
                PGC_CUDA(cudaMemcpyAsync(stg.ci.ptr, col_idx, (size_t)nnz * 4,
                                         cudaMemcpyHostToDevice, stream));
            d_ci = stg.ci.as<int>();
        }
    }
    if (host_col) {
        if (pgc_status s = stg.col.ensure((size_t)n * 4)) return s;
        d_col = stg.col.as<int>();
    }
    if (o.flags & PGC_VALIDATE) {
        if (nnz > 0 && !d_ci) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx with row_ptr[n] > 0");
        if (pgc_status s = validate::symmetric_csr(d_rp, d_ci, n, cx->dev, stream)) return s;
    }
    SingleView view{d_rp, d_ci};
    const Upload up{col_idx, row_ptr, stg.ci.as<int>()};
    pgc_status s = cx->run(view, n, nnz, d_col, nullptr, nullptr, seed, o, stream, rounds,
                           num_colors, overlap ? &up : nullptr);
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
