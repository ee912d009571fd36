// batch.cu -- pgc_color_d1_batch: many independent graphs in one launch.
//
// The graphs are flattened into one vertex range; ids, degrees and the
// priority hash stay graph-local (d1::BatchView), so each graph's colors,
// rounds and color count are exactly those of coloring it alone.  One CUDA
// graph launch runs the setup and the device-side round loop for all of
// them; per-graph round and color counts are kept with atomics.  An
// optional autotuner (PGC_AUTOTUNE) times a few launch configurations --
// block size and the tier thresholds of detection -- on the first batch of
// a size class and reuses the fastest one afterwards; colors do not depend
// on the choice.
#include "d1_engine.cuh"
#include "tune_cache.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>

namespace pgc {
namespace d1 {

// graph id of every vertex, and per-graph outputs initialised
__global__ void batch_prep(int G, const long long* __restrict__ vtx_off, int* gid,
                           int* g_rounds, int* g_colors) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const long long a = vtx_off[g], b = vtx_off[g + 1];
        for (long long v = a + threadIdx.x; v < b; v += blockDim.x) gid[v] = g;
        if (threadIdx.x == 0) {
            g_rounds[g] = b > a ? 1 : 0;
            g_colors[g] = 0;
        }
    }
}

// PGC_VALIDATE: per graph, local offsets start at 0, do not decrease, end at
// the graph's entry count; then every local id is in [0, n_g).
__global__ void batch_validate(int G, const long long* __restrict__ vtx_off,
                               const long long* __restrict__ nnz_off, const int* __restrict__ rp,
                               const int* __restrict__ ci, int* bad) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const long long a = vtx_off[g], b = vtx_off[g + 1];
        const int ng = (int)(b - a);
        const int* r = rp + a + g;
        const long long e0 = nnz_off[g], m = nnz_off[g + 1] - e0;
        if (b < a || m < 0) {
            atomicOr(bad, 1);
            continue;
        }
        int ok = 1;
        if (threadIdx.x == 0 && (r[0] != 0 || r[ng] != m)) ok = 0;
        for (int v = threadIdx.x; v < ng; v += blockDim.x)
            if (r[v + 1] < r[v]) ok = 0;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(bad, 1);
            continue;
        }
        for (long long e = threadIdx.x; e < m; e += blockDim.x)
            if ((unsigned)ci[e0 + e] >= (unsigned)ng) atomicOr(bad, 2);
    }
}

struct BatchBufs {
    DevBuf gid, vo, no, rp, ci, col, gr, gc, flag;
    HostBuf h;
    void release() {
        for (DevBuf* b : {&gid, &vo, &no, &rp, &ci, &col, &gr, &gc, &flag}) b->release();
        h.release();
    }
};

static BatchBufs& bufs_for(int device) {
    static std::mutex mu;
    static std::unordered_map<int, std::unique_ptr<BatchBufs>> m;
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
    auto e = std::make_unique<BatchBufs>();
    BatchBufs* p = e.get();
    m.emplace(device, std::move(e));
    return *p;
}

// --------------------------------------------------------------------------
// autotuner: candidates, size classes, an in-memory cache mirrored to the
// file named by PGC_TUNE_FILE (lines "key block mid hub")
// --------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::string, Tuned>& tune_cache() {
    static std::map<std::string, Tuned> m;
    static bool loaded = false;
    if (!loaded) {
        loaded = true;
        if (const char* f = std::getenv("PGC_TUNE_FILE")) {
            if (FILE* fp = std::fopen(f, "r")) {
                tune_file_read(fp, m);
                std::fclose(fp);
            }
        }
    }
    return m;
}

static void tune_store(const std::string& key, const Tuned& t) {
    tune_cache()[key] = t;
    if (const char* f = std::getenv("PGC_TUNE_FILE")) {
        if (FILE* fp = std::fopen(f, "a")) {
            tune_file_append(fp, key, t);
            std::fclose(fp);
        }
    }
}

static pgc_status color_batch(int32_t G, const int64_t* vtx_off, const int64_t* nnz_off,
                              const int32_t* row_ptr, const int32_t* col_idx, uint64_t seed,
                              int32_t* colors, int32_t* rounds_per_g, int32_t* ncolors_per_g,
                              int32_t* rounds_total, const pgc_opts* opts, void* stream_v) {
    if (G < 0) return fail(PGC_ERR_INVALID_ARG, "G < 0");
    Opts o;
    if (pgc_status s = read_opts(opts, &o)) return s;
    if (rounds_total) *rounds_total = 0;
    if (G == 0) return PGC_OK;
    if (!vtx_off || !nnz_off || !row_ptr || !colors || !rounds_per_g || !ncolors_per_g)
        return fail(PGC_ERR_INVALID_ARG, "NULL array");
    cudaStream_t stream = (cudaStream_t)stream_v;
    DeviceInfo dev;
    if (pgc_status s = current_device(&dev)) return s;
    Engine<BatchView>* E = engine_for<BatchView>(dev.device);
    std::lock_guard<std::mutex> lk(E->mu);
    E->dev = dev;
    BatchBufs& B = bufs_for(dev.device);

    // offsets to the host (for sizes) and to the device (for the kernels)
    if (pgc_status s = B.h.ensure((size_t)(G + 1) * 16 + 64)) return s;
    long long* h_vo = B.h.as<long long>();
    long long* h_no = h_vo + (G + 1);
    const bool host_vo = is_host_pointer(vtx_off), host_no = is_host_pointer(nnz_off);
    if (host_vo) std::memcpy(h_vo, vtx_off, (size_t)(G + 1) * 8);
    else PGC_CUDA(cudaMemcpyAsync(h_vo, vtx_off, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost, stream));
    if (host_no) std::memcpy(h_no, nnz_off, (size_t)(G + 1) * 8);
    else PGC_CUDA(cudaMemcpyAsync(h_no, nnz_off, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost, stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    const long long N = h_vo[G], NNZ = h_no[G];
    if (h_vo[0] != 0 || h_no[0] != 0 || N < 0 || NNZ < 0)
        return fail(PGC_ERR_INVALID_ARG, "offsets must start at 0");
    for (int g = 0; g < G; ++g)
        if (h_vo[g + 1] < h_vo[g] || h_no[g + 1] < h_no[g])
            return fail(PGC_ERR_INVALID_ARG, "offsets must not decrease");
    if (N >= INT32_MAX) return fail(PGC_ERR_INVALID_ARG, "more than 2^31-1 vertices in a batch");
    if (N == 0) {   // only empty graphs
        for (int32_t* a : {rounds_per_g, ncolors_per_g}) {
            if (is_host_pointer(a)) std::memset(a, 0, (size_t)G * 4);
            else PGC_CUDA(cudaMemsetAsync(a, 0, (size_t)G * 4, stream));
        }
        PGC_CUDA(cudaStreamSynchronize(stream));
        return PGC_OK;
    }
    if (NNZ > 0 && !col_idx) return fail(PGC_ERR_INVALID_ARG, "NULL col_idx");

    auto dev_array = [&](DevBuf& buf, const void* src, size_t bytes, const void** out) {
        if (!is_host_pointer(src)) {
            *out = src;
            return PGC_OK;
        }
        if (pgc_status s = buf.ensure(std::max<size_t>(bytes, 4))) return s;
        if (bytes) {
            cudaError_t e = cudaMemcpyAsync(buf.ptr, src, bytes, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        }
        *out = buf.ptr;
        return PGC_OK;
    };
    const void *d_vo, *d_no, *d_rp, *d_ci = col_idx;
    if (pgc_status s = dev_array(B.vo, vtx_off, (size_t)(G + 1) * 8, &d_vo)) return s;
    if (pgc_status s = dev_array(B.no, nnz_off, (size_t)(G + 1) * 8, &d_no)) return s;
    if (pgc_status s = dev_array(B.rp, row_ptr, (size_t)(N + G) * 4, &d_rp)) return s;
    if (NNZ > 0)
        if (pgc_status s = dev_array(B.ci, col_idx, (size_t)NNZ * 4, &d_ci)) return s;
    const bool host_col = is_host_pointer(colors);
    const bool host_gr = is_host_pointer(rounds_per_g), host_gc = is_host_pointer(ncolors_per_g);
    int* d_col = colors;
    if (host_col) {
        if (pgc_status s = B.col.ensure((size_t)N * 4)) return s;
        d_col = B.col.as<int>();
    }
    int* d_gr = rounds_per_g;
    int* d_gc = ncolors_per_g;
    if (host_gr) {
        if (pgc_status s = B.gr.ensure((size_t)G * 4)) return s;
        d_gr = B.gr.as<int>();
    }
    if (host_gc) {
        if (pgc_status s = B.gc.ensure((size_t)G * 4)) return s;
        d_gc = B.gc.as<int>();
    }
    if (o.flags & PGC_VALIDATE) {
        if (pgc_status s = B.flag.ensure(4)) return s;
        PGC_CUDA(cudaMemsetAsync(B.flag.ptr, 0, 4, stream));
        batch_validate<<<std::min(G, dev.num_sms * 8), 256, 0, stream>>>(
            G, (const long long*)d_vo, (const long long*)d_no, (const int*)d_rp, (const int*)d_ci,
            B.flag.as<int>());
        PGC_CUDA(cudaGetLastError());
        int* hb = (int*)(h_no + G + 1);
        PGC_CUDA(cudaMemcpyAsync(hb, B.flag.ptr, 4, cudaMemcpyDeviceToHost, stream));
        PGC_CUDA(cudaStreamSynchronize(stream));
        if (*hb) return fail(PGC_ERR_INVALID_ARG, (*hb & 1) ? "a graph's row_ptr is malformed"
                                                             : "a column id is out of its graph");
    }
    if (pgc_status s = B.gid.ensure((size_t)N * 4)) return s;
    batch_prep<<<std::min(G, dev.num_sms * 8), 256, 0, stream>>>(G, (const long long*)d_vo,
                                                                 B.gid.as<int>(), d_gr, d_gc);
    PGC_CUDA(cudaGetLastError());
    BatchView view{(const long long*)d_vo, (const long long*)d_no, (const int*)d_rp,
                   (const int*)d_ci, B.gid.as<int>()};

    int rounds = 0, ncolors = 0;
    if (o.flags & PGC_AUTOTUNE) {
        const std::string key = tune_size_class(N, NNZ, G, !(o.flags & PGC_NO_DEGREE_RULE));
        Tuned best{0, 0, 0};
        bool have = false;
        {
            std::lock_guard<std::mutex> tl(g_tune_mu);
            auto it = tune_cache().find(key);
            if (it != tune_cache().end()) {
                best = it->second;
                have = true;
            }
        }
        if (!have) {
            static const Tuned cand[] = {{128, 16, 256},  {256, 16, 256},   {256, 32, 1024},
                                         {512, 32, 1024}, {256, 64, 4096},  {512, 64, 4096},
                                         {256, 64, 16384}, {256, 128, 16384}};
            cudaEvent_t a, b;
            PGC_CUDA(cudaEventCreate(&a));
            PGC_CUDA(cudaEventCreate(&b));
            float best_ms = 1e30f;
            for (const Tuned& c : cand) {
                Opts oc = o;
                oc.block = c.block;
                oc.mid_degree = c.mid;
                oc.hub_degree = c.hub;
                oc.flags &= ~PGC_HOST_LOOP;
                oc.profile = nullptr;
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {   // first run warms buffers and the graph
                    PGC_CUDA(cudaEventRecord(a, stream));
                    if (pgc_status s = E->run(view, (int)N, NNZ, d_col, d_gr, d_gc, seed, oc,
                                              stream, &rounds, &ncolors)) {
                        cudaEventDestroy(a);
                        cudaEventDestroy(b);
                        return s;
                    }
                    PGC_CUDA(cudaEventRecord(b, stream));
                    PGC_CUDA(cudaEventSynchronize(b));
                    PGC_CUDA(cudaEventElapsedTime(&ms, a, b));
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            std::lock_guard<std::mutex> tl(g_tune_mu);
            tune_store(key, best);
        }
        o.block = best.block;
        o.mid_degree = best.mid;
        o.hub_degree = best.hub;
    }
    if (pgc_status s = E->run(view, (int)N, NNZ, d_col, d_gr, d_gc, seed, o, stream, &rounds,
                              &ncolors))
        return s;
    if (rounds_total) *rounds_total = rounds;
    if (host_col)
        PGC_CUDA(cudaMemcpyAsync(colors, d_col, (size_t)N * 4, cudaMemcpyDeviceToHost, stream));
    if (host_gr)
        PGC_CUDA(cudaMemcpyAsync(rounds_per_g, d_gr, (size_t)G * 4, cudaMemcpyDeviceToHost, stream));
    if (host_gc)
        PGC_CUDA(cudaMemcpyAsync(ncolors_per_g, d_gc, (size_t)G * 4, cudaMemcpyDeviceToHost, stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    return PGC_OK;
}

}  // namespace d1
}  // namespace pgc

extern "C" pgc_status pgc_color_d1_batch(int32_t G, const int64_t* vtx_off, const int64_t* nnz_off,
                                         const int32_t* row_ptr, const int32_t* col_idx,
                                         uint64_t seed, int32_t* colors, int32_t* rounds_per_g,
                                         int32_t* ncolors_per_g, int32_t* rounds,
                                         const pgc_opts* opts, void* stream) {
    try {
        return pgc::d1::color_batch(G, vtx_off, nnz_off, row_ptr, col_idx, seed, colors,
                                    rounds_per_g, ncolors_per_g, rounds, opts, stream);
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    } catch (...) {
        return pgc::fail(PGC_ERR_CUDA, "unknown exception");
    }
}
