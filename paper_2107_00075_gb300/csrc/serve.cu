// serve.cu -- a coloring server with continuous batching.
//
// Requests (distance-1 graphs or partial distance-2 patterns) are queued by
// any host thread and admitted by one engine thread, first come first
// served, when two things are free: an execution slot and room for the
// request's whole device footprint (inputs, colors and scratch) in the
// server's HBM arena.  Each admitted request gets its own CUDA stream and
// runs the device-side round loop (one CUDA graph per slot), so the rounds of
// all active requests overlap on the GPU, and requests that arrive while
// others run are admitted as soon as a slot and memory free up.  Its CSR and
// color state stay on the device for all rounds; only the input upload and
// the color download cross the bus.  Colors are the same as those of
// pgc_color_d1 / pgc_color_pd2 on the request alone: every request is
// computed by its own instance of the same engine, with graph-local state.
#include "d1_engine.cuh"
#include "arena.h"

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

namespace pgc {
namespace serve {

static long long now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

enum Kind { KIND_D1 = 1, KIND_PD2 = 3 };

// PD2 requests first run with masks for colors 1..128; a request that needs
// more is re-queued at the head with the window count of its exact color
// bound (the run is deterministic, so the retry gives the same colors).
constexpr int kFirstWindows = 2;

struct Request {
    long long id = 0;
    int kind = KIND_D1;
    int n = 0, n_rows = 0, n_cols = 0;   // n = colored vertices
    long long nnz = 0;
    const int *rp = nullptr, *ci = nullptr, *cp = nullptr, *ri = nullptr;
    int* out = nullptr;
    bool out_on_device = false;   // device memory: copied device to device
    bool out_pinned = false;      // pinned host memory: copied directly
    uint64_t seed = 1;
    int windows = 1;
    size_t bytes = 0, off = 0;
    int slot = -1;
    bool done = false;
    pgc_status status = PGC_OK;
    int rounds = 0, num_colors = 0;
    long long t_submit = 0, t_admit = 0, t_done = 0;
};

// max over columns v of sum over v's rows of (row length - 1): a first-fit
// color never exceeds this + 1.
static int pd2_windows(const Request& r) {
    long long bound = 0;
    for (int v = 0; v < r.n_cols; ++v) {
        long long b = 0;
        for (int e = r.cp[v]; e < r.cp[v + 1]; ++e) {
            const int row = r.ri[e];
            b += r.rp[row + 1] - r.rp[row] - 1;
        }
        bound = std::max(bound, b);
    }
    return (int)std::max<long long>(1, std::min<long long>(64, (bound + 1 + 63) / 64));
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    d1::Engine<d1::SingleView> d1e;
    void* nete = nullptr;
    HostBuf colors;   // pinned staging for host outputs
    Request* req = nullptr;
};

struct Server {
    int device = 0;
    size_t budget = 0;
    DevBuf arena_mem;
    Arena arena;
    std::vector<std::unique_ptr<Slot>> slots;
    std::deque<Request*> queue;
    std::map<long long, Request*> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread engine;
    bool stop = false;
    long long next_id = 1;
    long long submitted = 0, completed = 0, rejected = 0;
    size_t peak_bytes = 0;
    int max_active_seen = 0, active = 0;
    std::string engine_error;
};

// Device bytes a request needs while it is active.
static size_t footprint(const Request& r) {
    if (r.kind == KIND_D1) {
        return al((size_t)(r.n + 1) * 4) + al((size_t)std::max<long long>(r.nnz, 1) * 4) +
               al((size_t)r.n * 4) + d1::scratch_sizes(r.n, r.nnz).total();
    }
    return al((size_t)(r.n_rows + 1) * 4) + al((size_t)(r.n_cols + 1) * 4) +
           2 * al((size_t)std::max<long long>(r.nnz, 1) * 4) + al((size_t)r.n_cols * 4) +
           net::scratch_bytes(r.n_cols, r.n_rows, r.windows);
}

// Uploads the request into its arena block and enqueues the coloring.
static pgc_status start(Server& S, Slot& sl, Request& r) {
    char* base = static_cast<char*>(S.arena_mem.ptr) + r.off;
    char* p = base;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += al(bytes);
        return q;
    };
    cudaStream_t st = sl.stream;
    int* d_col;
    if (r.kind == KIND_D1) {
        int* d_rp = reinterpret_cast<int*>(take((size_t)(r.n + 1) * 4));
        int* d_ci = reinterpret_cast<int*>(take((size_t)std::max<long long>(r.nnz, 1) * 4));
        d_col = reinterpret_cast<int*>(take((size_t)r.n * 4));
        PGC_CUDA(cudaMemcpyAsync(d_rp, r.rp, (size_t)(r.n + 1) * 4, cudaMemcpyDefault, st));
        if (r.nnz)
            PGC_CUDA(cudaMemcpyAsync(d_ci, r.ci, (size_t)r.nnz * 4, cudaMemcpyDefault, st));
        d1::Scratch sc = d1::carve_scratch(p, r.n, r.nnz);
        Opts o;
        if (pgc_status s = sl.d1e.launch(sc, d1::SingleView{d_rp, d_ci}, r.n, r.nnz, d_col,
                                         nullptr, nullptr, r.seed, o, st))
            return s;
    } else {
        int* d_rp = reinterpret_cast<int*>(take((size_t)(r.n_rows + 1) * 4));
        int* d_cp = reinterpret_cast<int*>(take((size_t)(r.n_cols + 1) * 4));
        int* d_ci = reinterpret_cast<int*>(take((size_t)std::max<long long>(r.nnz, 1) * 4));
        int* d_ri = reinterpret_cast<int*>(take((size_t)std::max<long long>(r.nnz, 1) * 4));
        d_col = reinterpret_cast<int*>(take((size_t)r.n_cols * 4));
        PGC_CUDA(cudaMemcpyAsync(d_rp, r.rp, (size_t)(r.n_rows + 1) * 4, cudaMemcpyDefault, st));
        PGC_CUDA(cudaMemcpyAsync(d_cp, r.cp, (size_t)(r.n_cols + 1) * 4, cudaMemcpyDefault, st));
        if (r.nnz) {
            PGC_CUDA(cudaMemcpyAsync(d_ci, r.ci, (size_t)r.nnz * 4, cudaMemcpyDefault, st));
            PGC_CUDA(cudaMemcpyAsync(d_ri, r.ri, (size_t)r.nnz * 4, cudaMemcpyDefault, st));
        }
        if (!sl.nete) sl.nete = net::slot_create();
        if (pgc_status s = net::slot_launch_pd2(sl.nete, p, r.n_rows, r.n_cols, d_rp, d_ci, d_cp,
                                                d_ri, d_col, r.windows, r.seed, st))
            return s;
    }
    if (r.out_on_device || r.out_pinned) {
        PGC_CUDA(cudaMemcpyAsync(r.out, d_col, (size_t)r.n * 4, cudaMemcpyDefault, st));
    } else {
        if (pgc_status s = sl.colors.ensure((size_t)r.n * 4)) return s;
        PGC_CUDA(cudaMemcpyAsync(sl.colors.ptr, d_col, (size_t)r.n * 4, cudaMemcpyDeviceToHost, st));
    }
    PGC_CUDA(cudaEventRecord(sl.done, st));
    return PGC_OK;
}

static void complete(Server& S, Slot& sl, pgc_status launch_status) {
    Request& r = *sl.req;
    pgc_status s = launch_status;
    if (s == PGC_OK) {
        const cudaError_t e = cudaEventSynchronize(sl.done);
        if (e != cudaSuccess) s = cuda_fail(e, "request stream");
    }
    if (s == PGC_OK) {
        s = r.kind == KIND_D1 ? sl.d1e.finish(Opts(), &r.rounds, &r.num_colors)
                              : net::slot_finish(sl.nete, &r.rounds, &r.num_colors);
    }
    if (s == PGC_ERR_NO_CONVERGE && r.kind == KIND_PD2 && r.windows == kFirstWindows &&
        net::slot_overflowed(sl.nete)) {
        // more than 128 colors: retry with masks sized by the exact bound
        const int w = pd2_windows(r);
        std::lock_guard<std::mutex> lk(S.mu);
        S.arena.release(r.off, r.bytes);
        sl.req = nullptr;
        S.active -= 1;
        r.windows = std::max(w, kFirstWindows + 1);
        r.bytes = footprint(r);
        if (r.bytes > S.budget) {
            r.status = fail(PGC_ERR_BUSY, "request footprint exceeds the server's HBM budget");
            r.done = true;
            r.t_done = now_ns();
            S.completed += 1;
            S.cv_done.notify_all();
        } else {
            S.queue.push_front(&r);
        }
        return;
    }
    if (s == PGC_OK && !r.out_on_device && !r.out_pinned)
        std::memcpy(r.out, sl.colors.ptr, (size_t)r.n * 4);
    std::lock_guard<std::mutex> lk(S.mu);
    r.status = s;
    r.done = true;
    r.t_done = now_ns();
    S.arena.release(r.off, r.bytes);
    sl.req = nullptr;
    S.active -= 1;
    S.completed += 1;
    S.cv_done.notify_all();
}

static void engine_loop(Server* Sp) {
    Server& S = *Sp;
    cudaSetDevice(S.device);
    for (;;) {
        bool progressed = false;
        // completions
        for (auto& slp : S.slots) {
            Slot& sl = *slp;
            Request* r;
            {
                std::lock_guard<std::mutex> lk(S.mu);
                r = sl.req;
            }
            if (!r) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            complete(S, sl, PGC_OK);
            progressed = true;
        }
        // admission, first come first served, at this step boundary
        for (;;) {
            Slot* free_slot = nullptr;
            Request* r = nullptr;
            {
                std::unique_lock<std::mutex> lk(S.mu);
                if (S.queue.empty()) break;
                int idx = 0;
                for (auto& slp : S.slots) {
                    if (!slp->req) {
                        free_slot = slp.get();
                        break;
                    }
                    ++idx;
                }
                if (!free_slot) break;
                r = S.queue.front();
                if (!S.arena.alloc(r->bytes, &r->off)) break;   // wait for memory
                S.queue.pop_front();
                free_slot->req = r;
                r->slot = idx;
                r->t_admit = now_ns();
                S.active += 1;
                S.max_active_seen = std::max(S.max_active_seen, S.active);
                S.peak_bytes = std::max(S.peak_bytes, S.arena.used());
            }
            const pgc_status s = start(S, *free_slot, *r);
            if (s != PGC_OK) {
                cudaStreamSynchronize(free_slot->stream);
                complete(S, *free_slot, s);
            }
            progressed = true;
        }
        std::unique_lock<std::mutex> lk(S.mu);
        if (S.stop && S.queue.empty() && S.active == 0) return;
        if (!progressed) {
            if (S.active == 0 && S.queue.empty())
                S.cv_work.wait(lk, [&] { return S.stop || !S.queue.empty(); });
            else
                S.cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

static pgc_status submit(Server* S, Request* r, long long* req_id) {
    r->bytes = footprint(*r);
    r->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
        delete r;
        return fail(PGC_ERR_INVALID_ARG, "server is shutting down");
    }
    if (r->bytes > S->budget) {
        S->rejected += 1;
        delete r;
        return fail(PGC_ERR_BUSY, "request footprint exceeds the server's HBM budget");
    }
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    S->submitted += 1;
    *req_id = r->id;
    S->cv_work.notify_one();
    return PGC_OK;
}

static void classify_output(Request* r, int* colors) {
    r->out = colors;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, colors) != cudaSuccess) {
        cudaGetLastError();
        a.type = cudaMemoryTypeUnregistered;
    }
    r->out_on_device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    r->out_pinned = a.type == cudaMemoryTypeHost;
}

static void fill_info(const Request& r, pgc_request_info* info) {
    if (!info) return;
    info->status = r.status;
    info->rounds = r.rounds;
    info->num_colors = r.num_colors;
    info->t_submit_ns = r.t_submit;
    info->t_admit_ns = r.t_admit;
    info->t_done_ns = r.t_done;
    info->footprint_bytes = (int64_t)r.bytes;
}

}  // namespace serve
}  // namespace pgc

using pgc::serve::Request;
using pgc::serve::Server;

struct pgc_server {
    Server impl;
};

extern "C" {

pgc_status pgc_server_create(size_t hbm_budget_bytes, int32_t max_active, pgc_server** out) {
    if (!out) return pgc::fail(PGC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_active < 1 || max_active > 256)
        return pgc::fail(PGC_ERR_INVALID_ARG, "max_active must be in [1, 256]");
    if (hbm_budget_bytes < 4096) return pgc::fail(PGC_ERR_INVALID_ARG, "budget too small");
    try {
        auto* srv = new pgc_server();
        Server& S = srv->impl;
        if (cudaGetDevice(&S.device) != cudaSuccess) {
            delete srv;
            return pgc::fail(PGC_ERR_CUDA, "no current device");
        }
        S.budget = hbm_budget_bytes;
        if (pgc_status s = S.arena_mem.ensure(hbm_budget_bytes)) {
            delete srv;
            return s;
        }
        S.arena.init(hbm_budget_bytes);
        for (int i = 0; i < max_active; ++i) S.slots.push_back(std::make_unique<pgc::serve::Slot>());
        for (auto& slp : S.slots) {
            auto& sl = *slp;
            cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
            sl.d1e.dev.device = S.device;
            cudaDeviceGetAttribute(&sl.d1e.dev.num_sms, cudaDevAttrMultiProcessorCount, S.device);
        }
        S.engine = std::thread(pgc::serve::engine_loop, &S);
        *out = srv;
        return PGC_OK;
    } catch (const std::exception& e) {
        return pgc::fail(PGC_ERR_CUDA, e.what());
    }
}

pgc_status pgc_server_submit_d1(pgc_server* srv, int32_t n, const int32_t* row_ptr,
                                const int32_t* col_idx, uint64_t seed, int32_t* colors,
                                int64_t* req_id) {
    if (!srv || !req_id || n < 1 || !row_ptr || !colors)
        return pgc::fail(PGC_ERR_INVALID_ARG, "bad server request");
    const bool host_rp = pgc::is_host_pointer(row_ptr);
    long long nnz = 0;
    if (host_rp) {
        nnz = row_ptr[n];
    } else {
        int v = 0;
        if (cudaMemcpy(&v, row_ptr + n, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return pgc::fail(PGC_ERR_INVALID_ARG, "row_ptr not readable");
        nnz = v;
    }
    if (nnz < 0 || (nnz > 0 && !col_idx)) return pgc::fail(PGC_ERR_INVALID_ARG, "bad CSR");
    auto* r = new Request();
    r->kind = pgc::serve::KIND_D1;
    r->n = n;
    r->nnz = nnz;
    r->rp = row_ptr;
    r->ci = col_idx;
    pgc::serve::classify_output(r, colors);
    r->seed = seed;
    long long id = 0;
    pgc_status s = pgc::serve::submit(&srv->impl, r, &id);
    *req_id = id;
    return s;
}

pgc_status pgc_server_submit_pd2(pgc_server* srv, int32_t n_rows, int32_t n_cols,
                                 const int32_t* row_ptr, const int32_t* col_idx,
                                 const int32_t* col_ptr, const int32_t* row_idx, uint64_t seed,
                                 int32_t* colors, int64_t* req_id) {
    if (!srv || !req_id || n_rows < 0 || n_cols < 1 || !row_ptr || !col_ptr || !colors)
        return pgc::fail(PGC_ERR_INVALID_ARG, "bad server request");
    if (!pgc::is_host_pointer(row_ptr) || !pgc::is_host_pointer(col_ptr) ||
        !pgc::is_host_pointer(col_idx) || !pgc::is_host_pointer(row_idx))
        return pgc::fail(PGC_ERR_INVALID_ARG, "server PD2 inputs must be host memory");
    const long long nnz = row_ptr[n_rows];
    if (nnz != col_ptr[n_cols] || nnz < 0) return pgc::fail(PGC_ERR_INVALID_ARG, "CSR/CSC mismatch");
    auto* r = new Request();
    r->kind = pgc::serve::KIND_PD2;
    r->n = n_cols;
    r->n_rows = n_rows;
    r->n_cols = n_cols;
    r->nnz = nnz;
    r->rp = row_ptr;
    r->ci = col_idx;
    r->cp = col_ptr;
    r->ri = row_idx;
    pgc::serve::classify_output(r, colors);
    r->seed = seed;
    r->windows = pgc::serve::kFirstWindows;
    long long id = 0;
    pgc_status s = pgc::serve::submit(&srv->impl, r, &id);
    *req_id = id;
    return s;
}

pgc_status pgc_server_poll(pgc_server* srv, int64_t req_id, int32_t* done,
                           pgc_request_info* info) {
    if (!srv || !done) return pgc::fail(PGC_ERR_INVALID_ARG, "NULL argument");
    Server& S = srv->impl;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(req_id);
    if (it == S.reqs.end()) return pgc::fail(PGC_ERR_NOT_FOUND, "unknown request id");
    Request* r = it->second;
    *done = r->done ? 1 : 0;
    if (r->done) {
        pgc::serve::fill_info(*r, info);
        const pgc_status s = r->status;
        S.reqs.erase(it);
        delete r;
        return s;
    }
    return PGC_OK;
}

pgc_status pgc_server_wait(pgc_server* srv, int64_t req_id, int32_t timeout_ms,
                           pgc_request_info* info) {
    if (!srv) return pgc::fail(PGC_ERR_INVALID_ARG, "NULL server");
    Server& S = srv->impl;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(req_id);
    if (it == S.reqs.end()) return pgc::fail(PGC_ERR_NOT_FOUND, "unknown request id");
    Request* r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) S.cv_done.wait(lk, pred);
    else if (!S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return pgc::fail(PGC_ERR_TIMEOUT, "request not finished within timeout_ms");
    pgc::serve::fill_info(*r, info);
    const pgc_status s = r->status;
    S.reqs.erase(req_id);
    delete r;
    if (s != PGC_OK) return pgc::fail(s, "request failed");
    return PGC_OK;
}

pgc_status pgc_server_stats(pgc_server* srv, pgc_server_counters* out) {
    if (!srv || !out) return pgc::fail(PGC_ERR_INVALID_ARG, "NULL argument");
    Server& S = srv->impl;
    std::lock_guard<std::mutex> lk(S.mu);
    out->submitted = S.submitted;
    out->completed = S.completed;
    out->rejected = S.rejected;
    out->active = S.active;
    out->queued = (int32_t)S.queue.size();
    out->bytes_in_use = (int64_t)S.arena.used();
    out->peak_bytes = (int64_t)S.peak_bytes;
    out->budget_bytes = (int64_t)S.budget;
    out->max_active_seen = S.max_active_seen;
    return PGC_OK;
}

pgc_status pgc_server_destroy(pgc_server* srv) {
    if (!srv) return PGC_OK;
    Server& S = srv->impl;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
        S.cv_work.notify_all();
    }
    if (S.engine.joinable()) S.engine.join();
    for (auto& kv : S.reqs) delete kv.second;
    S.reqs.clear();
    for (auto& slp : S.slots) {
        auto& sl = *slp;
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        sl.d1e.release();
        if (sl.nete) pgc::net::slot_destroy(sl.nete);
        sl.colors.release();
    }
    S.arena_mem.release();
    delete srv;
    return PGC_OK;
}

}  // extern "C"
