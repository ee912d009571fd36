// validate.cu -- input checks behind PGC_VALIDATE.
//
// The coloring assumes (Sec. 2.1) an undirected graph given as a symmetric
// CSR (D1, D2) or one pattern given twice, as CSR and as CSC (PD2).  These
// kernels check that before any coloring work is launched:
//   * offsets start at 0 and never decrease; every id is in range;
//   * symmetry: the multiset of entries (v, u) equals the multiset of
//     (u, v); CSR/CSC: the multiset of (row, column) pairs read from the
//     CSR equals the one read from the CSC.
// Multiset equality is tested by comparing two sums of a 64-bit mix of
// each pair (one sum per side): equal multisets always give equal sums; an
// unequal pair of sums proves a mismatch, and a mismatch goes unnoticed only
// if the two sums collide by chance.  When every row is sorted, each entry is
// also looked up by binary search in the other side (an exact existence
// check that needs no hashing).
#include "runtime.h"
#include "device_common.cuh"

#include <functional>
#include <memory>
#include <unordered_map>

namespace pgc {
std::vector<std::function<void()>>& release_hooks();

namespace validate {

enum : int { BAD_OFFSETS = 1, BAD_IDS = 2, UNSORTED = 4, MISSING = 8 };

struct Words {
    int flags;
    int pad;
    unsigned long long sum_a;   // mix of (row, col) over the first array
    unsigned long long sum_b;   // mix of (row, col) over the second array
};

// MurmurHash3's 64-bit finaliser (Appleby) applied to the ordered pair.
__device__ __forceinline__ unsigned long long pair_mix(unsigned r, unsigned c) {
    unsigned long long k = ((unsigned long long)r << 32 | c) ^ 0x5bd1e9955bd1e995ull;
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__global__ void check_offsets(const int* __restrict__ p, int n, int* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (p[v + 1] < p[v]) atomicOr(flags, BAD_OFFSETS);
    if (blockIdx.x == 0 && threadIdx.x == 0 && p[0] != 0) atomicOr(flags, BAD_OFFSETS);
}

// Ids in [0, bound); rows sorted (non-decreasing).  Launched only after the
// offsets passed, so every e < p[n] is inside idx.
__global__ void check_ids(const int* __restrict__ p, const int* __restrict__ idx, int n,
                          int bound, int* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int prev = -1;
        for (int e = p[v]; e < p[v + 1]; ++e) {
            const int u = idx[e];
            if ((unsigned)u >= (unsigned)bound) atomicOr(flags, BAD_IDS);
            if (u < prev) atomicOr(flags, UNSORTED);
            prev = u;
        }
    }
}

// Adds pair_mix(v, u) (swap = false) or pair_mix(u, v) (swap = true) over
// every entry u of row v into *sum.
__global__ void pair_sum(const int* __restrict__ p, const int* __restrict__ idx, int n, bool swap,
                         unsigned long long* sum) {
    unsigned long long acc = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        for (int e = p[v]; e < p[v + 1]; ++e) {
            const unsigned u = (unsigned)idx[e];
            acc += swap ? pair_mix(u, (unsigned)v) : pair_mix((unsigned)v, u);
        }
    acc = warp_sum(acc);
    if (lane_id() == 0 && acc) atomicAdd(sum, acc);
}

// Sorted rows only: every entry u of row v of (p, idx) must find v in row u
// of (q, jdx).
__global__ void find_reverse(const int* __restrict__ p, const int* __restrict__ idx, int n,
                             const int* __restrict__ q, const int* __restrict__ jdx, int* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        for (int e = p[v]; e < p[v + 1]; ++e) {
            const int u = idx[e];
            int lo = q[u], hi = q[u + 1];
            while (lo < hi) {
                const int mid = lo + (hi - lo) / 2;
                if (jdx[mid] < (int)v) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= q[u + 1] || jdx[lo] != (int)v) atomicOr(flags, MISSING);
        }
}

struct Buffers {
    DevBuf words;
    HostBuf host;
};

static Buffers& buffers_for(int device) {
    static std::mutex mu;
    static std::unordered_map<int, std::unique_ptr<Buffers>> m;
    std::lock_guard<std::mutex> lk(mu);
    auto it = m.find(device);
    if (it != m.end()) return *it->second;
    if (m.empty()) {
        release_hooks().push_back([] {
            std::lock_guard<std::mutex> lk2(mu);
            int cur = 0;
            cudaGetDevice(&cur);
            auto f = m.find(cur);
            if (f != m.end()) {
                f->second->words.release();
                f->second->host.release();
            }
        });
    }
    auto b = std::make_unique<Buffers>();
    Buffers* p = b.get();
    m.emplace(device, std::move(b));
    return *p;
}

static pgc_status read_words(Buffers& b, cudaStream_t stream, Words* out) {
    PGC_CUDA(cudaMemcpyAsync(b.host.ptr, b.words.ptr, sizeof(Words), cudaMemcpyDeviceToHost,
                             stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    *out = *b.host.as<Words>();
    return PGC_OK;
}

// Offsets, then ids (and sortedness) of one compressed array.
static pgc_status check_array(Buffers& b, const int* p, const int* idx, int n, int bound,
                              const DeviceInfo& dev, cudaStream_t stream, const char* what,
                              bool* sorted) {
    Words w;
    PGC_CUDA(cudaMemsetAsync(b.words.ptr, 0, sizeof(Words), stream));
    check_offsets<<<dev.num_sms * 4, 256, 0, stream>>>(p, n, &b.words.as<Words>()->flags);
    PGC_CUDA(cudaGetLastError());
    if (pgc_status s = read_words(b, stream, &w)) return s;
    if (w.flags & BAD_OFFSETS)
        return fail(PGC_ERR_INVALID_ARG, std::string(what) + ": offsets are not a valid offset array");
    int nnz = 0;
    PGC_CUDA(cudaMemcpyAsync(b.host.ptr, p + n, 4, cudaMemcpyDeviceToHost, stream));
    PGC_CUDA(cudaStreamSynchronize(stream));
    nnz = *b.host.as<int>();
    if (nnz > 0 && !idx) return fail(PGC_ERR_INVALID_ARG, std::string(what) + ": NULL ids");
    if (nnz > 0) {
        check_ids<<<dev.num_sms * 4, 256, 0, stream>>>(p, idx, n, bound,
                                                       &b.words.as<Words>()->flags);
        PGC_CUDA(cudaGetLastError());
        if (pgc_status s = read_words(b, stream, &w)) return s;
        if (w.flags & BAD_IDS)
            return fail(PGC_ERR_INVALID_ARG, std::string(what) + ": an id is out of range");
    }
    *sorted = !(w.flags & UNSORTED);
    return PGC_OK;
}

// Equal pair multisets of (p, idx) read as (row, col) and (q, jdx) read as
// (col, row) (q = p for the symmetry test), plus the exact reverse lookup
// when both are sorted.
static pgc_status check_pairs(Buffers& b, const int* p, const int* idx, int n, const int* q,
                              const int* jdx, int m, bool sorted, const DeviceInfo& dev,
                              cudaStream_t stream, const char* what) {
    Words w;
    PGC_CUDA(cudaMemsetAsync(b.words.ptr, 0, sizeof(Words), stream));
    Words* dw = b.words.as<Words>();
    pair_sum<<<dev.num_sms * 4, 256, 0, stream>>>(p, idx, n, false, &dw->sum_a);
    pair_sum<<<dev.num_sms * 4, 256, 0, stream>>>(q, jdx, m, true, &dw->sum_b);
    if (sorted) find_reverse<<<dev.num_sms * 4, 256, 0, stream>>>(p, idx, n, q, jdx, &dw->flags);
    PGC_CUDA(cudaGetLastError());
    if (pgc_status s = read_words(b, stream, &w)) return s;
    if (w.sum_a != w.sum_b || (w.flags & MISSING)) return fail(PGC_ERR_INVALID_ARG, what);
    return PGC_OK;
}

pgc_status symmetric_csr(const int* rp, const int* ci, int n, const DeviceInfo& dev,
                         cudaStream_t stream) {
    Buffers& b = buffers_for(dev.device);
    if (pgc_status s = b.words.ensure(sizeof(Words))) return s;
    if (pgc_status s = b.host.ensure(sizeof(Words))) return s;
    bool sorted = false;
    if (pgc_status s = check_array(b, rp, ci, n, n, dev, stream, "row_ptr/col_idx", &sorted))
        return s;
    return check_pairs(b, rp, ci, n, rp, ci, n, sorted, dev, stream,
                       "the graph is not symmetric (u in N(v) but v not in N(u))");
}

pgc_status csr_csc_pair(const int* rp, const int* ci, int n_rows, const int* cp, const int* ri,
                        int n_cols, const DeviceInfo& dev, cudaStream_t stream) {
    Buffers& b = buffers_for(dev.device);
    if (pgc_status s = b.words.ensure(sizeof(Words))) return s;
    if (pgc_status s = b.host.ensure(sizeof(Words))) return s;
    bool s1 = false, s2 = false;
    if (pgc_status s = check_array(b, rp, ci, n_rows, n_cols, dev, stream,
                                   "row_ptr/col_idx (CSR)", &s1))
        return s;
    if (pgc_status s = check_array(b, cp, ri, n_cols, n_rows, dev, stream,
                                   "col_ptr/row_idx (CSC)", &s2))
        return s;
    return check_pairs(b, rp, ci, n_rows, cp, ri, n_cols, s1 && s2, dev, stream,
                       "the CSR and the CSC do not describe the same pattern");
}

}  // namespace validate
}  // namespace pgc
