// tune_cache.h -- the batch autotuner's saved choices (host only).
//
// pgc_color_d1_batch with PGC_AUTOTUNE times a few launch configurations on
// the first batch of a size class and keeps the fastest.  The choices live
// in memory and, when $PGC_TUNE_FILE names a file, are appended to it as
// lines "key block mid hub" and read back by the next process.  A line
// that does not parse, or whose configuration fails the checks that
// pgc_opts values get, is skipped, so a damaged file can cost tuning time
// but never a bad launch.  Plain C++ (no CUDA), so the host-side tests
// compile it on its own.
#pragma once
#include <cmath>
#include <cstdio>
#include <map>
#include <string>

namespace pgc {
namespace d1 {

struct Tuned {
    int block, mid, hub;   // threads per block, warp-tier and block-tier list lengths
};

// Same limits as pgc_opts: block a multiple of 32 in [128, 1024], tier
// thresholds positive and ordered.
inline bool tuned_valid(const Tuned& t) {
    return t.block >= 128 && t.block <= 1024 && t.block % 32 == 0 && t.mid >= 1 &&
           t.hub >= t.mid;
}

// Reads every valid "key block mid hub" line of fp into m (later lines win).
inline void tune_file_read(std::FILE* fp, std::map<std::string, Tuned>& m) {
    char line[256];
    while (std::fgets(line, sizeof line, fp)) {
        char key[128];
        Tuned t;
        char extra;
        if (std::sscanf(line, "%127s %d %d %d %c", key, &t.block, &t.mid, &t.hub, &extra) == 4 &&
            tuned_valid(t))
            m[key] = t;
    }
}

inline void tune_file_append(std::FILE* fp, const std::string& key, const Tuned& t) {
    std::fprintf(fp, "%s %d %d %d\n", key.c_str(), t.block, t.mid, t.hub);
}

// Size class: log2 (rounded) of the vertex count, of the mean degree and of
// the graph count, plus the priority rule (it changes the detection lists).
inline std::string tune_size_class(long long n, long long nnz, int G, bool use_deg) {
    auto lg = [](double x) { return x <= 1 ? 0 : (int)std::lround(std::log2(x)); };
    char buf[96];
    std::snprintf(buf, sizeof buf, "d1b:n%d:d%d:g%d:r%d", lg((double)n),
                  lg((double)nnz / (double)(n > 1 ? n : 1)), lg((double)G), use_deg ? 1 : 0);
    return buf;
}

}  // namespace d1
}  // namespace pgc
