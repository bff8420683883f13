// tune.cu -- the autotuner and its cache (not in the paper).
//
// Every FP64-EFT tile gives the same, k-sequential result, and every batch
// policy the same C_i, so the choice between them is a matter of speed only
// and is made by measurement.  Choices are remembered per device (name and
// SM count), per precision and per shape bucket (m, n, k each rounded up to
// a power of two) for single products, and per exact list of problem shapes
// for batches.  They live in memory and, when MPGEMM_TUNE_CACHE names a
// file, in that file as JSON: read at the first lookup (or the first after
// mpgemm_tune_cache_reset), rewritten after every new choice through a
// temporary file and a rename.  The file holds one entry per line,
//
//   {
//    "version": 1,
//    "entries": {
//     "NVIDIA GB300/152|gemm:2:7:7:7": {"choice": 7, "ms": 0.0902},
//     "NVIDIA GB300/152|batch:4:512:9f86d081884c7d65": {"choice": 2, "ms": 551.1}
//    }
//   }
//
// and lines that do not parse as an entry are ignored.
#include "mpgemm.h"
#include "internal.h"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

namespace mpg {

namespace {

struct TuneEntry {
    int choice;
    float ms;
};

struct TuneCache {
    std::mutex mu;
    bool loaded = false;
    std::string path;                            // empty: memory only
    std::map<std::string, TuneEntry> entries;
};

TuneCache& cache()
{
    static TuneCache c;
    return c;
}

// "name/SMs" of the current device (looked up once per device), or "none"
// without one.
std::string device_id()
{
    static std::mutex mu;
    static std::string ids[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();                      // no device: nothing sticky left behind
        return "none";
    }
    std::lock_guard<std::mutex> lock(mu);
    if (ids[dev].empty()) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return "none";
        }
        char buf[320];
        std::snprintf(buf, sizeof(buf), "%s/%d", prop.name, prop.multiProcessorCount);
        ids[dev] = buf;
    }
    return ids[dev];
}

// Parses one line `"key": {"choice": N, "ms": X}` (a trailing comma allowed).
bool parse_entry(const char* line, std::string& key, TuneEntry& e)
{
    const char* q0 = std::strchr(line, '"');
    if (!q0) return false;
    const char* q1 = std::strchr(q0 + 1, '"');
    if (!q1) return false;
    const char* rest = q1 + 1;
    int choice = 0;
    float ms = 0.f;
    if (std::sscanf(rest, " : { \"choice\" : %d , \"ms\" : %f }", &choice, &ms) != 2) return false;
    key.assign(q0 + 1, q1);
    e.choice = choice;
    e.ms = ms;
    return true;
}

// With the cache's mutex held.
void load_locked(TuneCache& c)
{
    if (c.loaded) return;
    c.loaded = true;
    const char* p = std::getenv("MPGEMM_TUNE_CACHE");
    c.path = p ? p : "";
    if (c.path.empty()) return;
    FILE* f = std::fopen(c.path.c_str(), "r");
    if (!f) return;                              // no file yet
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        std::string key;
        TuneEntry e;
        if (parse_entry(line, key, e)) c.entries[key] = e;
    }
    std::fclose(f);
}

// With the cache's mutex held.  Failures to write leave the choices in
// memory (a read-only location is not an error).
void save_locked(TuneCache& c)
{
    if (c.path.empty()) return;
    const std::string tmp = c.path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n \"version\": 1,\n \"entries\": {\n");
    size_t i = 0;
    for (const auto& kv : c.entries) {
        std::fprintf(f, "  \"%s\": {\"choice\": %d, \"ms\": %.6g}%s\n", kv.first.c_str(), kv.second.choice,
                     static_cast<double>(kv.second.ms), ++i < c.entries.size() ? "," : "");
    }
    std::fprintf(f, " }\n}\n");
    const bool ok = std::fclose(f) == 0;
    if (ok) std::rename(tmp.c_str(), c.path.c_str());
    else std::remove(tmp.c_str());
}

}  // namespace

int tune_bucket(int64_t x)
{
    int b = 0;
    while (b < 62 && (int64_t{1} << b) < x) ++b;
    return b;
}

void gemm_tune_key(int P, int64_t m, int64_t n, int64_t k, char* out, size_t cap)
{
    std::snprintf(out, cap, "%s|gemm:%d:%d:%d:%d", device_id().c_str(), P, tune_bucket(m), tune_bucket(n),
                  tune_bucket(k));
}

void batch_tune_key(int P, int count, uint64_t shapes_hash, char* out, size_t cap)
{
    std::snprintf(out, cap, "%s|batch:%d:%d:%016llx", device_id().c_str(), P, count,
                  static_cast<unsigned long long>(shapes_hash));
}

bool tune_lookup(const char* key, int* choice, float* ms)
{
    TuneCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    load_locked(c);
    const auto it = c.entries.find(key);
    if (it == c.entries.end()) return false;
    if (choice) *choice = it->second.choice;
    if (ms) *ms = it->second.ms;
    return true;
}

void tune_store(const char* key, int choice, float ms)
{
    TuneCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    load_locked(c);
    c.entries[key] = TuneEntry{choice, ms};
    save_locked(c);
}

// The remembered 0-based tile of (P, m, n, k), or -1.  Without any
// remembered choice this costs a lock and no device query.
int tuned_tile_index(int P, int64_t m, int64_t n, int64_t k, int ntiles)
{
    {
        TuneCache& c = cache();
        std::lock_guard<std::mutex> lock(c.mu);
        load_locked(c);
        if (c.entries.empty()) return -1;
    }
    char key[512];
    gemm_tune_key(P, m, n, k, key, sizeof(key));
    int choice = 0;
    if (!tune_lookup(key, &choice, nullptr)) return -1;
    return choice >= 1 && choice <= ntiles ? choice - 1 : -1;
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_autotune(int P, int64_t m, int64_t n, int64_t k, const double* const* A, int64_t lda,
                    const double* const* B, int64_t ldb, double* const* C, int64_t ldc, int reps, int* best_tile,
                    float* best_ms)
{
    clear_error();
    if (!best_tile) return set_error(MPG_EINVAL, "best_tile must not be NULL");
    const int nt = mpgemm_num_tiles(P);
    if (nt <= 0) return set_error(MPG_EINVAL, "P must be 1, 2, 3 or 4");
    if (reps < 1) reps = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return set_error(MPG_ECUDA, "event creation failed");
    }
    const cudaStream_t s = current_stream();
    float best = 0.f;
    int arg = 0, rc = MPG_OK;
    char why[256] = "";
    for (int t = 1; t <= nt && rc == MPG_OK; ++t) {
        mpgemm_opts o;
        std::memset(&o, 0, sizeof(o));
        o.algo = MPG_ALGO_FP64_EFT;
        o.tile = t;
        rc = mpgemm_ex(P, &o, m, n, k, A, lda, B, ldb, C, ldc);             // warm-up, and the checks
        if (rc == MPG_EINVAL) {                                              // this tile cannot run the call
            std::snprintf(why, sizeof(why), "%s", mpgemm_last_error());
            rc = MPG_OK;
            continue;
        }
        if (rc != MPG_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && rc == MPG_OK; ++r) rc = mpgemm_ex(P, &o, m, n, k, A, lda, B, ldb, C, ldc);
        cudaEventRecord(e1, s);
        if (rc == MPG_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(MPG_ECUDA, "timing failed");
        if (rc == MPG_OK) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= static_cast<float>(reps);
            if (arg == 0 || ms < best) {
                best = ms;
                arg = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MPG_OK) return rc;
    if (arg == 0) {
        char msg[320];
        std::snprintf(msg, sizeof(msg), "no tile can run this call (%s)", why);
        return set_error(MPG_EINVAL, msg);
    }
    clear_error();
    char key[512];
    gemm_tune_key(P, m, n, k, key, sizeof(key));
    tune_store(key, arg, best);
    *best_tile = arg;
    if (best_ms) *best_ms = best;
    return MPG_OK;
}

int mpgemm_tuned_tile(int P, int64_t m, int64_t n, int64_t k)
{
    const int nt = mpgemm_num_tiles(P);
    if (nt <= 0 || m < 0 || n < 0 || k < 0) return 0;
    return tuned_tile_index(P, m, n, k, nt) + 1;
}

void mpgemm_tune_cache_reset(void)
{
    TuneCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    c.entries.clear();
    c.loaded = false;
    c.path.clear();
}

}  // extern "C"
