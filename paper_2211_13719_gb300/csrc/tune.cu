// Autotuner for launch variants that change only how work is mapped onto the
// GPU, never the arithmetic of an output element: a kernel family offers a
// few variants (here the site-tile shapes of the FP32 stencils), and the first
// eager launch for a (kernel, lattice extents, RHS count) key times each
// variant with CUDA events on the launching stream.  The choice, cached for
// the rest of the process and savable to / loadable from a text file, is the
// fastest variant if it beats the default (variant 0) by more than 3 %, else
// the default.  Launches made while the stream is being captured into a CUDA
// graph never tune: they use the cached choice or variant 0.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg);

namespace {

struct TuneKey {
    std::string kernel;
    int dims[4];
    int n;
    bool operator<(const TuneKey &o) const {
        if (kernel != o.kernel) return kernel < o.kernel;
        for (int i = 0; i < 4; ++i)
            if (dims[i] != o.dims[i]) return dims[i] < o.dims[i];
        return n < o.n;
    }
};

struct TuneVal {
    int variant = 0;
    int nvariants = 1;
    float best_ms = 0.f;
    float default_ms = 0.f;
};

struct Tuner {
    std::mutex mu;
    std::map<TuneKey, TuneVal> cache;
    std::vector<TuneKey> order;  // insertion order, for mrhs_tune_get
    int enabled = -1;            // -1: from MRHS_AUTOTUNE on first use (default on)
};

Tuner &tuner() {
    static Tuner t;
    return t;
}

bool tuning_enabled(Tuner &t) {
    if (t.enabled < 0) {
        const char *e = std::getenv("MRHS_AUTOTUNE");
        t.enabled = (e && std::strcmp(e, "0") == 0) ? 0 : 1;
    }
    return t.enabled == 1;
}

void insert(Tuner &t, const TuneKey &k, const TuneVal &v) {
    auto it = t.cache.find(k);
    if (it == t.cache.end()) t.order.push_back(k);
    t.cache[k] = v;
}

}  // namespace

int tune_pick(const char *kernel, const int dims[4], int n, int nvariants, const std::function<void(int)> &launch,
              cudaStream_t s) {
    if (nvariants <= 1) return 0;
    Tuner &t = tuner();
    TuneKey key{kernel, {dims[0], dims[1], dims[2], dims[3]}, n};
    {
        std::lock_guard<std::mutex> lk(t.mu);
        auto it = t.cache.find(key);
        if (it != t.cache.end() && it->second.variant < nvariants) return it->second.variant;
        if (!tuning_enabled(t)) return 0;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MRHS_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MRHS_CUDA(cudaEventCreate(&e0));
    MRHS_CUDA(cudaEventCreate(&e1));
    constexpr int reps = 3;
    TuneVal v;
    v.nvariants = nvariants;
    std::vector<float> ms(nvariants, 0.f);
    try {
        for (int i = 0; i < nvariants; ++i) {
            launch(i);  // warm-up
            MRHS_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r) launch(i);
            MRHS_CUDA(cudaEventRecord(e1, s));
            MRHS_CUDA(cudaEventSynchronize(e1));
            MRHS_CUDA(cudaEventElapsedTime(&ms[i], e0, e1));
            ms[i] /= reps;
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 1; i < nvariants; ++i)
        if (ms[i] < ms[v.variant]) v.variant = i;
    // keep the default unless another variant is clearly faster: differences
    // within the run-to-run spread of a few launches are not a reason to switch
    constexpr float kMargin = 0.03f;
    if (ms[v.variant] > (1.f - kMargin) * ms[0]) v.variant = 0;
    v.best_ms = ms[v.variant];
    v.default_ms = ms[0];
    std::lock_guard<std::mutex> lk(t.mu);
    insert(t, key, v);
    return v.variant;
}

}  // namespace mrhs

using namespace mrhs;

void mrhs_tune_set_enabled(int enabled) {
    Tuner &t = tuner();
    std::lock_guard<std::mutex> lk(t.mu);
    t.enabled = enabled ? 1 : 0;
}

void mrhs_tune_clear(void) {
    Tuner &t = tuner();
    std::lock_guard<std::mutex> lk(t.mu);
    t.cache.clear();
    t.order.clear();
}

int mrhs_tune_count(void) {
    Tuner &t = tuner();
    std::lock_guard<std::mutex> lk(t.mu);
    return (int)t.order.size();
}

mrhs_status mrhs_tune_get(int index, mrhs_tune_entry *out) {
    Tuner &t = tuner();
    std::lock_guard<std::mutex> lk(t.mu);
    if (!out || index < 0 || index >= (int)t.order.size())
        return api_record(MRHS_ERR_INVALID, "tune entry index out of range or output null");
    const TuneKey &k = t.order[(size_t)index];
    const TuneVal &v = t.cache[k];
    std::memset(out, 0, sizeof(*out));
    std::snprintf(out->kernel, sizeof(out->kernel), "%s", k.kernel.c_str());
    for (int i = 0; i < 4; ++i) out->dims[i] = k.dims[i];
    out->nrhs = k.n;
    out->variant = v.variant;
    out->nvariants = v.nvariants;
    out->best_ms = v.best_ms;
    out->default_ms = v.default_ms;
    return MRHS_OK;
}

mrhs_status mrhs_tune_save(const char *path) {
    if (!path) return api_record(MRHS_ERR_INVALID, "path must be non-null");
    Tuner &t = tuner();
    std::lock_guard<std::mutex> lk(t.mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return api_record(MRHS_ERR_INVALID, std::string("cannot open ") + path + " for writing");
    std::fprintf(f, "# kernel Lx Ly Lz Lt nrhs variant nvariants best_ms default_ms\n");
    for (const TuneKey &k : t.order) {
        const TuneVal &v = t.cache[k];
        std::fprintf(f, "%s %d %d %d %d %d %d %d %.6f %.6f\n", k.kernel.c_str(), k.dims[0], k.dims[1], k.dims[2],
                     k.dims[3], k.n, v.variant, v.nvariants, v.best_ms, v.default_ms);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? MRHS_OK : api_record(MRHS_ERR_INVALID, std::string("cannot write ") + path);
}

mrhs_status mrhs_tune_load(const char *path) {
    if (!path) return api_record(MRHS_ERR_INVALID, "path must be non-null");
    FILE *f = std::fopen(path, "r");
    if (!f) return api_record(MRHS_ERR_NOT_FOUND, std::string("cannot open ") + path);
    Tuner &t = tuner();
    std::lock_guard<std::mutex> lk(t.mu);
    char line[512];
    int lineno = 0;
    mrhs_status st = MRHS_OK;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        if (line[0] == '#' || line[0] == '\n') continue;
        char name[64];
        TuneKey k;
        TuneVal v;
        if (std::sscanf(line, "%63s %d %d %d %d %d %d %d %f %f", name, &k.dims[0], &k.dims[1], &k.dims[2], &k.dims[3],
                        &k.n, &v.variant, &v.nvariants, &v.best_ms, &v.default_ms) != 10 ||
            v.variant < 0 || v.nvariants < 1 || v.variant >= v.nvariants) {
            st = api_record(MRHS_ERR_INVALID, std::string(path) + ": malformed line " + std::to_string(lineno));
            break;
        }
        k.kernel = name;
        insert(t, k, v);
    }
    std::fclose(f);
    return st;
}
