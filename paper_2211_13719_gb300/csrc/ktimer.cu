// Event timing of one kernel's launches (mrhs_kernel_timer_start / _stop), for
// measurement harnesses that need a kernel's own duration inside a larger
// timed region: the launches happen inside the library on its streams, where
// the caller cannot place events.  Nothing on the compute path depends on it.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg);

namespace {
struct TimerState {
    std::mutex mu;
    std::atomic<bool> active{false};
    std::string name;
    std::vector<cudaEvent_t> ev;  // (start, stop) pairs, reused across timings
    int used = 0;                 // pairs recorded in this timing
    int64_t captured = 0;         // launches captured into graphs (not timed)
};
TimerState &state() {
    static TimerState s;
    return s;
}
}  // namespace

KernelTimerScope::KernelTimerScope(const char *name, cudaStream_t s) {
    TimerState &t = state();
    if (!t.active.load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lock(t.mu);
    if (!t.active.load(std::memory_order_relaxed) || t.name != name) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    if (cs != cudaStreamCaptureStatusNone) {
        ++t.captured;
        return;
    }
    if (2 * t.used + 2 > (int)t.ev.size()) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            (void)cudaGetLastError();
            if (a) cudaEventDestroy(a);
            return;
        }
        t.ev.push_back(a);
        t.ev.push_back(b);
    }
    if (cudaEventRecord(t.ev[2 * t.used], s) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    slot = t.used++;
    stream = s;
}

KernelTimerScope::~KernelTimerScope() {
    if (slot < 0) return;
    TimerState &t = state();
    std::lock_guard<std::mutex> lock(t.mu);
    if (cudaEventRecord(t.ev[2 * slot + 1], stream) != cudaSuccess) (void)cudaGetLastError();
}

}  // namespace mrhs

using namespace mrhs;

extern "C" {

mrhs_status mrhs_kernel_timer_start(const char *kernel_name) {
    if (!kernel_name || !*kernel_name) return api_record(MRHS_ERR_INVALID, "kernel_name must be non-empty");
    TimerState &t = state();
    std::lock_guard<std::mutex> lock(t.mu);
    if (t.active.load()) return api_record(MRHS_ERR_INVALID, "a kernel timing is already active");
    t.name = kernel_name;
    t.used = 0;
    t.captured = 0;
    t.active.store(true, std::memory_order_release);
    return api_record(MRHS_OK, "");
}

mrhs_status mrhs_kernel_timer_stop(double *total_ms, int64_t *timed_launches, int64_t *captured_launches) {
    TimerState &t = state();
    std::lock_guard<std::mutex> lock(t.mu);
    if (!t.active.load()) return api_record(MRHS_ERR_INVALID, "no kernel timing is active");
    t.active.store(false, std::memory_order_release);
    double ms = 0.0;
    for (int i = 0; i < t.used; ++i) {
        float e = 0.f;
        cudaError_t r = cudaEventSynchronize(t.ev[2 * i + 1]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&e, t.ev[2 * i], t.ev[2 * i + 1]);
        if (r != cudaSuccess) {
            (void)cudaGetLastError();
            return api_record(MRHS_ERR_CUDA, std::string("kernel timer: ") + cudaGetErrorString(r));
        }
        ms += e;
    }
    if (total_ms) *total_ms = ms;
    if (timed_launches) *timed_launches = t.used;
    if (captured_launches) *captured_launches = t.captured;
    return api_record(MRHS_OK, "");
}

}  // extern "C"
