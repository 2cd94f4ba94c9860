// Internal helpers shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "../../include/mrhs.h"

namespace mrhs {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    mrhs_status code;
    Error(mrhs_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(mrhs_status c, const std::string &m) { throw Error(c, m); }

inline void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (e == cudaErrorMemoryAllocation)
            fail(MRHS_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
        fail(MRHS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}
#define MRHS_CUDA(call) ::mrhs::cuda_check((call), #call)
// counts kernel launches (diagnostic) and checks the launch
void count_launches(uint64_t k);
#define MRHS_LAUNCHED(name) (::mrhs::count_launches(1), ::mrhs::cuda_check(cudaGetLastError(), name))

// Event timing of one kernel's launches for measurement harnesses
// (mrhs_kernel_timer_start / _stop): declared just before a launch, the scope
// records an event on the launching stream before the launch and another when
// the scope closes, if that kernel is being timed and the stream is not being
// captured into a graph (captured launches are only counted).
struct KernelTimerScope {
    int slot = -1;
    cudaStream_t stream = nullptr;
    KernelTimerScope(const char *name, cudaStream_t s);
    ~KernelTimerScope();
    KernelTimerScope(const KernelTimerScope &) = delete;
    KernelTimerScope &operator=(const KernelTimerScope &) = delete;
};
#define MRHS_TIMED(name, stream) ::mrhs::KernelTimerScope mrhs_timer_scope_(name, stream)

// -------------------------------------------------------- device buffers
struct DeviceBuffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    DeviceBuffer() = default;
    explicit DeviceBuffer(size_t b) { alloc(b); }
    DeviceBuffer(const DeviceBuffer &) = delete;
    DeviceBuffer &operator=(const DeviceBuffer &) = delete;
    DeviceBuffer(DeviceBuffer &&o) noexcept : ptr(o.ptr), bytes(o.bytes) { o.ptr = nullptr; o.bytes = 0; }
    DeviceBuffer &operator=(DeviceBuffer &&o) noexcept {
        if (this != &o) { release(); ptr = o.ptr; bytes = o.bytes; o.ptr = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DeviceBuffer() { release(); }
    void alloc(size_t b) {
        release();
        if (b == 0) return;
        cudaError_t e = cudaMalloc(&ptr, b);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            ptr = nullptr;
            fail(MRHS_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
        }
        bytes = b;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// ------------------------------------------------------------- complex
template <typename T> struct cplx { T re, im; };

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T r, T i) { return {r, i}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
// i * a and -i * a
template <typename T> __host__ __device__ __forceinline__ cplx<T> ti(cplx<T> a) { return {-a.im, a.re}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> tmi(cplx<T> a) { return {a.im, -a.re}; }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
// acc += a * b ; acc += conj(a) * b
template <typename T> __device__ __forceinline__ void cmac(cplx<T> &acc, cplx<T> a, cplx<T> b) {
    acc.re = fmadd(a.re, b.re, acc.re); acc.re = fmadd(-a.im, b.im, acc.re);
    acc.im = fmadd(a.re, b.im, acc.im); acc.im = fmadd(a.im, b.re, acc.im);
}
template <typename T> __device__ __forceinline__ void cmac_conj(cplx<T> &acc, cplx<T> a, cplx<T> b) {
    acc.re = fmadd(a.re, b.re, acc.re); acc.re = fmadd(a.im, b.im, acc.re);
    acc.im = fmadd(a.re, b.im, acc.im); acc.im = fmadd(-a.im, b.re, acc.im);
}

template <typename T> struct real_of;
template <> struct real_of<float> { using type = float; };
template <> struct real_of<double> { using type = double; };

// precision enum -> bytes of one complex
inline size_t complex_bytes(mrhs_precision p) {
    return p == MRHS_FP64 ? 16 : (p == MRHS_FP32 ? 8 : 4);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// --------------------------------------------------------- device query
int sm_count(int device);

// ---------------------------------------------------- lattice geometry
struct Geom {
    int L[4];
    int64_t V;
    int tb;  // +1 periodic / -1 antiperiodic in t
};

// site index <-> coordinates (x fastest)
__host__ __device__ __forceinline__ void site_to_coords(int64_t s, const int L[4], int c[4]) {
    c[0] = (int)(s % L[0]);
    int64_t q = s / L[0];
    c[1] = (int)(q % L[1]);
    q /= L[1];
    c[2] = (int)(q % L[2]);
    c[3] = (int)(q / L[2]);
}
__host__ __device__ __forceinline__ int64_t coords_to_site(const int c[4], const int L[4]) {
    return c[0] + (int64_t)L[0] * (c[1] + (int64_t)L[1] * (c[2] + (int64_t)L[2] * c[3]));
}

// neighbour of `site` in direction d of the 9-point coarse stencil (Sec. 6): d = 0 the site
// itself, d = 1..4 the forward neighbours in x, y, z, t, d = 5..8 the backward ones (periodic)
__host__ __device__ __forceinline__ int64_t stencil_nb_site(int64_t site, const int L[4], int d) {
    if (d == 0) return site;
    int c[4];
    site_to_coords(site, L, c);
    const int mu = d <= 4 ? d - 1 : d - 5;
    const int step = d <= 4 ? 1 : -1;
    c[mu] = (c[mu] + step + L[mu]) % L[mu];
    return coords_to_site(c, L);
}

}  // namespace mrhs
