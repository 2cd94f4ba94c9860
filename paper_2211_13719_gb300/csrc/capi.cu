// C ABI entry points (include/mrhs.h): argument validation, device
// selection, error translation.  Every call catches the library's internal
// exceptions and returns an mrhs_status; nothing aborts the host process.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace mrhs;

namespace {

thread_local std::string g_last_error;

mrhs_status record(mrhs_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

// Makes `device` current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            (void)cudaGetLastError();
            prev = -1;
        }
        if (prev != device) MRHS_CUDA(cudaSetDevice(device));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

std::mutex g_scratch_mu;
std::map<std::pair<int, cudaStream_t>, Scratch> g_scratch;

Scratch &stream_scratch(cudaStream_t s) {
    int dev = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    return g_scratch[{dev, s}];
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

#define MRHS_API_BEGIN try {
#define MRHS_API_END                                                   \
    }                                                                  \
    catch (const mrhs::Error &e) { return record(e.code, e.what()); }  \
    catch (const std::bad_alloc &) { return record(MRHS_ERR_OOM, "host allocation failed"); } \
    catch (const std::exception &e) { return record(MRHS_ERR_CUDA, e.what()); } \
    g_last_error.clear();                                              \
    return MRHS_OK;

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg) { return record(code, msg); }
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}

extern "C" {

const char *mrhs_last_error(void) { return g_last_error.c_str(); }

uint64_t mrhs_kernel_launch_count(void) { return mrhs::g_launches.load(); }

mrhs_status mrhs_create_lattice(const int dims[4], int t_boundary, int device, mrhs_lattice **out) {
    MRHS_API_BEGIN
    if (!dims || !out) fail(MRHS_ERR_INVALID, "dims and out must be non-null");
    *out = nullptr;
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 1) fail(MRHS_ERR_INVALID, "lattice extents must be >= 1");
    if (t_boundary != 1 && t_boundary != -1) fail(MRHS_ERR_INVALID, "t_boundary must be +1 or -1");
    int ndev = 0;
    MRHS_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) fail(MRHS_ERR_INVALID, "no such CUDA device");
    DeviceGuard dg(device);
    auto lat = std::make_unique<mrhs_lattice>();
    for (int mu = 0; mu < 4; ++mu) lat->g.L[mu] = dims[mu];
    lat->g.V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    lat->g.tb = t_boundary;
    lat->device = device;
    const size_t V = (size_t)lat->g.V;
    lat->U64.alloc(V * 36 * sizeof(double2));
    lat->U32.alloc(V * 36 * sizeof(float2));
    lat->C64.alloc(V * 36 * sizeof(double2));
    lat->C32.alloc(V * 36 * sizeof(float2));
    lat->Udf.alloc(V * 36 * sizeof(float4));
    lat->Cdf.alloc(V * 36 * sizeof(float4));
    lat->Cinv64.alloc(V * 36 * sizeof(double2));
    lat->Cinv32.alloc(V * 36 * sizeof(float2));
    lat->U32a.alloc(V * 36 * sizeof(float2));
    lat->C32a.alloc(V * 36 * sizeof(float2));
    lat->Cinv32a.alloc(V * 36 * sizeof(float2));
    lat->CinvErr.alloc(sizeof(int));
    *out = lat.release();
    MRHS_API_END
}

void mrhs_destroy_lattice(mrhs_lattice *lat) {
    if (!lat) return;
    try {
        DeviceGuard dg(lat->device);
        cudaDeviceSynchronize();
        delete lat;
    } catch (...) {
        delete lat;
    }
}

mrhs_status mrhs_load_gauge(mrhs_lattice *lat, const double *U_host) {
    MRHS_API_BEGIN
    if (!lat || !U_host) fail(MRHS_ERR_INVALID, "lattice and gauge field must be non-null");
    DeviceGuard dg(lat->device);
    const size_t bytes = (size_t)lat->g.V * 36 * sizeof(double2);
    DeviceBuffer tmp(bytes);
    MRHS_CUDA(cudaMemcpy(tmp.ptr, U_host, bytes, cudaMemcpyHostToDevice));
    gauge_to_soa(*lat, tmp.as<double>(), 0);
    MRHS_CUDA(cudaDeviceSynchronize());
    lat->has_gauge = true;
    lat->has_clover = false;
    MRHS_API_END
}

mrhs_status mrhs_build_clover(mrhs_lattice *lat, double mass, double csw) {
    MRHS_API_BEGIN
    if (!lat) fail(MRHS_ERR_INVALID, "lattice must be non-null");
    if (!lat->has_gauge) fail(MRHS_ERR_INVALID, "gauge field not loaded");
    DeviceGuard dg(lat->device);
    build_clover(*lat, mass, csw, 0);
    MRHS_CUDA(cudaDeviceSynchronize());
    lat->cinv_singular = clover_inverse_error(*lat) != 0;
    lat->mass = mass;
    lat->csw = csw;
    lat->has_clover = true;
    MRHS_API_END
}

mrhs_status mrhs_get_clover(mrhs_lattice *lat, double *clover_host) {
    MRHS_API_BEGIN
    if (!lat || !clover_host) fail(MRHS_ERR_INVALID, "lattice and output must be non-null");
    if (!lat->has_clover) fail(MRHS_ERR_INVALID, "clover term not built");
    DeviceGuard dg(lat->device);
    const int64_t V = lat->g.V;
    std::vector<double2> soa((size_t)V * 36);
    MRHS_CUDA(cudaMemcpy(soa.data(), lat->C64.ptr, soa.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    for (int64_t x = 0; x < V; ++x) {
        for (int chi = 0; chi < 2; ++chi) {
            double *o = clover_host + (x * 2 + chi) * 36;
            for (int q = 0; q < 3; ++q) {
                const double2 d = soa[(size_t)(chi * 18 + q) * V + x];
                o[2 * q] = d.x;
                o[2 * q + 1] = d.y;
            }
            for (int q = 3; q < 18; ++q) {
                const double2 l = soa[(size_t)(chi * 18 + q) * V + x];
                o[6 + 2 * (q - 3)] = l.x;
                o[6 + 2 * (q - 3) + 1] = l.y;
            }
        }
    }
    MRHS_API_END
}

static void check_apply(mrhs_lattice *lat, const void *in, const void *out, int nrhs, mrhs_precision prec) {
    if (!lat) fail(MRHS_ERR_INVALID, "lattice must be non-null");
    if (!in || !out) fail(MRHS_ERR_INVALID, "in and out must be non-null");
    if (in == out) fail(MRHS_ERR_INVALID, "in and out must not overlap");
    if (nrhs < 1) fail(MRHS_ERR_INVALID, "nrhs must be >= 1");
    if (prec != MRHS_FP32 && prec != MRHS_FP64 && prec != MRHS_DF64)
        fail(MRHS_ERR_INVALID, "precision must be FP32, FP64 or DF64");
    if (!aligned16(in) || !aligned16(out)) fail(MRHS_ERR_INVALID, "fields must be 16-byte aligned");
    if (!lat->has_clover) fail(MRHS_ERR_INVALID, "clover term not built");
}

// input precision of an operator computing in `prec`: float-float takes FP32 fields
static mrhs_precision input_prec(mrhs_precision prec) { return prec == MRHS_DF64 ? MRHS_FP32 : prec; }

mrhs_status mrhs_apply_D(mrhs_lattice *lat, const void *in_dev, void *out_dev, int nrhs, mrhs_precision prec,
                         void *stream) {
    MRHS_API_BEGIN
    check_apply(lat, in_dev, out_dev, nrhs, prec);
    DeviceGuard dg(lat->device);
    dslash(*lat, prec, input_prec(prec), in_dev, out_dev, nullptr, nrhs, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

mrhs_status mrhs_residual_D(mrhs_lattice *lat, const void *in_dev, const void *y_dev, void *out_dev, int nrhs,
                            mrhs_precision prec, void *stream) {
    MRHS_API_BEGIN
    check_apply(lat, in_dev, out_dev, nrhs, prec);
    if (!y_dev || !aligned16(y_dev)) fail(MRHS_ERR_INVALID, "y must be non-null and 16-byte aligned");
    DeviceGuard dg(lat->device);
    dslash(*lat, prec, input_prec(prec), in_dev, out_dev, y_dev, nrhs, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

mrhs_status mrhs_apply_D_batch(const mrhs_apply_item *items, int count, void *stream) {
    MRHS_API_BEGIN
    if (!items || count < 1 || count > 8) fail(MRHS_ERR_INVALID, "items must be non-null and count in 1..8");
    std::vector<BatchItemHost> h((size_t)count);
    for (int i = 0; i < count; ++i) {
        const mrhs_apply_item &it = items[i];
        if (!it.lat) fail(MRHS_ERR_INVALID, "every batch item needs a lattice");
        check_apply(it.lat, it.in_dev, it.out_dev, it.nrhs, MRHS_FP32);
        if (it.y_dev && (reinterpret_cast<uintptr_t>(it.y_dev) & 7u))
            fail(MRHS_ERR_INVALID, "y must be 8-byte aligned");
        h[(size_t)i] = BatchItemHost{it.lat, it.in_dev, it.out_dev, it.y_dev, it.nrhs};
    }
    DeviceGuard dg(items[0].lat->device);
    dslash_batch(h.data(), count, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

mrhs_status mrhs_apply_hop_eo(mrhs_lattice *lat, int out_parity, const void *in_dev, void *out_dev, int nrhs,
                              void *stream) {
    MRHS_API_BEGIN
    check_apply(lat, in_dev, out_dev, nrhs, MRHS_FP32);
    if (out_parity != 0 && out_parity != 1) fail(MRHS_ERR_INVALID, "out_parity must be 0 (even) or 1 (odd)");
    DeviceGuard dg(lat->device);
    hop_eo(*lat, out_parity, in_dev, out_dev, nrhs, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

mrhs_status mrhs_apply_schur(mrhs_lattice *lat, const void *in_dev, void *out_dev, int nrhs, void *stream) {
    MRHS_API_BEGIN
    check_apply(lat, in_dev, out_dev, nrhs, MRHS_FP32);
    DeviceGuard dg(lat->device);
    const size_t half = sizeof(float2) * (size_t)(lat->g.V / 2) * 12 * nrhs;
    if (lat->EOtmp.bytes < half) {
        MRHS_CUDA(cudaDeviceSynchronize());  // the old scratch may still be in use by earlier calls
        lat->EOtmp.alloc(half);
    }
    schur_apply(*lat, in_dev, out_dev, nrhs, lat->EOtmp.ptr, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

mrhs_status mrhs_sap_smooth(mrhs_lattice *lat, const void *v_dev, void *z_dev, int nrhs, const int block[4],
                            int cycles, int mr_steps, void *stream) {
    MRHS_API_BEGIN
    check_apply(lat, v_dev, z_dev, nrhs, MRHS_FP32);
    if (!block) fail(MRHS_ERR_INVALID, "block extents must be non-null");
    if (!sap_supported(*lat, block, nrhs))
        fail(MRHS_ERR_INVALID, "SAP needs an even nrhs, block extents dividing the lattice into an even number of "
                               "blocks per direction, at most 256 sites per block and 32-bit field indexing");
    DeviceGuard dg(lat->device);
    const size_t full = sizeof(float2) * (size_t)lat->g.V * 12 * nrhs;
    if (lat->SAPtmp.bytes < full) {
        MRHS_CUDA(cudaDeviceSynchronize());  // the old scratch may still be in use by earlier calls
        lat->SAPtmp.alloc(full);
    }
    sap_smooth(*lat, v_dev, z_dev, nrhs, block, cycles, mr_steps, lat->SAPtmp.ptr, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

static void check_blas(const void *p, int64_t rows, int nrhs, mrhs_precision prec) {
    if (!p) fail(MRHS_ERR_INVALID, "field pointer must be non-null");
    if (rows < 1) fail(MRHS_ERR_INVALID, "rows must be >= 1");
    if (nrhs < 1 || nrhs > 256) fail(MRHS_ERR_INVALID, "nrhs must be in 1..256");
    if (prec != MRHS_FP32 && prec != MRHS_FP64) fail(MRHS_ERR_INVALID, "precision must be FP32 or FP64");
}

mrhs_status mrhs_blas_multi_dot(const void *basis_dev, int k, const void *w_dev, int64_t rows, int nrhs,
                                mrhs_precision prec, void *out_dev, void *stream) {
    MRHS_API_BEGIN
    check_blas(basis_dev, rows, nrhs, prec);
    check_blas(w_dev, rows, nrhs, prec);
    if (k < 1 || !out_dev) fail(MRHS_ERR_INVALID, "k >= 1 and a non-null output required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    multi_dot(prec, basis_dev, rows * nrhs, k, w_dev, rows, nrhs, static_cast<double2 *>(out_dev),
              stream_scratch(s), s);
    MRHS_API_END
}

mrhs_status mrhs_blas_norm2(const void *w_dev, int64_t rows, int nrhs, mrhs_precision prec, double *out_dev,
                            void *stream) {
    MRHS_API_BEGIN
    check_blas(w_dev, rows, nrhs, prec);
    if (!out_dev) fail(MRHS_ERR_INVALID, "output must be non-null");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    norm2(prec, w_dev, rows, nrhs, out_dev, stream_scratch(s), s);
    MRHS_API_END
}

mrhs_status mrhs_blas_lincomb(void *w_dev, const void *basis_dev, int k, const void *coef_dev, double alpha,
                              int64_t rows, int nrhs, mrhs_precision prec, void *stream) {
    MRHS_API_BEGIN
    check_blas(w_dev, rows, nrhs, prec);
    check_blas(basis_dev, rows, nrhs, prec);
    if (k < 1 || !coef_dev) fail(MRHS_ERR_INVALID, "k >= 1 and coefficients required");
    lincomb(prec, w_dev, prec, basis_dev, rows * nrhs, k, static_cast<const double2 *>(coef_dev), alpha, rows,
            nrhs, static_cast<cudaStream_t>(stream));
    MRHS_API_END
}

}  // extern "C"
