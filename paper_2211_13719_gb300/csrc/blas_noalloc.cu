// mrhs_blas_multi_dot_noalloc: the batched multi-dot with its reduction
// scratch in statically allocated device memory instead of cudaMalloc.
//
// Who needs it: callers that must not allocate device memory while they run,
// e.g. code recording work into a CUDA graph (cudaMalloc / cudaFree are not
// stream operations and may synchronise the device), real-time or embedded
// hosts that reserve all device memory up front, or programs whose memory is
// owned by another allocator.  The regular mrhs_blas_multi_dot grows a
// per-stream scratch buffer with cudaMalloc on first use; this variant never
// allocates.
//
// Scratch: one file-scope array shared by every call in the process (each
// GPU that loads the library holds its own copy until exit).  Every call
// looks its device address up (cudaGetSymbolAddress, which allocates
// nothing) with the caller's device current, so the address stays right
// after a device reset or a new primary context.  The first call on a
// device may also load the library's module onto it: make that first call
// before any stream capture.  Calls that overlap on the GPU (other streams,
// other host threads) race on the shared scratch: order them on one stream.
#include "internal.cuh"

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg);
}

using namespace mrhs;

namespace {

constexpr int NOALLOC_MAX_RHS = 64;
constexpr int NOALLOC_MAX_BLOCKS = 512;
// per-block partials plus one total per group of 32 blocks: 4.1 MiB of double2
constexpr size_t NOALLOC_PARTIALS = (size_t)(NOALLOC_MAX_BLOCKS + NOALLOC_MAX_BLOCKS / 32) * KCHUNK * NOALLOC_MAX_RHS;

static __device__ __align__(256) double2 g_noalloc_partials[NOALLOC_PARTIALS];
static __device__ __align__(256) unsigned int g_noalloc_counter[64];

struct DevScratch {
    double2 *partials = nullptr;
    unsigned int *counter = nullptr;
};

// the device addresses of the two arrays on the current device
DevScratch noalloc_scratch() {
    DevScratch d;
    void *p = nullptr, *c = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(MRHS_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    e = cudaGetSymbolAddress(&c, g_noalloc_counter);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(MRHS_ERR_CUDA, std::string("cudaGetSymbolAddress(counter): ") + cudaGetErrorString(e));
    }
    d.partials = static_cast<double2 *>(p);
    d.counter = static_cast<unsigned int *>(c);
    return d;
}

}  // namespace

extern "C" mrhs_status mrhs_blas_multi_dot_noalloc(const void *basis_dev, int k, const void *w_dev, int64_t rows,
                                                   int nrhs, mrhs_precision prec, void *out_dev, void *stream) {
    try {
        if (!basis_dev || !w_dev || !out_dev) fail(MRHS_ERR_INVALID, "basis, w and out must be non-null");
        if (k < 1) fail(MRHS_ERR_INVALID, "k must be >= 1");
        if (rows < 1) fail(MRHS_ERR_INVALID, "rows must be >= 1");
        if (nrhs < 1 || nrhs > NOALLOC_MAX_RHS)
            fail(MRHS_ERR_INVALID, "nrhs must be in 1..64 for the no-allocation multi-dot (static scratch limit)");
        if (prec != MRHS_FP32 && prec != MRHS_FP64) fail(MRHS_ERR_INVALID, "precision must be FP32 or FP64");
        const DevScratch d = noalloc_scratch();
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        // the completion counter must start at zero (a previous call that failed
        // part-way could have left it set)
        MRHS_CUDA(cudaMemsetAsync(d.counter, 0, sizeof(unsigned int) * 64, s));
        multi_dot_fixed_scratch(prec, basis_dev, rows * nrhs, k, w_dev, rows, nrhs, static_cast<double2 *>(out_dev),
                                d.partials, d.counter, NOALLOC_MAX_BLOCKS, s);
    } catch (const mrhs::Error &e) {
        return api_record(e.code, e.what());
    } catch (const std::exception &e) {
        return api_record(MRHS_ERR_CUDA, e.what());
    }
    api_record(MRHS_OK, "");
    return MRHS_OK;
}
