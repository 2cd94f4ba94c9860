// GCRO-DR on the coarsest level (paper Sec. 9 outlook: a recycling coarsest
// solver): the per-RHS small dense work of each cycle on the device.
//
// The fields (Arnoldi basis V, recycle space U, C = A U) are batched over the
// RHS like every other Krylov vector (solver.cu drives them with the batched
// stencil and BLAS kernels); what is per RHS and small -- the Hessenberg H,
// the block B = C^H A V, the least-squares problem, the harmonic Ritz
// eigenproblem and the QR factorisations -- runs here, one CTA per RHS whose
// first thread calls the FP64 drivers of gcro_small.cuh with its workspace in
// shared memory.  The kernels below also move dots from the batched layout
// ([index][n]) into the per-RHS matrices ([n][LD][LD]) and the drivers'
// results back into the coefficient layout of the batched linear combination.
#include "gcro_small.cuh"
#include "mg.cuh"

namespace mrhs {

namespace {

using gcro::LD;
using gcro::zc;

__device__ __forceinline__ zc toz(double2 v) { return zc{v.x, v.y}; }
__device__ __forceinline__ double2 fromz(zc v) { return make_double2(v.re, v.im); }

// column j of a per-RHS Hessenberg: H[r][i][j] = hcol[i][r] (i <= j), H[r][j+1][j] = beta
// (sqrt(hn2), rescaled like the Givens update when the normalisation fix-up ran)
__global__ void k_gcro_store_col(double2 *__restrict__ H, const double2 *__restrict__ hcol,
                                 const double *__restrict__ hn2, const double *__restrict__ nn, int j, int row0,
                                 int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 *Hr = H + (int64_t)r * LD * LD;
    for (int i = 0; i <= j; ++i) Hr[(row0 + i) * LD + j] = hcol[(int64_t)i * n + r];
    double beta = sqrt(fmax(hn2[r], 0.0));
    if (nn) {
        const double f = nn[r];
        if (f > 0.0 && fabs(f - 1.0) > 1e-2) beta *= sqrt(f);
        if (f == 0.0) beta = 0.0;
    }
    Hr[(row0 + j + 1) * LD + j] = make_double2(beta, 0.0);
}

// M[r][row0 + i][col] = d[i][r], i < cnt (a column of dots into the per-RHS matrices)
__global__ void k_gcro_put_col(double2 *__restrict__ M, const double2 *__restrict__ d, int cnt, int row0, int col,
                               int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int i = 0; i < cnt; ++i) M[(int64_t)r * LD * LD + (row0 + i) * LD + col] = d[(int64_t)i * n + r];
}

// v[r][off + i] = d[i][r] (double2) or |.|^2 source nrm2[i][r] into un2 (double)
__global__ void k_gcro_put_vec(double2 *__restrict__ v, const double2 *__restrict__ d, int cnt, int off, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int i = 0; i < cnt; ++i) v[(int64_t)r * LD + off + i] = d[(int64_t)i * n + r];
}
__global__ void k_gcro_put_norm(double *__restrict__ un2, const double *__restrict__ nrm2, int i, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    un2[(int64_t)r * LD + i] = nrm2[r];
}

// one CTA per RHS; thread 0 runs the driver with its workspace in dynamic shared memory
__global__ void k_gcro_seed(const double2 *__restrict__ H, const double *__restrict__ beta2, int m, int k,
                            double2 *__restrict__ Y, double2 *__restrict__ QC, double2 *__restrict__ PU,
                            int *__restrict__ err) {
    extern __shared__ double2 wsd[];
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    zc *ws = reinterpret_cast<zc *>(wsd);
    const zc *Hr = reinterpret_cast<const zc *>(H + (int64_t)r * LD * LD);
    zc *y = reinterpret_cast<zc *>(Y + (int64_t)r * LD);
    zc *qc = reinterpret_cast<zc *>(QC + (int64_t)r * LD * LD);
    zc *pu = reinterpret_cast<zc *>(PU + (int64_t)r * LD * LD);
    if (!gcro::gcro_seed(Hr, sqrt(fmax(beta2[r], 0.0)), m, k, y, qc, pu, ws)) atomicExch(err, 1);
}

__global__ void k_gcro_cycle(const double2 *__restrict__ H, const double2 *__restrict__ B,
                             const double *__restrict__ UN2, const double2 *__restrict__ WR,
                             const double2 *__restrict__ WU, int m, int k, double2 *__restrict__ Y,
                             double2 *__restrict__ QC, double2 *__restrict__ PU, int *__restrict__ err) {
    extern __shared__ double2 wsd[];
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    zc *ws = reinterpret_cast<zc *>(wsd);
    const zc *Hr = reinterpret_cast<const zc *>(H + (int64_t)r * LD * LD);
    const zc *Br = reinterpret_cast<const zc *>(B + (int64_t)r * LD * LD);
    const zc *wr = reinterpret_cast<const zc *>(WR + (int64_t)r * LD);
    const zc *wu = reinterpret_cast<const zc *>(WU + (int64_t)r * LD * LD);
    zc *y = reinterpret_cast<zc *>(Y + (int64_t)r * LD);
    zc *qc = reinterpret_cast<zc *>(QC + (int64_t)r * LD * LD);
    zc *pu = reinterpret_cast<zc *>(PU + (int64_t)r * LD * LD);
    if (!gcro::gcro_cycle(Hr, Br, UN2 + (int64_t)r * LD, wr, wu, m, k, y, qc, pu, ws)) atomicExch(err, 1);
}

// coefficient arrays of the batched linear combination, coef[j][r] (j < cnt):
// from a per-RHS vector (v[r][off + j]) or a column of a per-RHS matrix (M[r][off + j][col]),
// times sign
__global__ void k_gcro_coef_vec(double2 *__restrict__ coef, const double2 *__restrict__ v, int off, int cnt,
                                double sign, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int j = 0; j < cnt; ++j) {
        const double2 a = v[(int64_t)r * LD + off + j];
        coef[(int64_t)j * n + r] = make_double2(sign * a.x, sign * a.y);
    }
}
__global__ void k_gcro_coef_col(double2 *__restrict__ coef, const double2 *__restrict__ M, int off, int cnt, int col,
                                double sign, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int j = 0; j < cnt; ++j) {
        const double2 a = M[(int64_t)r * LD * LD + (off + j) * LD + col];
        coef[(int64_t)j * n + r] = make_double2(sign * a.x, sign * a.y);
    }
}

}  // namespace

constexpr size_t kGcroSmem = sizeof(double2) * gcro::GCRO_WS * gcro::LD * gcro::LD;

void gcro_store_col(double2 *H, const double2 *hcol, const double *hn2, const double *nn, int j, int row0, int n,
                    cudaStream_t s) {
    k_gcro_store_col<<<ceil_div(n, 64), 64, 0, s>>>(H, hcol, hn2, nn, j, row0, n);
    MRHS_LAUNCHED("k_gcro_store_col");
}

void gcro_put_col(double2 *M, const double2 *d, int cnt, int row0, int col, int n, cudaStream_t s) {
    k_gcro_put_col<<<ceil_div(n, 64), 64, 0, s>>>(M, d, cnt, row0, col, n);
    MRHS_LAUNCHED("k_gcro_put_col");
}

void gcro_put_vec(double2 *v, const double2 *d, int cnt, int off, int n, cudaStream_t s) {
    k_gcro_put_vec<<<ceil_div(n, 64), 64, 0, s>>>(v, d, cnt, off, n);
    MRHS_LAUNCHED("k_gcro_put_vec");
}

void gcro_put_norm(double *un2, const double *nrm2, int i, int n, cudaStream_t s) {
    k_gcro_put_norm<<<ceil_div(n, 64), 64, 0, s>>>(un2, nrm2, i, n);
    MRHS_LAUNCHED("k_gcro_put_norm");
}

static void smem_attr(const void *kern) {
    MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGcroSmem));
}

void gcro_seed_small(const double2 *H, const double *beta2, int m, int k, double2 *Y, double2 *QC, double2 *PU,
                     int *err, int n, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        smem_attr(reinterpret_cast<const void *>(k_gcro_seed));
        attr = true;
    }
    k_gcro_seed<<<n, 32, kGcroSmem, s>>>(H, beta2, m, k, Y, QC, PU, err);
    MRHS_LAUNCHED("k_gcro_seed");
}

void gcro_cycle_small(const double2 *H, const double2 *B, const double *UN2, const double2 *WR, const double2 *WU,
                      int m, int k, double2 *Y, double2 *QC, double2 *PU, int *err, int n, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        smem_attr(reinterpret_cast<const void *>(k_gcro_cycle));
        attr = true;
    }
    k_gcro_cycle<<<n, 32, kGcroSmem, s>>>(H, B, UN2, WR, WU, m, k, Y, QC, PU, err);
    MRHS_LAUNCHED("k_gcro_cycle");
}

void gcro_coef_vec(double2 *coef, const double2 *v, int off, int cnt, double sign, int n, cudaStream_t s) {
    k_gcro_coef_vec<<<ceil_div(n, 64), 64, 0, s>>>(coef, v, off, cnt, sign, n);
    MRHS_LAUNCHED("k_gcro_coef_vec");
}

void gcro_coef_col(double2 *coef, const double2 *M, int off, int cnt, int col, double sign, int n, cudaStream_t s) {
    k_gcro_coef_col<<<ceil_div(n, 64), 64, 0, s>>>(coef, M, off, cnt, col, sign, n);
    MRHS_LAUNCHED("k_gcro_coef_col");
}

}  // namespace mrhs
