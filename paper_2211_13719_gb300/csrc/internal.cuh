// Internal declarations shared by the library's translation units.
#pragma once

#include <functional>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"

// ----------------------------------------------------------------- lattice
struct mrhs_lattice {
    mrhs::Geom g;
    int device = 0;
    // links, link-major SoA: element (mu*9 + a*3 + b) of site x at [(mu*9+a*3+b)*V + x]
    mrhs::DeviceBuffer U64, U32;
    // compact clover + mass, SoA: [(chi*18 + q)*V + x], q < 3 packs diagonal
    // pairs (d_{2q}, d_{2q+1}); q >= 3 is lower-triangle entry q - 3
    mrhs::DeviceBuffer C64, C32;
    // the same links and clover as float-float pairs (float4 per complex:
    // re hi, re lo, im hi, im lo) for the float-float operator
    mrhs::DeviceBuffer Udf, Cdf;
    // inverse of the site matrix C per site, same compact layout as C (for the
    // even-odd decomposition); CinvErr: int, set when a block was singular
    mrhs::DeviceBuffer Cinv64, Cinv32, CinvErr;
    // site-major FP32 copies for the paired-FP32 stencils at 16 RHS and more:
    // links [V][4][9], clover and its inverse [V][36] (entry chi * 18 + q)
    mrhs::DeviceBuffer U32a, C32a, Cinv32a;
    mrhs::DeviceBuffer EOtmp;  // half-lattice scratch of the Schur operator
    mrhs::DeviceBuffer SAPtmp; // full-lattice residual scratch of mrhs_sap_smooth
    bool has_gauge = false, has_clover = false;
    bool cinv_singular = false;  // a block of C was singular (no even-odd inverse)
    double mass = 0.0, csw = 0.0;
};

namespace mrhs {

// Autotuner: the variant (0 .. nvariants-1) to launch for this key; at the first
// eager call it runs launch(v) for every variant, timed with events on s.
int tune_pick(const char *kernel, const int dims[4], int n, int nvariants, const std::function<void(int)> &launch,
              cudaStream_t s);

// --------------------------------------------------------- fine operator
// Selection of terms for the Galerkin construction (setup only).
struct HopMask {
    int diag;   // include the clover + mass diagonal
    int dir;    // -1: all hops; else only stencil direction d in 1..8 (1+mu: +mu, 5+mu: -mu)
    int cross;  // 0: all selected hops; 1: only hops leaving the aggregate; 2: only hops staying in
    int B[4];   // aggregate extents
};

void gauge_to_soa(mrhs_lattice &lat, const double *aos_dev, cudaStream_t s);
// Even-odd decomposition, FP32, even n, half-lattice fields [V/2][12][n]
// (sites of one parity in lexicographic order, site s at index s / 2):
// out = H in from the other parity (M_eooe), and out_o = D_hat in_o =
// C_oo in_o - 1/4 H_oe C_ee^-1 H_eo in_o; clover_inverse_error: nonzero if a
// block of C was singular when the inverse was built.
void hop_eo(const mrhs_lattice &lat, int out_parity, const void *in, void *out, int n, cudaStream_t s);
// tmp_even: a half field of n RHS, overwritten
void schur_apply(const mrhs_lattice &lat, const void *in_odd, void *out_odd, int n, void *tmp_even, cudaStream_t s);
int clover_inverse_error(const mrhs_lattice &lat);
// even-odd solution pieces (FP32, even n): eo_supported tells whether the lattice
// and n allow them; eo_split: r (full) -> r_e, r_o, t_e = C_ee^-1 r_e (halves);
// eo_axpy_hop: out = self + 1/2 H in onto out_parity (cinv: C^-1 of that)
bool eo_supported(const mrhs_lattice &lat, int n);
void eo_split(const mrhs_lattice &lat, const void *r, void *re, void *ro, void *te, int n, cudaStream_t s);
// r = y - D x (FP32) straight into the halves r_e, r_o and te = C_ee^-1 r_e: the residual and
// eo_split in one pass, for 16, 24, 32, 48 or 64 RHS (false: not applicable, nothing launched)
bool residual_eo_split(const mrhs_lattice &lat, const void *x, const void *y, void *re, void *ro, void *te, int n,
                       cudaStream_t s);
void eo_axpy_hop(const mrhs_lattice &lat, int out_parity, const void *self, const void *in, void *out, bool cinv,
                 int n, cudaStream_t s);
// the smoother's last step in one pass: z_e += C_ee^-1 (r_e + 1/2 H_eo d_o), z_o += d_o;
// scratch_half: an even half field the autotuner may overwrite
void eo_cinv_axpy_hop_merge(const mrhs_lattice &lat, const void *r_e, const void *d_o, void *z, void *scratch_half,
                            int n, cudaStream_t s);
// SAP smoother (FP32, even n): `cycles` cycles of the block-coloured Schwarz
// alternating procedure for D z = v, each block system by `mr_steps` MR steps
// in shared memory; r_tmp: a full FP32 field of n RHS, overwritten.
// sap_supported tells whether the lattice, block extents and n allow it.
bool sap_supported(const mrhs_lattice &lat, const int B[4], int n);
void sap_smooth(const mrhs_lattice &lat, const void *v, void *z, int n, const int B[4], int cycles, int mr_steps,
                void *r_tmp, cudaStream_t s);
// dst[i] = (hi, lo) float pairs of the FP64 complex src[i], i < count
void split_df(const void *src_c128, void *dst_f4, int64_t count, cudaStream_t s);
// out = D in (y == nullptr) or y - D in; `in` FP32, out and y FP64, float-float arithmetic
void dslash_df(const mrhs_lattice &lat, const void *in, void *out, const void *y, int n, cudaStream_t s);
void build_clover(mrhs_lattice &lat, double mass, double csw, cudaStream_t s);
// One problem of a fused batch: out = D in (y == nullptr) or y - D in, FP32
// fields [V][12][n] of lattice `lat`.
struct BatchItemHost {
    const mrhs_lattice *lat;
    const void *in;
    void *out;
    const void *y;
    int n;
};
// The fine operator on up to 8 problems of different volumes and RHS counts
// (same device) in one persistent launch.
void dslash_batch(const BatchItemHost *items, int count, cudaStream_t s);
// out = D in (y == nullptr) or out = y - D in; compute in `compute` precision,
// input in `in_prec` (FP32 input allowed with FP64 compute); out and y in `compute`.
void dslash(const mrhs_lattice &lat, mrhs_precision compute, mrhs_precision in_prec,
            const void *in, void *out, const void *y, int n, cudaStream_t s,
            const HopMask *mask = nullptr);

// ------------------------------------------------------------------ BLAS
// Reduction scratch: per-block partial sums and a completion counter.
struct Scratch {
    DeviceBuffer partials;   // double2 [max_blocks][kchunk][n]
    DeviceBuffer counter;    // unsigned int
    int max_blocks = 0;
    int max_cols = 0;        // kchunk * n capacity per block
    void ensure(int blocks, int cols);
};

constexpr int KCHUNK = 8;  // basis vectors per multi-dot pass

void multi_dot(mrhs_precision p, const void *basis, int64_t stride, int k, const void *w,
               int64_t rows, int n, double2 *out, Scratch &sc, cudaStream_t s, bool accumulate = false);
void norm2(mrhs_precision p, const void *w, int64_t rows, int n, double *out, Scratch &sc, cudaStream_t s);
// *flag = 0 if all `bytes` bytes at p (a multiple of 16, 16-byte aligned) are zero, else nonzero
void any_nonzero(const void *p, int64_t bytes, unsigned *flag, cudaStream_t s);
// multi_dot with caller-provided reduction scratch: `partials` holds at least
// (max_blocks + ceil(max_blocks / 32)) * KCHUNK * n double2, `counter` holds
// 64 unsigned ints that are zero on entry (the kernel leaves them zero);
// the grid is capped at max_blocks (at most 2016).
void multi_dot_fixed_scratch(mrhs_precision p, const void *basis, int64_t stride, int k, const void *w, int64_t rows,
                             int n, double2 *out, double2 *partials, unsigned int *counter, int max_blocks,
                             cudaStream_t s);
// w += alpha * sum_j coef[j][r] basis_j ; basis may be FP32 while w is FP64.
// If norm_out != nullptr, also writes ||w_new||^2 per RHS (needs sc).
void lincomb(mrhs_precision pw, void *w, mrhs_precision pb, const void *basis, int64_t stride, int k,
             const double2 *coef, double alpha, int64_t rows, int n, cudaStream_t s,
             double *norm_out = nullptr, Scratch *sc = nullptr);
// dst = src / sqrt(nrm2[r]) (0 where nrm2 == 0); dst may equal src
void scale_inv_sqrt(mrhs_precision p, void *dst, const void *src, const double *nrm2, int64_t rows, int n,
                    cudaStream_t s);
// device-to-device copy by a kernel (bytes a multiple of 4), never queued behind the copy engines
void copy_on_sms(void *dst, const void *src, size_t bytes, cudaStream_t s);
// zero `bytes` (a multiple of 4) of device memory by a kernel
void zero_on_sms(void *dst, size_t bytes, cudaStream_t s);
// device -> page-locked host memory (cudaMallocHost) by a kernel; the caller synchronises s
void read_back(void *pinned_host, const void *dev, size_t bytes, cudaStream_t s);
// a page-locked int[4] of the calling host thread, for flag read-backs
int *pinned_flag_slot();
// dst (pd) = src (ps) elementwise conversion
void cast(mrhs_precision pd, void *dst, mrhs_precision ps, const void *src, int64_t count, cudaStream_t s);
// y = a*x + y with real a, same precision
void axpy(mrhs_precision p, double a, const void *x, void *y, int64_t count, cudaStream_t s);
// x *= a (real a)
void scale_real(mrhs_precision p, double a, void *x, int64_t count, cudaStream_t s);

// ----------------------------------------------- per-RHS small Krylov state
// Hessenberg / Givens state for n RHS and restart length m (device arrays).
struct KrylovState {
    int m = 0, n = 0;
    DeviceBuffer R;      // double2 [n][m+1][m] rotated Hessenberg (upper triangular part)
    DeviceBuffer cs;     // double  [n][m]
    DeviceBuffer sn;     // double2 [n][m]
    DeviceBuffer g;      // double2 [n][m+1]
    DeviceBuffer y;      // double2 [m][n]  (layout of lincomb coefficients)
    DeviceBuffer hcol;   // double2 [m+1][n] current Arnoldi column (pass 1 + pass 2)
    DeviceBuffer h2;     // double2 [m+1][n] second-pass coefficients
    DeviceBuffer hn2;    // double  [n]      ||w||^2 after orthogonalisation
    DeviceBuffer nrm2w;  // double  [n]      ||w||^2 before orthogonalisation (single-pass scheme)
    DeviceBuffer nn;     // double  [n]      ||v_{j+1}||^2 after normalisation (single-pass scheme)
    DeviceBuffer beta2;  // double  [n]      ||r0||^2
    DeviceBuffer res;    // double  [n]      current residual estimate |g_{j+1}|
    void init(int m_, int n_);
};
// g = (sqrt(beta2), 0, ...), clears rotations
void krylov_start(KrylovState &ks, int n, cudaStream_t s);
// fold column j (hcol[0..j] (+ h2 for two-pass Gram-Schmidt), hn2) into R with
// Givens rotations; updates g, res.  single_pass: h2 unused, beta corrected by nn.
void krylov_givens(KrylovState &ks, int j, int n, cudaStream_t s, bool single_pass = false);
// One Gram-Schmidt step against an orthonormal basis in two passes over the data:
// h = V^H w and ||w||^2 together, then w <- (w - V h) / beta with
// beta^2 = ||w||^2 - |h|^2 (hn2 <- beta^2), nn <- ||w_new||^2, and a fix-up that
// rescales columns whose new norm is off by more than 1% (cancellation).
// need_vector false: only h, ||w||^2, hn2 (Pythagoras) and nn = 1 -- for a last step
// whose new basis vector is never read; w is left as it was.
void orthonormalize_step(mrhs_precision p, const void *basis, int64_t stride, int k, void *w, int64_t rows, int n,
                         double2 *h, double *nrm2, double *hn2, double *nn, Scratch &sc, cudaStream_t s,
                         bool need_vector = true);
// y = R^{-1} g for the first `j` columns
void krylov_solve(KrylovState &ks, int j, int n, cudaStream_t s);

// -------------------------------------------------------------- RNG
// Gaussian complex numbers from splitmix64 (Steele, Lea, Flood, OOPSLA 2014)
// + Box-Muller; deterministic in (seed, index).
void fill_gaussian(mrhs_precision p, void *dst, int64_t count, uint64_t seed, cudaStream_t s);

}  // namespace mrhs
