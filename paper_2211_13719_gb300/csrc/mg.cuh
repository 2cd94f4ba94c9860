// Multigrid hierarchy: levels, intergrid kernels, coarse stencil, setup.
#pragma once

#include <functional>
#include <map>
#include <memory>
#include <vector>

#include "internal.cuh"

namespace mrhs {

// Transfer from one level to the next and the operator of coarse levels.
struct Level {
    int L[4] = {1, 1, 1, 1};
    int64_t V = 0;
    int dof = 12;          // components per site (12 on the fine level, nc on coarse levels)
    // transfer to the next level (l < n_levels - 1)
    int B[4] = {1, 1, 1, 1};
    int N = 0;             // null vectors; the next level has nc = 2N
    int64_t asize = 0;     // sites per aggregate
    DeviceBuffer P32;      // [V][dof][N] chirally split, block-orthonormal vectors (FP32)
    DeviceBuffer P64;      // same in FP64 (kept for export)
    // coarse operator (l >= 1): 9-point stencil
    DeviceBuffer A32;      // [V][9][dof][dof] complex FP32
    DeviceBuffer Abf;      // tensor-core layout in BF16 (dof == 64), see coarse_tc.cu
    DeviceBuffer PhiBf;    // packed 16-bit input field of the tensor-core stencil
    DeviceBuffer TcErr;    // int: set by the tensor-core stencil when a bounded wait expired
    DeviceBuffer LinkScale;  // float [V]: per-site scale of the 16-bit links
    DeviceBuffer ColScale;   // float [64]: per-RHS scale of the packed input (max |component|)
    int tc_fmt = 0;          // MRHS_FP16 or MRHS_BF16 when the 16-bit links exist
    // tensor-core transfer to the next level (16-bit hierarchies): packed P tiles
    DeviceBuffer PA;         // prolongation A tiles [Vc][2][tiles] 128 x 64 FP16
    DeviceBuffer RB;         // restriction B tiles [Vc][2][chunks] 64 x 64 FP16
    DeviceBuffer RBlo;       // their FP16 rounding errors (split-precision restriction of the Galerkin build)
    DeviceBuffer IgErr;      // int: set when a tensor-core transfer gave up waiting
    DeviceBuffer IgBound;    // float [2][64]: ones (unit-norm inputs), then the column maxima of the last input
    bool tc_intergrid = false;
    // coarse even-odd decomposition (16-bit tensor-core levels with even extents):
    // inverse self blocks A_0(x)^-1 as 16-bit tiles [V] with a per-site scale
    DeviceBuffer AinvBf, AinvScale, EoErr;
    int64_t rows() const { return V * dof; }
};

// Term selection of the coarse stencil for the Galerkin construction.
struct StencilMask {
    int diag;   // include the d = 0 (self) block
    int dir;    // -1 all, else only direction d in 1..8
    int cross;  // 0 all; 1 only hops leaving the aggregate; 2 only hops staying inside
    int B[4];
};

// c = P^dagger psi: fine [V][dof][n] -> coarse [Vc][2N][n] (coarse site stride `ostride` complex)
void restrict_fields(const Level &f, const Level &c, const float2 *fine, float2 *coarse, int n,
                     int64_t ostride, cudaStream_t s);
// psi = P c
void prolong_fields(const Level &f, const Level &c, const float2 *coarse, float2 *fine, int n, cudaStream_t s);
// out = A in (or y - A in) with FP32 links; optional mask (setup)
void coarse_apply_fp32(const Level &c, const float2 *in, float2 *out, const float2 *y, int n, cudaStream_t s,
                       const StencilMask *mask = nullptr);
// BF16 tensor-core stencil (dof == 64): out = A in (or y - A in)
void coarse_apply_bf16(const Level &c, const float2 *in, float2 *out, const float2 *y, int n, cudaStream_t s);
bool coarse_bf16_supported(const Level &c);
// nonzero if a tensor-core stencil launch on this level gave up waiting (reads the
// flag after the work queued on s, synchronising s)
int coarse_tc_error(const Level &c, cudaStream_t s);
void coarse_links_to_16bit(Level &c, mrhs_precision fmt, cudaStream_t s);
// try_wait rounds of the first operand wait of the next tensor-core coarse launch on s:
// the normal bound, or 0 while mrhs_debug_expire_waits has eager launches left to expire
uint32_t tc_first_wait_limit(cudaStream_t s);
// Coarse even-odd decomposition (Sec. 6, M_eooe) on 16-bit tensor-core levels with
// even extents; half fields [V/2][64][n] hold the sites of one parity (site s at s / 2).
bool coarse_eo_supported(const Level &c);
// inverts every self block A_0(x) (FP64 Gauss-Jordan) and stores it as 16-bit tiles
void coarse_eo_prepare(Level &c, cudaStream_t s);
// out = H in (or y - H in): the 8 hop terms onto the sites of out_parity
void coarse_eo_hop(const Level &c, int out_parity, const float2 *in_half, float2 *out_half, const float2 *y_half,
                   int n, cudaStream_t s);
// out = A_0 in or A_0^-1 in on the sites of `parity`
void coarse_eo_self(const Level &c, bool inverse, int parity, const float2 *in_half, float2 *out_half, int n,
                    cudaStream_t s);
// out_o = D_hat in_o = A_oo in_o - H_oe A_ee^-1 H_eo in_o; tmp_e1, tmp_e2: even half fields
void coarse_schur_apply(const Level &c, const float2 *in_o, float2 *out_o, float2 *tmp_e1, float2 *tmp_e2, int n,
                        cudaStream_t s);
void coarse_parity_split(const Level &c, const float2 *full, float2 *he, float2 *ho, int n, cudaStream_t s);
void coarse_parity_merge_add(const Level &c, const float2 *he, const float2 *ho, float2 *full, int n,
                             cudaStream_t s);
// tensor-core restriction / prolongation (FP16, <= 32 null vectors, <= 64 RHS)
bool intergrid_tc_supported(const Level &f);
// packs the prolongation and restriction tiles once (a second call adds only what is missing);
// split: also the FP16 rounding errors of the restriction tiles
void intergrid_tc_prepare(Level &f, const Level &c, cudaStream_t s, bool split = false);
// unit_norm: every RHS column of `fine` has norm <= 1 (its components are then bounded by 1).
// split: every operand as the sum of two FP16 numbers, three MMA terms (FP32-level accuracy,
// for the Galerkin construction); needs intergrid_tc_prepare(..., split = true)
void restrict_fields_tc(const Level &f, const Level &c, const float2 *fine, float2 *coarse, int n, int64_t ostride,
                        bool unit_norm, cudaStream_t s, bool split = false);
void prolong_fields_tc(const Level &f, const Level &c, const float2 *coarse, float2 *fine, int n, cudaStream_t s);
int intergrid_tc_error(const Level &f, cudaStream_t s);
// FP64 modified Gram-Schmidt (twice) of the chiral halves of `vecs` per aggregate, in place
void block_orthonormalize(const Level &f, double2 *vecs, cudaStream_t s);
// P [V][dof][N] -> Pexp [V][dof][2N] with column K = chi*N + k nonzero only on chirality chi
void expand_chiral(const Level &f, const float2 *P, float2 *Pexp, cudaStream_t s);

// GCRO-DR small dense work per RHS (gcrodr.cu).  Per-RHS matrices are
// [n][17][17] double2 (row-major, leading dimension 17), vectors [n][17].
void gcro_store_col(double2 *H, const double2 *hcol, const double *hn2, const double *nn, int j, int row0, int n,
                    cudaStream_t s);
void gcro_put_col(double2 *M, const double2 *d, int cnt, int row0, int col, int n, cudaStream_t s);
void gcro_put_vec(double2 *v, const double2 *d, int cnt, int off, int n, cudaStream_t s);
void gcro_put_norm(double *un2, const double *nrm2, int i, int n, cudaStream_t s);
void gcro_seed_small(const double2 *H, const double *beta2, int m, int k, double2 *Y, double2 *QC, double2 *PU,
                     int *err, int n, cudaStream_t s);
void gcro_cycle_small(const double2 *H, const double2 *B, const double *UN2, const double2 *WR, const double2 *WU,
                      int m, int k, double2 *Y, double2 *QC, double2 *PU, int *err, int n, cudaStream_t s);
void gcro_coef_vec(double2 *coef, const double2 *v, int off, int cnt, double sign, int n, cudaStream_t s);
void gcro_coef_col(double2 *coef, const double2 *M, int off, int cnt, int col, double sign, int n, cudaStream_t s);

// The coarsest level's GMRES(m) cycle from x = 0 as one persistent cooperative kernel
// (coarsest_fused.cu): 16-bit tensor-core levels with 64 dof, <= 64 RHS, m <= 16, every
// CTA resident at once, each owning up to max_sites_per_cta sites.
struct CoarsestFused {
    int m = 0, nmax = 0, G = 0, S = 0;  // restart length, RHS bound, CTAs, sites per CTA
    DeviceBuffer part, npart, hcol, sig, R, cs, sn, g, y, sync;
    static size_t smem_bytes(int n);
    // CTAs of the kernel sized for nmax RHS that can be resident at once on `device` (0: no
    // tensor-core level or no cooperative launch); the kernel needs one per coarsest site
    static int resident_ctas(const Level &c, int nmax, int device);
    // sites one CTA can own: one tensor-memory accumulator each
    static int max_sites_per_cta(int nmax);
    static bool supported(const Level &c, int nmax, int m, int device);
    void init(const Level &c, int m, int nmax, int device);
    // x = GMRES_m(A_c) b on level c (x overwritten); Vbasis: m + 1 fields of workspace.
    // Uses the level's packed-input buffer and records expired waits in its TcErr.
    void solve(const Level &c, float2 *Vbasis, const float2 *b, float2 *x, int n, cudaStream_t s);
};

// Solver entry used by the C ABI and the server (solver.cu).
bool mg_solve(mrhs_mg &mg, const double2 *b, double2 *x, int n, const double *tols, double *rel_out,
              mrhs_solve_stats *st, cudaStream_t s, int max_outer,
              const std::function<bool(const double *, int)> &stop);
int mg_max_rhs(const mrhs_mg *mg);
int64_t mg_fine_rows(const mrhs_mg *mg);
int mg_device(const mrhs_mg *mg);
int mg_outer_m(const mrhs_mg *mg);

}  // namespace mrhs
