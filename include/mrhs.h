/*
 * mrhs.h - C ABI of the GB300 multiple-right-hand-side (MRHS) multigrid
 * solver for the Wilson-clover Dirac equation (arXiv:2211.13719).
 *
 * The library solves D x = b for many right-hand sides (RHS) at once on one
 * GPU (Sec. 1-2 of the paper: MRHS turns the many independent solves into
 * one batched solve, reusing every gauge link and coarse link for all RHS).
 *
 * Conventions used by every call below
 * ------------------------------------
 * Lattice        dims = {Lx, Ly, Lz, Lt}; site index x + Lx*(y + Ly*(z + Lz*t)).
 * Gauge field    [V][4][3][3] complex, interleaved (re, im); U[x][mu] is the
 *                link from x to x + mu_hat, mu = 0..3 = x, y, z, t.
 * Spinor fields  [V][12][nrhs] complex, component s*3 + c (spin s, colour c),
 *                RHS index innermost (Sec. 2: one link load serves all RHS).
 * Gamma basis    chiral: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *                gamma_t = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).
 * Operator       D = (4 + m) - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) delta_{x+mu}
 *                    + (1 + gamma_mu) U_mu(x - mu)^dagger delta_{x-mu}]
 *                    + c_sw (i/4) sum_{mu nu} sigma_{mu nu} F_{mu nu}(x)
 *                (Sec. 4 hopping and clover terms), F from the clover leaf
 *                (Q - Q^dagger)/8, sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu].
 * Coarse fields  [Vc][nc][nrhs] complex, nc = 2 * (number of null vectors),
 *                coarse dof K = chi*N + k with chi = 0 for the upper spins
 *                (Sec. 5: "nbasis" is twice the number of basis vectors).
 * Coarse links   [Vc][9][nc][nc] complex; block d = 0 self, 1 + mu for the
 *                neighbour at +mu, 5 + mu for the neighbour at -mu (Sec. 6).
 * Complex        float2 / double2 (interleaved), bf16 pairs where stated.
 *
 * Pointers named *_dev are device pointers owned by the caller; *_host are
 * host pointers owned by the caller.  Handles (mrhs_lattice, mrhs_mg,
 * mrhs_server) own every device buffer they allocate (gauge field, clover
 * term, MG hierarchy, Krylov workspace) until destroyed.  `stream` is a
 * cudaStream_t passed as void* (NULL = the legacy default stream); kernels are
 * enqueued on it and the call returns without synchronising unless stated.
 *
 * Errors: every call returns an mrhs_status and never aborts.  Arguments are
 * validated on the host before any launch; a failed CUDA call returns
 * MRHS_ERR_CUDA.  mrhs_last_error() gives a message for the calling thread.
 * There is no CPU fallback: without a usable CUDA device every call that
 * needs one fails with MRHS_ERR_CUDA.
 */
#ifndef MRHS_H
#define MRHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MRHS_OK = 0,
    MRHS_PENDING = 1,
    MRHS_ERR_INVALID = -1,
    MRHS_ERR_OOM = -2,
    MRHS_ERR_CUDA = -3,
    MRHS_ERR_NOT_CONVERGED = -4,
    MRHS_ERR_TIMEOUT = -5,
    MRHS_ERR_BUSY = -6,
    MRHS_ERR_NOT_FOUND = -7
} mrhs_status;

typedef enum {
    MRHS_FP32 = 0,
    MRHS_FP64 = 1,
    MRHS_BF16 = 2,
    MRHS_FP16 = 3,
    /* float-float: each real carried as an unevaluated sum of two floats
     * (48 significant bits), evaluated on the FP32 units; only for the fine
     * operator, which then reads an FP32 field and writes an FP64 field */
    MRHS_DF64 = 4
} mrhs_precision;

typedef struct mrhs_lattice mrhs_lattice;
typedef struct mrhs_mg mrhs_mg;
typedef struct mrhs_server mrhs_server;

#define MRHS_MAX_LEVELS 3

/* Message of the last failed call on this thread ("" if none). */
const char *mrhs_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (a replayed CUDA graph counts its kernel nodes).  Diagnostic only. */
uint64_t mrhs_kernel_launch_count(void);

/* Event timing of one kernel, for measurement harnesses (no effect on any
 * result).  After mrhs_kernel_timer_start(name), every launch of the kernel
 * `name` ("k_dslash_x2", "k_eo_x2", "k_sap_mr", "k_dslash", "k_dots_norm", "k_lincomb_scale",
 * "k_lincomb", "k_multi_dot", "k_norm2", "k_restrict_tc", "k_prolong_tc",
 * "k_coarse_tc") that is not being captured into a CUDA graph is bracketed by
 * two CUDA events recorded on its launching stream; launches captured into a
 * graph are only counted.  mrhs_kernel_timer_stop waits for the recorded
 * events, writes the summed event time of the timed launches (ms), their
 * number and the number of captured launches (each pointer may be NULL), and
 * ends the timing.  One timing at a time: start while one is active, or stop
 * while none is, returns MRHS_ERR_INVALID.  The events are created on the
 * device current at the launch. */
mrhs_status mrhs_kernel_timer_start(const char *kernel_name);
mrhs_status mrhs_kernel_timer_stop(double *total_ms, int64_t *timed_launches, int64_t *captured_launches);

/* Autotuner (no counterpart in the paper; it only changes how work is mapped
 * onto the GPU, never an output value).  Kernels with launch variants (the
 * site-tile shapes of the FP32 fine and even-odd stencils) time every variant
 * with CUDA events on their stream at the first eager launch for a (kernel,
 * lattice extents, nrhs) key and keep the fastest for the process (the
 * default variant 0 unless another is more than 3 % faster); a launch
 * made while its stream is captured into a CUDA graph never tunes (cached
 * choice or the default variant 0).  Tuning is on unless the environment sets
 * MRHS_AUTOTUNE=0 or mrhs_tune_set_enabled(0) is called.  mrhs_tune_save /
 * mrhs_tune_load write / read the cache as text lines "kernel Lx Ly Lz Lt nrhs
 * variant nvariants best_ms default_ms" (a load keeps the lines before a
 * malformed one and returns MRHS_ERR_INVALID; a missing file gives
 * MRHS_ERR_NOT_FOUND). */
typedef struct {
    char kernel[32];
    int dims[4];
    int nrhs;
    int variant;       /* chosen variant, 0 = default            */
    int nvariants;
    float best_ms;     /* event time per launch of the choice    */
    float default_ms;  /* event time per launch of variant 0     */
} mrhs_tune_entry;
void mrhs_tune_set_enabled(int enabled);
void mrhs_tune_clear(void);
int mrhs_tune_count(void);
mrhs_status mrhs_tune_get(int index, mrhs_tune_entry *out);
mrhs_status mrhs_tune_save(const char *path);
mrhs_status mrhs_tune_load(const char *path);

/* ------------------------------------------------------------------ */
/* Lattice, gauge field, clover term                                   */
/* ------------------------------------------------------------------ */

/* Create a lattice on CUDA device `device`.  dims[mu] >= 1.  t_boundary is
 * +1 (periodic) or -1 (antiperiodic fermion boundary in t: every hop that
 * crosses t = Lt-1 <-> 0 gets a factor -1).  Paper: Sec. 4 (operator). */
mrhs_status mrhs_create_lattice(const int dims[4], int t_boundary, int device,
                                mrhs_lattice **out);
void mrhs_destroy_lattice(mrhs_lattice *lat);

/* Copy the gauge field (host, FP64, layout above) to the device; the
 * library keeps FP64 and FP32 copies in its own link-major layout. */
mrhs_status mrhs_load_gauge(mrhs_lattice *lat, const double *U_host);

/* Build the clover term from the clover-leaf field strength (Sec. 4, the
 * "compact" clover: two Hermitian 6x6 blocks per site in the chiral basis)
 * with the mass folded into its diagonal: 4 + m + c_sw (i/4) sigma F.
 * Requires a loaded gauge field. */
mrhs_status mrhs_build_clover(mrhs_lattice *lat, double mass, double csw);

/* Copy the compact clover term to the host: [V][2][36] doubles; per
 * chirality block the 6 diagonal reals, then the 15 strictly-lower
 * entries (row i > col j, order i*(i-1)/2 + j) as (re, im); component
 * index within a block is s_local*3 + c. */
mrhs_status mrhs_get_clover(mrhs_lattice *lat, double *clover_host);

/* out_dev = D in_dev for nrhs >= 1 RHS (Sec. 4: hopping + clover fused),
 * both [V][12][nrhs] complex in precision `prec` (MRHS_FP32 or MRHS_FP64);
 * with MRHS_DF64 in_dev is FP32 and out_dev FP64, computed in float-float
 * arithmetic (within about 2^-48 of the largest term of each sum).
 * in and out must not overlap. */
mrhs_status mrhs_apply_D(mrhs_lattice *lat, const void *in_dev, void *out_dev,
                         int nrhs, mrhs_precision prec, void *stream);

/* out_dev = y_dev - D in_dev (the fused residual used by the solvers). */
mrhs_status mrhs_residual_D(mrhs_lattice *lat, const void *in_dev, const void *y_dev,
                            void *out_dev, int nrhs, mrhs_precision prec, void *stream);

/* One problem of a fused batch: out = D in (y_dev NULL) or out = y - D in,
 * FP32 device fields [V][12][nrhs] of `lat` (layout of mrhs_apply_D). */
typedef struct {
    mrhs_lattice *lat;
    const void *in_dev;
    void *out_dev;
    const void *y_dev;      /* NULL or FP32 [V][12][nrhs] */
    int nrhs;               /* 1..256 (the fused kernel compiles 16/24/32/48/64) */
} mrhs_apply_item;

/* The FP32 fine operator (hop + clover + axpy of the residual form, Sec. 4)
 * on 1..8 problems of different lattice volumes and RHS counts in one
 * persistent launch: the problems' work is concatenated and one occupancy
 * wave of CTAs walks it, so small or uneven MRHS blocks share the GPU
 * instead of each paying a launch and a partial wave.  Every output equals
 * the single-problem mrhs_apply_D / mrhs_residual_D result of the same
 * problem (the same arithmetic per element).  All lattices on one device;
 * out must not alias in.  MRHS_ERR_INVALID on bad counts or arguments. */
mrhs_status mrhs_apply_D_batch(const mrhs_apply_item *items, int count, void *stream);


/* Even-odd decomposition (Sec. 4, M_eooe: the hopping term between the
 * checkerboarded lattices).  Half-lattice fields are [V/2][12][nrhs] complex
 * FP32 holding the sites of one parity p = (x + y + z + t) mod 2 in
 * increasing lexicographic order (site s at index s / 2).  All four lattice
 * extents must be even and nrhs even (MRHS_ERR_INVALID otherwise); in and out
 * must not overlap and be 16-byte aligned.  With D = C - 1/2 H (C the clover +
 * mass term, H the hopping term):
 * mrhs_apply_hop_eo: out_dev (parity out_parity) = H in_dev (the other parity),
 *   without the -1/2 factor.
 * mrhs_apply_schur: out_o = D_hat in_o = C_oo in_o - 1/4 H_oe C_ee^-1 H_eo in_o,
 *   the Schur complement of D on the odd sites.  C^-1 is built by
 *   mrhs_build_clover (FP64 Gauss-Jordan per 6x6 chirality block); if a block is
 *   singular the call fails with MRHS_ERR_INVALID.  Uses a half-lattice scratch
 *   field owned by the lattice (allocated on first use). */
mrhs_status mrhs_apply_hop_eo(mrhs_lattice *lat, int out_parity, const void *in_dev, void *out_dev, int nrhs,
                              void *stream);
mrhs_status mrhs_apply_schur(mrhs_lattice *lat, const void *in_dev, void *out_dev, int nrhs, void *stream);

/* SAP smoother (Schwarz alternating procedure; the smoother the paper's
 * Sec. 9 outlook names next), FP32 fields [V][12][nrhs], z_dev updated in
 * place: `cycles` SAP cycles for D z = v.  The lattice is cut into blocks of
 * extents block[4] (each dividing the lattice extent an even number of
 * times; at most 256 sites per block) coloured by block parity
 * (sum_mu x_mu / block_mu) mod 2; per cycle, for colour 0 then 1: r = v - D z,
 * then z += e with e_B approximating D_BB^{-1} r_B on every block of that
 * colour by `mr_steps` minimal-residual steps from zero with inner products
 * over the block (D_BB: D with the hops that leave the block dropped).
 * nrhs even; v, z 16-byte aligned and not overlapping (MRHS_ERR_INVALID
 * otherwise).  Uses a full-lattice residual field owned by the lattice
 * (allocated on first use). */
mrhs_status mrhs_sap_smooth(mrhs_lattice *lat, const void *v_dev, void *z_dev, int nrhs, const int block[4],
                            int cycles, int mr_steps, void *stream);

/* ------------------------------------------------------------------ */
/* Batched BLAS-1 over the RHS index (Sec. 7, "simultaneous" inner      */
/* products).  A field is `rows` rows of `nrhs` complex values, RHS     */
/* innermost (rows = sites * dof).  Results are complex double (double2) */
/* on the device, one per RHS; sums run in a fixed order per RHS.       */
/* ------------------------------------------------------------------ */

/* out_dev[j*nrhs + r] = sum_i conj(basis_j[i][r]) w[i][r] for j < k, where
 * basis_j = basis_dev + j * rows * nrhs (k fields stored back to back). */
mrhs_status mrhs_blas_multi_dot(const void *basis_dev, int k, const void *w_dev,
                                int64_t rows, int nrhs, mrhs_precision prec,
                                void *out_dev, void *stream);

/* out_dev[r] = sum_i |w[i][r]|^2 (double, one per RHS). */
mrhs_status mrhs_blas_norm2(const void *w_dev, int64_t rows, int nrhs,
                            mrhs_precision prec, double *out_dev, void *stream);

/* w[i][r] += alpha * sum_j coef[j*nrhs + r] * basis_j[i][r]  (coef: double2). */
mrhs_status mrhs_blas_lincomb(void *w_dev, const void *basis_dev, int k,
                              const void *coef_dev, double alpha, int64_t rows,
                              int nrhs, mrhs_precision prec, void *stream);

/* The paper has no counterpart to this entry point.  It computes exactly
 * what mrhs_blas_multi_dot computes, for callers that must not allocate
 * device memory while they run (code being recorded into a CUDA graph,
 * hosts that reserve all device memory up front, programs whose memory
 * belongs to another allocator): it never calls cudaMalloc or cudaFree.
 * Its reduction scratch is a statically allocated 4.1 MiB device array shared
 * by all calls; nrhs is limited to 1..64 (MRHS_ERR_INVALID beyond).  Every
 * call looks the array up (cudaGetSymbolAddress, no allocation) on the
 * caller's current device, so a device reset does not leave a stale address.
 * The first call on a device may load the library's module there: make it
 * before any stream capture.  Calls that overlap on the GPU race on the
 * shared scratch; order them on one stream. */
mrhs_status mrhs_blas_multi_dot_noalloc(const void *basis_dev, int k, const void *w_dev,
                                        int64_t rows, int nrhs, mrhs_precision prec,
                                        void *out_dev, void *stream);

/* ------------------------------------------------------------------ */
/* Multigrid hierarchy                                                  */
/* ------------------------------------------------------------------ */

typedef struct {
    int n_levels;                          /* 2 or 3                              */
    int block[MRHS_MAX_LEVELS - 1][4];     /* aggregate extents, level l -> l+1   */
    int n_vec[MRHS_MAX_LEVELS - 1];        /* null vectors N (nc = 2N), even <= 64 */
    int setup_sweeps;                      /* GMRES cycles on A v = 0 per vector  */
    int setup_m;                           /* their restart length                */
    int smooth_m;                          /* post-smoothing GMRES iterations     */
    int coarse_m;                          /* coarsest GMRES restart length       */
    int coarse_cycles;                     /* coarsest GMRES cycles per V-cycle   */
    int inter_m;                           /* intermediate FGMRES iterations      */
    int inner_m;                           /* FP32 MG-FGMRES restart length       */
    int inner_max_iters;                   /* FP32 MG-FGMRES iteration cap        */
    double inner_tol;                      /* FP32 inner relative tolerance       */
    int outer_m;                           /* FP64 outer FGMRES restart length    */
    int max_outer_iters;                   /* FP64 outer iteration cap            */
    int coarse_precision;                  /* MRHS_FP32, MRHS_FP16 or MRHS_BF16   */
    int max_rhs;                           /* largest nrhs a solve may use        */
    int use_graph;                         /* replay the V-cycle as a CUDA graph  */
    int outer_op_precision;                /* outer Arnoldi applies D z: MRHS_DF64
                                              (float-float) or MRHS_FP64; the
                                              true residual is always FP64        */
    int smoother_evenodd;                  /* 1: the fine post-smoother runs GMRES on
                                              the even-odd Schur complement D_hat
                                              (even extents and nrhs; otherwise,
                                              and with 0, GMRES on D)             */
    uint64_t seed;                         /* start vectors when none supplied    */
    /* Optional host start vectors per level, [V_l][dof_l][n_vec[l]] complex
     * FP64 (dof_0 = 12, dof_l = nc of level l).  NULL entries: random. */
    const double *init_vecs[MRHS_MAX_LEVELS - 1];
    int smoother_sap;                      /* 1: the fine post-smoother is sap_cycles
                                              SAP cycles (mrhs_sap_smooth) instead
                                              of GMRES; takes precedence over
                                              smoother_evenodd where SAP applies  */
    int sap_block[4];                      /* SAP block extents                   */
    int sap_cycles;                        /* SAP cycles per post-smoothing       */
    int sap_mr;                            /* MR steps per SAP block solve        */
    int coarse_smoother_evenodd;           /* 1: intermediate levels post-smooth with
                                              smooth_m GMRES steps on the coarse
                                              even-odd Schur complement (16-bit
                                              tensor-core levels with even extents;
                                              otherwise GMRES on the level operator) */
    int coarse_solver;                     /* coarsest level: 0 GMRES(coarse_m),
                                              1 GCRO-DR(coarse_m, coarse_recycle)
                                              with a recycle space kept per RHS
                                              from one V-cycle to the next
                                              (coarse_m <= 16)                    */
    int coarse_recycle;                    /* GCRO-DR recycle vectors k < coarse_m */
    int coarse_fused;                      /* 1: the coarsest GMRES cycle runs as one
                                              persistent cooperative kernel (16-bit
                                              tensor-core coarsest level with 64 dof,
                                              coarse_m <= 16, every coarsest site's
                                              CTA resident); else, and with 0, one
                                              launch per operation                */
    int galerkin_tc;                       /* the restriction R = P^dagger of the
                                              Galerkin build R D P: on the tensor
                                              cores with every operand split into two
                                              FP16 numbers, three MMA terms, FP32
                                              accumulation (<= 32 null vectors; the
                                              links to about 1e-5 relative) -- 1: on
                                              16-bit hierarchies, whose links are
                                              rounded to 16 bits afterwards; 2: on
                                              every hierarchy; 0: never (CUDA cores,
                                              FP32)                                */
} mrhs_mg_params;

/* Fill `p` with the defaults used for the 24^3x64 three-level workload. */
void mrhs_mg_default_params(mrhs_mg_params *p);

/* Build the hierarchy (Sec. 5 prolongators, Sec. 6 coarse operators):
 * null vectors relaxed in FP32, chirally split and block-orthonormalised in
 * FP64, Galerkin coarse links R D P, cast to the coarse precision.  The
 * lattice must have gauge + clover and must outlive the hierarchy. */
mrhs_status mrhs_setup_mg(mrhs_lattice *lat, const mrhs_mg_params *params,
                          mrhs_mg **out);
void mrhs_destroy_mg(mrhs_mg *mg);

/* Level geometry: dims of level `level` (0 = fine) and its dof per site. */
mrhs_status mrhs_mg_level_info(mrhs_mg *mg, int level, int dims[4], int *dof);

/* Copy the block-orthonormalised, chirally split null vectors of level
 * `level` -> level+1 to the host: [V_l][dof_l][N] complex FP64.  Column
 * (chi, k) of the prolongator is this array restricted to the components
 * of chirality chi and to one aggregate. */
mrhs_status mrhs_mg_get_prolongator(mrhs_mg *mg, int level, double *host_out);

/* Copy the coarse links of level `level` (>= 1) to the host as FP64,
 * [Vc][9][nc][nc] complex (Sec. 6 stencil, layout above). */
mrhs_status mrhs_mg_get_coarse_links(mrhs_mg *mg, int level, double *host_out);

/* Restriction c = P^dagger psi from level `level` to level+1 (Sec. 5),
 * FP32 fields (level-l layout in, coarse layout out).  Hierarchies built
 * with coarse_precision FP16 or BF16 compute it on the tensor cores (FP16
 * operands scaled per RHS, FP32 accumulation, nrhs <= 64); FP32 hierarchies
 * on CUDA cores. */
mrhs_status mrhs_restrict(mrhs_mg *mg, int level, const void *fine_dev,
                          void *coarse_dev, int nrhs, void *stream);
/* The tensor-core forms of mrhs_restrict, mrhs_prolong and mrhs_coarse_apply,
 * and mrhs_vcycle, read the kernels' bounded-wait flag after the launch, so
 * they return only after their GPU work on `stream` is done; a wait that
 * gave up (an operand copy that never landed) returns MRHS_ERR_TIMEOUT and
 * clears the flag, the output then being incomplete. */

/* Prolongation psi = P c from level+1 to level `level` (Sec. 5), FP32
 * fields, on the tensor cores or CUDA cores as for mrhs_restrict. */
mrhs_status mrhs_prolong(mrhs_mg *mg, int level, const void *coarse_dev,
                         void *fine_dev, int nrhs, void *stream);

/* Coarse 9-point stencil out = D_c in on level `level` >= 1 (Sec. 6), FP32
 * fields; links_prec MRHS_FP32 (CUDA cores) or the level's 16-bit tensor-core
 * format MRHS_FP16 / MRHS_BF16 (FP32 accumulation; requires nc = 64 and the
 * hierarchy built with that coarse_precision).  The 16-bit path stores each
 * site's links scaled by their largest component and packs the input with
 * one scale per RHS column, so FP16 neither overflows nor underflows. */
mrhs_status mrhs_coarse_apply(mrhs_mg *mg, int level, const void *in_dev, void *out_dev,
                              int nrhs, mrhs_precision links_prec, void *stream);

/* Coarse even-odd Schur complement (Sec. 6, coarse M_eooe) on level `level`
 * (>= 1, a 16-bit tensor-core level with even extents, prepared at setup with
 * coarse_smoother_evenodd = 1): out_o = D_hat in_o = A_oo in_o - H_oe A_ee^-1
 * H_eo in_o, with A the 9-point stencil's self blocks and H its hops, on odd
 * half fields [Vc/2][64][nrhs] FP32 (the odd sites in lexicographic order).
 * A_ee^-1 is inverted per site in FP64 at setup and applied, like A and H, on
 * the tensor cores in the level's 16-bit format with FP32 accumulation.
 * Allocates two even half fields of scratch per call; returns after the work
 * on `stream` (it reads the kernels' bounded-wait flag). */
mrhs_status mrhs_coarse_apply_schur(mrhs_mg *mg, int level, const void *in_dev, void *out_dev, int nrhs,
                                    void *stream);

/* The coarsest level's solve as the V-cycle runs it: coarse_cycles cycles
 * of GMRES(coarse_m), or of GCRO-DR(coarse_m, coarse_recycle) with
 * coarse_solver = 1 (Sec. 9 outlook: a recycling coarsest solver), from
 * x = 0, on FP32 coarsest-level fields [Vc][nc][nrhs].  GCRO-DR keeps one
 * recycle space per RHS column in the hierarchy: a solve enters with the
 * space the previous solve (or V-cycle) left, and mrhs_coarsest_reset
 * drops it.  The per-RHS small dense work (least squares, harmonic Ritz
 * eigenproblem, QR) runs in FP64 on the device.  Returns after the work on
 * `stream`; MRHS_ERR_CUDA if a harmonic Ritz eigenproblem did not converge. */
mrhs_status mrhs_coarsest_solve(mrhs_mg *mg, const void *b_dev, void *x_dev, int nrhs, void *stream);
mrhs_status mrhs_coarsest_reset(mrhs_mg *mg);
/* Setup time of the transfer level -> level + 1 (milliseconds, CUDA events
 * on the setup stream, recorded by mrhs_setup_mg): [0] null-vector
 * relaxation (Sec. 5, the N vectors as N right-hand sides), [1] chiral split
 * and FP64 block orthonormalisation, [2] Galerkin coarse operator (Sec. 6),
 * [3] 16-bit links, tensor-core transfer tiles and coarse even-odd inverses.
 * MRHS_ERR_INVALID unless 0 <= level < n_levels - 1. */
mrhs_status mrhs_mg_setup_times(mrhs_mg *mg, int level, double out_ms[4]);

/* Whether the coarsest solve runs as the persistent kernel (coarse_fused):
 * *in_use 1 if it does; *resident_ctas the kernel's CTAs that fit on the
 * device at once (one per SM: it holds tensor memory; 0 without a 16-bit
 * tensor-core coarsest level); *sites the coarsest level's sites, which the
 * CTAs share, up to 2 each (each staged in shared memory). */
mrhs_status mrhs_coarsest_fused_info(mrhs_mg *mg, int *in_use, int *resident_ctas, int *sites);

/* One MG V-cycle z = M^{-1} v on the fine level (Sec. 8 preconditioner),
 * FP32 fields [V][12][nrhs]. */
mrhs_status mrhs_vcycle(mrhs_mg *mg, const void *v_dev, void *z_dev, int nrhs, void *stream);

typedef struct {
    int outer_iters;        /* FP64 FGMRES iterations                          */
    int inner_iters;        /* FP32 MG-FGMRES iterations, summed               */
    int vcycles;            /* V-cycles applied                                */
    double seconds;         /* wall time of the solve                          */
    double t_fine;          /* fine-level smoother + fine FP32 applies (s)     */
    double t_restrict;      /* restriction (s)                                 */
    double t_prolong;       /* prolongation (s)                                */
    double t_coarse;        /* coarse-level solves (s)                         */
    double t_outer;         /* FP64 outer work: residuals, Arnoldi (s)         */
    double max_rel_residual;/* max over RHS of ||b - D x|| / ||b||, FP64 D     */
} mrhs_solve_stats;

/* Solve D x = b for nrhs <= max_rhs RHS to a relative true residual `tol`
 * (checked with the FP64 operator).  b_dev, x_dev: FP64 device fields
 * [V][12][nrhs]; x_dev is the start vector on entry (set it to zero for a
 * cold start) and the solution on exit.  rel_res_host (optional, [nrhs])
 * receives each RHS's final relative residual.  Synchronises `stream`.
 * Returns MRHS_ERR_NOT_CONVERGED (x = best iterate) if the outer cap is
 * reached first.  Component timing in `stats` (optional) follows the
 * breakdown of the paper's Sec. 8 table. */
mrhs_status mrhs_solve(mrhs_mg *mg, const void *b_dev, void *x_dev, int nrhs, double tol,
                       double *rel_res_host, mrhs_solve_stats *stats, void *stream);
/* A solve also returns MRHS_ERR_TIMEOUT when a tensor-core kernel's bounded
 * mbarrier wait gave up (the flags are read after every inner FGMRES cycle
 * and at the end); x then holds an incomplete iterate.  The flags are
 * cleared, so the next call on the same hierarchy starts clean. */

/* Testing hook, not part of the paper's method: the next `launches` launches
 * of the 16-bit tensor-core coarse stencil (or of the persistent coarsest
 * GMRES kernel, which contains it) that are not being recorded into
 * a CUDA graph give up their first operand wait at once (zero try_wait
 * rounds) instead of after the normal bound.  The kernel still waits for
 * every copy it has issued before it frees its tensor memory and returns,
 * so nothing is left in flight; the call that launched it returns
 * MRHS_ERR_TIMEOUT.  0 cancels.  MRHS_ERR_INVALID for launches < 0. */
mrhs_status mrhs_debug_expire_waits(int launches);

/* Testing hook, not part of the paper's method: the next `launches` launches
 * of the half-line ring form of the even-odd hop (an autotuner variant of the
 * two launches of mrhs_apply_schur's D_hat) that are not being recorded into
 * a CUDA graph run with a zero try_wait bound on the first wait of every
 * compute warp.  Each warp then reads its neighbours from global memory
 * instead of the shared-memory ring (the same values: the output is bitwise
 * unchanged), and the copy-issuing warp stops issuing and waits for the
 * copies it has already issued before it returns, so nothing is left in
 * flight.  0 cancels.  MRHS_ERR_INVALID for launches < 0. */
mrhs_status mrhs_debug_expire_ring_waits(int launches);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of solve requests                      */
/* ------------------------------------------------------------------ */

typedef struct {
    int max_queue;          /* pending requests accepted before MRHS_ERR_BUSY  */
    double hbm_reserve_gb;  /* free HBM to keep when admitting a config        */
} mrhs_server_params;

typedef struct {
    int state;              /* MRHS_PENDING, MRHS_OK or an error status        */
    double latency_s;       /* submit -> completion                            */
    double queue_s;         /* submit -> first slot admission                  */
    int outer_iters;        /* outer iterations the request took part in      */
    double max_rel_residual;
} mrhs_request_stats;

mrhs_status mrhs_server_create(const mrhs_server_params *params, mrhs_server **out);
/* Make a resident hierarchy servable with `slots` RHS slots (<= max_rhs of
 * its params); its Krylov workspace is sized for `slots`.  Admission fails
 * with MRHS_ERR_OOM if free HBM minus the reserve cannot hold the slot
 * block (two FP64 fields of `slots` columns). */
mrhs_status mrhs_server_add_config(mrhs_server *srv, mrhs_mg *mg, int slots, int *config_id);
/* Queue nrhs sources b_host ([V][12][nrhs] FP64, copied before return);
 * x_host receives the solutions and must stay valid until mrhs_poll
 * reports completion.  Requests are admitted to free slots in FIFO order
 * per config, and each only when its device staging (V * 12 * nrhs FP64
 * complex, held until it completes) fits into free HBM above the reserve
 * (cudaMemGetInfo at admission); otherwise it waits for running requests
 * to release theirs.  MRHS_ERR_OOM at submit if the staging exceeds the
 * device's memory above the reserve; a request that still cannot be
 * staged while no other request holds staging completes with
 * MRHS_ERR_OOM. */
mrhs_status mrhs_submit(mrhs_server *srv, int config_id, const double *b_host, double *x_host,
                        int nrhs, double tol, uint64_t *req_id);
/* MRHS_PENDING while queued or running, MRHS_OK when x_host is written,
 * an error status if the request failed; `stats` optional. */
mrhs_status mrhs_poll(mrhs_server *srv, uint64_t req_id, mrhs_request_stats *stats);
/* Block until every submitted request has completed. */
mrhs_status mrhs_server_drain(mrhs_server *srv);
/* Change the HBM the server keeps free when it admits requests (GB, >= 0);
 * takes effect at the next admission. */
mrhs_status mrhs_server_set_reserve(mrhs_server *srv, double hbm_reserve_gb);
/* Admissions deferred or refused so far because free HBM above the reserve
 * could not hold a request's staging. */
mrhs_status mrhs_server_memory_waits(mrhs_server *srv, uint64_t *count);
void mrhs_server_destroy(mrhs_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* MRHS_H */
