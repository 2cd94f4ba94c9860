// Multigrid setup, V-cycle and the mixed-precision MRHS solve (paper Sec. 5-8).
//
// Every RHS keeps its own Krylov space: operator applications and inner
// products are batched over the RHS index, while the small Hessenberg /
// Givens / least-squares work runs per RHS on the device (blas.cu).  The
// V-cycle therefore contains no host synchronisation and is replayed as a
// CUDA graph.
//
// Solve structure (FGMRES preconditioned by MG, Sec. 8; precision split):
//   outer  FGMRES(outer_m) in FP64: true residual b - D x, its inner
//          products and norms in FP64;
//   inner  preconditioner of each outer step = FP32 FGMRES(inner_m) on D,
//          preconditioned by the V-cycle, to relative tolerance inner_tol;
//   V-cycle on level l: restrict, approximate coarse solve (GMRES on the
//          coarsest level, FGMRES preconditioned by the next V-cycle on an
//          intermediate level), prolong, post-smooth with smooth_m GMRES
//          iterations (FP32; coarse stencil FP32 or BF16 tensor cores).
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "mg.cuh"

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg);
}

using namespace mrhs;

namespace mrhs {
void check_wait_flags(const Level &L, cudaStream_t s);
void check_all_wait_flags(const mrhs_mg &mg, cudaStream_t s);
}

namespace {

int current_sm_count() {
    int dev = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    return sm_count(dev);
}

// ------------------------------------------------------------ operators
struct Op {
    int64_t rows = 0;
    virtual ~Op() = default;
    virtual void apply(const float2 *in, float2 *out, int n, cudaStream_t s) = 0;
    // r = b - A x
    virtual void residual(const float2 *x, const float2 *b, float2 *r, int n, cudaStream_t s) = 0;
};

struct FineOp : Op {
    const mrhs_lattice *lat;
    explicit FineOp(const mrhs_lattice *l) : lat(l) { rows = l->g.V * 12; }
    void apply(const float2 *in, float2 *out, int n, cudaStream_t s) override {
        dslash(*lat, MRHS_FP32, MRHS_FP32, in, out, nullptr, n, s);
    }
    void residual(const float2 *x, const float2 *b, float2 *r, int n, cudaStream_t s) override {
        dslash(*lat, MRHS_FP32, MRHS_FP32, x, r, b, n, s);
    }
};

struct CoarseOp : Op {
    const Level *lev;
    bool bf16;
    CoarseOp(const Level *l, bool use_bf16) : lev(l), bf16(use_bf16) { rows = l->rows(); }
    void apply(const float2 *in, float2 *out, int n, cudaStream_t s) override {
        if (bf16) coarse_apply_bf16(*lev, in, out, nullptr, n, s);
        else coarse_apply_fp32(*lev, in, out, nullptr, n, s);
    }
    void residual(const float2 *x, const float2 *b, float2 *r, int n, cudaStream_t s) override {
        if (bf16) coarse_apply_bf16(*lev, x, r, b, n, s);
        else coarse_apply_fp32(*lev, x, r, b, n, s);
    }
};

// D_hat = C_oo - 1/4 H_oe C_ee^-1 H_eo on odd half-lattice fields (the fine
// level's even-odd Schur complement); `tmp` is its own half-field scratch
struct SchurOp : Op {
    const mrhs_lattice *lat;
    DeviceBuffer tmp;
    SchurOp(const mrhs_lattice *l, int nmax) : lat(l) {
        rows = l->g.V / 2 * 12;
        tmp.alloc(sizeof(float2) * (size_t)rows * nmax);
    }
    void apply(const float2 *in, float2 *out, int n, cudaStream_t s) override {
        schur_apply(*lat, in, out, n, tmp.ptr, s);
    }
    void residual(const float2 *x, const float2 *b, float2 *r, int n, cudaStream_t s) override {
        schur_apply(*lat, x, r, n, tmp.ptr, s);
        scale_real(MRHS_FP32, -1.0, r, rows * n, s);
        axpy(MRHS_FP32, 1.0, b, r, rows * n, s);
    }
};

// D_hat = A_oo - H_oe A_ee^-1 H_eo on the odd half fields of a coarse level
// (the coarse even-odd Schur complement, tensor cores); t1, t2: even half scratch
struct CoarseSchurOp : Op {
    const Level *lev;
    DeviceBuffer t1, t2;
    CoarseSchurOp(const Level *l, int nmax) : lev(l) {
        rows = l->V / 2 * l->dof;
        t1.alloc(sizeof(float2) * (size_t)rows * nmax);
        t2.alloc(sizeof(float2) * (size_t)rows * nmax);
    }
    void apply(const float2 *in, float2 *out, int n, cudaStream_t s) override {
        coarse_schur_apply(*lev, in, out, t1.as<float2>(), t2.as<float2>(), n, s);
    }
    void residual(const float2 *x, const float2 *b, float2 *r, int n, cudaStream_t s) override {
        apply(x, r, n, s);
        scale_real(MRHS_FP32, -1.0, r, rows * n, s);
        axpy(MRHS_FP32, 1.0, b, r, rows * n, s);
    }
};

struct Precond {
    virtual ~Precond() = default;
    virtual void apply(const float2 *v, float2 *z, int n, cudaStream_t s) = 0;
};

// ------------------------------------------------------- Krylov workspace
struct KWork {
    int m = 0, nmax = 0;
    int64_t rows = 0;
    bool flexible = false;
    DeviceBuffer V, Z;
    KrylovState ks;
    Scratch sc;
    void init(int m_, int64_t rows_, int nmax_, bool flex) {
        m = m_;
        rows = rows_;
        nmax = nmax_;
        flexible = flex;
        V.alloc(sizeof(float2) * (size_t)(m + 1) * rows * nmax);
        if (flex) Z.alloc(sizeof(float2) * (size_t)m * rows * nmax);
        ks.init(m, nmax);
        sc.ensure(current_sm_count() * 8, KCHUNK * nmax);
    }
    float2 *Vj(int j, int n) const { return V.as<float2>() + (size_t)j * rows * n; }
    float2 *Zj(int j, int n) const { return Z.as<float2>() + (size_t)j * rows * n; }
};

// Per-iteration convergence test on the host (outer / inner solves only).
struct HostCheck {
    const double *target;  // host, [n] absolute residual targets
    double *res_host;      // pinned, [n]
    bool done = false;
    bool test(KrylovState &ks, int n, cudaStream_t s) {
        read_back(res_host, ks.res.ptr, sizeof(double) * n, s);
        MRHS_CUDA(cudaStreamSynchronize(s));
        for (int r = 0; r < n; ++r)
            if (!(res_host[r] <= target[r])) return false;
        done = true;
        return true;
    }
};

// One cycle of GMRES(m) (FGMRES(m) if M is given) for A x = b, updating x.
// b == nullptr stands for b = 0; x_zero: x is zero on entry.
// Returns the number of Arnoldi steps taken.
int krylov_cycle(Op &A, Precond *M, const float2 *b, float2 *x, int n, int m, KWork &w, cudaStream_t s, bool x_zero,
                 HostCheck *chk) {
    const int64_t rows = A.rows;
    const int64_t F = rows * n;
    float2 *V0 = w.Vj(0, n);
    const float2 *r0 = V0;  // the initial residual; from a zero x it is b itself, normalised into V0 directly
    if (x_zero) {
        zero_on_sms(x, sizeof(float2) * F, s);
        if (b) r0 = b;
        else zero_on_sms(V0, sizeof(float2) * F, s);
    } else if (b) {
        A.residual(x, b, V0, n, s);
    } else {
        A.apply(x, V0, n, s);
        scale_real(MRHS_FP32, -1.0, V0, F, s);
    }
    KrylovState &ks = w.ks;
    norm2(MRHS_FP32, r0, rows, n, ks.beta2.as<double>(), w.sc, s);
    krylov_start(ks, n, s);
    scale_inv_sqrt(MRHS_FP32, V0, r0, ks.beta2.as<double>(), rows, n, s);
    int steps = m;
    for (int j = 0; j < m; ++j) {
        const float2 *vj = w.Vj(j, n);
        const float2 *zj = vj;
        if (M) {
            float2 *z = w.Zj(j, n);
            M->apply(vj, z, n, s);
            zj = z;
        }
        float2 *wj = w.Vj(j + 1, n);
        A.apply(zj, wj, n, s);
        // a fixed-length cycle (no convergence check) never reads v_m: its last step needs only
        // h_{m,m-1}, from Pythagoras, and skips the subtract-and-normalise pass
        const bool need_vector = chk || j + 1 < m;
        orthonormalize_step(MRHS_FP32, V0, F, j + 1, wj, rows, n, ks.hcol.as<double2>(), ks.nrm2w.as<double>(),
                            ks.hn2.as<double>(), ks.nn.as<double>(), w.sc, s, need_vector);
        krylov_givens(ks, j, n, s, true);
        if (chk && chk->test(ks, n, s)) {
            steps = j + 1;
            break;
        }
    }
    krylov_solve(ks, steps, n, s);
    lincomb(MRHS_FP32, x, MRHS_FP32, M ? w.Zj(0, n) : V0, F, steps, ks.y.as<double2>(), 1.0, rows, n, s);
    return steps;
}

// ------------------------------------------------ GCRO-DR (coarsest level)
// GCRO with deflated restarting (Sec. 9 outlook names it for the coarsest
// level), per RHS, every cycle from the true residual; the recycle space (U,
// C = A U, k vectors per RHS) carries over from one coarsest solve (one
// V-cycle) to the next.  Fields are FP32 and batched over the RHS; the small
// dense work runs per RHS in FP64 on the device (gcrodr.cu).  Readings:
// the residual entering a cycle is orthogonal to C up to rounding (GCRO-DR
// keeps it so), hence W^H V_p = [0; I] is used for the Arnoldi columns of
// W^H V^, while W^H U and W^H r are formed as inner products.
struct GcroWork {
    int m = 0, k = 0, nmax = 0;
    int64_t rows = 0;
    bool has_recycle = false;
    int last_n = 0;  // RHS count the recycle fields are laid out for
    DeviceBuffer V, U, C, U2, C2, AU, r;           // fields [rows][n]
    DeviceBuffer H, B, WU, QC, PU;                 // per RHS [n][17][17] double2
    DeviceBuffer WR, Y, UN2;                       // per RHS [n][17] (UN2 double)
    DeviceBuffer dots, coef, nrm2, hn2, nn, beta2, rin2, err;
    Scratch sc;
    void init(int m_, int k_, int64_t rows_, int nmax_) {
        m = m_;
        k = k_;
        rows = rows_;
        nmax = nmax_;
        const size_t f = sizeof(float2) * (size_t)rows * nmax;
        V.alloc(f * (m + 1));
        r.alloc(f);
        if (k > 0) {
            U.alloc(f * k);
            C.alloc(f * k);
            U2.alloc(f * k);
            C2.alloc(f * k);
            AU.alloc(f * k);
        }
        const size_t mat = sizeof(double2) * (size_t)nmax * 17 * 17, vec = sizeof(double2) * (size_t)nmax * 17;
        H.alloc(mat);
        B.alloc(mat);
        WU.alloc(mat);
        QC.alloc(mat);
        PU.alloc(mat);
        WR.alloc(vec);
        Y.alloc(vec);
        UN2.alloc(sizeof(double) * (size_t)nmax * 17);
        dots.alloc(sizeof(double2) * (size_t)(m + 1) * nmax);
        coef.alloc(sizeof(double2) * (size_t)(m + 1) * nmax);
        for (DeviceBuffer *b : {&nrm2, &hn2, &nn, &beta2, &rin2}) b->alloc(sizeof(double) * nmax * 17);
        err.alloc(sizeof(int));
        MRHS_CUDA(cudaMemset(err.ptr, 0, sizeof(int)));
        MRHS_CUDA(cudaMemset(H.ptr, 0, mat));
        MRHS_CUDA(cudaMemset(B.ptr, 0, mat));
        sc.ensure(current_sm_count() * 8, KCHUNK * nmax);
    }
    float2 *fld(const DeviceBuffer &b, int i, int n) const { return b.as<float2>() + (size_t)i * rows * n; }
};

// One Arnoldi step on field j+1 = A field j against fields 0..j of `V`, storing column j of the
// per-RHS Hessenberg (rows row0..row0+j+1); with C (k > 0), first w -= C (C^H w), B column j.
void gcro_arnoldi_step(Op &A, GcroWork &g, int j, int row0, bool project, int n, cudaStream_t s) {
    float2 *vj = g.fld(g.V, j, n), *w = g.fld(g.V, j + 1, n);
    const int64_t F = g.rows * n;
    A.apply(vj, w, n, s);
    if (project) {
        multi_dot(MRHS_FP32, g.C.ptr, F, g.k, w, g.rows, n, g.dots.as<double2>(), g.sc, s);
        gcro_put_col(g.B.as<double2>(), g.dots.as<double2>(), g.k, 0, j, n, s);
        lincomb(MRHS_FP32, w, MRHS_FP32, g.C.ptr, F, g.k, g.dots.as<double2>(), -1.0, g.rows, n, s);
    }
    orthonormalize_step(MRHS_FP32, g.V.ptr, F, j + 1, w, g.rows, n, g.dots.as<double2>(), g.nrm2.as<double>(),
                        g.hn2.as<double>(), g.nn.as<double>(), g.sc, s);
    gcro_store_col(g.H.as<double2>(), g.dots.as<double2>(), g.hn2.as<double>(), g.nn.as<double>(), j, row0, n, s);
}

// out_i = sum_j coef_i[j] basis_j for the k outputs, out fields zeroed first; coefficients from column i
// of the per-RHS matrix M (rows off..off+cnt-1)
void gcro_combine(GcroWork &g, const DeviceBuffer &M, const void *basis, int off, int cnt, DeviceBuffer &out, int i,
                  int n, cudaStream_t s) {
    gcro_coef_col(g.coef.as<double2>(), M.as<double2>(), off, cnt, i, 1.0, n, s);
    lincomb(MRHS_FP32, g.fld(out, i, n), MRHS_FP32, basis, g.rows * n, cnt, g.coef.as<double2>(), 1.0, g.rows, n,
            s);
}

// Solve A x = b approximately by `cycles` GCRO-DR(m, k) cycles from x = 0.
void gcro_solve(Op &A, GcroWork &g, const float2 *b, float2 *x, int n, int cycles, cudaStream_t s) {
    const int m = g.m, k = g.k, p = m - k;
    const int64_t F = g.rows * n;
    float2 *r = g.r.as<float2>();
    if (n != g.last_n) g.has_recycle = false;  // the recycle fields hold another RHS count's layout
    g.last_n = n;
    zero_on_sms(x, sizeof(float2) * F, s);
    copy_on_sms(r, b, sizeof(float2) * F, s);
    if (g.has_recycle && k > 0) {
        // C = Q, U = U R^{-1} from A U = Q R (Gram-Schmidt on the batched fields)
        for (int i = 0; i < k; ++i) A.apply(g.fld(g.U, i, n), g.fld(g.AU, i, n), n, s);
        for (int i = 0; i < k; ++i) {
            float2 *ci = g.fld(g.C, i, n);
            copy_on_sms(ci, g.fld(g.AU, i, n), sizeof(float2) * F, s);
            double *rii2 = g.rin2.as<double>() + (size_t)i * n;
            if (i == 0) {
                norm2(MRHS_FP32, ci, g.rows, n, rii2, g.sc, s);
                scale_inv_sqrt(MRHS_FP32, ci, ci, rii2, g.rows, n, s);
            } else {
                orthonormalize_step(MRHS_FP32, g.C.ptr, F, i, ci, g.rows, n, g.dots.as<double2>(),
                                    g.nrm2.as<double>(), rii2, g.nn.as<double>(), g.sc, s);
                // u_i <- (u_i - sum_{j<i} R_ji u_j) / R_ii, the u_j already replaced
                lincomb(MRHS_FP32, g.fld(g.U, i, n), MRHS_FP32, g.U.ptr, F, i, g.dots.as<double2>(), -1.0, g.rows,
                        n, s);
            }
            scale_inv_sqrt(MRHS_FP32, g.fld(g.U, i, n), g.fld(g.U, i, n), rii2, g.rows, n, s);
        }
        // x = U C^H r, r = b - A x
        multi_dot(MRHS_FP32, g.C.ptr, F, k, r, g.rows, n, g.dots.as<double2>(), g.sc, s);
        lincomb(MRHS_FP32, x, MRHS_FP32, g.U.ptr, F, k, g.dots.as<double2>(), 1.0, g.rows, n, s);
        A.residual(x, b, r, n, s);
    }
    for (int c = 0; c < cycles; ++c) {
        norm2(MRHS_FP32, r, g.rows, n, g.beta2.as<double>(), g.sc, s);
        scale_inv_sqrt(MRHS_FP32, g.fld(g.V, 0, n), r, g.beta2.as<double>(), g.rows, n, s);
        if (!g.has_recycle || k == 0) {
            // a GMRES(m) cycle that seeds the recycle space
            for (int j = 0; j < m; ++j) gcro_arnoldi_step(A, g, j, 0, false, n, s);
            gcro_seed_small(g.H.as<double2>(), g.beta2.as<double>(), m, k, g.Y.as<double2>(), g.QC.as<double2>(),
                            g.PU.as<double2>(), g.err.as<int>(), n, s);
            gcro_coef_vec(g.coef.as<double2>(), g.Y.as<double2>(), 0, m, 1.0, n, s);
            lincomb(MRHS_FP32, x, MRHS_FP32, g.V.ptr, F, m, g.coef.as<double2>(), 1.0, g.rows, n, s);
            if (k > 0) {
                zero_on_sms(g.C.ptr, sizeof(float2) * F * k, s);
                zero_on_sms(g.U.ptr, sizeof(float2) * F * k, s);
                for (int i = 0; i < k; ++i) {
                    gcro_combine(g, g.QC, g.V.ptr, 0, m + 1, g.C, i, n, s);
                    gcro_combine(g, g.PU, g.V.ptr, 0, m, g.U, i, n, s);
                }
                g.has_recycle = true;
            }
        } else {
            // a cycle with the recycle space: p Arnoldi steps of (I - C C^H) A
            for (int j = 0; j < p; ++j) gcro_arnoldi_step(A, g, j, 0, true, n, s);
            for (int i = 0; i < k; ++i) {
                norm2(MRHS_FP32, g.fld(g.U, i, n), g.rows, n, g.nrm2.as<double>(), g.sc, s);
                gcro_put_norm(g.UN2.as<double>(), g.nrm2.as<double>(), i, n, s);
                // W^H u_i = [C^H u_i ; V^H u_i]
                multi_dot(MRHS_FP32, g.C.ptr, F, k, g.fld(g.U, i, n), g.rows, n, g.dots.as<double2>(), g.sc, s);
                gcro_put_col(g.WU.as<double2>(), g.dots.as<double2>(), k, 0, i, n, s);
                multi_dot(MRHS_FP32, g.V.ptr, F, p + 1, g.fld(g.U, i, n), g.rows, n, g.dots.as<double2>(), g.sc, s);
                gcro_put_col(g.WU.as<double2>(), g.dots.as<double2>(), p + 1, k, i, n, s);
            }
            multi_dot(MRHS_FP32, g.C.ptr, F, k, r, g.rows, n, g.dots.as<double2>(), g.sc, s);
            gcro_put_vec(g.WR.as<double2>(), g.dots.as<double2>(), k, 0, n, s);
            multi_dot(MRHS_FP32, g.V.ptr, F, p + 1, r, g.rows, n, g.dots.as<double2>(), g.sc, s);
            gcro_put_vec(g.WR.as<double2>(), g.dots.as<double2>(), p + 1, k, n, s);
            gcro_cycle_small(g.H.as<double2>(), g.B.as<double2>(), g.UN2.as<double>(), g.WR.as<double2>(),
                             g.WU.as<double2>(), m, k, g.Y.as<double2>(), g.QC.as<double2>(), g.PU.as<double2>(),
                             g.err.as<int>(), n, s);
            // x += U (D y_U) + V_p y_V
            gcro_coef_vec(g.coef.as<double2>(), g.Y.as<double2>(), 0, k, 1.0, n, s);
            lincomb(MRHS_FP32, x, MRHS_FP32, g.U.ptr, F, k, g.coef.as<double2>(), 1.0, g.rows, n, s);
            gcro_coef_vec(g.coef.as<double2>(), g.Y.as<double2>(), k, p, 1.0, n, s);
            lincomb(MRHS_FP32, x, MRHS_FP32, g.V.ptr, F, p, g.coef.as<double2>(), 1.0, g.rows, n, s);
            // C <- [C, V_{p+1}] Q, U <- [U D, V_p] P R^{-1}
            zero_on_sms(g.C2.ptr, sizeof(float2) * F * k, s);
            zero_on_sms(g.U2.ptr, sizeof(float2) * F * k, s);
            for (int i = 0; i < k; ++i) {
                gcro_combine(g, g.QC, g.C.ptr, 0, k, g.C2, i, n, s);
                gcro_combine(g, g.QC, g.V.ptr, k, p + 1, g.C2, i, n, s);
                gcro_combine(g, g.PU, g.U.ptr, 0, k, g.U2, i, n, s);
                gcro_combine(g, g.PU, g.V.ptr, k, p, g.U2, i, n, s);
            }
            copy_on_sms(g.C.ptr, g.C2.ptr, sizeof(float2) * F * k, s);
            copy_on_sms(g.U.ptr, g.U2.ptr, sizeof(float2) * F * k, s);
        }
        A.residual(x, b, r, n, s);
    }
}

// ------------------------------------------------------- level workspace
struct LevelWork {
    DeviceBuffer rhs, sol;  // coarse levels: restricted residual and coarse solution
    KWork solve;            // coarse levels: GMRES (coarsest) or FGMRES (intermediate)
    KWork smooth;           // levels with a coarser level: post-smoother GMRES
    // fine level, even-odd smoother: full residual, half fields r_e, r_o,
    // C_ee^-1 r_e, b_hat, delta_e, delta_o, and GMRES on D_hat
    DeviceBuffer eo_r, eo_re, eo_ro, eo_te, eo_bh, eo_de, eo_do;
    KWork eo_smooth;
    DeviceBuffer sap_r;  // fine level, SAP smoother: its residual field
    // intermediate coarse levels, even-odd smoother: residual, its halves, A_ee^-1 r_e,
    // b_hat, the corrections and GMRES on the coarse Schur complement
    DeviceBuffer ceo_r, ceo_re, ceo_ro, ceo_te, ceo_bh, ceo_de, ceo_do;
    KWork ceo_smooth;
    std::unique_ptr<CoarseSchurOp> ceo_op;
    std::unique_ptr<GcroWork> gcro;  // coarsest level with the GCRO-DR solver
    // coarsest level, GMRES as one persistent kernel; fused_r, fused_e: residual and
    // correction fields of the cycles after the first
    std::unique_ptr<CoarsestFused> fused;
    DeviceBuffer fused_r, fused_e;
};

struct GraphKey {
    int n;
    const void *in;
    void *out;
    bool operator<(const GraphKey &o) const {
        if (n != o.n) return n < o.n;
        if (in != o.in) return in < o.in;
        return out < o.out;
    }
};

}  // namespace

// --------------------------------------------------------------- handle
struct mrhs_mg {
    mrhs_lattice *lat = nullptr;
    mrhs_mg_params p{};
    int nlev = 0;
    int nmax = 0;
    std::vector<Level> lev;
    std::vector<LevelWork> work;
    std::vector<std::unique_ptr<Op>> ops;
    std::unique_ptr<SchurOp> schur;  // the fine level's even-odd smoother operator (when enabled)
    bool bf16 = false;
    // inner FP32 MG-FGMRES on the fine level
    KWork inner;
    DeviceBuffer inner_b;
    // outer FP64 FGMRES
    int om = 0;
    DeviceBuffer oV, oZ;  // FP64 [(om+1)][rows][nmax], FP32 [om][rows][nmax]
    KrylovState oks;
    Scratch osc;
    DeviceBuffer obn2;    // double [nmax]
    double *pinned = nullptr;  // host staging, 4*nmax doubles
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, uint64_t> graph_kernels;  // kernel nodes per graph
    // component timing (profiled, non-graph solves only)
    bool profile = false;
    double t_fine = 0, t_restrict = 0, t_prolong = 0, t_coarse = 0;
    // setup phases per transfer l -> l+1 (milliseconds, CUDA events on the setup stream): null
    // vectors, chiral split + orthonormalisation, Galerkin operator, 16-bit / tensor-core preparation
    double setup_ms[MRHS_MAX_LEVELS - 1][4] = {};
    int vcycles = 0;
    // the solver's own stream: graphs cannot be captured on the legacy default stream
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    ~mrhs_mg() {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
        if (pinned) cudaFreeHost(pinned);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (own) cudaStreamDestroy(own);
    }
};

namespace {

struct EventTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    double *acc;
    bool on;
    EventTimer(bool enabled, cudaStream_t st, double *accum) : s(st), acc(accum), on(enabled) {
        if (!on) return;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    ~EventTimer() {
        if (!on) return;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        *acc += ms * 1e-3;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// The coarsest level's solve x = A^-1 b as the V-cycle runs it: coarse_cycles
// cycles of GCRO-DR, of GMRES as one persistent kernel, or of GMRES one launch
// per operation, from x = 0.
void coarsest_solve(mrhs_mg &mg, const float2 *b, float2 *x, int n, cudaStream_t s) {
    const int l = mg.nlev - 1;
    LevelWork &W = mg.work[l];
    Op &A = *mg.ops[l];
    if (W.gcro) {
        gcro_solve(A, *W.gcro, b, x, n, mg.p.coarse_cycles, s);
    } else if (W.fused) {
        const Level &C = mg.lev[l];
        W.fused->solve(C, W.solve.Vj(0, n), b, x, n, s);
        for (int c = 1; c < mg.p.coarse_cycles; ++c) {
            A.residual(x, b, W.fused_r.as<float2>(), n, s);
            W.fused->solve(C, W.solve.Vj(0, n), W.fused_r.as<float2>(), W.fused_e.as<float2>(), n, s);
            axpy(MRHS_FP32, 1.0, W.fused_e.ptr, x, C.rows() * n, s);
        }
    } else {
        for (int c = 0; c < mg.p.coarse_cycles; ++c)
            krylov_cycle(A, nullptr, b, x, n, mg.p.coarse_m, W.solve, s, c == 0, nullptr);
    }
}

// unit_norm: every RHS column of v has norm <= 1 (true for the Arnoldi vectors
// the preconditioned Krylov cycles pass in)
void vcycle(mrhs_mg &mg, int l, const float2 *v, float2 *z, int n, cudaStream_t s, bool unit_norm = true);

struct VcyclePrecond : Precond {
    mrhs_mg *mg;
    int level;
    VcyclePrecond(mrhs_mg *g, int l) : mg(g), level(l) {}
    void apply(const float2 *v, float2 *z, int n, cudaStream_t s) override { vcycle(*mg, level, v, z, n, s); }
};

void vcycle(mrhs_mg &mg, int l, const float2 *v, float2 *z, int n, cudaStream_t s, bool unit_norm) {
    Level &F = mg.lev[l];
    Level &Cl = mg.lev[l + 1];
    LevelWork &WC = mg.work[l + 1];
    const bool prof = mg.profile && l == 0;
    {
        EventTimer t(prof, s, &mg.t_restrict);
        if (F.tc_intergrid) restrict_fields_tc(F, Cl, v, WC.rhs.as<float2>(), n, (int64_t)Cl.dof * n, unit_norm, s);
        else restrict_fields(F, Cl, v, WC.rhs.as<float2>(), n, (int64_t)Cl.dof * n, s);
    }
    {
        EventTimer t(prof, s, &mg.t_coarse);
        Op &Ac = *mg.ops[l + 1];
        float2 *sol = WC.sol.as<float2>();
        if (l + 1 == mg.nlev - 1) {
            coarsest_solve(mg, WC.rhs.as<float2>(), sol, n, s);
        } else {
            VcyclePrecond M(&mg, l + 1);
            krylov_cycle(Ac, &M, WC.rhs.as<float2>(), sol, n, mg.p.inter_m, WC.solve, s, true, nullptr);
        }
    }
    {
        EventTimer t(prof, s, &mg.t_prolong);
        if (F.tc_intergrid) prolong_fields_tc(F, Cl, WC.sol.as<float2>(), z, n, s);
        else prolong_fields(F, Cl, WC.sol.as<float2>(), z, n, s);
    }
    {
        EventTimer t(prof, s, &mg.t_fine);
        if (l == 0 && mg.p.smoother_sap && sap_supported(*mg.lat, mg.p.sap_block, n)) {
            // SAP smoother: sap_cycles cycles of block-coloured Schwarz on D z = v from the
            // coarse-corrected z, each block system by sap_mr MR steps
            sap_smooth(*mg.lat, v, z, n, mg.p.sap_block, mg.p.sap_cycles, mg.p.sap_mr, mg.work[0].sap_r.ptr, s);
        } else if (l == 0 && mg.schur && eo_supported(*mg.lat, n)) {
            // even-odd smoother: z += delta, D delta ~= r = v - D z through smooth_m GMRES
            // steps on D_hat delta_o = b_hat = r_o + 1/2 H_oe C_ee^-1 r_e from 0, then
            // delta_e = C_ee^-1 (r_e + 1/2 H_eo delta_o), both added to z in one pass
            LevelWork &W = mg.work[0];
            if (!residual_eo_split(*mg.lat, z, v, W.eo_re.ptr, W.eo_ro.ptr, W.eo_te.ptr, n, s)) {
                mg.ops[0]->residual(z, v, W.eo_r.as<float2>(), n, s);
                eo_split(*mg.lat, W.eo_r.ptr, W.eo_re.ptr, W.eo_ro.ptr, W.eo_te.ptr, n, s);
            }
            eo_axpy_hop(*mg.lat, 1, W.eo_ro.ptr, W.eo_te.ptr, W.eo_bh.ptr, false, n, s);
            krylov_cycle(*mg.schur, nullptr, W.eo_bh.as<float2>(), W.eo_do.as<float2>(), n, mg.p.smooth_m,
                         W.eo_smooth, s, true, nullptr);
            eo_cinv_axpy_hop_merge(*mg.lat, W.eo_re.ptr, W.eo_do.ptr, z, W.eo_de.ptr, n, s);
        } else if (l > 0 && mg.work[l].ceo_op) {
            // coarse even-odd smoother: z += delta, delta from smooth_m GMRES steps on
            // D_hat delta_o = b_hat = r_o - H_oe A_ee^-1 r_e (r = v - A z), then
            // delta_e = A_ee^-1 (r_e - H_eo delta_o)
            LevelWork &W = mg.work[l];
            mg.ops[l]->residual(z, v, W.ceo_r.as<float2>(), n, s);
            coarse_parity_split(F, W.ceo_r.as<float2>(), W.ceo_re.as<float2>(), W.ceo_ro.as<float2>(), n, s);
            coarse_eo_self(F, true, 0, W.ceo_re.as<float2>(), W.ceo_te.as<float2>(), n, s);
            coarse_eo_hop(F, 1, W.ceo_te.as<float2>(), W.ceo_bh.as<float2>(), W.ceo_ro.as<float2>(), n, s);
            krylov_cycle(*W.ceo_op, nullptr, W.ceo_bh.as<float2>(), W.ceo_do.as<float2>(), n, mg.p.smooth_m,
                         W.ceo_smooth, s, true, nullptr);
            coarse_eo_hop(F, 0, W.ceo_do.as<float2>(), W.ceo_te.as<float2>(), W.ceo_re.as<float2>(), n, s);
            coarse_eo_self(F, true, 0, W.ceo_te.as<float2>(), W.ceo_de.as<float2>(), n, s);
            coarse_parity_merge_add(F, W.ceo_de.as<float2>(), W.ceo_do.as<float2>(), z, n, s);
        } else {
            krylov_cycle(*mg.ops[l], nullptr, v, z, n, mg.p.smooth_m, mg.work[l].smooth, s, false, nullptr);
        }
    }
    if (l == 0) mg.vcycles++;
}

// V-cycle on the fine level, replayed from a CUDA graph per (n, in, out).
struct FinePrecond : Precond {
    mrhs_mg *mg;
    explicit FinePrecond(mrhs_mg *g) : mg(g) {}
    void apply(const float2 *v, float2 *z, int n, cudaStream_t s) override {
        if (!mg->p.use_graph || mg->profile) {
            vcycle(*mg, 0, v, z, n, s);
            return;
        }
        GraphKey key{n, v, z};
        auto it = mg->graphs.find(key);
        if (it == mg->graphs.end()) {
            // first use: run once eagerly (sizes every lazily configured kernel), then capture
            vcycle(*mg, 0, v, z, n, s);
            cudaGraph_t g = nullptr;
            MRHS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            try {
                vcycle(*mg, 0, v, z, n, s);
            } catch (...) {
                cudaStreamEndCapture(s, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            MRHS_CUDA(cudaStreamEndCapture(s, &g));
            cudaGraphExec_t ex = nullptr;
            MRHS_CUDA(cudaGraphInstantiate(&ex, g, 0));
            size_t nn = 0;
            MRHS_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            if (nn) MRHS_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
            uint64_t kern = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
            }
            cudaGraphDestroy(g);
            mg->graph_kernels[key] = kern;
            it = mg->graphs.emplace(key, ex).first;
            return;  // the eager run already produced z
        }
        MRHS_CUDA(cudaGraphLaunch(it->second, s));
        count_launches(mg->graph_kernels[key]);
        mg->vcycles++;
    }
};

// FP32 MG-preconditioned FGMRES on the fine level: x = approx D^{-1} b.
// rel[r]: relative residual reduction asked of RHS r (the inner FGMRES stops
// when every RHS has reached its own)
int inner_solve(mrhs_mg &mg, const float2 *b, float2 *x, int n, const std::vector<double> &rel, cudaStream_t s) {
    Op &A = *mg.ops[0];
    FinePrecond M(&mg);
    const int64_t F = A.rows * n;
    zero_on_sms(x, sizeof(float2) * F, s);
    double *bn = mg.pinned + 2 * mg.nmax;
    double *target = mg.pinned + 3 * mg.nmax;
    norm2(MRHS_FP32, b, A.rows, n, mg.inner.ks.beta2.as<double>(), mg.inner.sc, s);
    read_back(bn, mg.inner.ks.beta2.ptr, sizeof(double) * n, s);
    MRHS_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < n; ++r) target[r] = rel[r] * std::sqrt(bn[r]);
    HostCheck chk{target, mg.pinned + mg.nmax};
    int total = 0;
    bool first = true;
    while (total < mg.p.inner_max_iters && !chk.done) {
        const int m = std::min(mg.p.inner_m, mg.p.inner_max_iters - total);
        total += krylov_cycle(A, &M, b, x, n, m, mg.inner, s, first, &chk);
        first = false;
        // a tensor-core wait that gave up leaves a V-cycle without an operand: stop here
        check_all_wait_flags(mg, s);
    }
    return total;
}

void validate_params(const mrhs_lattice *lat, const mrhs_mg_params &p) {
    if (p.n_levels < 2 || p.n_levels > MRHS_MAX_LEVELS) fail(MRHS_ERR_INVALID, "n_levels must be 2 or 3");
    int L[4] = {lat->g.L[0], lat->g.L[1], lat->g.L[2], lat->g.L[3]};
    int dof = 12;
    for (int l = 0; l < p.n_levels - 1; ++l) {
        for (int mu = 0; mu < 4; ++mu) {
            if (p.block[l][mu] < 1 || L[mu] % p.block[l][mu])
                fail(MRHS_ERR_INVALID, "aggregate extents must divide the level's lattice extents");
            L[mu] /= p.block[l][mu];
        }
        const int N = p.n_vec[l];
        if (N < 1 || N > 32) fail(MRHS_ERR_INVALID, "n_vec must be in 1..32");
        int64_t asize = (int64_t)p.block[l][0] * p.block[l][1] * p.block[l][2] * p.block[l][3];
        if (asize * (dof / 2) < N) fail(MRHS_ERR_INVALID, "aggregate too small for n_vec vectors per chirality");
        dof = 2 * N;
    }
    if (p.smooth_m < 1 || p.smooth_m > 64 || p.coarse_m < 1 || p.coarse_m > 64 || p.inner_m < 1 || p.inner_m > 64 ||
        p.outer_m < 1 || p.outer_m > 64 || p.setup_m < 1 || p.setup_m > 64 || p.inter_m < 1 || p.inter_m > 64)
        fail(MRHS_ERR_INVALID, "Krylov lengths must be in 1..64");
    if (p.coarse_cycles < 1 || p.setup_sweeps < 0 || p.inner_max_iters < 1 || p.max_outer_iters < 1)
        fail(MRHS_ERR_INVALID, "iteration counts must be positive");
    if (p.max_rhs < 1 || p.max_rhs > 64) fail(MRHS_ERR_INVALID, "max_rhs must be in 1..64");
    if (p.coarse_precision != MRHS_FP32 && p.coarse_precision != MRHS_BF16 && p.coarse_precision != MRHS_FP16)
        fail(MRHS_ERR_INVALID, "coarse_precision must be FP32, FP16 or BF16");
    if (p.outer_op_precision != MRHS_DF64 && p.outer_op_precision != MRHS_FP64)
        fail(MRHS_ERR_INVALID, "outer_op_precision must be DF64 or FP64");
    if (p.smoother_evenodd != 0 && p.smoother_evenodd != 1) fail(MRHS_ERR_INVALID, "smoother_evenodd must be 0 or 1");
    if (p.smoother_sap != 0 && p.smoother_sap != 1) fail(MRHS_ERR_INVALID, "smoother_sap must be 0 or 1");
    if (p.smoother_sap && (p.sap_cycles < 1 || p.sap_cycles > 16 || p.sap_mr < 1 || p.sap_mr > 64))
        fail(MRHS_ERR_INVALID, "sap_cycles must be in 1..16 and sap_mr in 1..64");
    if (p.coarse_smoother_evenodd != 0 && p.coarse_smoother_evenodd != 1)
        fail(MRHS_ERR_INVALID, "coarse_smoother_evenodd must be 0 or 1");
    if (p.coarse_solver != 0 && p.coarse_solver != 1) fail(MRHS_ERR_INVALID, "coarse_solver must be 0 or 1");
    if (p.coarse_fused != 0 && p.coarse_fused != 1) fail(MRHS_ERR_INVALID, "coarse_fused must be 0 or 1");
    if (p.galerkin_tc < 0 || p.galerkin_tc > 2) fail(MRHS_ERR_INVALID, "galerkin_tc must be 0, 1 or 2");
    if (p.coarse_solver == 1 && (p.coarse_m > 16 || p.coarse_recycle < 0 || p.coarse_recycle >= p.coarse_m))
        fail(MRHS_ERR_INVALID, "GCRO-DR needs coarse_m <= 16 and 0 <= coarse_recycle < coarse_m");
    if (!(p.inner_tol > 0 && p.inner_tol < 1)) fail(MRHS_ERR_INVALID, "inner_tol must be in (0, 1)");
}

// CUDA events marking the setup phases of one level on the setup stream
struct PhaseEvents {
    std::vector<cudaEvent_t> ev;
    void mark(cudaStream_t s) {
        cudaEvent_t e = nullptr;
        MRHS_CUDA(cudaEventCreate(&e));
        ev.push_back(e);
        MRHS_CUDA(cudaEventRecord(e, s));
    }
    // milliseconds between consecutive marks (after the stream has finished them)
    void read(double *out, int count) {
        for (int i = 0; i < count && i + 1 < (int)ev.size(); ++i) {
            float ms = 0.f;
            MRHS_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            out[i] = ms;
        }
    }
    ~PhaseEvents() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

void setup_level(mrhs_mg &mg, int l, cudaStream_t s, PhaseEvents &ph) {
    Level &F = mg.lev[l];
    Level &Cl = mg.lev[l + 1];
    const int N = F.N;
    const int64_t count = F.V * F.dof * N;
    // start vectors
    DeviceBuffer v64(sizeof(double2) * count);
    DeviceBuffer v32(sizeof(float2) * count);
    if (mg.p.init_vecs[l]) {
        MRHS_CUDA(cudaMemcpyAsync(v64.ptr, mg.p.init_vecs[l], sizeof(double2) * count, cudaMemcpyHostToDevice, s));
        cast(MRHS_FP32, v32.ptr, MRHS_FP64, v64.ptr, count, s);
    } else {
        fill_gaussian(MRHS_FP32, v32.ptr, count, mg.p.seed * 0x9E3779B9ull + (uint64_t)l, s);
    }
    // relaxation of A v = 0, the N vectors as N right-hand sides
    ph.mark(s);
    if (mg.p.setup_sweeps > 0) {
        KWork rw;
        rw.init(mg.p.setup_m, F.rows(), N, false);
        for (int sweep = 0; sweep < mg.p.setup_sweeps; ++sweep) {
            krylov_cycle(*mg.ops[l], nullptr, nullptr, v32.as<float2>(), N, mg.p.setup_m, rw, s, false, nullptr);
            norm2(MRHS_FP32, v32.ptr, F.rows(), N, rw.ks.beta2.as<double>(), rw.sc, s);
            scale_inv_sqrt(MRHS_FP32, v32.ptr, v32.ptr, rw.ks.beta2.as<double>(), F.rows(), N, s);
        }
        cast(MRHS_FP64, v64.ptr, MRHS_FP32, v32.ptr, count, s);
    } else if (!mg.p.init_vecs[l]) {
        cast(MRHS_FP64, v64.ptr, MRHS_FP32, v32.ptr, count, s);
    }
    // chiral split + FP64 block orthonormalisation
    ph.mark(s);
    block_orthonormalize(F, v64.as<double2>(), s);
    F.P64 = std::move(v64);
    F.P32.alloc(sizeof(float2) * count);
    cast(MRHS_FP32, F.P32.ptr, MRHS_FP64, F.P64.ptr, count, s);
    v32.release();
    // Galerkin coarse operator R A P, stencil block by stencil block; the restriction R = P^dagger
    // on the tensor cores in split FP16 (FP32-level accuracy) where the transfer tiles apply
    ph.mark(s);
    const int nc = 2 * N;
    const bool bit16 = mg.p.coarse_precision == MRHS_FP16 || mg.p.coarse_precision == MRHS_BF16;
    const bool tc_galerkin = (mg.p.galerkin_tc == 2 || (mg.p.galerkin_tc == 1 && bit16)) &&
                             intergrid_tc_supported(F) && nc <= 64;
    if (tc_galerkin) intergrid_tc_prepare(F, Cl, s, true);
    Cl.A32.alloc(sizeof(float2) * (size_t)Cl.V * 9 * nc * nc);
    DeviceBuffer Pe(sizeof(float2) * (size_t)F.V * F.dof * nc);
    DeviceBuffer H(sizeof(float2) * (size_t)F.V * F.dof * nc);
    expand_chiral(F, F.P32.as<float2>(), Pe.as<float2>(), s);
    const int64_t ostride = (int64_t)9 * nc * nc;
    for (int d = 0; d < 9; ++d) {
        if (l == 0) {
            HopMask m{d == 0 ? 1 : 0, d == 0 ? -1 : d, d == 0 ? 2 : 1, {F.B[0], F.B[1], F.B[2], F.B[3]}};
            dslash(*mg.lat, MRHS_FP32, MRHS_FP32, Pe.ptr, H.ptr, nullptr, nc, s, &m);
        } else {
            StencilMask m{d == 0 ? 1 : 0, d == 0 ? -1 : d, d == 0 ? 2 : 1, {F.B[0], F.B[1], F.B[2], F.B[3]}};
            coarse_apply_fp32(F, Pe.as<float2>(), H.as<float2>(), nullptr, nc, s, &m);
        }
        if (tc_galerkin)
            restrict_fields_tc(F, Cl, H.as<float2>(), Cl.A32.as<float2>() + (size_t)d * nc * nc, nc, ostride, false, s,
                               true);
        else
            restrict_fields(F, Cl, H.as<float2>(), Cl.A32.as<float2>() + (size_t)d * nc * nc, nc, ostride, s);
    }
    ph.mark(s);
    if (tc_galerkin && intergrid_tc_error(F, s))
        fail(MRHS_ERR_TIMEOUT, "setup: a tensor-core restriction of the Galerkin build gave up waiting");
    MRHS_CUDA(cudaStreamSynchronize(s));
}

void alloc_workspace(mrhs_mg &mg) {
    const int nmax = mg.nmax;
    mg.work.resize(mg.nlev);
    for (int l = 0; l < mg.nlev; ++l) {
        Level &L = mg.lev[l];
        LevelWork &W = mg.work[l];
        if (l >= 1) {
            W.rhs.alloc(sizeof(float2) * (size_t)L.rows() * nmax);
            W.sol.alloc(sizeof(float2) * (size_t)L.rows() * nmax);
            if (l == mg.nlev - 1) W.solve.init(mg.p.coarse_m, L.rows(), nmax, false);
            else W.solve.init(mg.p.inter_m, L.rows(), nmax, true);
            if (l == mg.nlev - 1 && mg.p.coarse_solver == 1) {
                W.gcro.reset(new GcroWork());
                W.gcro->init(mg.p.coarse_m, mg.p.coarse_recycle, L.rows(), nmax);
            } else if (l == mg.nlev - 1 && mg.p.coarse_fused &&
                       CoarsestFused::supported(L, nmax, mg.p.coarse_m, mg.lat->device)) {
                W.fused.reset(new CoarsestFused());
                W.fused->init(L, mg.p.coarse_m, nmax, mg.lat->device);
                if (mg.p.coarse_cycles > 1) {
                    W.fused_r.alloc(sizeof(float2) * (size_t)L.rows() * nmax);
                    W.fused_e.alloc(sizeof(float2) * (size_t)L.rows() * nmax);
                }
            }
        }
        if (l < mg.nlev - 1) W.smooth.init(mg.p.smooth_m, L.rows(), nmax, false);
    }
    if (mg.p.smoother_evenodd && eo_supported(*mg.lat, 2)) {
        LevelWork &W = mg.work[0];
        const int64_t hrows = mg.lat->g.V / 2 * 12;
        const size_t hb = sizeof(float2) * (size_t)hrows * nmax;
        W.eo_r.alloc(2 * hb);
        for (DeviceBuffer *b : {&W.eo_re, &W.eo_ro, &W.eo_te, &W.eo_bh, &W.eo_de, &W.eo_do}) b->alloc(hb);
        W.eo_smooth.init(mg.p.smooth_m, hrows, nmax, false);
        mg.schur.reset(new SchurOp(mg.lat, nmax));
    }
    if (mg.p.smoother_sap && sap_supported(*mg.lat, mg.p.sap_block, 2))
        mg.work[0].sap_r.alloc(sizeof(float2) * (size_t)mg.lev[0].rows() * nmax);
    // coarse even-odd smoother on the intermediate levels that have the inverse self blocks
    for (int l = 1; l + 1 < mg.nlev; ++l) {
        Level &L = mg.lev[l];
        if (!L.AinvBf.ptr) continue;
        LevelWork &W = mg.work[l];
        const size_t half = sizeof(float2) * (size_t)(L.V / 2) * L.dof * nmax;
        W.ceo_r.alloc(2 * half);
        for (DeviceBuffer *b : {&W.ceo_re, &W.ceo_ro, &W.ceo_te, &W.ceo_bh, &W.ceo_de, &W.ceo_do}) b->alloc(half);
        W.ceo_smooth.init(mg.p.smooth_m, L.V / 2 * L.dof, nmax, false);
        W.ceo_op.reset(new CoarseSchurOp(&L, nmax));
    }
    const int64_t rows = mg.lev[0].rows();
    mg.inner.init(mg.p.inner_m, rows, nmax, true);
    mg.inner_b.alloc(sizeof(float2) * (size_t)rows * nmax);
    mg.om = mg.p.outer_m;
    mg.oV.alloc(sizeof(double2) * (size_t)(mg.om + 1) * rows * nmax);
    mg.oZ.alloc(sizeof(float2) * (size_t)mg.om * rows * nmax);
    mg.oks.init(mg.om, nmax);
    mg.osc.ensure(current_sm_count() * 8, KCHUNK * nmax);
    mg.obn2.alloc(sizeof(double) * nmax);
    MRHS_CUDA(cudaMallocHost(&mg.pinned, sizeof(double) * 4 * nmax));
}

}  // namespace

// ------------------------------------------------------------- solve
namespace mrhs {

// The tensor-core kernels record a bounded mbarrier wait that gave up in a
// per-level flag (their result then lacks an operand).  Read the flags of
// level l's coarse stencil and of its transfer to level l + 1 after the work
// queued on s, clear them, and fail with MRHS_ERR_TIMEOUT if one was set.
void check_wait_flags(const Level &L, cudaStream_t s) {
    if (coarse_tc_error(L, s)) {
        zero_on_sms(L.TcErr.ptr, sizeof(int), s);
        MRHS_CUDA(cudaStreamSynchronize(s));
        fail(MRHS_ERR_TIMEOUT, "tensor-core coarse stencil gave up waiting for its operands");
    }
    if (intergrid_tc_error(L, s)) {
        zero_on_sms(L.IgErr.ptr, sizeof(int), s);
        MRHS_CUDA(cudaStreamSynchronize(s));
        fail(MRHS_ERR_TIMEOUT, "tensor-core restriction / prolongation gave up waiting");
    }
}

void check_all_wait_flags(const mrhs_mg &mg, cudaStream_t s) {
    for (int l = 0; l < mg.nlev; ++l) check_wait_flags(mg.lev[l], s);
}

void clear_all_wait_flags(const mrhs_mg &mg, cudaStream_t s) {
    for (int l = 0; l < mg.nlev; ++l) {
        if (mg.lev[l].TcErr.ptr) zero_on_sms(mg.lev[l].TcErr.ptr, sizeof(int), s);
        if (mg.lev[l].IgErr.ptr) zero_on_sms(mg.lev[l].IgErr.ptr, sizeof(int), s);
    }
}

// Outer FP64 FGMRES; returns true if every RHS r reached tols[r].
// max_outer > 0 caps the outer iterations of this call (else the params' cap);
// stop(res, n) is asked after every outer iteration with the per-RHS residual
// estimates and may end the cycle early (used by the server to free slots).
bool mg_solve(mrhs_mg &mg, const double2 *b, double2 *x, int n, const double *tols, double *rel_out,
              mrhs_solve_stats *st, cudaStream_t s, int max_outer, const std::function<bool(const double *, int)> &stop) {
    const auto t0 = std::chrono::steady_clock::now();
    const mrhs_lattice &lat = *mg.lat;
    const int64_t rows = mg.lev[0].rows();
    const int64_t F = rows * n;
    double2 *V0 = mg.oV.as<double2>();
    float2 *Z0 = mg.oZ.as<float2>();
    double *hbn2 = mg.pinned;          // ||b||^2
    double *hres = mg.pinned + mg.nmax;
    std::vector<double> target(n), rel(n, 0.0), relest(n, 0.0), cur_res(n, 0.0), inner_rel(n, 0.0);
    mg.vcycles = 0;
    int outer = 0, inner_total = 0;
    clear_all_wait_flags(mg, s);
    norm2(MRHS_FP64, b, rows, n, mg.obn2.as<double>(), mg.osc, s);
    read_back(hbn2, mg.obn2.ptr, sizeof(double) * n, s);
    MRHS_CUDA(cudaStreamSynchronize(s));
    std::vector<double> bn2(hbn2, hbn2 + n);
    for (int r = 0; r < n; ++r) target[r] = 0.5 * tols[r] * std::sqrt(bn2[r]);
    const int cap = max_outer > 0 ? max_outer : mg.p.max_outer_iters;
    bool converged = false;
    // a zero start vector (the usual cold start) makes the first residual b itself:
    // skip that FP64 operator application
    bool x_zero = false;
    {
        unsigned *flag = reinterpret_cast<unsigned *>(mg.oks.nn.as<double>());
        any_nonzero(x, sizeof(double2) * F, flag, s);
        unsigned *hflag = reinterpret_cast<unsigned *>(hres);
        read_back(hflag, flag, sizeof(unsigned), s);
        MRHS_CUDA(cudaStreamSynchronize(s));
        x_zero = *hflag == 0u;
    }
    while (true) {
        // true residual in FP64 (for x = 0 it is b, whose norms are known)
        if (x_zero) {
            copy_on_sms(V0, b, sizeof(double2) * F, s);
            copy_on_sms(mg.oks.beta2.ptr, mg.obn2.ptr, sizeof(double) * n, s);
            x_zero = false;
        } else {
            dslash(lat, MRHS_FP64, MRHS_FP64, x, V0, b, n, s);
            norm2(MRHS_FP64, V0, rows, n, mg.oks.beta2.as<double>(), mg.osc, s);
        }
        read_back(hres, mg.oks.beta2.ptr, sizeof(double) * n, s);
        MRHS_CUDA(cudaStreamSynchronize(s));
        converged = true;
        for (int r = 0; r < n; ++r) {
            rel[r] = bn2[r] > 0 ? std::sqrt(hres[r] / bn2[r]) : std::sqrt(hres[r]);
            if (!(rel[r] <= tols[r])) converged = false;
        }
        if (converged || outer >= cap) break;
        krylov_start(mg.oks, n, s);
        scale_inv_sqrt(MRHS_FP64, V0, V0, mg.oks.beta2.as<double>(), rows, n, s);
        for (int r = 0; r < n; ++r) cur_res[r] = std::sqrt(hres[r]);
        int steps = mg.om;
        for (int j = 0; j < mg.om; ++j) {
            float2 *zj = Z0 + (size_t)j * F;
            double2 *vj = V0 + (size_t)j * F;
            double2 *wj = V0 + (size_t)(j + 1) * F;
            cast(MRHS_FP32, mg.inner_b.ptr, MRHS_FP64, vj, F, s);
            // inner accuracy per RHS: inner_tol on the first outer step; later, the
            // reduction that takes RHS r from its current residual to its target
            // (clamped to [inner_tol / 4, 0.1]): looser when earlier steps overshot,
            // tighter when one more step must finish the solve
            for (int r = 0; r < n; ++r) {
                if (outer == 0 || !(cur_res[r] > 0.0)) {
                    inner_rel[r] = mg.p.inner_tol;
                } else {
                    inner_rel[r] = std::min(0.1, std::max(0.25 * mg.p.inner_tol, target[r] / cur_res[r]));
                }
            }
            inner_total += inner_solve(mg, mg.inner_b.as<float2>(), zj, n, inner_rel, s);
            // w = D z_j: z_j is FP32, w FP64 (float-float or FP64 arithmetic)
            dslash(lat, mg.p.outer_op_precision == MRHS_DF64 ? MRHS_DF64 : MRHS_FP64, MRHS_FP32, zj, wj, nullptr, n,
                   s);
            // one pass of classical Gram-Schmidt with the Pythagorean norm (and the
            // cancellation fix-up), as in the FP32 cycles: the outer basis has at most
            // outer_m vectors and FP64 keeps its loss of orthogonality far below tol
            orthonormalize_step(MRHS_FP64, V0, F, j + 1, wj, rows, n, mg.oks.hcol.as<double2>(),
                                mg.oks.nrm2w.as<double>(), mg.oks.hn2.as<double>(), mg.oks.nn.as<double>(), mg.osc,
                                s);
            krylov_givens(mg.oks, j, n, s, true);
            ++outer;
            HostCheck chk{target.data(), hres};
            bool halt = chk.test(mg.oks, n, s) || outer >= cap;
            for (int r = 0; r < n; ++r) cur_res[r] = hres[r];
            if (!halt && stop) {
                for (int r = 0; r < n; ++r) relest[r] = bn2[r] > 0 ? hres[r] / std::sqrt(bn2[r]) : 0.0;
                halt = stop(relest.data(), n);
            }
            if (halt) {
                steps = j + 1;
                break;
            }
        }
        krylov_solve(mg.oks, steps, n, s);
        lincomb(MRHS_FP64, x, MRHS_FP32, Z0, F, steps, mg.oks.y.as<double2>(), 1.0, rows, n, s);
    }
    check_all_wait_flags(mg, s);
    if (rel_out)
        for (int r = 0; r < n; ++r) rel_out[r] = rel[r];
    if (st) {
        st->outer_iters = outer;
        st->inner_iters = inner_total;
        st->vcycles = mg.vcycles;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        double mx = 0;
        for (int r = 0; r < n; ++r) mx = std::max(mx, rel[r]);
        st->max_rel_residual = mx;
    }
    return converged;
}

int mg_max_rhs(const mrhs_mg *mg) { return mg->nmax; }
int64_t mg_fine_rows(const mrhs_mg *mg) { return mg->lev[0].rows(); }
int mg_device(const mrhs_mg *mg) { return mg->lat->device; }
int mg_outer_m(const mrhs_mg *mg) { return mg->p.outer_m; }

}  // namespace mrhs

// ------------------------------------------------------------- C ABI
namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            (void)cudaGetLastError();
            prev = -1;
        }
        if (prev != d) MRHS_CUDA(cudaSetDevice(d));
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

mrhs_status ok() {
    api_record(MRHS_OK, "");
    return MRHS_OK;
}

#define API_TRY try {
#define API_CATCH                                                                   \
    }                                                                               \
    catch (const mrhs::Error &e) { return api_record(e.code, e.what()); }           \
    catch (const std::bad_alloc &) { return api_record(MRHS_ERR_OOM, "host allocation failed"); } \
    catch (const std::exception &e) { return api_record(MRHS_ERR_CUDA, e.what()); }

void check_level(mrhs_mg *mg, int level, int min_level, int max_level) {
    if (!mg) fail(MRHS_ERR_INVALID, "mg must be non-null");
    if (level < min_level || level > max_level) fail(MRHS_ERR_INVALID, "level out of range");
}

void check_n(mrhs_mg *mg, int nrhs) {
    if (nrhs < 1 || nrhs > mg->nmax) fail(MRHS_ERR_INVALID, "nrhs must be in 1..max_rhs");
}

}  // namespace

extern "C" {

void mrhs_mg_default_params(mrhs_mg_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n_levels = 3;
    for (int mu = 0; mu < 4; ++mu) {
        p->block[0][mu] = 4;
        p->block[1][mu] = 2;
    }
    p->n_vec[0] = 32;
    p->n_vec[1] = 32;
    p->setup_sweeps = 6;
    p->setup_m = 8;
    p->smooth_m = 3;
    p->coarse_m = 14;
    p->coarse_cycles = 1;
    p->inter_m = 4;
    p->inner_m = 8;
    p->inner_max_iters = 200;
    p->inner_tol = 1e-5;
    p->outer_m = 4;
    p->max_outer_iters = 30;
    p->coarse_precision = MRHS_FP16;
    p->max_rhs = 48;
    p->use_graph = 1;
    p->outer_op_precision = MRHS_DF64;
    p->smoother_evenodd = 1;
    p->seed = 1234;
    p->smoother_sap = 0;
    for (int mu = 0; mu < 4; ++mu) p->sap_block[mu] = 4;
    p->sap_cycles = 1;
    p->sap_mr = 4;
    p->coarse_smoother_evenodd = 0;
    p->coarse_solver = 0;
    p->coarse_recycle = 4;
    p->coarse_fused = 1;
    p->galerkin_tc = 1;
}

mrhs_status mrhs_setup_mg(mrhs_lattice *lat, const mrhs_mg_params *params, mrhs_mg **out) {
    API_TRY
    if (!lat || !params || !out) fail(MRHS_ERR_INVALID, "lattice, params and out must be non-null");
    *out = nullptr;
    if (!lat->has_clover) fail(MRHS_ERR_INVALID, "clover term not built");
    validate_params(lat, *params);
    DevGuard dg(lat->device);
    auto mg = std::make_unique<mrhs_mg>();
    mg->lat = lat;
    mg->p = *params;
    mg->nlev = params->n_levels;
    mg->nmax = params->max_rhs;
    mg->profile = std::getenv("MRHS_PROFILE") && std::atoi(std::getenv("MRHS_PROFILE")) != 0;
    mg->lev.resize(mg->nlev);
    // geometry
    Level &f = mg->lev[0];
    for (int mu = 0; mu < 4; ++mu) f.L[mu] = lat->g.L[mu];
    f.V = lat->g.V;
    f.dof = 12;
    for (int l = 0; l < mg->nlev - 1; ++l) {
        Level &F = mg->lev[l];
        Level &C = mg->lev[l + 1];
        for (int mu = 0; mu < 4; ++mu) {
            F.B[mu] = params->block[l][mu];
            C.L[mu] = F.L[mu] / F.B[mu];
        }
        F.N = params->n_vec[l];
        F.asize = (int64_t)F.B[0] * F.B[1] * F.B[2] * F.B[3];
        C.V = (int64_t)C.L[0] * C.L[1] * C.L[2] * C.L[3];
        C.dof = 2 * F.N;
    }
    mg->ops.emplace_back(new FineOp(lat));
    cudaStream_t s = nullptr;
    MRHS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    try {
        for (int l = 0; l < mg->nlev - 1; ++l) {
            PhaseEvents ph;
            setup_level(*mg, l, s, ph);
            Level &C = mg->lev[l + 1];
            const bool use_tc = (params->coarse_precision == MRHS_BF16 || params->coarse_precision == MRHS_FP16) &&
                                coarse_bf16_supported(C);
            if (use_tc) coarse_links_to_16bit(C, (mrhs_precision)params->coarse_precision, s);
            // coarse even-odd smoother: intermediate levels (those that post-smooth) only
            if (use_tc && params->coarse_smoother_evenodd && l + 2 < mg->nlev && coarse_eo_supported(C))
                coarse_eo_prepare(C, s);
            // 16-bit hierarchies also move fields between levels on the tensor cores
            Level &F = mg->lev[l];
            if ((params->coarse_precision == MRHS_BF16 || params->coarse_precision == MRHS_FP16) &&
                intergrid_tc_supported(F)) {
                intergrid_tc_prepare(F, C, s);
                F.tc_intergrid = true;
            }
            ph.mark(s);
            MRHS_CUDA(cudaStreamSynchronize(s));
            ph.read(mg->setup_ms[l], 4);
            mg->ops.emplace_back(new CoarseOp(&C, use_tc));
        }
        MRHS_CUDA(cudaStreamSynchronize(s));
        alloc_workspace(*mg);
        MRHS_CUDA(cudaStreamCreateWithFlags(&mg->own, cudaStreamNonBlocking));
        MRHS_CUDA(cudaEventCreateWithFlags(&mg->ev_in, cudaEventDisableTiming));
        MRHS_CUDA(cudaEventCreateWithFlags(&mg->ev_out, cudaEventDisableTiming));
    } catch (...) {
        cudaStreamDestroy(s);
        throw;
    }
    cudaStreamDestroy(s);
    *out = mg.release();
    return ok();
    API_CATCH
}

void mrhs_destroy_mg(mrhs_mg *mg) {
    if (!mg) return;
    try {
        DevGuard dg(mg->lat->device);
        cudaDeviceSynchronize();
        delete mg;
    } catch (...) {
        delete mg;
    }
}

mrhs_status mrhs_mg_level_info(mrhs_mg *mg, int level, int dims[4], int *dof) {
    API_TRY
    check_level(mg, level, 0, mg ? mg->nlev - 1 : 0);
    if (!dims || !dof) fail(MRHS_ERR_INVALID, "outputs must be non-null");
    for (int mu = 0; mu < 4; ++mu) dims[mu] = mg->lev[level].L[mu];
    *dof = mg->lev[level].dof;
    return ok();
    API_CATCH
}

mrhs_status mrhs_mg_get_prolongator(mrhs_mg *mg, int level, double *host_out) {
    API_TRY
    check_level(mg, level, 0, mg ? mg->nlev - 2 : 0);
    if (!host_out) fail(MRHS_ERR_INVALID, "output must be non-null");
    DevGuard dg(mg->lat->device);
    const Level &F = mg->lev[level];
    MRHS_CUDA(cudaMemcpy(host_out, F.P64.ptr, sizeof(double2) * F.V * F.dof * F.N, cudaMemcpyDeviceToHost));
    return ok();
    API_CATCH
}

mrhs_status mrhs_mg_get_coarse_links(mrhs_mg *mg, int level, double *host_out) {
    API_TRY
    check_level(mg, level, 1, mg ? mg->nlev - 1 : 1);
    if (!host_out) fail(MRHS_ERR_INVALID, "output must be non-null");
    DevGuard dg(mg->lat->device);
    const Level &C = mg->lev[level];
    const size_t count = (size_t)C.V * 9 * C.dof * C.dof;
    std::vector<float2> tmp(count);
    MRHS_CUDA(cudaMemcpy(tmp.data(), C.A32.ptr, sizeof(float2) * count, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < count; ++i) {
        host_out[2 * i] = tmp[i].x;
        host_out[2 * i + 1] = tmp[i].y;
    }
    return ok();
    API_CATCH
}

mrhs_status mrhs_restrict(mrhs_mg *mg, int level, const void *fine_dev, void *coarse_dev, int nrhs, void *stream) {
    API_TRY
    check_level(mg, level, 0, mg ? mg->nlev - 2 : 0);
    check_n(mg, nrhs);
    if (!fine_dev || !coarse_dev) fail(MRHS_ERR_INVALID, "fields must be non-null");
    DevGuard dg(mg->lat->device);
    const Level &C = mg->lev[level + 1];
    const Level &F = mg->lev[level];
    if (F.tc_intergrid) {
        restrict_fields_tc(F, C, static_cast<const float2 *>(fine_dev), static_cast<float2 *>(coarse_dev), nrhs,
                           (int64_t)C.dof * nrhs, false, static_cast<cudaStream_t>(stream));
        check_wait_flags(F, static_cast<cudaStream_t>(stream));
    } else
        restrict_fields(F, C, static_cast<const float2 *>(fine_dev), static_cast<float2 *>(coarse_dev), nrhs,
                        (int64_t)C.dof * nrhs, static_cast<cudaStream_t>(stream));
    return ok();
    API_CATCH
}

mrhs_status mrhs_prolong(mrhs_mg *mg, int level, const void *coarse_dev, void *fine_dev, int nrhs, void *stream) {
    API_TRY
    check_level(mg, level, 0, mg ? mg->nlev - 2 : 0);
    check_n(mg, nrhs);
    if (!fine_dev || !coarse_dev) fail(MRHS_ERR_INVALID, "fields must be non-null");
    DevGuard dg(mg->lat->device);
    if (mg->lev[level].tc_intergrid) {
        prolong_fields_tc(mg->lev[level], mg->lev[level + 1], static_cast<const float2 *>(coarse_dev),
                          static_cast<float2 *>(fine_dev), nrhs, static_cast<cudaStream_t>(stream));
        check_wait_flags(mg->lev[level], static_cast<cudaStream_t>(stream));
    } else
        prolong_fields(mg->lev[level], mg->lev[level + 1], static_cast<const float2 *>(coarse_dev),
                       static_cast<float2 *>(fine_dev), nrhs, static_cast<cudaStream_t>(stream));
    return ok();
    API_CATCH
}

mrhs_status mrhs_coarse_apply(mrhs_mg *mg, int level, const void *in_dev, void *out_dev, int nrhs,
                              mrhs_precision links_prec, void *stream) {
    API_TRY
    check_level(mg, level, 1, mg ? mg->nlev - 1 : 1);
    if (nrhs < 1 || nrhs > 64) fail(MRHS_ERR_INVALID, "nrhs must be in 1..64");
    if (!in_dev || !out_dev || in_dev == out_dev) fail(MRHS_ERR_INVALID, "distinct non-null fields required");
    DevGuard dg(mg->lat->device);
    const Level &C = mg->lev[level];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (links_prec == MRHS_FP32) {
        coarse_apply_fp32(C, static_cast<const float2 *>(in_dev), static_cast<float2 *>(out_dev), nullptr, nrhs, s);
    } else if (links_prec == MRHS_BF16 || links_prec == MRHS_FP16) {
        if (!C.Abf.ptr || C.tc_fmt != links_prec)
            fail(MRHS_ERR_INVALID, "no 16-bit links of this format on this level (needs nc = 64 and that coarse_precision)");
        coarse_apply_bf16(C, static_cast<const float2 *>(in_dev), static_cast<float2 *>(out_dev), nullptr, nrhs, s);
        check_wait_flags(C, s);
    } else {
        fail(MRHS_ERR_INVALID, "links precision must be FP32 or BF16");
    }
    return ok();
    API_CATCH
}

mrhs_status mrhs_coarse_apply_schur(mrhs_mg *mg, int level, const void *in_dev, void *out_dev, int nrhs,
                                    void *stream) {
    API_TRY
    check_level(mg, level, 1, mg ? mg->nlev - 1 : 1);
    if (nrhs < 1 || nrhs > 64) fail(MRHS_ERR_INVALID, "nrhs must be in 1..64");
    if (!in_dev || !out_dev || in_dev == out_dev) fail(MRHS_ERR_INVALID, "distinct non-null fields required");
    DevGuard dg(mg->lat->device);
    const Level &C = mg->lev[level];
    if (!C.AinvBf.ptr)
        fail(MRHS_ERR_INVALID, "no coarse even-odd decomposition on this level (needs coarse_smoother_evenodd, "
                               "16-bit links and even coarse extents on an intermediate level)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t half = sizeof(float2) * (size_t)(C.V / 2) * C.dof * nrhs;
    DeviceBuffer t1(half), t2(half);
    coarse_schur_apply(C, static_cast<const float2 *>(in_dev), static_cast<float2 *>(out_dev), t1.as<float2>(),
                       t2.as<float2>(), nrhs, s);
    check_wait_flags(C, s);
    return ok();
    API_CATCH
}

mrhs_status mrhs_coarsest_solve(mrhs_mg *mg, const void *b_dev, void *x_dev, int nrhs, void *stream) {
    API_TRY
    if (!mg) fail(MRHS_ERR_INVALID, "mg must be non-null");
    check_n(mg, nrhs);
    if (!b_dev || !x_dev || b_dev == x_dev) fail(MRHS_ERR_INVALID, "distinct non-null fields required");
    DevGuard dg(mg->lat->device);
    const int l = mg->nlev - 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LevelWork &W = mg->work[l];
    const float2 *b = static_cast<const float2 *>(b_dev);
    float2 *x = static_cast<float2 *>(x_dev);
    coarsest_solve(*mg, b, x, nrhs, s);
    if (W.gcro) {
        int *e = pinned_flag_slot();
        read_back(e, W.gcro->err.ptr, sizeof(int), s);
        MRHS_CUDA(cudaStreamSynchronize(s));
        if (*e) {
            MRHS_CUDA(cudaMemset(W.gcro->err.ptr, 0, sizeof(int)));
            fail(MRHS_ERR_CUDA, "GCRO-DR: the QR algorithm of a harmonic Ritz problem did not converge");
        }
    }
    check_wait_flags(mg->lev[l], s);
    return ok();
    API_CATCH
}

mrhs_status mrhs_mg_setup_times(mrhs_mg *mg, int level, double out_ms[4]) {
    API_TRY
    if (!mg || !out_ms) fail(MRHS_ERR_INVALID, "non-null mg and output required");
    if (level < 0 || level >= mg->nlev - 1) fail(MRHS_ERR_INVALID, "level must name a transfer l -> l+1");
    for (int i = 0; i < 4; ++i) out_ms[i] = mg->setup_ms[level][i];
    return ok();
    API_CATCH
}

mrhs_status mrhs_coarsest_fused_info(mrhs_mg *mg, int *in_use, int *resident_ctas, int *sites) {
    API_TRY
    if (!mg || !in_use || !resident_ctas || !sites) fail(MRHS_ERR_INVALID, "non-null mg and outputs required");
    DevGuard dg(mg->lat->device);
    const int l = mg->nlev - 1;
    *in_use = mg->work[l].fused ? 1 : 0;
    *resident_ctas = l >= 1 ? CoarsestFused::resident_ctas(mg->lev[l], mg->nmax, mg->lat->device) : 0;
    *sites = (int)mg->lev[l].V;
    return ok();
    API_CATCH
}

mrhs_status mrhs_coarsest_reset(mrhs_mg *mg) {
    API_TRY
    if (!mg) fail(MRHS_ERR_INVALID, "mg must be non-null");
    LevelWork &W = mg->work[mg->nlev - 1];
    if (W.gcro) W.gcro->has_recycle = false;
    return ok();
    API_CATCH
}

mrhs_status mrhs_vcycle(mrhs_mg *mg, const void *v_dev, void *z_dev, int nrhs, void *stream) {
    API_TRY
    check_level(mg, 0, 0, 0);
    check_n(mg, nrhs);
    if (!v_dev || !z_dev || v_dev == z_dev) fail(MRHS_ERR_INVALID, "distinct non-null fields required");
    DevGuard dg(mg->lat->device);
    vcycle(*mg, 0, static_cast<const float2 *>(v_dev), static_cast<float2 *>(z_dev), nrhs,
           static_cast<cudaStream_t>(stream), false);
    check_all_wait_flags(*mg, static_cast<cudaStream_t>(stream));
    return ok();
    API_CATCH
}

mrhs_status mrhs_solve(mrhs_mg *mg, const void *b_dev, void *x_dev, int nrhs, double tol, double *rel_res_host,
                       mrhs_solve_stats *stats, void *stream) {
    API_TRY
    if (!mg) fail(MRHS_ERR_INVALID, "mg must be non-null");
    check_n(mg, nrhs);
    if (!b_dev || !x_dev || b_dev == x_dev) fail(MRHS_ERR_INVALID, "distinct non-null b and x required");
    if (!(tol > 0 && tol < 1)) fail(MRHS_ERR_INVALID, "tol must be in (0, 1)");
    DevGuard dg(mg->lat->device);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    mg->t_fine = mg->t_restrict = mg->t_prolong = mg->t_coarse = 0;
    std::vector<double> tols(nrhs, tol);
    // order the solve after the caller's prior work on `stream`, run it on the
    // solver's own stream, and order the caller's later work after it
    MRHS_CUDA(cudaEventRecord(mg->ev_in, user));
    MRHS_CUDA(cudaStreamWaitEvent(mg->own, mg->ev_in, 0));
    const bool conv = mg_solve(*mg, static_cast<const double2 *>(b_dev), static_cast<double2 *>(x_dev), nrhs,
                               tols.data(), rel_res_host, stats, mg->own, 0, nullptr);
    MRHS_CUDA(cudaEventRecord(mg->ev_out, mg->own));
    MRHS_CUDA(cudaStreamWaitEvent(user, mg->ev_out, 0));
    MRHS_CUDA(cudaStreamSynchronize(mg->own));
    if (stats) {
        stats->t_fine = mg->t_fine;
        stats->t_restrict = mg->t_restrict;
        stats->t_prolong = mg->t_prolong;
        stats->t_coarse = mg->t_coarse;
    }
    if (!conv) return api_record(MRHS_ERR_NOT_CONVERGED, "outer iteration cap reached before tol");
    return ok();
    API_CATCH
}

}  // extern "C"
