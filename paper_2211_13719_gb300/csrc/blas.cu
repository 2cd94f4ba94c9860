// Batched BLAS-1 over the RHS index (paper Sec. 7: inner products of many
// RHS computed "simultaneously" in one pass instead of one after another).
//
// A field is `rows` rows of `n` complex values, RHS innermost.  A block of
// n * rpb threads (rpb = rows per block pass) gives each thread one RHS
// column and a strided set of rows, so every warp load is contiguous in
// memory.  Each thread accumulates its rows; the block reduces over its
// row-threads in a fixed order into a per-block partial; the last block to
// finish (atomic ticket) sums the partials in block order.  The sum order of
// RHS r therefore depends only on (rows, n, grid), never on the values of
// other RHS: batching does not change a result beyond that fixed order.
//
// FP32 fields are accumulated in FP32 per thread and in FP64 from the block
// level up; FP64 fields in FP64 throughout.  Outputs are FP64.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace mrhs {

static int g_sm_count[64] = {0};

int sm_count(int device) {
    if (device < 0 || device >= 64) return 148;
    if (!g_sm_count[device]) {
        int v = 0;
        MRHS_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device));
        g_sm_count[device] = v > 0 ? v : 148;
    }
    return g_sm_count[device];
}

static int current_sms() {
    int dev = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    return sm_count(dev);
}

void Scratch::ensure(int blocks, int cols) {
    if (!counter.ptr) {
        counter.alloc(sizeof(unsigned int) * 4);
        MRHS_CUDA(cudaMemset(counter.ptr, 0, sizeof(unsigned int) * 4));
    }
    if (blocks > max_blocks || cols > max_cols) {
        const int b = std::max(blocks, max_blocks);
        const int c = std::max(cols, max_cols);
        partials.alloc(sizeof(double2) * (size_t)b * (size_t)c);
        max_blocks = b;
        max_cols = c;
    }
}

struct RedGeom {
    int rpb;      // rows per block pass
    int threads;  // n * rpb
    int blocks;
};

static RedGeom red_geom(int64_t rows, int n) {
    RedGeom r;
    r.rpb = n >= 256 ? 1 : 256 / n;
    r.threads = n * r.rpb;
    // at least 32 rows per thread, at most 4 blocks per SM: enough loads in
    // flight for HBM on large fields, few partials for the last block to sum
    // on the small coarse-level fields
    const int64_t need = (rows + 32 * r.rpb - 1) / (32 * r.rpb);
    const int64_t cap = (int64_t)current_sms() * 4;
    r.blocks = (int)std::max<int64_t>(1, std::min(need, cap));
    return r;
}

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

template <typename T> __device__ __forceinline__ cplx<T> ldv(const T *p, int64_t i) {
    const typename vec2<T>::type v = reinterpret_cast<const typename vec2<T>::type *>(p)[i];
    return {v.x, v.y};
}
template <typename T> __device__ __forceinline__ void stv(T *p, int64_t i, cplx<T> v) {
    typename vec2<T>::type o;
    o.x = v.re;
    o.y = v.im;
    reinterpret_cast<typename vec2<T>::type *>(p)[i] = o;
}

// Block-level fixed-order reduction of `cols` complex values per thread
// (vals[c] for c < cols), then the cross-block finish by the last block.
// smem: double2 [rpb][cols][n] laid out as [(rsub*cols + c)*n + col].
// With real_only the single column goes to out_real; with real_tail the
// first cols-1 columns go to out and the last column's real part to out_real.
__device__ void block_finish(double2 *smem, const double2 *vals, int cols, int n, int rpb, int col, int rsub,
                             double2 *partials, unsigned int *counter, double2 *out, bool accumulate,
                             bool real_only, double *out_real, bool real_tail = false) {
    for (int c = 0; c < cols; ++c) smem[((int64_t)rsub * cols + c) * n + col] = vals[c];
    __syncthreads();
    const int tid = threadIdx.x;
    const int nout = cols * n;
    for (int o = tid; o < nout; o += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < rpb; ++q) {
            const double2 v = smem[(int64_t)q * nout + o];
            s.x += v.x;
            s.y += v.y;
        }
        partials[(int64_t)blockIdx.x * nout + o] = s;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int ticket = atomicAdd(counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int o = tid; o < nout; o += blockDim.x) {
        // fixed order: four interleaved partial sums over the blocks, then combined
        double2 q[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                        make_double2(0.0, 0.0)};
        const int nb = (int)gridDim.x;
        int b = 0;
        for (; b + 4 <= nb; b += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double2 v = __ldcg(&partials[(int64_t)(b + u) * nout + o]);
                q[u].x += v.x;
                q[u].y += v.y;
            }
        }
        for (; b < nb; ++b) {
            const double2 v = __ldcg(&partials[(int64_t)b * nout + o]);
            q[0].x += v.x;
            q[0].y += v.y;
        }
        double2 s = make_double2((q[0].x + q[1].x) + (q[2].x + q[3].x), (q[0].y + q[1].y) + (q[2].y + q[3].y));
        if (real_only) {
            out_real[o] = s.x;
        } else if (real_tail && o >= (cols - 1) * n) {
            out_real[o - (cols - 1) * n] = s.x;
        } else if (accumulate) {
            double2 prev = out[o];
            out[o] = make_double2(prev.x + s.x, prev.y + s.y);
        } else {
            out[o] = s;
        }
    }
    if (tid == 0) *counter = 0u;
}

// out[j][r] = sum_i conj(b_j[i][r]) w[i][r], j < k <= KCHUNK
template <typename T>
__global__ void k_multi_dot(const T *__restrict__ basis, int64_t stride, int k, const T *__restrict__ w,
                            int64_t rows, int n, int rpb, double2 *partials, unsigned int *counter,
                            double2 *out, int accumulate) {
    extern __shared__ double2 smem[];
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    cplx<T> acc[KCHUNK];
#pragma unroll
    for (int j = 0; j < KCHUNK; ++j) acc[j] = {0, 0};
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        const cplx<T> x = ldv(w, e);
#pragma unroll
        for (int j = 0; j < KCHUNK; ++j)
            if (j < k) cmac_conj(acc[j], ldv(basis, e + j * stride), x);
    }
    double2 vals[KCHUNK];
#pragma unroll
    for (int j = 0; j < KCHUNK; ++j) vals[j] = make_double2((double)acc[j].re, (double)acc[j].im);
    block_finish(smem, vals, k, n, rpb, col, rsub, partials, counter, out, accumulate != 0, false, nullptr);
}

template <typename T>
__global__ void k_norm2(const T *__restrict__ w, int64_t rows, int n, int rpb, double2 *partials,
                        unsigned int *counter, double *out) {
    extern __shared__ double2 smem[];
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    T acc = 0;
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const cplx<T> x = ldv(w, row * n + col);
        acc = fmadd(x.re, x.re, acc);
        acc = fmadd(x.im, x.im, acc);
    }
    double2 v = make_double2((double)acc, 0.0);
    block_finish(smem, &v, 1, n, rpb, col, rsub, partials, counter, nullptr, false, true, out);
}

// w += alpha * sum_j coef[j][r] b_j ; optional ||w||^2 per RHS
template <typename TW, typename TB, bool NORM>
__global__ void k_lincomb(TW *__restrict__ w, const TB *__restrict__ basis, int64_t stride, int k,
                          const double2 *__restrict__ coef, double alpha, int64_t rows, int n, int rpb,
                          double2 *partials, unsigned int *counter, double *norm_out) {
    extern __shared__ double2 smem[];
    // coefficients of this thread's column, scaled by alpha, in the basis precision
    using TC = typename std::conditional<sizeof(TW) == 8 || sizeof(TB) == 8, double, float>::type;
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    cplx<TC> cf[KCHUNK];
#pragma unroll
    for (int j = 0; j < KCHUNK; ++j) {
        if (j < k) {
            const double2 c = coef[(int64_t)j * n + col];
            cf[j] = {(TC)(alpha * c.x), (TC)(alpha * c.y)};
        } else {
            cf[j] = {0, 0};
        }
    }
    TW nacc = 0;
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        cplx<TC> s = {0, 0};
#pragma unroll
        for (int j = 0; j < KCHUNK; ++j) {
            if (j < k) {
                const cplx<TB> b = ldv(basis, e + j * stride);
                cmac(s, cf[j], cplx<TC>{(TC)b.re, (TC)b.im});
            }
        }
        cplx<TW> x = ldv(w, e);
        x.re += (TW)s.re;
        x.im += (TW)s.im;
        stv(w, e, x);
        if (NORM) {
            nacc = fmadd(x.re, x.re, nacc);
            nacc = fmadd(x.im, x.im, nacc);
        }
    }
    if (NORM) {
        double2 v = make_double2((double)nacc, 0.0);
        block_finish(smem, &v, 1, n, rpb, col, rsub, partials, counter, nullptr, false, true, norm_out);
    }
}

// dst = src / sqrt(nrm2[col]); one RHS column per thread, factor computed once
template <typename T>
__global__ void k_scale_inv_sqrt(T *dst, const T *src, const double *nrm2, int64_t rows, int n, int rpb) {
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    const double v = nrm2[col];
    const T f = v > 0.0 ? (T)(1.0 / sqrt(v)) : (T)0;
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        const cplx<T> x = ldv(src, e);
        stv(dst, e, cplx<T>{x.re * f, x.im * f});
    }
}

template <typename TD, typename TS>
__global__ void k_cast(TD *dst, const TS *src, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const cplx<TS> x = ldv(src, i);
    stv(dst, i, cplx<TD>{(TD)x.re, (TD)x.im});
}

template <typename T>
__global__ void k_axpy(T a, const T *x, T *y, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const cplx<T> u = ldv(x, i);
    cplx<T> v = ldv(y, i);
    v.re = fmadd(a, u.re, v.re);
    v.im = fmadd(a, u.im, v.im);
    stv(y, i, v);
}

// out[j][r] = <b_j, w>_r for j < k (k < KCHUNK) and nrm2[r] = ||w_r||^2, one pass over w
template <typename T>
__global__ void k_dots_norm(const T *__restrict__ basis, int64_t stride, int k, const T *__restrict__ w,
                            int64_t rows, int n, int rpb, double2 *partials, unsigned int *counter, double2 *out,
                            double *nrm2) {
    extern __shared__ double2 smem[];
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    cplx<T> acc[KCHUNK];
#pragma unroll
    for (int j = 0; j < KCHUNK; ++j) acc[j] = {0, 0};
    T nacc = 0;
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        const cplx<T> x = ldv(w, e);
        nacc = fmadd(x.re, x.re, nacc);
        nacc = fmadd(x.im, x.im, nacc);
#pragma unroll
        for (int j = 0; j < KCHUNK - 1; ++j)
            if (j < k) cmac_conj(acc[j], ldv(basis, e + j * stride), x);
    }
    double2 vals[KCHUNK];
#pragma unroll
    for (int j = 0; j < KCHUNK; ++j) vals[j] = make_double2((double)acc[j].re, (double)acc[j].im);
    vals[k] = make_double2((double)nacc, 0.0);
    block_finish(smem, vals, k + 1, n, rpb, col, rsub, partials, counter, out, false, false, nrm2, true);
}

// w <- (w - sum_{j<k} h_j b_j) / beta with beta^2 = max(||w||^2 - sum_{all j<kall} |h_j|^2, 1e-6 ||w||^2)
// (Pythagoras for an orthonormal basis); writes beta^2 to hn2 and ||w_new||^2 to nn.
// `coef` points at the first of the k coefficients handled here, `hall` at all kall of them.
template <typename T>
__global__ void k_lincomb_scale(T *__restrict__ w, const T *__restrict__ basis, int64_t stride, int k,
                                const double2 *__restrict__ coef, const double2 *__restrict__ hall, int kall,
                                const double *__restrict__ nrm2, double *__restrict__ hn2, int64_t rows, int n,
                                int rpb, double2 *partials, unsigned int *counter, double *nn) {
    extern __shared__ double2 smem[];
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    double hh = 0.0;
    for (int j = 0; j < kall; ++j) {
        const double2 c = hall[(int64_t)j * n + col];
        hh += c.x * c.x + c.y * c.y;
    }
    const double w2 = nrm2[col];
    const double b2 = fmax(w2 - hh, 1e-6 * w2);
    const double inv = b2 > 0.0 ? 1.0 / sqrt(b2) : 0.0;
    if (blockIdx.x == 0 && rsub == 0) hn2[col] = b2;
    cplx<T> cf[KCHUNK];
#pragma unroll
    for (int j = 0; j < KCHUNK; ++j) {
        if (j < k) {
            const double2 c = coef[(int64_t)j * n + col];
            cf[j] = {(T)(-c.x), (T)(-c.y)};
        } else {
            cf[j] = {0, 0};
        }
    }
    const T f = (T)inv;
    T nacc = 0;
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        cplx<T> x = ldv(w, e);
#pragma unroll
        for (int j = 0; j < KCHUNK; ++j)
            if (j < k) cmac(x, cf[j], ldv(basis, e + j * stride));
        x.re *= f;
        x.im *= f;
        stv(w, e, x);
        nacc = fmadd(x.re, x.re, nacc);
        nacc = fmadd(x.im, x.im, nacc);
    }
    double2 v = make_double2((double)nacc, 0.0);
    block_finish(smem, &v, 1, n, rpb, col, rsub, partials, counter, nullptr, false, true, nn);
}

// columns whose new basis vector is not unit length (cancellation in the
// Pythagorean norm) are rescaled; the Givens step applies the same factor to beta
// columns whose new basis vector is not unit length (cancellation in the
// Pythagorean norm) are rescaled; the Givens step applies the same factor to
// beta.  One column per thread: unflagged columns return without touching data.
template <typename T>
__global__ void k_norm_fixup(T *__restrict__ w, const double *__restrict__ nn, int64_t rows, int n, int rpb) {
    const int col = threadIdx.x % n;
    const int rsub = threadIdx.x / n;
    const double f = nn[col];
    if (!(f > 0.0 && fabs(f - 1.0) > 1e-2)) return;
    const T sc = (T)(1.0 / sqrt(f));
    const int64_t step = (int64_t)gridDim.x * rpb;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        const cplx<T> x = ldv(w, e);
        stv(w, e, cplx<T>{x.re * sc, x.im * sc});
    }
}

// ------------------------------------------------------------- launchers
static void check_n(int n) {
    if (n < 1 || n > 256) fail(MRHS_ERR_INVALID, "batched BLAS supports 1 <= nrhs <= 256");
}

void multi_dot(mrhs_precision p, const void *basis, int64_t stride, int k, const void *w, int64_t rows, int n,
               double2 *out, Scratch &sc, cudaStream_t s, bool accumulate) {
    check_n(n);
    if (k <= 0) return;
    const RedGeom g = red_geom(rows, n);
    for (int j0 = 0; j0 < k; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        sc.ensure(g.blocks, kk * n);
        const size_t smem = sizeof(double2) * (size_t)g.rpb * kk * n;
        if (p == MRHS_FP32) {
            k_multi_dot<float><<<g.blocks, g.threads, smem, s>>>(
                static_cast<const float *>(basis) + 2 * j0 * stride, stride, kk, static_cast<const float *>(w), rows, n,
                g.rpb, sc.partials.as<double2>(), sc.counter.as<unsigned int>(), out + (int64_t)j0 * n, accumulate);
        } else if (p == MRHS_FP64) {
            k_multi_dot<double><<<g.blocks, g.threads, smem, s>>>(
                static_cast<const double *>(basis) + 2 * j0 * stride, stride, kk, static_cast<const double *>(w), rows,
                n, g.rpb, sc.partials.as<double2>(), sc.counter.as<unsigned int>(), out + (int64_t)j0 * n, accumulate);
        } else {
            fail(MRHS_ERR_INVALID, "multi_dot: FP32 or FP64 fields");
        }
        MRHS_LAUNCHED("k_multi_dot");
    }
}

void orthonormalize_step(mrhs_precision p, const void *basis, int64_t stride, int k, void *w, int64_t rows, int n,
                         double2 *h, double *nrm2, double *hn2, double *nn, Scratch &sc, cudaStream_t s) {
    check_n(n);
    const RedGeom g = red_geom(rows, n);
    const bool f32 = p == MRHS_FP32;
    if (!f32 && p != MRHS_FP64) fail(MRHS_ERR_INVALID, "orthonormalize: FP32 or FP64 fields");
    // dots (and ||w||^2 with the last chunk)
    for (int j0 = 0; j0 < k || j0 == 0; j0 += KCHUNK - 1) {
        const int kk = std::min(KCHUNK - 1, k - j0);
        const bool last = j0 + kk >= k;
        const size_t esz = f32 ? 8 : 16;
        if (last) {
            sc.ensure(g.blocks, (kk + 1) * n);
            const size_t smem = sizeof(double2) * (size_t)g.rpb * (kk + 1) * n;
            if (f32)
                k_dots_norm<float><<<g.blocks, g.threads, smem, s>>>(
                    static_cast<const float *>(basis) + 2 * j0 * stride, stride, kk, static_cast<const float *>(w),
                    rows, n, g.rpb, sc.partials.as<double2>(), sc.counter.as<unsigned int>(), h + (int64_t)j0 * n, nrm2);
            else
                k_dots_norm<double><<<g.blocks, g.threads, smem, s>>>(
                    static_cast<const double *>(basis) + 2 * j0 * stride, stride, kk, static_cast<const double *>(w),
                    rows, n, g.rpb, sc.partials.as<double2>(), sc.counter.as<unsigned int>(), h + (int64_t)j0 * n, nrm2);
            MRHS_LAUNCHED("k_dots_norm");
            break;
        }
        multi_dot(p, static_cast<const char *>(basis) + esz * j0 * stride, stride, kk, w, rows, n,
                  h + (int64_t)j0 * n, sc, s);
    }
    // subtract, normalise
    for (int j0 = 0; j0 < k || j0 == 0; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        const bool last = j0 + kk >= k;
        const size_t esz = f32 ? 8 : 16;
        if (!last) {
            lincomb(p, w, p, static_cast<const char *>(basis) + esz * j0 * stride, stride, kk, h + (int64_t)j0 * n,
                    -1.0, rows, n, s);
            continue;
        }
        sc.ensure(g.blocks, n);
        const size_t smem = sizeof(double2) * (size_t)g.rpb * n;
        if (f32)
            k_lincomb_scale<float><<<g.blocks, g.threads, smem, s>>>(
                static_cast<float *>(w), static_cast<const float *>(basis) + 2 * j0 * stride, stride, kk,
                h + (int64_t)j0 * n, h, k, nrm2, hn2, rows, n, g.rpb, sc.partials.as<double2>(),
                sc.counter.as<unsigned int>(), nn);
        else
            k_lincomb_scale<double><<<g.blocks, g.threads, smem, s>>>(
                static_cast<double *>(w), static_cast<const double *>(basis) + 2 * j0 * stride, stride, kk,
                h + (int64_t)j0 * n, h, k, nrm2, hn2, rows, n, g.rpb, sc.partials.as<double2>(),
                sc.counter.as<unsigned int>(), nn);
        MRHS_LAUNCHED("k_lincomb_scale");
        break;
    }
    if (f32)
        k_norm_fixup<float><<<g.blocks, g.threads, 0, s>>>(static_cast<float *>(w), nn, rows, n, g.rpb);
    else
        k_norm_fixup<double><<<g.blocks, g.threads, 0, s>>>(static_cast<double *>(w), nn, rows, n, g.rpb);
    MRHS_LAUNCHED("k_norm_fixup");
}

void multi_dot_fixed_scratch(mrhs_precision p, const void *basis, int64_t stride, int k, const void *w, int64_t rows,
                             int n, double2 *out, double2 *partials, unsigned int *counter, int max_blocks,
                             cudaStream_t s) {
    check_n(n);
    RedGeom g = red_geom(rows, n);
    g.blocks = std::min(g.blocks, max_blocks);
    for (int j0 = 0; j0 < k; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        const size_t smem = sizeof(double2) * (size_t)g.rpb * kk * n;
        if (p == MRHS_FP32)
            k_multi_dot<float><<<g.blocks, g.threads, smem, s>>>(
                static_cast<const float *>(basis) + 2 * j0 * stride, stride, kk, static_cast<const float *>(w), rows, n,
                g.rpb, partials, counter, out + (int64_t)j0 * n, 0);
        else
            k_multi_dot<double><<<g.blocks, g.threads, smem, s>>>(
                static_cast<const double *>(basis) + 2 * j0 * stride, stride, kk, static_cast<const double *>(w), rows,
                n, g.rpb, partials, counter, out + (int64_t)j0 * n, 0);
        MRHS_LAUNCHED("k_multi_dot");
    }
}

void norm2(mrhs_precision p, const void *w, int64_t rows, int n, double *out, Scratch &sc, cudaStream_t s) {
    check_n(n);
    const RedGeom g = red_geom(rows, n);
    sc.ensure(g.blocks, n);
    const size_t smem = sizeof(double2) * (size_t)g.rpb * n;
    if (p == MRHS_FP32)
        k_norm2<float><<<g.blocks, g.threads, smem, s>>>(static_cast<const float *>(w), rows, n, g.rpb,
                                                         sc.partials.as<double2>(), sc.counter.as<unsigned int>(), out);
    else if (p == MRHS_FP64)
        k_norm2<double><<<g.blocks, g.threads, smem, s>>>(static_cast<const double *>(w), rows, n, g.rpb,
                                                          sc.partials.as<double2>(), sc.counter.as<unsigned int>(), out);
    else
        fail(MRHS_ERR_INVALID, "norm2: FP32 or FP64 fields");
    MRHS_LAUNCHED("k_norm2");
}

template <typename TW, typename TB>
static void lincomb_t(void *w, const void *basis, int64_t stride, int k, const double2 *coef, double alpha,
                      int64_t rows, int n, cudaStream_t s, double *norm_out, Scratch *sc) {
    const RedGeom g = red_geom(rows, n);
    for (int j0 = 0; j0 < k; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        const bool last_chunk = j0 + kk >= k;
        const bool want_norm = norm_out != nullptr && last_chunk;
        const TB *b = static_cast<const TB *>(basis) + 2 * j0 * stride;
        const double2 *c = coef + (int64_t)j0 * n;
        if (want_norm) {
            if (!sc) fail(MRHS_ERR_INVALID, "lincomb with norm needs scratch");
            sc->ensure(g.blocks, n);
            const size_t smem = sizeof(double2) * (size_t)g.rpb * n;
            k_lincomb<TW, TB, true><<<g.blocks, g.threads, smem, s>>>(
                static_cast<TW *>(w), b, stride, kk, c, alpha, rows, n, g.rpb, sc->partials.as<double2>(),
                sc->counter.as<unsigned int>(), norm_out);
        } else {
            k_lincomb<TW, TB, false><<<g.blocks, g.threads, 0, s>>>(static_cast<TW *>(w), b, stride, kk, c, alpha,
                                                                    rows, n, g.rpb, nullptr, nullptr, nullptr);
        }
        MRHS_LAUNCHED("k_lincomb");
    }
}

void lincomb(mrhs_precision pw, void *w, mrhs_precision pb, const void *basis, int64_t stride, int k,
             const double2 *coef, double alpha, int64_t rows, int n, cudaStream_t s, double *norm_out, Scratch *sc) {
    check_n(n);
    if (k <= 0) {
        if (norm_out) norm2(pw, w, rows, n, norm_out, *sc, s);
        return;
    }
    if (pw == MRHS_FP32 && pb == MRHS_FP32) lincomb_t<float, float>(w, basis, stride, k, coef, alpha, rows, n, s, norm_out, sc);
    else if (pw == MRHS_FP64 && pb == MRHS_FP64) lincomb_t<double, double>(w, basis, stride, k, coef, alpha, rows, n, s, norm_out, sc);
    else if (pw == MRHS_FP64 && pb == MRHS_FP32) lincomb_t<double, float>(w, basis, stride, k, coef, alpha, rows, n, s, norm_out, sc);
    else fail(MRHS_ERR_INVALID, "lincomb: unsupported precision pair");
}

void scale_inv_sqrt(mrhs_precision p, void *dst, const void *src, const double *nrm2, int64_t rows, int n,
                    cudaStream_t s) {
    check_n(n);
    const RedGeom g = red_geom(rows, n);
    if (p == MRHS_FP32)
        k_scale_inv_sqrt<float><<<g.blocks, g.threads, 0, s>>>(static_cast<float *>(dst),
                                                              static_cast<const float *>(src), nrm2, rows, n, g.rpb);
    else
        k_scale_inv_sqrt<double><<<g.blocks, g.threads, 0, s>>>(static_cast<double *>(dst),
                                                               static_cast<const double *>(src), nrm2, rows, n, g.rpb);
    MRHS_LAUNCHED("k_scale_inv_sqrt");
}

void cast(mrhs_precision pd, void *dst, mrhs_precision ps, const void *src, int64_t count, cudaStream_t s) {
    const int nb = ceil_div(count, 256);
    if (pd == MRHS_FP32 && ps == MRHS_FP64)
        k_cast<float, double><<<nb, 256, 0, s>>>(static_cast<float *>(dst), static_cast<const double *>(src), count);
    else if (pd == MRHS_FP64 && ps == MRHS_FP32)
        k_cast<double, float><<<nb, 256, 0, s>>>(static_cast<double *>(dst), static_cast<const float *>(src), count);
    else if (pd == ps) {
        MRHS_CUDA(cudaMemcpyAsync(dst, src, count * complex_bytes(pd), cudaMemcpyDeviceToDevice, s));
        return;
    } else
        fail(MRHS_ERR_INVALID, "cast: unsupported precision pair");
    MRHS_LAUNCHED("k_cast");
}

void axpy(mrhs_precision p, double a, const void *x, void *y, int64_t count, cudaStream_t s) {
    const int nb = ceil_div(count, 256);
    if (p == MRHS_FP32)
        k_axpy<float><<<nb, 256, 0, s>>>((float)a, static_cast<const float *>(x), static_cast<float *>(y), count);
    else
        k_axpy<double><<<nb, 256, 0, s>>>(a, static_cast<const double *>(x), static_cast<double *>(y), count);
    MRHS_LAUNCHED("k_axpy");
}

template <typename T>
__global__ void k_scale_real(T a, T *x, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    cplx<T> v = ldv(x, i);
    stv(x, i, cplx<T>{a * v.re, a * v.im});
}

void scale_real(mrhs_precision p, double a, void *x, int64_t count, cudaStream_t s) {
    const int nb = ceil_div(count, 256);
    if (p == MRHS_FP32)
        k_scale_real<float><<<nb, 256, 0, s>>>((float)a, static_cast<float *>(x), count);
    else
        k_scale_real<double><<<nb, 256, 0, s>>>(a, static_cast<double *>(x), count);
    MRHS_LAUNCHED("k_scale_real");
}

// ------------------------------------------------- per-RHS Givens / solve
void KrylovState::init(int m_, int n_) {
    m = m_;
    n = n_;
    R.alloc(sizeof(double2) * (size_t)n * (m + 1) * m);
    cs.alloc(sizeof(double) * (size_t)n * m);
    sn.alloc(sizeof(double2) * (size_t)n * m);
    g.alloc(sizeof(double2) * (size_t)n * (m + 1));
    y.alloc(sizeof(double2) * (size_t)m * n);
    hcol.alloc(sizeof(double2) * (size_t)(m + 1) * n);
    h2.alloc(sizeof(double2) * (size_t)(m + 1) * n);
    hn2.alloc(sizeof(double) * (size_t)n);
    nrm2w.alloc(sizeof(double) * (size_t)n);
    nn.alloc(sizeof(double) * (size_t)n);
    beta2.alloc(sizeof(double) * (size_t)n);
    res.alloc(sizeof(double) * (size_t)n);
}

__global__ void k_krylov_start(double2 *g, const double *beta2, double *res, int n, int m) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double b = sqrt(fmax(beta2[r], 0.0));
    g[(int64_t)r * (m + 1)] = make_double2(b, 0.0);
    for (int i = 1; i <= m; ++i) g[(int64_t)r * (m + 1) + i] = make_double2(0.0, 0.0);
    res[r] = b;
}

// Complex Givens rotation G = [[c, s], [-conj(s), c]] (c real) with
// G [a; b] = [rho; 0]: c = |a|/t, s = (a/|a|) conj(b)/t, t = sqrt(|a|^2+|b|^2);
// for a = 0: c = 0, s = conj(b)/|b|.
__global__ void k_krylov_givens(double2 *R, double *cs, double2 *sn, double2 *g, const double2 *hcol,
                                const double2 *h2, const double *hn2, const double *nn, double *res, int j, int n,
                                int m) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 col[65];
    for (int i = 0; i <= j; ++i) {
        const double2 a = hcol[(int64_t)i * n + r];
        const double2 b = h2 ? h2[(int64_t)i * n + r] : make_double2(0.0, 0.0);
        col[i] = make_double2(a.x + b.x, a.y + b.y);
    }
    double beta = sqrt(fmax(hn2[r], 0.0));
    if (nn) {  // basis vector rescaled by the fix-up (same test as k_norm_fixup)
        const double f = nn[r];
        if (f > 0.0 && fabs(f - 1.0) > 1e-2) beta *= sqrt(f);
        if (f == 0.0) beta = 0.0;
    }
    col[j + 1] = make_double2(beta, 0.0);
    for (int i = 0; i < j; ++i) {
        const double c = cs[(int64_t)r * m + i];
        const double2 s = sn[(int64_t)r * m + i];
        const double2 a = col[i], b = col[i + 1];
        // c a + s b
        col[i] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
        // -conj(s) a + c b
        col[i + 1] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    const double2 a = col[j], b = col[j + 1];
    const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
    double c;
    double2 s;
    if (nb == 0.0) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
    } else if (na == 0.0) {
        c = 0.0;
        s = make_double2(b.x / nb, -b.y / nb);
    } else {
        const double t = hypot(na, nb);
        c = na / t;
        const double2 ph = make_double2(a.x / na, a.y / na);
        const double2 cb = make_double2(b.x / t, -b.y / t);
        s = make_double2(ph.x * cb.x - ph.y * cb.y, ph.x * cb.y + ph.y * cb.x);
    }
    cs[(int64_t)r * m + j] = c;
    sn[(int64_t)r * m + j] = s;
    col[j] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    for (int i = 0; i <= j; ++i) R[((int64_t)r * (m + 1) + i) * m + j] = col[i];
    const double2 gj = g[(int64_t)r * (m + 1) + j];
    g[(int64_t)r * (m + 1) + j] = make_double2(c * gj.x, c * gj.y);
    const double2 gj1 = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[(int64_t)r * (m + 1) + j + 1] = gj1;
    res[r] = hypot(gj1.x, gj1.y);
}

__global__ void k_krylov_solve(const double2 *R, const double2 *g, double2 *y, int j, int n, int m) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 yy[64];
    for (int i = j - 1; i >= 0; --i) {
        double2 acc = g[(int64_t)r * (m + 1) + i];
        for (int l = i + 1; l < j; ++l) {
            const double2 rv = R[((int64_t)r * (m + 1) + i) * m + l];
            acc.x -= rv.x * yy[l].x - rv.y * yy[l].y;
            acc.y -= rv.x * yy[l].y + rv.y * yy[l].x;
        }
        const double2 d = R[((int64_t)r * (m + 1) + i) * m + i];
        const double dd = d.x * d.x + d.y * d.y;
        if (dd > 0.0) {
            yy[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
        } else {
            yy[i] = make_double2(0.0, 0.0);
        }
    }
    for (int i = 0; i < j; ++i) y[(int64_t)i * n + r] = yy[i];
}

void krylov_start(KrylovState &ks, int n, cudaStream_t s) {
    k_krylov_start<<<ceil_div(n, 64), 64, 0, s>>>(ks.g.as<double2>(), ks.beta2.as<double>(), ks.res.as<double>(), n, ks.m);
    MRHS_LAUNCHED("k_krylov_start");
}

void krylov_givens(KrylovState &ks, int j, int n, cudaStream_t s, bool single_pass) {
    if (ks.m > 64) fail(MRHS_ERR_INVALID, "Krylov restart length above 64");
    k_krylov_givens<<<ceil_div(n, 64), 64, 0, s>>>(
        ks.R.as<double2>(), ks.cs.as<double>(), ks.sn.as<double2>(), ks.g.as<double2>(), ks.hcol.as<double2>(),
        single_pass ? nullptr : ks.h2.as<double2>(), ks.hn2.as<double>(), single_pass ? ks.nn.as<double>() : nullptr,
        ks.res.as<double>(), j, n, ks.m);
    MRHS_LAUNCHED("k_krylov_givens");
}

void krylov_solve(KrylovState &ks, int j, int n, cudaStream_t s) {
    k_krylov_solve<<<ceil_div(n, 64), 64, 0, s>>>(ks.R.as<double2>(), ks.g.as<double2>(), ks.y.as<double2>(), j, n, ks.m);
    MRHS_LAUNCHED("k_krylov_solve");
}

// ------------------------------------------------------------------- RNG
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

template <typename T>
__global__ void k_fill_gaussian(T *dst, int64_t count, uint64_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t a = splitmix64(seed ^ splitmix64((uint64_t)i));
    const uint64_t b = splitmix64(a);
    const float u1 = ((float)(a >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = (float)(b >> 40) * (1.0f / 16777216.0f);
    const float rad = sqrtf(-2.0f * logf(u1));
    float sn, cn;
    sincosf(6.283185307179586f * u2, &sn, &cn);
    stv(dst, i, cplx<T>{(T)(rad * cn), (T)(rad * sn)});
}

void fill_gaussian(mrhs_precision p, void *dst, int64_t count, uint64_t seed, cudaStream_t s) {
    if (p == MRHS_FP32)
        k_fill_gaussian<float><<<ceil_div(count, 256), 256, 0, s>>>(static_cast<float *>(dst), count, seed);
    else
        k_fill_gaussian<double><<<ceil_div(count, 256), 256, 0, s>>>(static_cast<double *>(dst), count, seed);
    MRHS_LAUNCHED("k_fill_gaussian");
}

}  // namespace mrhs
