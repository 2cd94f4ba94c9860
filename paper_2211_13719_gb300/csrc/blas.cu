// Batched BLAS-1 over the RHS index (paper Sec. 7: inner products of many
// RHS computed "simultaneously" in one pass instead of one after another).
//
// A field is `rows` rows of `n` complex values, RHS innermost.  A block of
// (n / W) * rpb threads (rpb = rows per block pass) gives each thread W
// adjacent RHS columns (W = 2 for FP32 fields with even n: one 16-byte load
// per row) and a strided set of rows, so every warp load is contiguous in
// memory.  Each thread accumulates its rows; the block reduces over its
// row-threads in a fixed order into a per-block partial; the last block of
// each group of 32 (atomic ticket) sums its group's partials in block order
// and the last group sums the group totals in group order.  The sum order of
// RHS r therefore depends only on (rows, n, grid), never on the values of
// other RHS: batching does not change a result beyond that fixed order.
//
// FP32 fields are accumulated in FP32 per thread and in FP64 from the block
// level up; FP64 fields in FP64 throughout.  Outputs are FP64.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
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
        counter.alloc(sizeof(unsigned int) * 64);
        MRHS_CUDA(cudaMemset(counter.ptr, 0, sizeof(unsigned int) * 64));
    }
    if (blocks > max_blocks || cols > max_cols) {
        const int b = std::max(blocks, max_blocks);
        const int c = std::max(cols, max_cols);
        // per-block partials, then one total per group of 32 blocks
        partials.alloc(sizeof(double2) * (size_t)(b + (b + 31) / 32) * (size_t)c);
        max_blocks = b;
        max_cols = c;
    }
}

struct RedGeom {
    int w;        // RHS columns per thread (2: FP32 pairs moved as float4)
    int rpb;      // rows per block pass
    int threads;  // (n / w) * rpb
    int blocks;
};

constexpr int RED_GROUP = 32;  // blocks per first-level group of the cross-block sum

// rpt: at least this many rows per thread (the autotuner's grid variants below)
static RedGeom red_geom(int64_t rows, int n, int w = 1, int rpt = 4) {
    RedGeom r;
    r.w = w;
    const int nw = n / w;
    const int target = w == 2 ? 128 : 256;
    r.rpb = nw >= target ? 1 : target / nw;
    r.threads = nw * r.rpb;
    // at least rpt rows per thread, at most one wave of resident blocks (fit_wave):
    // large fields run one full wave, small ones spread over many blocks so that
    // no thread walks a long chain of dependent row loads
    const int64_t need = (rows + (int64_t)rpt * r.rpb - 1) / ((int64_t)rpt * r.rpb);
    const int64_t cap = (int64_t)current_sms() * (w == 2 ? 8 : 4);
    r.blocks = (int)std::max<int64_t>(1, std::min(need, cap));
    return r;
}

// Caps the grid at one full wave: the blocks of `kernel` (block size
// g.threads, `smem` dynamic bytes) that are resident on all SMs at once.
// Rows are split evenly over the blocks, so a partial second wave would
// leave most SMs idle for its duration.
template <typename K> static void fit_wave(RedGeom &g, K kernel, size_t smem) {
    // resident blocks per SM for (kernel, block size, smem), computed once per key
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t>, int> cache;
    const auto key = std::make_tuple(reinterpret_cast<const void *>(kernel), g.threads, smem);
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) per_sm = it->second;
    }
    if (per_sm == 0) {
        MRHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, g.threads, smem));
        per_sm = std::max(1, per_sm);
        std::lock_guard<std::mutex> lock(mu);
        cache[key] = per_sm;
    }
    g.blocks = std::min(g.blocks, per_sm * current_sms());
}

// Grid variants of the reductions for the autotuner: the minimum rows per
// thread.  4 (variant 0) spreads small fields over many blocks; on small
// coarse-level fields (a few MB) that many blocks write per-block partial
// sums nearly as large as the field, which 16 or 64 rows per thread avoid.
constexpr int kRptVariants[] = {4, 16, 64};
constexpr int kNumRpt = 3;

// tuner key of a reduction over `rows` x n complex values (k basis vectors)
static void blas_key(int64_t rows, int n, int k, int w, mrhs_precision p, int dims[4]) {
    dims[0] = (int)(rows & 0x3fffffff);
    dims[1] = (int)(rows >> 30);
    dims[2] = k;
    dims[3] = w * 16 + (int)p;
}

// FP32 fields take the paired path when n is even and every field pointer
// (and the basis stride) keeps the 16-byte alignment of a float4
static int pair_width(mrhs_precision p, int n, std::initializer_list<const void *> ptrs, int64_t stride = 0) {
    if (p != MRHS_FP32 || n % 2 != 0 || stride % 2 != 0) return 1;
    for (const void *q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) & 15u) return 1;
    return 2;
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
// W consecutive complex values starting at element e (e even when W == 2)
template <int W, typename T> __device__ __forceinline__ void ldw(const T *p, int64_t e, cplx<T> (&x)[W]) {
    if constexpr (W == 2) {
        static_assert(std::is_same<T, float>::value, "paired access is FP32");
        const float4 v = *reinterpret_cast<const float4 *>(p + 2 * e);
        x[0] = {v.x, v.y};
        x[1] = {v.z, v.w};
    } else {
        x[0] = ldv(p, e);
    }
}
template <int W, typename T> __device__ __forceinline__ void stw(T *p, int64_t e, const cplx<T> (&x)[W]) {
    if constexpr (W == 2) {
        *reinterpret_cast<float4 *>(p + 2 * e) = make_float4(x[0].re, x[0].im, x[1].re, x[1].im);
    } else {
        stv(p, e, x[0]);
    }
}

// as ldw, zeros when !ok (the second row of a pair past the end)
template <int W, typename T> __device__ __forceinline__ void ldw_if(const T *p, int64_t e, bool ok, cplx<T> (&x)[W]) {
    if (ok) {
        ldw<W>(p, e, x);
    } else {
#pragma unroll
        for (int v = 0; v < W; ++v) x[v] = {0, 0};
    }
}

// fixed-order sum of count values p[0], p[stride], ... (four interleaved partial sums)
__device__ __forceinline__ double2 ordered_sum(const double2 *p, int count, int stride) {
    double2 q[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    int b = 0;
    for (; b + 4 <= count; b += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 v = __ldcg(&p[(int64_t)(b + u) * stride]);
            q[u].x += v.x;
            q[u].y += v.y;
        }
    }
    for (; b < count; ++b) {
        const double2 v = __ldcg(&p[(int64_t)b * stride]);
        q[0].x += v.x;
        q[0].y += v.y;
    }
    return make_double2((q[0].x + q[1].x) + (q[2].x + q[3].x), (q[0].y + q[1].y) + (q[2].y + q[3].y));
}

struct FinishOut {
    double2 *out;
    bool accumulate;
    bool real_only;   // the single column goes to out_real
    double *out_real;
    bool real_tail;   // the first cols - 1 columns go to out, the last column's real part to out_real
};

__device__ __forceinline__ void finish_emit(const FinishOut &f, int cols, int n, int o, double2 s) {
    if (f.real_only) {
        f.out_real[o] = s.x;
    } else if (f.real_tail && o >= (cols - 1) * n) {
        f.out_real[o - (cols - 1) * n] = s.x;
    } else if (f.accumulate) {
        const double2 prev = f.out[o];
        f.out[o] = make_double2(prev.x + s.x, prev.y + s.y);
    } else {
        f.out[o] = s;
    }
}

// Block-level fixed-order reduction of `cols` quantities for the thread's W
// columns col..col+W-1 (vals[c * W + w]), then the cross-block finish: the last
// block of each group of RED_GROUP consecutive blocks sums the group's partials
// in block order, the last group sums the group totals in group order.  Every
// sum has a fixed order, so no result depends on the order blocks finish in.
// smem: double2 [rpb][cols][n] as [(rsub * cols + c) * n + col]; partials hold
// (blocks + groups) * cols * n; counter[0..groups] is zero on entry and left zero.
template <int W>
__device__ void block_finish(double2 *smem, const double2 *vals, int cols, int n, int rpb, int col, int rsub,
                             double2 *partials, unsigned int *counter, const FinishOut &f) {
    for (int c = 0; c < cols; ++c)
#pragma unroll
        for (int w = 0; w < W; ++w) smem[((int64_t)rsub * cols + c) * n + col + w] = vals[c * W + w];
    __syncthreads();
    const int tid = threadIdx.x;
    const int nout = cols * n;
    const int nb = (int)gridDim.x;
    for (int o = tid; o < nout; o += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < rpb; ++q) {
            const double2 v = smem[(int64_t)q * nout + o];
            s.x += v.x;
            s.y += v.y;
        }
        partials[(int64_t)blockIdx.x * nout + o] = s;
    }
    const int g = (int)blockIdx.x / RED_GROUP;
    const int groups = (nb + RED_GROUP - 1) / RED_GROUP;
    const int gb0 = g * RED_GROUP, gsize = min(RED_GROUP, nb - gb0);
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&counter[g], 1u) == (unsigned)(gsize - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 *gpart = partials + (int64_t)nb * nout;
    for (int o = tid; o < nout; o += blockDim.x) {
        const double2 s = ordered_sum(partials + (int64_t)gb0 * nout + o, gsize, nout);
        if (groups == 1) finish_emit(f, cols, n, o, s);
        else gpart[(int64_t)g * nout + o] = s;
    }
    if (groups == 1) {
        if (tid == 0) counter[g] = 0u;
        return;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        counter[g] = 0u;
        last = atomicAdd(&counter[groups], 1u) == (unsigned)(groups - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int o = tid; o < nout; o += blockDim.x) finish_emit(f, cols, n, o, ordered_sum(gpart + o, groups, nout));
    if (tid == 0) counter[groups] = 0u;
}

// thread geometry shared by the reductions: W columns per thread, rpb row-threads per block
#define RED_THREAD_GEOMETRY                    \
    const int nw = n / W;                      \
    const int col = (int)(threadIdx.x % nw) * W; \
    const int rsub = (int)(threadIdx.x / nw);   \
    const int64_t step = (int64_t)gridDim.x * rpb

// Kernels with a basis loop take KM, a compile-time bound on the number k of
// basis vectors (KM in {1, 2, 4, 8}, the smallest >= k): the unrolled loop then
// issues no work for the slots j >= k, which matters at GB300's FP64 rate.
// U = 2 walks a thread's rows two at a time into two partial sums (independent
// FMA chains, added in a fixed order at the end); used where the FMA latency
// chain, not memory, would bound the kernel (FP64, and FP32 with KM <= 2).

// out[j][r] = sum_i conj(b_j[i][r]) w[i][r], j < k <= KM
template <typename T, int W, int KM, int U>
__global__ void k_multi_dot(const T *__restrict__ basis, int64_t stride, int k, const T *__restrict__ w,
                            int64_t rows, int n, int rpb, double2 *partials, unsigned int *counter,
                            double2 *out, int accumulate) {
    extern __shared__ double2 smem[];
    RED_THREAD_GEOMETRY;
    cplx<T> acc[U][KM][W];
#pragma unroll
    for (int h = 0; h < U; ++h)
#pragma unroll
        for (int j = 0; j < KM; ++j)
#pragma unroll
            for (int v = 0; v < W; ++v) acc[h][j][v] = {0, 0};
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += U * step) {
        cplx<T> x[U][W];
        int64_t e[U];
        bool ok[U];
#pragma unroll
        for (int h = 0; h < U; ++h) {
            e[h] = (row + h * step) * n + col;
            ok[h] = h == 0 || row + h * step < rows;
            ldw_if<W>(w, e[h], ok[h], x[h]);
        }
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            if (j < k) {
#pragma unroll
                for (int h = 0; h < U; ++h) {
                    cplx<T> b[W];
                    ldw_if<W>(basis + 2 * j * stride, e[h], ok[h], b);
#pragma unroll
                    for (int v = 0; v < W; ++v) cmac_conj(acc[h][j][v], b[v], x[h][v]);
                }
            }
        }
    }
    double2 vals[KM * W];
#pragma unroll
    for (int j = 0; j < KM; ++j)
#pragma unroll
        for (int v = 0; v < W; ++v) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int h = 0; h < U; ++h) {
                re += (double)acc[h][j][v].re;
                im += (double)acc[h][j][v].im;
            }
            vals[j * W + v] = make_double2(re, im);
        }
    block_finish<W>(smem, vals, k, n, rpb, col, rsub, partials, counter,
                    FinishOut{out, accumulate != 0, false, nullptr, false});
}

template <typename T, int W>
__global__ void k_norm2(const T *__restrict__ w, int64_t rows, int n, int rpb, double2 *partials,
                        unsigned int *counter, double *out) {
    extern __shared__ double2 smem[];
    RED_THREAD_GEOMETRY;
    T acc[2][W];
#pragma unroll
    for (int v = 0; v < W; ++v) acc[0][v] = acc[1][v] = 0;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += 2 * step) {
        cplx<T> x0[W], x1[W];
        ldw<W>(w, row * n + col, x0);
        ldw_if<W>(w, (row + step) * n + col, row + step < rows, x1);
#pragma unroll
        for (int v = 0; v < W; ++v) {
            acc[0][v] = fmadd(x0[v].re, x0[v].re, acc[0][v]);
            acc[0][v] = fmadd(x0[v].im, x0[v].im, acc[0][v]);
            acc[1][v] = fmadd(x1[v].re, x1[v].re, acc[1][v]);
            acc[1][v] = fmadd(x1[v].im, x1[v].im, acc[1][v]);
        }
    }
    double2 vals[W];
#pragma unroll
    for (int v = 0; v < W; ++v) vals[v] = make_double2((double)acc[0][v] + (double)acc[1][v], 0.0);
    block_finish<W>(smem, vals, 1, n, rpb, col, rsub, partials, counter, FinishOut{nullptr, false, true, out, false});
}

// w += alpha * sum_j coef[j][r] b_j (k <= KM) ; optional ||w||^2 per RHS
template <typename TW, typename TB, bool NORM, int W, int KM>
__global__ void k_lincomb(TW *__restrict__ w, const TB *__restrict__ basis, int64_t stride, int k,
                          const double2 *__restrict__ coef, double alpha, int64_t rows, int n, int rpb,
                          double2 *partials, unsigned int *counter, double *norm_out) {
    extern __shared__ double2 smem[];
    // coefficients of this thread's columns, scaled by alpha, in the basis precision
    using TC = typename std::conditional<sizeof(TW) == 8 || sizeof(TB) == 8, double, float>::type;
    RED_THREAD_GEOMETRY;
    cplx<TC> cf[KM][W];
#pragma unroll
    for (int j = 0; j < KM; ++j) {
#pragma unroll
        for (int v = 0; v < W; ++v) {
            if (j < k) {
                const double2 c = coef[(int64_t)j * n + col + v];
                cf[j][v] = {(TC)(alpha * c.x), (TC)(alpha * c.y)};
            } else {
                cf[j][v] = {0, 0};
            }
        }
    }
    // rows two at a time: independent work per row, two norm accumulators
    TW nacc[2][W];
#pragma unroll
    for (int v = 0; v < W; ++v) nacc[0][v] = nacc[1][v] = 0;
    for (int64_t row0 = (int64_t)blockIdx.x * rpb + rsub; row0 < rows; row0 += 2 * step) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t row = row0 + h * step;
            if (h == 1 && row >= rows) break;
            const int64_t e = row * n + col;
            cplx<TC> s[W];
#pragma unroll
            for (int v = 0; v < W; ++v) s[v] = {0, 0};
#pragma unroll
            for (int j = 0; j < KM; ++j) {
                if (j < k) {
                    cplx<TB> b[W];
                    ldw<W>(basis + 2 * j * stride, e, b);
#pragma unroll
                    for (int v = 0; v < W; ++v) cmac(s[v], cf[j][v], cplx<TC>{(TC)b[v].re, (TC)b[v].im});
                }
            }
            cplx<TW> x[W];
            ldw<W>(w, e, x);
#pragma unroll
            for (int v = 0; v < W; ++v) {
                x[v].re += (TW)s[v].re;
                x[v].im += (TW)s[v].im;
                if (NORM) {
                    nacc[h][v] = fmadd(x[v].re, x[v].re, nacc[h][v]);
                    nacc[h][v] = fmadd(x[v].im, x[v].im, nacc[h][v]);
                }
            }
            stw<W>(w, e, x);
        }
    }
    if (NORM) {
        double2 vals[W];
#pragma unroll
        for (int v = 0; v < W; ++v) vals[v] = make_double2((double)nacc[0][v] + (double)nacc[1][v], 0.0);
        block_finish<W>(smem, vals, 1, n, rpb, col, rsub, partials, counter,
                        FinishOut{nullptr, false, true, norm_out, false});
    }
}

// dst = src / sqrt(nrm2[col]); factors computed once per thread
template <typename T, int W>
__global__ void k_scale_inv_sqrt(T *dst, const T *src, const double *nrm2, int64_t rows, int n, int rpb) {
    RED_THREAD_GEOMETRY;
    T f[W];
#pragma unroll
    for (int v = 0; v < W; ++v) {
        const double q = nrm2[col + v];
        f[v] = q > 0.0 ? (T)(1.0 / sqrt(q)) : (T)0;
    }
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        cplx<T> x[W];
        ldw<W>(src, e, x);
#pragma unroll
        for (int v = 0; v < W; ++v) x[v] = {x[v].re * f[v], x[v].im * f[v]};
        stw<W>(dst, e, x);
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

// out[j][r] = <b_j, w>_r for j < k (k <= KM, k < KCHUNK) and nrm2[r] = ||w_r||^2, one pass over w
template <typename T, int W, int KM, int U>
__global__ void k_dots_norm(const T *__restrict__ basis, int64_t stride, int k, const T *__restrict__ w,
                            int64_t rows, int n, int rpb, double2 *partials, unsigned int *counter, double2 *out,
                            double *nrm2) {
    extern __shared__ double2 smem[];
    RED_THREAD_GEOMETRY;
    cplx<T> acc[U][KM][W];
    T nacc[U][W];
#pragma unroll
    for (int h = 0; h < U; ++h)
#pragma unroll
        for (int v = 0; v < W; ++v) {
            nacc[h][v] = 0;
#pragma unroll
            for (int j = 0; j < KM; ++j) acc[h][j][v] = {0, 0};
        }
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += U * step) {
        cplx<T> x[U][W];
        int64_t e[U];
        bool ok[U];
#pragma unroll
        for (int h = 0; h < U; ++h) {
            e[h] = (row + h * step) * n + col;
            ok[h] = h == 0 || row + h * step < rows;
            ldw_if<W>(w, e[h], ok[h], x[h]);
#pragma unroll
            for (int v = 0; v < W; ++v) {
                nacc[h][v] = fmadd(x[h][v].re, x[h][v].re, nacc[h][v]);
                nacc[h][v] = fmadd(x[h][v].im, x[h][v].im, nacc[h][v]);
            }
        }
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            if (j < k) {
#pragma unroll
                for (int h = 0; h < U; ++h) {
                    cplx<T> b[W];
                    ldw_if<W>(basis + 2 * j * stride, e[h], ok[h], b);
#pragma unroll
                    for (int v = 0; v < W; ++v) cmac_conj(acc[h][j][v], b[v], x[h][v]);
                }
            }
        }
    }
    double2 vals[(KM + 1) * W];
#pragma unroll
    for (int j = 0; j < KM; ++j)
#pragma unroll
        for (int v = 0; v < W; ++v) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int h = 0; h < U; ++h) {
                re += (double)acc[h][j][v].re;
                im += (double)acc[h][j][v].im;
            }
            vals[j * W + v] = make_double2(re, im);
        }
#pragma unroll
    for (int v = 0; v < W; ++v) {
        double q = 0.0;
#pragma unroll
        for (int h = 0; h < U; ++h) q += (double)nacc[h][v];
        vals[k * W + v] = make_double2(q, 0.0);
    }
    block_finish<W>(smem, vals, k + 1, n, rpb, col, rsub, partials, counter, FinishOut{out, false, false, nrm2, true});
}

// w <- (w - sum_{j<k} h_j b_j) / beta with beta^2 = max(||w||^2 - sum_{all j<kall} |h_j|^2, 1e-6 ||w||^2)
// (Pythagoras for an orthonormal basis); writes beta^2 to hn2 and ||w_new||^2 to nn.
// `coef` points at the first of the k coefficients handled here, `hall` at all kall of them.
template <typename T, int W, int KM>
__global__ void k_lincomb_scale(T *__restrict__ w, const T *__restrict__ basis, int64_t stride, int k,
                                const double2 *__restrict__ coef, const double2 *__restrict__ hall, int kall,
                                const double *__restrict__ nrm2, double *__restrict__ hn2, int64_t rows, int n,
                                int rpb, double2 *partials, unsigned int *counter, double *nn) {
    extern __shared__ double2 smem[];
    RED_THREAD_GEOMETRY;
    cplx<T> cf[KM][W];
    T f[W];
#pragma unroll
    for (int v = 0; v < W; ++v) {
        double hh = 0.0;
        for (int j = 0; j < kall; ++j) {
            const double2 c = hall[(int64_t)j * n + col + v];
            hh += c.x * c.x + c.y * c.y;
        }
        const double w2 = nrm2[col + v];
        const double b2 = fmax(w2 - hh, 1e-6 * w2);
        f[v] = (T)(b2 > 0.0 ? 1.0 / sqrt(b2) : 0.0);
        if (blockIdx.x == 0 && rsub == 0) hn2[col + v] = b2;
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            if (j < k) {
                const double2 c = coef[(int64_t)j * n + col + v];
                cf[j][v] = {(T)(-c.x), (T)(-c.y)};
            } else {
                cf[j][v] = {0, 0};
            }
        }
    }
    // rows two at a time: two independent norm accumulators
    T nacc[2][W];
#pragma unroll
    for (int v = 0; v < W; ++v) nacc[0][v] = nacc[1][v] = 0;
    for (int64_t row0 = (int64_t)blockIdx.x * rpb + rsub; row0 < rows; row0 += 2 * step) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t row = row0 + h * step;
            if (h == 1 && row >= rows) break;
            const int64_t e = row * n + col;
            cplx<T> x[W];
            ldw<W>(w, e, x);
#pragma unroll
            for (int j = 0; j < KM; ++j) {
                if (j < k) {
                    cplx<T> b[W];
                    ldw<W>(basis + 2 * j * stride, e, b);
#pragma unroll
                    for (int v = 0; v < W; ++v) cmac(x[v], cf[j][v], b[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < W; ++v) {
                x[v].re *= f[v];
                x[v].im *= f[v];
                nacc[h][v] = fmadd(x[v].re, x[v].re, nacc[h][v]);
                nacc[h][v] = fmadd(x[v].im, x[v].im, nacc[h][v]);
            }
            stw<W>(w, e, x);
        }
    }
    double2 vals[W];
#pragma unroll
    for (int v = 0; v < W; ++v) vals[v] = make_double2((double)nacc[0][v] + (double)nacc[1][v], 0.0);
    block_finish<W>(smem, vals, 1, n, rpb, col, rsub, partials, counter, FinishOut{nullptr, false, true, nn, false});
}

// Columns whose new basis vector is not unit length (cancellation in the
// Pythagorean norm) are rescaled; the Givens step applies the same factor to
// beta.  Threads whose columns are all unflagged return without touching data.
template <typename T, int W>
__global__ void k_norm_fixup(T *__restrict__ w, const double *__restrict__ nn, int64_t rows, int n, int rpb) {
    RED_THREAD_GEOMETRY;
    T sc[W];
    bool any = false;
#pragma unroll
    for (int v = 0; v < W; ++v) {
        const double f = nn[col + v];
        const bool flag = f > 0.0 && fabs(f - 1.0) > 1e-2;
        sc[v] = flag ? (T)(1.0 / sqrt(f)) : (T)1;
        any = any || flag;
    }
    if (!any) return;
    for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += step) {
        const int64_t e = row * n + col;
        cplx<T> x[W];
        ldw<W>(w, e, x);
#pragma unroll
        for (int v = 0; v < W; ++v) x[v] = {x[v].re * sc[v], x[v].im * sc[v]};
        stw<W>(w, e, x);
    }
}

// ------------------------------------------------------------- launchers
static void check_n(int n) {
    if (n < 1 || n > 256) fail(MRHS_ERR_INVALID, "batched BLAS supports 1 <= nrhs <= 256");
}

// calls f(T{}, integral_constant<W>) for the field precision and column width
template <typename F> static void dispatch(mrhs_precision p, int w, const char *what, F &&f) {
    if (p == MRHS_FP32) {
        if (w == 2) f(float{}, std::integral_constant<int, 2>{});
        else f(float{}, std::integral_constant<int, 1>{});
    } else if (p == MRHS_FP64) {
        f(double{}, std::integral_constant<int, 1>{});
    } else {
        fail(MRHS_ERR_INVALID, std::string(what) + ": FP32 or FP64 fields");
    }
}

#define RED_TYPES(tT, tW)          \
    using T = decltype(tT);        \
    constexpr int W = decltype(tW)::value

// calls f(integral_constant<KM>) with KM in {1, 2, 4, 8}, the smallest >= k
template <typename F> static void with_kmax(int k, F &&f) {
    if (k <= 1) f(std::integral_constant<int, 1>{});
    else if (k <= 2) f(std::integral_constant<int, 2>{});
    else if (k <= 4) f(std::integral_constant<int, 4>{});
    else f(std::integral_constant<int, 8>{});
}
// rows two at a time where FMA latency chains would bound the kernel
template <typename T, int KM> constexpr int unroll_rows() { return (sizeof(T) == 8 || KM <= 2) ? 2 : 1; }

void multi_dot(mrhs_precision p, const void *basis, int64_t stride, int k, const void *w, int64_t rows, int n,
               double2 *out, Scratch &sc, cudaStream_t s, bool accumulate) {
    check_n(n);
    if (k <= 0) return;
    const RedGeom g0 = red_geom(rows, n, pair_width(p, n, {basis, w}, stride));
    for (int j0 = 0; j0 < k; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        const size_t smem = sizeof(double2) * (size_t)g0.rpb * kk * n;
        dispatch(p, g0.w, "multi_dot", [&](auto tT, auto tW) {
            RED_TYPES(tT, tW);
            with_kmax(kk, [&](auto tK) {
                constexpr int KM = decltype(tK)::value;
                auto kern = k_multi_dot<T, W, KM, unroll_rows<T, KM>()>;
                RedGeom g = g0;
                fit_wave(g, kern, smem);
                sc.ensure(g.blocks, kk * n);
                MRHS_TIMED("k_multi_dot", s);
                kern<<<g.blocks, g.threads, smem, s>>>(static_cast<const T *>(basis) + 2 * j0 * stride, stride, kk,
                                                       static_cast<const T *>(w), rows, n, g.rpb,
                                                       sc.partials.as<double2>(), sc.counter.as<unsigned int>(),
                                                       out + (int64_t)j0 * n, accumulate);
            });
        });
        MRHS_LAUNCHED("k_multi_dot");
    }
}

// hn2 = beta^2 = max(||w||^2 - sum_j |h_j|^2, 1e-6 ||w||^2) and nn = 1 per RHS: the Hessenberg
// entry of a last Arnoldi step whose normalised vector is never used
__global__ void k_pythag_norm(const double2 *__restrict__ h, int k, const double *__restrict__ nrm2,
                              double *__restrict__ hn2, double *__restrict__ nn, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double hh = 0.0;
    for (int j = 0; j < k; ++j) {
        const double2 c = h[(int64_t)j * n + r];
        hh += c.x * c.x + c.y * c.y;
    }
    const double w2 = nrm2[r];
    hn2[r] = fmax(w2 - hh, 1e-6 * w2);
    nn[r] = 1.0;
}

void orthonormalize_step(mrhs_precision p, const void *basis, int64_t stride, int k, void *w, int64_t rows, int n,
                         double2 *h, double *nrm2, double *hn2, double *nn, Scratch &sc, cudaStream_t s,
                         bool need_vector) {
    check_n(n);
    const int pw = pair_width(p, n, {basis, w}, stride);
    RedGeom g0 = red_geom(rows, n, pw);
    const bool f32 = p == MRHS_FP32;
    if (!f32 && p != MRHS_FP64) fail(MRHS_ERR_INVALID, "orthonormalize: FP32 or FP64 fields");
    const size_t esz = f32 ? 8 : 16;
    // dots (and ||w||^2 with the last chunk)
    for (int j0 = 0; j0 < k || j0 == 0; j0 += KCHUNK - 1) {
        const int kk = std::min(KCHUNK - 1, k - j0);
        if (j0 + kk < k) {
            multi_dot(p, static_cast<const char *>(basis) + esz * j0 * stride, stride, kk, w, rows, n,
                      h + (int64_t)j0 * n, sc, s);
            continue;
        }
        const size_t smem = sizeof(double2) * (size_t)g0.rpb * (kk + 1) * n;
        auto launch = [&](int v) {
            dispatch(p, g0.w, "orthonormalize", [&](auto tT, auto tW) {
                RED_TYPES(tT, tW);
                with_kmax(kk, [&](auto tK) {
                    constexpr int KM = decltype(tK)::value;
                    auto kern = k_dots_norm<T, W, KM, unroll_rows<T, KM>()>;
                    RedGeom g = red_geom(rows, n, pw, kRptVariants[v]);
                    fit_wave(g, kern, smem);
                    sc.ensure(g.blocks, (kk + 1) * n);
                    kern<<<g.blocks, g.threads, smem, s>>>(static_cast<const T *>(basis) + 2 * j0 * stride, stride,
                                                           kk, static_cast<const T *>(w), rows, n, g.rpb,
                                                           sc.partials.as<double2>(), sc.counter.as<unsigned int>(),
                                                           h + (int64_t)j0 * n, nrm2);
                });
            });
        };
        // the dots and the norm only read their inputs: the autotuner may repeat the launch
        int key[4];
        blas_key(rows, n, kk, pw, p, key);
        const int v = tune_pick("k_dots_norm", key, n, kNumRpt, launch, s);
        g0 = red_geom(rows, n, pw, kRptVariants[v]);
        {
            MRHS_TIMED("k_dots_norm", s);
            launch(v);
        }
        MRHS_LAUNCHED("k_dots_norm");
        break;
    }
    if (!need_vector) {
        k_pythag_norm<<<ceil_div(n, 64), 64, 0, s>>>(h, k, nrm2, hn2, nn, n);
        MRHS_LAUNCHED("k_pythag_norm");
        return;
    }
    // subtract, normalise
    for (int j0 = 0; j0 < k || j0 == 0; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        if (j0 + kk < k) {
            lincomb(p, w, p, static_cast<const char *>(basis) + esz * j0 * stride, stride, kk, h + (int64_t)j0 * n,
                    -1.0, rows, n, s);
            continue;
        }
        const size_t smem = sizeof(double2) * (size_t)g0.rpb * n;
        dispatch(p, g0.w, "orthonormalize", [&](auto tT, auto tW) {
            RED_TYPES(tT, tW);
            with_kmax(kk, [&](auto tK) {
                constexpr int KM = decltype(tK)::value;
                RedGeom g = g0;
                fit_wave(g, k_lincomb_scale<T, W, KM>, smem);
                sc.ensure(g.blocks, n);
                MRHS_TIMED("k_lincomb_scale", s);
                k_lincomb_scale<T, W, KM><<<g.blocks, g.threads, smem, s>>>(
                    static_cast<T *>(w), static_cast<const T *>(basis) + 2 * j0 * stride, stride, kk,
                    h + (int64_t)j0 * n, h, k, nrm2, hn2, rows, n, g.rpb, sc.partials.as<double2>(),
                    sc.counter.as<unsigned int>(), nn);
            });
        });
        MRHS_LAUNCHED("k_lincomb_scale");
        break;
    }
    dispatch(p, g0.w, "orthonormalize", [&](auto tT, auto tW) {
        RED_TYPES(tT, tW);
        RedGeom g = g0;
        fit_wave(g, k_norm_fixup<T, W>, 0);
        k_norm_fixup<T, W><<<g.blocks, g.threads, 0, s>>>(static_cast<T *>(w), nn, rows, n, g.rpb);
    });
    MRHS_LAUNCHED("k_norm_fixup");
}

void multi_dot_fixed_scratch(mrhs_precision p, const void *basis, int64_t stride, int k, const void *w, int64_t rows,
                             int n, double2 *out, double2 *partials, unsigned int *counter, int max_blocks,
                             cudaStream_t s) {
    check_n(n);
    RedGeom g0 = red_geom(rows, n, pair_width(p, n, {basis, w}, stride));
    g0.blocks = std::min(g0.blocks, max_blocks);
    for (int j0 = 0; j0 < k; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        const size_t smem = sizeof(double2) * (size_t)g0.rpb * kk * n;
        dispatch(p, g0.w, "multi_dot", [&](auto tT, auto tW) {
            RED_TYPES(tT, tW);
            with_kmax(kk, [&](auto tK) {
                constexpr int KM = decltype(tK)::value;
                auto kern = k_multi_dot<T, W, KM, unroll_rows<T, KM>()>;
                RedGeom g = g0;
                fit_wave(g, kern, smem);
                MRHS_TIMED("k_multi_dot", s);
                kern<<<g.blocks, g.threads, smem, s>>>(static_cast<const T *>(basis) + 2 * j0 * stride, stride, kk,
                                                       static_cast<const T *>(w), rows, n, g.rpb, partials, counter,
                                                       out + (int64_t)j0 * n, 0);
            });
        });
        MRHS_LAUNCHED("k_multi_dot");
    }
}

void norm2(mrhs_precision p, const void *w, int64_t rows, int n, double *out, Scratch &sc, cudaStream_t s) {
    check_n(n);
    const int pw = pair_width(p, n, {w});
    const RedGeom g0 = red_geom(rows, n, pw);
    const size_t smem = sizeof(double2) * (size_t)g0.rpb * n;
    auto launch = [&](int v) {
        dispatch(p, g0.w, "norm2", [&](auto tT, auto tW) {
            RED_TYPES(tT, tW);
            RedGeom g = red_geom(rows, n, pw, kRptVariants[v]);
            fit_wave(g, k_norm2<T, W>, smem);
            sc.ensure(g.blocks, n);
            k_norm2<T, W><<<g.blocks, g.threads, smem, s>>>(static_cast<const T *>(w), rows, n, g.rpb,
                                                            sc.partials.as<double2>(), sc.counter.as<unsigned int>(),
                                                            out);
        });
    };
    // an output that is also the input would not survive repeated launches
    int key[4];
    blas_key(rows, n, 0, pw, p, key);
    const int v = (const void *)out == w ? 0 : tune_pick("k_norm2", key, n, kNumRpt, launch, s);
    MRHS_TIMED("k_norm2", s);
    launch(v);
    MRHS_LAUNCHED("k_norm2");
}

template <typename TW, typename TB, int W>
static void lincomb_t(void *w, const void *basis, int64_t stride, int k, const double2 *coef, double alpha,
                      const RedGeom &g0, int64_t rows, int n, cudaStream_t s, double *norm_out, Scratch *sc) {
    for (int j0 = 0; j0 < k; j0 += KCHUNK) {
        const int kk = std::min(KCHUNK, k - j0);
        const bool want_norm = norm_out != nullptr && j0 + kk >= k;
        const TB *b = static_cast<const TB *>(basis) + 2 * j0 * stride;
        const double2 *c = coef + (int64_t)j0 * n;
        if (want_norm && !sc) fail(MRHS_ERR_INVALID, "lincomb with norm needs scratch");
        with_kmax(kk, [&](auto tK) {
            constexpr int KM = decltype(tK)::value;
            RedGeom g = g0;
            MRHS_TIMED("k_lincomb", s);
            if (want_norm) {
                const size_t smem = sizeof(double2) * (size_t)g0.rpb * n;
                fit_wave(g, k_lincomb<TW, TB, true, W, KM>, smem);
                sc->ensure(g.blocks, n);
                k_lincomb<TW, TB, true, W, KM><<<g.blocks, g.threads, smem, s>>>(
                    static_cast<TW *>(w), b, stride, kk, c, alpha, rows, n, g.rpb, sc->partials.as<double2>(),
                    sc->counter.as<unsigned int>(), norm_out);
            } else {
                fit_wave(g, k_lincomb<TW, TB, false, W, KM>, 0);
                k_lincomb<TW, TB, false, W, KM><<<g.blocks, g.threads, 0, s>>>(
                    static_cast<TW *>(w), b, stride, kk, c, alpha, rows, n, g.rpb, nullptr, nullptr, nullptr);
            }
        });
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
    if (pw == MRHS_FP32 && pb == MRHS_FP32) {
        const RedGeom g = red_geom(rows, n, pair_width(MRHS_FP32, n, {w, basis}, stride));
        if (g.w == 2) lincomb_t<float, float, 2>(w, basis, stride, k, coef, alpha, g, rows, n, s, norm_out, sc);
        else lincomb_t<float, float, 1>(w, basis, stride, k, coef, alpha, g, rows, n, s, norm_out, sc);
    } else if (pw == MRHS_FP64 && pb == MRHS_FP64) {
        lincomb_t<double, double, 1>(w, basis, stride, k, coef, alpha, red_geom(rows, n), rows, n, s, norm_out, sc);
    } else if (pw == MRHS_FP64 && pb == MRHS_FP32) {
        lincomb_t<double, float, 1>(w, basis, stride, k, coef, alpha, red_geom(rows, n), rows, n, s, norm_out, sc);
    } else {
        fail(MRHS_ERR_INVALID, "lincomb: unsupported precision pair");
    }
}

void scale_inv_sqrt(mrhs_precision p, void *dst, const void *src, const double *nrm2, int64_t rows, int n,
                    cudaStream_t s) {
    check_n(n);
    const RedGeom g0 = red_geom(rows, n, pair_width(p, n, {dst, src}));
    dispatch(p, g0.w, "scale_inv_sqrt", [&](auto tT, auto tW) {
        RED_TYPES(tT, tW);
        RedGeom g = g0;
        fit_wave(g, k_scale_inv_sqrt<T, W>, 0);
        k_scale_inv_sqrt<T, W><<<g.blocks, g.threads, 0, s>>>(static_cast<T *>(dst), static_cast<const T *>(src),
                                                              nrm2, rows, n, g.rpb);
    });
    MRHS_LAUNCHED("k_scale_inv_sqrt");
}

__global__ void k_any_nonzero(const uint4 *__restrict__ p, int64_t count, unsigned *flag) {
    unsigned acc = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldcs(p + i);
        acc |= v.x | v.y | v.z | v.w;
    }
    acc = __reduce_or_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(flag, 1u);
}

void any_nonzero(const void *p, int64_t bytes, unsigned *flag, cudaStream_t s) {
    zero_on_sms(flag, sizeof(unsigned), s);
    const int64_t count = bytes / 16;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)current_sms() * 8, ceil_div(count, 256)));
    k_any_nonzero<<<blocks, 256, 0, s>>>(static_cast<const uint4 *>(p), count, flag);
    MRHS_LAUNCHED("k_any_nonzero");
}

void cast(mrhs_precision pd, void *dst, mrhs_precision ps, const void *src, int64_t count, cudaStream_t s) {
    const int nb = ceil_div(count, 256);
    if (pd == MRHS_FP32 && ps == MRHS_FP64)
        k_cast<float, double><<<nb, 256, 0, s>>>(static_cast<float *>(dst), static_cast<const double *>(src), count);
    else if (pd == MRHS_FP64 && ps == MRHS_FP32)
        k_cast<double, float><<<nb, 256, 0, s>>>(static_cast<double *>(dst), static_cast<const float *>(src), count);
    else if (pd == ps) {
        copy_on_sms(dst, src, count * complex_bytes(pd), s);
        return;
    } else
        fail(MRHS_ERR_INVALID, "cast: unsupported precision pair");
    MRHS_LAUNCHED("k_cast");
}

// ------------------------------------------------- copies on the SMs
// Copies issued as kernels instead of cudaMemcpyAsync: they never wait behind
// the copy engines, which a caller's host transfers on other streams may hold
// for hundreds of milliseconds.
__global__ void k_copy16(uint4 *__restrict__ dst, const uint4 *__restrict__ src, int64_t n16) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void k_copy4(unsigned *__restrict__ dst, const unsigned *__restrict__ src, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

void copy_on_sms(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    if (bytes % 4) fail(MRHS_ERR_INVALID, "copy_on_sms: size must be a multiple of 4 bytes");
    const bool v16 = bytes % 16 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    const int64_t n = (int64_t)(v16 ? bytes / 16 : bytes / 4);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)current_sms() * 8, ceil_div(n, 256)));
    if (v16) k_copy16<<<blocks, 256, 0, s>>>(static_cast<uint4 *>(dst), static_cast<const uint4 *>(src), n);
    else k_copy4<<<blocks, 256, 0, s>>>(static_cast<unsigned *>(dst), static_cast<const unsigned *>(src), n);
    MRHS_CUDA(cudaGetLastError());
    MRHS_LAUNCHED("k_copy");
}

__global__ void k_zero4(unsigned *__restrict__ dst, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = 0u;
}
__global__ void k_zero16(uint4 *__restrict__ dst, int64_t n16) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = make_uint4(0u, 0u, 0u, 0u);
}

void zero_on_sms(void *dst, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    if (bytes % 4) fail(MRHS_ERR_INVALID, "zero_on_sms: size must be a multiple of 4 bytes");
    const bool v16 = bytes % 16 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
    const int64_t n = (int64_t)(v16 ? bytes / 16 : bytes / 4);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)current_sms() * 8, ceil_div(n, 256)));
    if (v16) k_zero16<<<blocks, 256, 0, s>>>(static_cast<uint4 *>(dst), n);
    else k_zero4<<<blocks, 256, 0, s>>>(static_cast<unsigned *>(dst), n);
    MRHS_CUDA(cudaGetLastError());
    MRHS_LAUNCHED("k_zero");
}

void read_back(void *pinned_host, const void *dev, size_t bytes, cudaStream_t s) {
    // page-locked host memory from cudaMallocHost is mapped at the same address on the device
    copy_on_sms(pinned_host, dev, bytes, s);
}

int *pinned_flag_slot() {
    struct Slot {
        int *p = nullptr;
        ~Slot() {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local Slot slot;
    if (!slot.p) MRHS_CUDA(cudaMallocHost(&slot.p, 4 * sizeof(int)));
    return slot.p;
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
