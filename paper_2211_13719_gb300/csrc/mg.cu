// Intergrid operators (paper Sec. 5), the coarse 9-point stencil on CUDA
// cores (Sec. 6) and the FP64 block orthonormalisation of the setup.
//
// Prolongator storage: the chirally split prolongator has, at every site and
// component d, nonzero entries only in the N columns of d's chirality, so it
// is stored as the N orthonormalised vectors themselves, [V][dof][N]; column
// K = chi*N + k of P is vector k restricted to the components of chirality
// chi (chi(d) = d / (dof/2): the upper spins on the fine level, the first
// half of the coarse dof on coarse levels).
#include <algorithm>

#include "mg.cuh"

namespace mrhs {

struct AggGeom {
    int L[4];
    int Lc[4];
    int B[4];
    int64_t asize;
    int dof, N, n;
};

static AggGeom agg_geom(const Level &f, const Level &c, int n) {
    AggGeom a;
    for (int mu = 0; mu < 4; ++mu) {
        a.L[mu] = f.L[mu];
        a.Lc[mu] = c.L[mu];
        a.B[mu] = f.B[mu];
    }
    a.asize = f.asize;
    a.dof = f.dof;
    a.N = f.N;
    a.n = n;
    return a;
}

// fine site of the i-th site (lexicographic inside the block) of aggregate xc
__device__ __forceinline__ int64_t agg_site(const AggGeom &a, int64_t xc, int64_t i) {
    int cc[4];
    site_to_coords(xc, a.Lc, cc);
    int f[4];
    f[0] = cc[0] * a.B[0] + (int)(i % a.B[0]);
    int64_t q = i / a.B[0];
    f[1] = cc[1] * a.B[1] + (int)(q % a.B[1]);
    q /= a.B[1];
    f[2] = cc[2] * a.B[2] + (int)(q % a.B[2]);
    f[3] = cc[3] * a.B[3] + (int)(q / a.B[2]);
    return coords_to_site(f, a.L);
}

__device__ __forceinline__ cplx<float> ld2(const float2 *p, int64_t i) {
    const float2 v = p[i];
    return {v.x, v.y};
}

// ---------------------------------------------------------------- restrict
// One block per coarse site (aggregate).  Each thread owns KG consecutive
// basis vectors k of one chirality and one RHS column r (up to MAXI such
// items); per round PSB fine sites of the aggregate are staged in shared
// memory (their prolongator rows [dof][N] and field rows [dof][n], both
// contiguous in global memory), and for every staged site and component of
// the item's chirality the thread loads one field value and KG prolongator
// values (shared-memory broadcasts) for KG complex multiply-adds.
constexpr int RESTRICT_MAXI = 4;

template <int KG>
__global__ void __launch_bounds__(1024) k_restrict(const float2 *__restrict__ fine, const float2 *__restrict__ P,
                                                  float2 *__restrict__ coarse, int64_t ostride, AggGeom a, int PSB) {
    extern __shared__ float2 sm[];
    float2 *Ps = sm;                                   // [PSB][dof][N]
    float2 *Fs = sm + (size_t)PSB * a.dof * a.N;       // [PSB][dof][n]
    const int64_t xc = blockIdx.x;
    const int half = a.dof / 2;
    const int kgroups = a.N / KG;
    const int items = 2 * kgroups * a.n;               // (chi, kgroup, r)
    const int tid = threadIdx.x, T = blockDim.x;
    cplx<float> acc[RESTRICT_MAXI][KG];
#pragma unroll
    for (int i = 0; i < RESTRICT_MAXI; ++i)
#pragma unroll
        for (int j = 0; j < KG; ++j) acc[i][j] = {0.f, 0.f};
    const int pw = a.dof * a.N, fw = a.dof * a.n;
    for (int64_t i0 = 0; i0 < a.asize; i0 += PSB) {
        const int nsb = (int)(a.asize - i0 < PSB ? a.asize - i0 : PSB);
        __syncthreads();
        for (int e = tid; e < nsb * pw; e += T) {
            const int sb = e / pw;
            Ps[e] = P[agg_site(a, xc, i0 + sb) * pw + (e - sb * pw)];
        }
        for (int e = tid; e < nsb * fw; e += T) {
            const int sb = e / fw;
            Fs[e] = fine[agg_site(a, xc, i0 + sb) * fw + (e - sb * fw)];
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < RESTRICT_MAXI; ++it) {
            const int item = tid + it * T;
            if (item < items) {
                const int r = item % a.n;
                const int q = item / a.n;
                const int chi = q / kgroups, k0 = (q - chi * kgroups) * KG;
                for (int sb = 0; sb < nsb; ++sb) {
                    const float2 *pp = Ps + (size_t)(sb * a.dof + chi * half) * a.N + k0;
                    const float2 *ff = Fs + (size_t)(sb * a.dof + chi * half) * a.n + r;
                    for (int d = 0; d < half; ++d) {
                        const cplx<float> f = ld2(ff, (int64_t)d * a.n);
#pragma unroll
                        for (int j = 0; j < KG; ++j) cmac_conj(acc[it][j], ld2(pp, (int64_t)d * a.N + j), f);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int it = 0; it < RESTRICT_MAXI; ++it) {
        const int item = tid + it * T;
        if (item < items) {
            const int r = item % a.n;
            const int q = item / a.n;
            const int chi = q / kgroups, k0 = (q - chi * kgroups) * KG;
#pragma unroll
            for (int j = 0; j < KG; ++j)
                coarse[xc * ostride + (int64_t)(chi * a.N + k0 + j) * a.n + r] = make_float2(acc[it][j].re, acc[it][j].im);
        }
    }
}

template <int KG>
static void launch_restrict(const AggGeom &a, int64_t Vc, const float2 *fine, const float2 *P, float2 *coarse,
                            int64_t ostride, cudaStream_t s) {
    const int items = 2 * (a.N / KG) * a.n;
    int T = std::min(1024, std::max(64, ((items + RESTRICT_MAXI - 1) / RESTRICT_MAXI + 31) / 32 * 32));
    if (T * RESTRICT_MAXI < items) fail(MRHS_ERR_INVALID, "restrict: nc * nrhs too large");
    const size_t per_site = sizeof(float2) * (size_t)a.dof * (a.N + a.n);
    int PSB = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_site));
    PSB = (int)std::min<int64_t>(PSB, a.asize);
    const size_t smem = per_site * PSB;
    if (smem > 200 * 1024) fail(MRHS_ERR_INVALID, "restrict: per-site data too large for shared memory");
    static bool attr = false;
    if (!attr) {
        MRHS_CUDA(cudaFuncSetAttribute(k_restrict<KG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    k_restrict<KG><<<(unsigned)Vc, T, smem, s>>>(fine, P, coarse, ostride, a, PSB);
    MRHS_LAUNCHED("k_restrict");
}

void restrict_fields(const Level &f, const Level &c, const float2 *fine, float2 *coarse, int n, int64_t ostride,
                     cudaStream_t s) {
    const AggGeom a = agg_geom(f, c, n);
    const float2 *P = f.P32.as<float2>();
    if (f.N % 4 == 0) launch_restrict<4>(a, c.V, fine, P, coarse, ostride, s);
    else if (f.N % 2 == 0) launch_restrict<2>(a, c.V, fine, P, coarse, ostride, s);
    else launch_restrict<1>(a, c.V, fine, P, coarse, ostride, s);
}

// ----------------------------------------------------------------- prolong
// One block per aggregate: the coarse block c[xc] ([nc][n]) is staged in
// shared memory once, the prolongator rows of PSB fine sites per round.  A
// thread item is (site, DG consecutive components of one chirality, RHS r):
// per basis vector k one coarse value and DG prolongator values (broadcast)
// feed DG complex multiply-adds; the DG outputs are stored contiguously in r.
template <int DG>
__global__ void __launch_bounds__(256) k_prolong(const float2 *__restrict__ coarse, const float2 *__restrict__ P,
                                                 float2 *__restrict__ fine, AggGeom a, int PSB) {
    extern __shared__ float2 sm[];
    const int nc = 2 * a.N;
    float2 *Cs = sm;                          // [nc][n]
    float2 *Ps = sm + (size_t)nc * a.n;       // [PSB][dof][N]
    const int64_t xc = blockIdx.x;
    const int half = a.dof / 2;
    const int tid = threadIdx.x, T = blockDim.x;
    for (int e = tid; e < nc * a.n; e += T) Cs[e] = coarse[xc * nc * a.n + e];
    const int dgroups = a.dof / DG;
    const int pw = a.dof * a.N;
    for (int64_t i0 = 0; i0 < a.asize; i0 += PSB) {
        const int nsb = (int)(a.asize - i0 < PSB ? a.asize - i0 : PSB);
        __syncthreads();
        for (int e = tid; e < nsb * pw; e += T) {
            const int sb = e / pw;
            Ps[e] = P[agg_site(a, xc, i0 + sb) * pw + (e - sb * pw)];
        }
        __syncthreads();
        const int items = nsb * dgroups * a.n;
        for (int item = tid; item < items; item += T) {
            const int r = item % a.n;
            const int q = item / a.n;
            const int sb = q / dgroups, g = q - sb * dgroups;
            const int d0 = g * DG;
            const int chi = d0 / half;
            cplx<float> acc[DG];
#pragma unroll
            for (int j = 0; j < DG; ++j) acc[j] = {0.f, 0.f};
            const float2 *pp = Ps + (size_t)(sb * a.dof + d0) * a.N;
            const float2 *cc = Cs + (size_t)(chi * a.N) * a.n + r;
            for (int k = 0; k < a.N; ++k) {
                const cplx<float> cv = ld2(cc, (int64_t)k * a.n);
#pragma unroll
                for (int j = 0; j < DG; ++j) cmac(acc[j], ld2(pp, (int64_t)j * a.N + k), cv);
            }
            const int64_t x = agg_site(a, xc, i0 + sb);
#pragma unroll
            for (int j = 0; j < DG; ++j)
                fine[(x * a.dof + d0 + j) * a.n + r] = make_float2(acc[j].re, acc[j].im);
        }
    }
}

template <int DG>
static void launch_prolong(const AggGeom &a, int64_t Vc, const float2 *coarse, const float2 *P, float2 *fine,
                           cudaStream_t s) {
    const size_t cbytes = sizeof(float2) * (size_t)2 * a.N * a.n;
    const size_t per_site = sizeof(float2) * (size_t)a.dof * a.N;
    int PSB = (int)std::max<size_t>(1, std::min<size_t>(16, (64 * 1024) / per_site));
    PSB = (int)std::min<int64_t>(PSB, a.asize);
    const size_t smem = cbytes + per_site * PSB;
    if (smem > 200 * 1024) fail(MRHS_ERR_INVALID, "prolong: coarse block too large for shared memory");
    static bool attr = false;
    if (!attr) {
        MRHS_CUDA(cudaFuncSetAttribute(k_prolong<DG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    k_prolong<DG><<<(unsigned)Vc, 256, smem, s>>>(coarse, P, fine, a, PSB);
    MRHS_LAUNCHED("k_prolong");
}

void prolong_fields(const Level &f, const Level &c, const float2 *coarse, float2 *fine, int n, cudaStream_t s) {
    const AggGeom a = agg_geom(f, c, n);
    const int half = f.dof / 2;
    const float2 *P = f.P32.as<float2>();
    if (half % 4 == 0) launch_prolong<4>(a, c.V, coarse, P, fine, s);
    else if (half % 3 == 0) launch_prolong<3>(a, c.V, coarse, P, fine, s);
    else if (half % 2 == 0) launch_prolong<2>(a, c.V, coarse, P, fine, s);
    else launch_prolong<1>(a, c.V, coarse, P, fine, s);
}

// ---------------------------------------------------- coarse stencil, FP32
// One block per coarse site; for each of the 9 stencil blocks the dense
// nc x nc link block and the neighbour's nc x n field block are staged in
// shared memory and the block's threads accumulate their (K, r) outputs.
struct CoarseArgs {
    int L[4];
    int64_t V;
    int nc, n;
};
constexpr int COARSE_MAXO = 16;

__device__ __forceinline__ int64_t stencil_nb(int64_t site, const int c[4], const int L[4], int d) {
    if (d == 0) return site;
    const int mu = d <= 4 ? d - 1 : d - 5;
    const int step = d <= 4 ? 1 : -1;
    int e[4] = {c[0], c[1], c[2], c[3]};
    e[mu] = (e[mu] + step + L[mu]) % L[mu];
    return coords_to_site(e, L);
}

__device__ __forceinline__ bool stencil_selected(const StencilMask &m, int d, const int c[4]) {
    if (d == 0) return m.diag != 0;
    if (m.dir >= 0 && m.dir != d) return false;
    if (m.cross == 0) return true;
    const int mu = d <= 4 ? d - 1 : d - 5;
    const int loc = c[mu] % m.B[mu];
    const bool crossing = d <= 4 ? (loc == m.B[mu] - 1) : (loc == 0);
    return m.cross == 1 ? crossing : !crossing;
}

__global__ void k_coarse_fp32(const float2 *__restrict__ A, const float2 *__restrict__ in, float2 *__restrict__ out,
                              const float2 *__restrict__ y, CoarseArgs a, StencilMask m, int general) {
    extern __shared__ float2 sm[];
    float2 *As = sm;
    float2 *Fs = sm + (size_t)a.nc * a.nc;
    const int64_t site = blockIdx.x;
    const int tid = threadIdx.x, T = blockDim.x;
    const int nout = a.nc * a.n;
    int c[4];
    site_to_coords(site, a.L, c);
    cplx<float> acc[COARSE_MAXO];
#pragma unroll
    for (int j = 0; j < COARSE_MAXO; ++j) acc[j] = {0.f, 0.f};
    const int blk = a.nc * a.nc, fw = a.nc * a.n;
    for (int d = 0; d < 9; ++d) {
        if (general && !stencil_selected(m, d, c)) continue;
        const int64_t nb = stencil_nb(site, c, a.L, d);
        __syncthreads();
        const float4 *A4 = reinterpret_cast<const float4 *>(A + (site * 9 + d) * blk);
        for (int e = tid; e < blk / 2; e += T) reinterpret_cast<float4 *>(As)[e] = __ldg(A4 + e);
        for (int e = tid; e < fw; e += T) Fs[e] = in[nb * fw + e];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < COARSE_MAXO; ++j) {
            const int o = tid + j * T;
            if (o < nout) {
                const int K = o / a.n, r = o - K * a.n;
                // each direction's nc-term sum in two interleaved partials, then added to
                // the site total: FP32 rounding of the 9 nc-term sums stays near 2e-7
                // relative per site at nc = 64 (one running sum over all 9 nc terms: 1e-6)
                cplx<float> s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
                const float2 *ar = As + (size_t)K * a.nc;
                for (int l = 0; l < a.nc; l += 2) {
                    cmac(s0, ld2(ar, l), ld2(Fs, (int64_t)l * a.n + r));
                    cmac(s1, ld2(ar, l + 1), ld2(Fs, (int64_t)(l + 1) * a.n + r));
                }
                acc[j] = acc[j] + (s0 + s1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < COARSE_MAXO; ++j) {
        const int o = tid + j * T;
        if (o < nout) {
            float2 v = make_float2(acc[j].re, acc[j].im);
            if (y) {
                const float2 yy = y[site * nout + o];
                v = make_float2(yy.x - v.x, yy.y - v.y);
            }
            out[site * nout + o] = v;
        }
    }
}

void coarse_apply_fp32(const Level &c, const float2 *in, float2 *out, const float2 *y, int n, cudaStream_t s,
                       const StencilMask *mask) {
    CoarseArgs a;
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = c.L[mu];
    a.V = c.V;
    a.nc = c.dof;
    a.n = n;
    if (a.nc % 2) fail(MRHS_ERR_INVALID, "coarse dof must be even");
    const int nout = a.nc * n;
    int T = ((nout + COARSE_MAXO - 1) / COARSE_MAXO + 31) / 32 * 32;
    T = std::max(64, std::min(1024, T));
    if ((int64_t)T * COARSE_MAXO < nout) fail(MRHS_ERR_INVALID, "coarse apply: nc * nrhs too large");
    const size_t smem = sizeof(float2) * ((size_t)a.nc * a.nc + (size_t)a.nc * n);
    if (smem > 220 * 1024) fail(MRHS_ERR_INVALID, "coarse apply: nc * nrhs too large for shared memory");
    static bool attr = false;
    if (!attr) {
        MRHS_CUDA(cudaFuncSetAttribute(k_coarse_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        attr = true;
    }
    StencilMask m{1, -1, 0, {1, 1, 1, 1}};
    if (mask) m = *mask;
    MRHS_TIMED("k_coarse_fp32", s);
    k_coarse_fp32<<<(unsigned)c.V, T, smem, s>>>(c.A32.as<float2>(), in, out, y, a, m, mask ? 1 : 0);
    MRHS_LAUNCHED("k_coarse_fp32");
}

// ---------------------------------------------------- chiral expansion
__global__ void k_expand_chiral(const float2 *__restrict__ P, float2 *__restrict__ Pe, int64_t V, int dof, int N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = 2 * N;
    if (i >= V * dof * nc) return;
    const int64_t xd = i / nc;
    const int K = (int)(i - xd * nc);
    const int d = (int)(xd % dof);
    const int chi_d = d / (dof / 2), chi_K = K / N;
    Pe[i] = chi_d == chi_K ? P[xd * N + (K - chi_K * N)] : make_float2(0.f, 0.f);
}

void expand_chiral(const Level &f, const float2 *P, float2 *Pexp, cudaStream_t s) {
    const int64_t count = f.V * f.dof * 2 * f.N;
    k_expand_chiral<<<ceil_div(count, 256), 256, 0, s>>>(P, Pexp, f.V, f.dof, f.N);
    MRHS_LAUNCHED("k_expand_chiral");
}

// --------------------------------------- FP64 block orthonormalisation
// One block per (aggregate, chirality).  The rows are the aggregate's sites
// times the components of that chirality; the N columns are processed in
// order with modified Gram-Schmidt applied twice, then normalised.
__device__ double2 block_sum(double2 v, double2 *red) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s.x += red[w].x;
            s.y += red[w].y;
        }
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

__global__ void k_block_orth(double2 *vecs, AggGeom a) {
    __shared__ double2 red[33];
    const int64_t xc = blockIdx.x;
    const int chi = blockIdx.y;
    const int half = a.dof / 2;
    const int64_t rows = a.asize * half;
    auto off = [&](int64_t row) -> int64_t {
        const int64_t i = row / half;
        const int d = chi * half + (int)(row - i * half);
        return (agg_site(a, xc, i) * a.dof + d) * a.N;
    };
    for (int k = 0; k < a.N; ++k) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = 0; j < k; ++j) {
                double2 h = make_double2(0.0, 0.0);
                for (int64_t row = threadIdx.x; row < rows; row += blockDim.x) {
                    const int64_t o = off(row);
                    const double2 q = vecs[o + j], v = vecs[o + k];
                    h.x += q.x * v.x + q.y * v.y;
                    h.y += q.x * v.y - q.y * v.x;
                }
                h = block_sum(h, red);
                for (int64_t row = threadIdx.x; row < rows; row += blockDim.x) {
                    const int64_t o = off(row);
                    const double2 q = vecs[o + j];
                    double2 v = vecs[o + k];
                    v.x -= h.x * q.x - h.y * q.y;
                    v.y -= h.x * q.y + h.y * q.x;
                    vecs[o + k] = v;
                }
            }
        }
        double2 nn = make_double2(0.0, 0.0);
        for (int64_t row = threadIdx.x; row < rows; row += blockDim.x) {
            const double2 v = vecs[off(row) + k];
            nn.x += v.x * v.x + v.y * v.y;
        }
        nn = block_sum(nn, red);
        const double inv = nn.x > 0.0 ? 1.0 / sqrt(nn.x) : 0.0;
        for (int64_t row = threadIdx.x; row < rows; row += blockDim.x) {
            const int64_t o = off(row) + k;
            const double2 v = vecs[o];
            vecs[o] = make_double2(v.x * inv, v.y * inv);
        }
    }
}

void block_orthonormalize(const Level &f, double2 *vecs, cudaStream_t s) {
    Level dummy;
    for (int mu = 0; mu < 4; ++mu) dummy.L[mu] = f.L[mu] / f.B[mu];
    const AggGeom a = agg_geom(f, dummy, 1);
    dim3 grid((unsigned)(f.V / f.asize), 2);
    k_block_orth<<<grid, 256, 0, s>>>(vecs, a);
    MRHS_LAUNCHED("k_block_orth");
}

}  // namespace mrhs
