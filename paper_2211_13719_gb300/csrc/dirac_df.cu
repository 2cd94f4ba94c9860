// Fine operator (paper Sec. 4) in float-float arithmetic for the outer
// solver's Arnoldi applies w = D z, z an FP32 field, w an FP64 field.
//
// GB300 executes FP32 at about 60 times its FP64 rate, so the FP64-accurate
// operator is evaluated on the FP32 units: every real value of the links and
// the clover is stored as hi + lo (two floats, hi = fl32(x), lo = fl32(x - hi),
// 48 significant bits), products of hi parts are made exact with one FMA
// (Dekker's product: a b = p + fma(a, b, -p)), sums of hi parts with Knuth's
// two-sum, and the low parts (errors and cross terms) are gathered in FP32.
// The result differs from an FP64 evaluation by about 2^-48 times the largest
// term; it is converted to FP64 on store.  The input z is exact in FP32; the
// spin projection psi_up -+ A psi_dn is formed exactly by a two-sum.
// Intrinsics (__fmul_rn, __fadd_rn, ...) keep the compiler from contracting or
// reordering these steps.
#include "internal.cuh"
#include "spin.cuh"

namespace mrhs {

namespace {

struct df {
    float hi, lo;
};
struct dfc {
    df re, im;
};

// a + b = s + e exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df neg(df a) { return {-a.hi, -a.lo}; }
// acc += a b
__device__ __forceinline__ void mac(df &acc, df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
// acc += a b, b a plain float
__device__ __forceinline__ void mac(df &acc, df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    const df s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void add(df &acc, df b) {
    const df s = two_sum(acc.hi, b.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, b.lo));
}

template <int F> __device__ __forceinline__ dfc fmul_df(dfc a) {
    if constexpr (F == FP) return a;
    else if constexpr (F == FM) return {neg(a.re), neg(a.im)};
    else if constexpr (F == FI) return {neg(a.im), a.re};
    else return {a.im, neg(a.re)};
}
__device__ __forceinline__ void cadd(dfc &acc, dfc b) {
    add(acc.re, b.re);
    add(acc.im, b.im);
}
// acc += u h
__device__ __forceinline__ void cmac_df(dfc &acc, dfc u, dfc h) {
    mac(acc.re, u.re, h.re);
    mac(acc.re, neg(u.im), h.im);
    mac(acc.im, u.re, h.im);
    mac(acc.im, u.im, h.re);
}
// acc += u v, v an FP32 complex
__device__ __forceinline__ void cmac_df(dfc &acc, dfc u, float2 v) {
    mac(acc.re, u.re, v.x);
    mac(acc.re, neg(u.im), v.y);
    mac(acc.im, u.re, v.y);
    mac(acc.im, u.im, v.x);
}
// acc += conj(u) v, v an FP32 complex
__device__ __forceinline__ void cmac_conj_df(dfc &acc, dfc u, float2 v) {
    mac(acc.re, u.re, v.x);
    mac(acc.re, u.im, v.y);
    mac(acc.im, u.re, v.y);
    mac(acc.im, neg(u.im), v.x);
}
__device__ __forceinline__ dfc ld_df(const float4 *__restrict__ p, int64_t i) {
    const float4 v = __ldg(p + i);
    return {{v.x, v.y}, {v.z, v.w}};
}
template <int F> __device__ __forceinline__ float2 fmul32(float2 a) {
    if constexpr (F == FP) return a;
    else if constexpr (F == FM) return make_float2(-a.x, -a.y);
    else if constexpr (F == FI) return make_float2(-a.y, a.x);
    else return make_float2(a.y, -a.x);
}

struct KArgsDF {
    Geom g;
    int n;
    int64_t stride[4];
};

template <int MU, bool FWD>
__device__ __forceinline__ void hop_df(dfc (&acc)[12], const float4 *__restrict__ U, const float2 *__restrict__ in,
                                       const KArgsDF &a, int64_t nb, int64_t link_site, bool flip, int r) {
    using P = Proj<MU>;
    constexpr int F0 = FWD ? P::F0 : neg_f<P::F0>::v;
    constexpr int F1 = FWD ? P::F1 : neg_f<P::F1>::v;
    constexpr int G2 = FWD ? P::G2 : neg_f<P::G2>::v;
    constexpr int G3 = FWD ? P::G3 : neg_f<P::G3>::v;
    const int64_t V = a.g.V;
    const int64_t base = nb * 12 * a.n + r;
    dfc h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 p0 = __ldg(in + base + (int64_t)(0 * 3 + c) * a.n);
        const float2 p1 = __ldg(in + base + (int64_t)(1 * 3 + c) * a.n);
        const float2 pa = fmul32<F0>(__ldg(in + base + (int64_t)(P::P0 * 3 + c) * a.n));
        const float2 pb = fmul32<F1>(__ldg(in + base + (int64_t)(P::P1 * 3 + c) * a.n));
        h0[c] = {two_sum(p0.x, pa.x), two_sum(p0.y, pa.y)};
        h1[c] = {two_sum(p1.x, pb.x), two_sum(p1.y, pb.y)};
        if (flip) {
            h0[c] = fmul_df<FM>(h0[c]);
            h1[c] = fmul_df<FM>(h1[c]);
        }
    }
#pragma unroll
    for (int row = 0; row < 3; ++row) {
        dfc s0 = {{0.f, 0.f}, {0.f, 0.f}}, s1 = s0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            // forward: row `row` of U_mu(x); backward: column `row` of U_mu(x - mu), conjugated
            dfc u = FWD ? ld_df(U, (int64_t)(MU * 9 + row * 3 + b) * V + link_site)
                        : ld_df(U, (int64_t)(MU * 9 + b * 3 + row) * V + link_site);
            if (!FWD) u.im = neg(u.im);
            cmac_df(s0, u, h0[b]);
            cmac_df(s1, u, h1[b]);
        }
        cadd(acc[0 * 3 + row], s0);
        cadd(acc[1 * 3 + row], s1);
        cadd(acc[2 * 3 + row], fmul_df<G2>(P::Q2 == 0 ? s0 : s1));
        cadd(acc[3 * 3 + row], fmul_df<G3>(P::Q3 == 0 ? s0 : s1));
    }
}

template <int MU>
__device__ __forceinline__ void hop_pair_df(dfc (&acc)[12], const float4 *__restrict__ U,
                                            const float2 *__restrict__ in, const KArgsDF &a, int64_t site,
                                            const int c[4], int r) {
    const int L = a.g.L[MU];
    const int64_t st = a.stride[MU];
    const bool wrapF = (c[MU] == L - 1), wrapB = (c[MU] == 0);
    const int64_t sf = wrapF ? site - st * (L - 1) : site + st;
    const int64_t sb = wrapB ? site + st * (L - 1) : site - st;
    const bool flipF = MU == 3 && wrapF && a.g.tb < 0;
    const bool flipB = MU == 3 && wrapB && a.g.tb < 0;
    hop_df<MU, true>(acc, U, in, a, sf, site, flipF, r);
    hop_df<MU, false>(acc, U, in, a, sb, sb, flipB, r);
}

__device__ __forceinline__ double to_f64(df v) { return (double)v.hi + (double)v.lo; }

// out = C psi - 1/2 sum(hops)  (RESID: out = y - that), FP32 psi, FP64 out
template <bool RESID>
__global__ void __launch_bounds__(128) k_dslash_df(const float4 *__restrict__ U, const float4 *__restrict__ C,
                                                    const float2 *__restrict__ in, double2 *__restrict__ out,
                                                    const double2 *__restrict__ y, KArgsDF a) {
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t site = item / a.n;
    if (site >= a.g.V) return;
    const int r = (int)(item - site * a.n);
    int c[4];
    site_to_coords(site, a.g.L, c);
    dfc acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {{0.f, 0.f}, {0.f, 0.f}};
    hop_pair_df<0>(acc, U, in, a, site, c, r);
    hop_pair_df<1>(acc, U, in, a, site, c, r);
    hop_pair_df<2>(acc, U, in, a, site, c, r);
    hop_pair_df<3>(acc, U, in, a, site, c, r);

    const int64_t V = a.g.V;
    const int64_t base = site * 12 * a.n + r;
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        float2 v[6];
        dfc o[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            v[i] = __ldg(in + base + (int64_t)(6 * chi + i) * a.n);
            o[i] = {{0.f, 0.f}, {0.f, 0.f}};
        }
        // diagonal pairs (d_{2q}, d_{2q+1}) stored as one complex entry
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const dfc d = ld_df(C, (int64_t)(chi * 18 + q) * V + site);
            mac(o[2 * q].re, d.re, v[2 * q].x);
            mac(o[2 * q].im, d.re, v[2 * q].y);
            mac(o[2 * q + 1].re, d.im, v[2 * q + 1].x);
            mac(o[2 * q + 1].im, d.im, v[2 * q + 1].y);
        }
        int q = 3;
#pragma unroll
        for (int i = 1; i < 6; ++i) {
#pragma unroll
            for (int j = 0; j < i; ++j, ++q) {
                const dfc l = ld_df(C, (int64_t)(chi * 18 + q) * V + site);
                cmac_df(o[i], l, v[j]);
                cmac_conj_df(o[j], l, v[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const dfc ai = acc[6 * chi + i];
            // o - acc / 2 in float-float (halving is exact), one conversion per real
            df re = o[i].re, im = o[i].im;
            add(re, {-0.5f * ai.re.hi, -0.5f * ai.re.lo});
            add(im, {-0.5f * ai.im.hi, -0.5f * ai.im.lo});
            const double dre = to_f64(re), dim = to_f64(im);
            const int64_t off = base + (int64_t)(6 * chi + i) * a.n;
            if constexpr (RESID) {
                const double2 yy = __ldg(y + off);
                out[off] = make_double2(yy.x - dre, yy.y - dim);
            } else {
                out[off] = make_double2(dre, dim);
            }
        }
    }
}

// FP64 complex -> (hi, lo) float pairs
__global__ void k_split_df(const double2 *__restrict__ src, float4 *__restrict__ dst, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double2 v = src[i];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    dst[i] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

}  // namespace

void split_df(const void *src_c128, void *dst_f4, int64_t count, cudaStream_t s) {
    k_split_df<<<ceil_div(count, 256), 256, 0, s>>>(static_cast<const double2 *>(src_c128),
                                                    static_cast<float4 *>(dst_f4), count);
    MRHS_LAUNCHED("k_split_df");
}

void dslash_df(const mrhs_lattice &lat, const void *in, void *out, const void *y, int n, cudaStream_t s) {
    if (!lat.has_clover || !lat.Udf.ptr || !lat.Cdf.ptr) fail(MRHS_ERR_INVALID, "clover term not built");
    KArgsDF a;
    a.g = lat.g;
    a.n = n;
    a.stride[0] = 1;
    a.stride[1] = a.g.L[0];
    a.stride[2] = (int64_t)a.g.L[0] * a.g.L[1];
    a.stride[3] = (int64_t)a.g.L[0] * a.g.L[1] * a.g.L[2];
    const int64_t items = a.g.V * n;
    const int threads = 128;
    const unsigned blocks = (unsigned)((items + threads - 1) / threads);
    const float4 *U = lat.Udf.as<float4>();
    const float4 *C = lat.Cdf.as<float4>();
    MRHS_TIMED("k_dslash_df", s);
    if (y)
        k_dslash_df<true><<<blocks, threads, 0, s>>>(U, C, static_cast<const float2 *>(in), static_cast<double2 *>(out),
                                                     static_cast<const double2 *>(y), a);
    else
        k_dslash_df<false><<<blocks, threads, 0, s>>>(U, C, static_cast<const float2 *>(in),
                                                      static_cast<double2 *>(out), nullptr, a);
    MRHS_LAUNCHED("k_dslash_df");
}

}  // namespace mrhs
