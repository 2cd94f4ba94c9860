// Paired-FP32 arithmetic shared by the FP32 stencil kernels (fine operator,
// even-odd operators, SAP block solves): two RHS per thread held as
// (Re r0, Re r1) / (Im r0, Im r1) pairs so that every multiply-add runs as
// one paired FP32 instruction (FFMA2 / FADD2 / FMUL2 on sm_100 and later).
#pragma once

#include "common.cuh"
#include "spin.cuh"

namespace mrhs {

struct P2 {
    float2 re, im;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ P2 p2add(P2 a, P2 b) { return {__fadd2_rn(a.re, b.re), __fadd2_rn(a.im, b.im)}; }
template <int F> __device__ __forceinline__ P2 p2f(P2 a) {
    if constexpr (F == FP) return a;
    else if constexpr (F == FM) return {neg2(a.re), neg2(a.im)};
    else if constexpr (F == FI) return {neg2(a.im), a.re};
    else return {a.im, neg2(a.re)};
}
__device__ __forceinline__ P2 ld_p2(const float2 *__restrict__ p, int64_t off) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p + off));
    return {make_float2(v.x, v.z), make_float2(v.y, v.w)};
}
// streaming store: the result is not read again by this kernel, keep it from
// displacing neighbour spinors in L2
__device__ __forceinline__ void st_p2(float2 *p, int64_t off, P2 v) {
    __stcs(reinterpret_cast<float4 *>(p + off), make_float4(v.re.x, v.im.x, v.re.y, v.im.y));
}
// acc += u * h  (u one complex number shared by both RHS)
__device__ __forceinline__ void p2mac(P2 &acc, float2 u, P2 h) {
    const float2 ur = make_float2(u.x, u.x), ui = make_float2(u.y, u.y), nui = make_float2(-u.y, -u.y);
    acc.re = __ffma2_rn(ur, h.re, acc.re);
    acc.re = __ffma2_rn(nui, h.im, acc.re);
    acc.im = __ffma2_rn(ur, h.im, acc.im);
    acc.im = __ffma2_rn(ui, h.re, acc.im);
}
// acc += conj(u) * h
__device__ __forceinline__ void p2mac_conj(P2 &acc, float2 u, P2 h) {
    const float2 ur = make_float2(u.x, u.x), ui = make_float2(u.y, u.y), nui = make_float2(-u.y, -u.y);
    acc.re = __ffma2_rn(ur, h.re, acc.re);
    acc.re = __ffma2_rn(ui, h.im, acc.re);
    acc.im = __ffma2_rn(ur, h.im, acc.im);
    acc.im = __ffma2_rn(nui, h.re, acc.im);
}

// o = M v for chirality block chi of a compact Hermitian site matrix M (the
// clover term C or its inverse): 3 diagonal pairs, then the 15 lower entries.
// AOS = false: entry (chi * 18 + q) of site x at M[(chi * 18 + q) * V + x]
// (entry-major); AOS = true: at M[x * 36 + chi * 18 + q] (site-major, so the
// 18 loads of a block are immediate offsets from one address).
template <bool AOS = false>
__device__ __forceinline__ void site_mat_x2(const float2 *__restrict__ M, int V, int site, int chi,
                                            const P2 (&v)[6], P2 (&o)[6]) {
    const float2 *Mp = AOS ? M + (int64_t)site * 36 + chi * 18 : M + (int64_t)chi * 18 * V + site;
    const int64_t st = AOS ? 1 : V;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float2 d = __ldg(Mp + q * st);
        const float2 d0 = make_float2(d.x, d.x), d1 = make_float2(d.y, d.y);
        o[2 * q] = {__fmul2_rn(d0, v[2 * q].re), __fmul2_rn(d0, v[2 * q].im)};
        o[2 * q + 1] = {__fmul2_rn(d1, v[2 * q + 1].re), __fmul2_rn(d1, v[2 * q + 1].im)};
    }
    int q = 3;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j, ++q) {
            const float2 l = __ldg(Mp + q * st);
            p2mac(o[i], l, v[j]);
            p2mac_conj(o[j], l, v[i]);
        }
    }
}

}  // namespace mrhs
