// Fine-level Wilson-clover operator (paper Sec. 4): fused hopping + compact
// clover (+ mass) with the RHS index innermost, plus the setup kernels that
// lay the gauge field out link-major and build the compact clover term.
//
// Work decomposition: one thread per (site, group of R consecutive RHS).
// Threads of one site are adjacent, so a warp reads each neighbour spinor
// component as one contiguous segment (16-byte vector loads for R = 2 in
// FP32) while every gauge link and clover entry is a single broadcast load
// shared by all RHS of the site: the MRHS reuse of Sec. 2.  With few RHS a
// warp spans many sites and the link-major (site-innermost) layout of U and
// of the clover keeps those loads coalesced as well; from 16 RHS on, where a
// warp covers one or two sites, the paired FP32 kernels read site-major
// copies instead, so the entries of one link or clover block are immediate
// offsets from one address.
//
// Spin projection (chiral basis, gamma_mu = [[0, A_mu], [A_mu^+, 0]] with
// A_k = -i sigma_k, A_t = 1): (1 -+ gamma_mu) psi has rank 2, so each hop
// forms a 2-spin half spinor h = psi_up -+ A psi_dn, multiplies it by the
// link, and rebuilds the lower spins from the two products.
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "internal.cuh"
#include "pair.cuh"
#include "spin.cuh"
#include "tc_common.cuh"

namespace mrhs {

// ------------------------------------------------------------ vector loads
// R consecutive complex values of the input field at complex offset `off`.
template <typename TIn, int R> struct Load;
template <> struct Load<float, 1> {
    template <typename Real> __device__ static void f(const void *p, int64_t off, cplx<Real> *v) {
        float2 a = __ldg(reinterpret_cast<const float2 *>(p) + off);
        v[0] = {(Real)a.x, (Real)a.y};
    }
};
template <> struct Load<float, 2> {
    template <typename Real> __device__ static void f(const void *p, int64_t off, cplx<Real> *v) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(p) + off));
        v[0] = {(Real)a.x, (Real)a.y};
        v[1] = {(Real)a.z, (Real)a.w};
    }
};
template <> struct Load<double, 1> {
    template <typename Real> __device__ static void f(const void *p, int64_t off, cplx<Real> *v) {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p) + off);
        v[0] = {(Real)a.x, (Real)a.y};
    }
};

template <typename Real, int R> struct Store;
template <> struct Store<float, 1> {
    __device__ static void f(void *p, int64_t off, const cplx<float> *v) {
        reinterpret_cast<float2 *>(p)[off] = make_float2(v[0].re, v[0].im);
    }
};
template <> struct Store<float, 2> {
    __device__ static void f(void *p, int64_t off, const cplx<float> *v) {
        *reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(p) + off) = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
    }
};
template <> struct Store<double, 1> {
    __device__ static void f(void *p, int64_t off, const cplx<double> *v) {
        reinterpret_cast<double2 *>(p)[off] = make_double2(v[0].re, v[0].im);
    }
};

template <typename Real> __device__ __forceinline__ cplx<Real> ldc(const cplx<Real> *p, int64_t i) {
    if constexpr (sizeof(Real) == 4) {
        float2 a = __ldg(reinterpret_cast<const float2 *>(p) + i);
        return {a.x, a.y};
    } else {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p) + i);
        return {a.x, a.y};
    }
}

struct KArgs {
    Geom g;
    int n;        // RHS count
    int G;        // RHS groups per site (n / R)
    int64_t stride[4];
};

// ------------------------------------------------------------ one direction
template <int MU, bool FWD, typename Real, typename TIn, int R>
__device__ __forceinline__ void hop(cplx<Real> (&acc)[12][R], const cplx<Real> *__restrict__ U,
                                    const TIn *__restrict__ in, const KArgs &a, int64_t nb,
                                    int64_t link_site, Real sign, int r0) {
    using P = Proj<MU>;
    constexpr int F0 = FWD ? P::F0 : neg_f<P::F0>::v;
    constexpr int F1 = FWD ? P::F1 : neg_f<P::F1>::v;
    constexpr int G2 = FWD ? P::G2 : neg_f<P::G2>::v;
    constexpr int G3 = FWD ? P::G3 : neg_f<P::G3>::v;
    const int64_t V = a.g.V;
    const int64_t base = nb * 12 * a.n + r0;
    cplx<Real> h0[3][R], h1[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cplx<Real> p0[R], p1[R], pa[R], pb[R];
        Load<TIn, R>::f(in, base + (int64_t)(0 * 3 + c) * a.n, p0);
        Load<TIn, R>::f(in, base + (int64_t)(1 * 3 + c) * a.n, p1);
        Load<TIn, R>::f(in, base + (int64_t)(P::P0 * 3 + c) * a.n, pa);
        Load<TIn, R>::f(in, base + (int64_t)(P::P1 * 3 + c) * a.n, pb);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            h0[c][r] = sign * (p0[r] + fmul<F0>(pa[r]));
            h1[c][r] = sign * (p1[r] + fmul<F1>(pb[r]));
        }
    }
#pragma unroll
    for (int row = 0; row < 3; ++row) {
        cplx<Real> u[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            // forward: row `row` of U_mu(x); backward: column `row` of U_mu(x - mu), conjugated
            u[b] = FWD ? ldc(U, (int64_t)(MU * 9 + row * 3 + b) * V + link_site)
                       : conj(ldc(U, (int64_t)(MU * 9 + b * 3 + row) * V + link_site));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cplx<Real> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                cmac(s0, u[b], h0[b][r]);
                cmac(s1, u[b], h1[b][r]);
            }
            acc[0 * 3 + row][r] = acc[0 * 3 + row][r] + s0;
            acc[1 * 3 + row][r] = acc[1 * 3 + row][r] + s1;
            const cplx<Real> q2 = P::Q2 == 0 ? s0 : s1;
            const cplx<Real> q3 = P::Q3 == 0 ? s0 : s1;
            acc[2 * 3 + row][r] = acc[2 * 3 + row][r] + fmul<G2>(q2);
            acc[3 * 3 + row][r] = acc[3 * 3 + row][r] + fmul<G3>(q3);
        }
    }
}

__device__ __forceinline__ bool hop_selected(const HopMask &m, int d, int loc, int B, bool fwd) {
    if (m.dir >= 0 && m.dir != d) return false;
    if (m.cross == 0) return true;
    const bool crossing = fwd ? (loc == B - 1) : (loc == 0);
    return m.cross == 1 ? crossing : !crossing;
}

template <int MU, typename Real, typename TIn, int R, bool GENERAL>
__device__ __forceinline__ void hop_pair(cplx<Real> (&acc)[12][R], const cplx<Real> *__restrict__ U,
                                         const TIn *__restrict__ in, const KArgs &a, int64_t site,
                                         const int c[4], int r0, const HopMask &mask) {
    const int L = a.g.L[MU];
    const int64_t st = a.stride[MU];
    const bool wrapF = (c[MU] == L - 1), wrapB = (c[MU] == 0);
    const int64_t sf = wrapF ? site - st * (L - 1) : site + st;
    const int64_t sb = wrapB ? site + st * (L - 1) : site - st;
    const Real sgnF = (MU == 3 && wrapF) ? (Real)a.g.tb : (Real)1;
    const Real sgnB = (MU == 3 && wrapB) ? (Real)a.g.tb : (Real)1;
    bool doF = true, doB = true;
    if constexpr (GENERAL) {
        const int loc = c[MU] % mask.B[MU];
        doF = hop_selected(mask, 1 + MU, loc, mask.B[MU], true);
        doB = hop_selected(mask, 5 + MU, loc, mask.B[MU], false);
    }
    if (doF) hop<MU, true, Real, TIn, R>(acc, U, in, a, sf, site, sgnF, r0);
    if (doB) hop<MU, false, Real, TIn, R>(acc, U, in, a, sb, sb, sgnB, r0);
}

// out = C psi - 1/2 sum(hops)  (RESID: out = y - that)
template <typename Real, typename TIn, int R, bool RESID, bool GENERAL>
__global__ void __launch_bounds__(128) k_dslash(const cplx<Real> *__restrict__ U, const cplx<Real> *__restrict__ C,
                                                 const TIn *__restrict__ in, Real *__restrict__ out,
                                                 const Real *__restrict__ y, KArgs a, HopMask mask) {
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t site = item / a.G;
    if (site >= a.g.V) return;
    const int r0 = (int)(item - site * a.G) * R;
    int c[4];
    site_to_coords(site, a.g.L, c);

    cplx<Real> acc[12][R];
#pragma unroll
    for (int i = 0; i < 12; ++i)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[i][r] = {0, 0};

    hop_pair<0, Real, TIn, R, GENERAL>(acc, U, in, a, site, c, r0, mask);
    hop_pair<1, Real, TIn, R, GENERAL>(acc, U, in, a, site, c, r0, mask);
    hop_pair<2, Real, TIn, R, GENERAL>(acc, U, in, a, site, c, r0, mask);
    hop_pair<3, Real, TIn, R, GENERAL>(acc, U, in, a, site, c, r0, mask);

    const bool diag = GENERAL ? (mask.diag != 0) : true;
    const int64_t V = a.g.V;
    const int64_t base = site * 12 * a.n + r0;
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        cplx<Real> v[6][R], o[6][R];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            Load<TIn, R>::f(in, base + (int64_t)(6 * chi + i) * a.n, v[i]);
#pragma unroll
            for (int r = 0; r < R; ++r) o[i][r] = {0, 0};
        }
        if (diag) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const cplx<Real> d = ldc(C, (int64_t)(chi * 18 + q) * V + site);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    o[2 * q][r] = d.re * v[2 * q][r];
                    o[2 * q + 1][r] = d.im * v[2 * q + 1][r];
                }
            }
            int q = 3;
#pragma unroll
            for (int i = 1; i < 6; ++i) {
#pragma unroll
                for (int j = 0; j < i; ++j, ++q) {
                    const cplx<Real> l = ldc(C, (int64_t)(chi * 18 + q) * V + site);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        cmac(o[i][r], l, v[j][r]);
                        cmac_conj(o[j][r], l, v[i][r]);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            cplx<Real> res[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                res[r] = o[i][r] - (Real)0.5 * acc[6 * chi + i][r];
            }
            const int64_t off = base + (int64_t)(6 * chi + i) * a.n;
            if constexpr (RESID) {
                cplx<Real> yy[R];
                Load<Real, R>::f(y, off, yy);
#pragma unroll
                for (int r = 0; r < R; ++r) res[r] = yy[r] - res[r];
            }
            Store<Real, R>::f(out, off, res);
        }
    }
}

// Sites are visited tile by tile: 4-D tiles of T[0] x T[1] x T[2] x T[3]
// sites (x fastest inside a tile), tiles in lexicographic order, x fastest.
// With T = 1 x 4 x 8 x 8 most neighbours of a site are visited a few hundred
// sites before or after it; measured on GB300 (24^3 x 64, 48 RHS) 18 % faster
// than visiting Lx x Ly x 8 x Lt bricks and 9-14 % faster than 4^4 tiles.
// Below 16 RHS the tiles span whole x rows (Lx x 4 x 8 x 8).
struct KArgs32 {
    int L[4];
    int V;
    int n, G;
    int stride[4];
    int tb;
    int T[4];     // tile extents (each divides L)
    int NT[3];    // tiles along x, y, z
    int tsites;   // sites per tile (mode 0) or per region (mode 1)
    // visit order: 0 = tiles of T, tiles x-fastest; 1 = x-regions of RX sites
    // (whole y, z, t extents), lexicographic inside a region (x fastest, t
    // slowest); 2 = RHS slabs of GS pairs, each slab a lexicographic sweep of
    // the whole lattice (t slowest).  Modes 1 and 2 keep the L2 window of a
    // sweep at about two t-layers of the region or slab.
    int mode;
    int RX;
    int GS;
    int occ8;  // host side: the one-RHS-per-thread build for 8 CTAs per SM (64 registers)
};

// Coordinates of the site a thread visits and its first RHS (r0) under the
// visit order of `a`; false for threads past the end.  `xpair`: the site
// index counts x pairs (one output site of a given parity per pair, even-odd
// kernels), the member of the pair is chosen by the caller.
__device__ __forceinline__ bool visit_coords(const KArgs32 &a, int item, int nvisit, bool xpair, int c[4],
                                             int &r0, int per_thread = 2) {
    int visit;
    if (a.mode == 2) {
        const int per_slab = nvisit * a.GS;
        const int slab = item / per_slab;
        const int rem = item - slab * per_slab;
        visit = rem / a.GS;
        if (slab * a.GS >= a.G) return false;
        r0 = (slab * a.GS + rem - visit * a.GS) * per_thread;
    } else {
        visit = item / a.G;
        if (visit >= nvisit) return false;
        r0 = (item - visit * a.G) * per_thread;
    }
    const int X = xpair ? a.L[0] / 2 : a.L[0];
    if (a.mode == 2) {
        int q = visit;
        c[0] = q % X;
        q /= X;
        c[1] = q % a.L[1];
        q /= a.L[1];
        c[2] = q % a.L[2];
        c[3] = q / a.L[2];
    } else if (a.mode == 1) {
        const int RX = xpair ? a.RX / 2 : a.RX;
        const int reg = visit / a.tsites;
        int q = visit - reg * a.tsites;
        c[0] = reg * RX + q % RX;
        q /= RX;
        c[1] = q % a.L[1];
        q /= a.L[1];
        c[2] = q % a.L[2];
        c[3] = q / a.L[2];
    } else {
        const int tile = visit / a.tsites;
        int q = visit - tile * a.tsites;
        int tq = tile;
        const int t0 = tq % a.NT[0];
        tq /= a.NT[0];
        const int t1 = tq % a.NT[1];
        tq /= a.NT[1];
        const int t2 = tq % a.NT[2];
        const int t3 = tq / a.NT[2];
        const int T0 = xpair ? 1 : a.T[0];
        c[0] = t0 * T0 + q % T0;
        q /= T0;
        c[1] = t1 * a.T[1] + q % a.T[1];
        q /= a.T[1];
        c[2] = t2 * a.T[2] + q % a.T[2];
        c[3] = t3 * a.T[3] + q / a.T[2];
    }
    return true;
}

// N: the RHS count as a compile-time constant (0: a.n at run time), so that
// the 12 component loads of a neighbour are immediate offsets from one
// address.  AOS: links site-major, [V][4][9] (the 9 entries of a link are
// immediate offsets), else link-major [(mu * 9 + e)][V].
template <int N> __device__ __forceinline__ int rhs_count(const KArgs32 &a) { return N ? N : a.n; }

template <int MU, bool FWD, int N, bool AOS>
__device__ __forceinline__ void hop_x2(P2 (&acc)[12], const float2 *__restrict__ U, const float2 *__restrict__ in,
                                      const KArgs32 &a, int nb, int link_site, bool flip, int r0) {
    using P = Proj<MU>;
    constexpr int F0 = FWD ? P::F0 : neg_f<P::F0>::v;
    constexpr int F1 = FWD ? P::F1 : neg_f<P::F1>::v;
    constexpr int G2 = FWD ? P::G2 : neg_f<P::G2>::v;
    constexpr int G3 = FWD ? P::G3 : neg_f<P::G3>::v;
    const int n = rhs_count<N>(a);
    const float2 *pin = in + ((int64_t)nb * 12 * n + r0);
    P2 h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const P2 p0 = ld_p2(pin, (0 * 3 + c) * n);
        const P2 p1 = ld_p2(pin, (1 * 3 + c) * n);
        const P2 pa = ld_p2(pin, (P::P0 * 3 + c) * n);
        const P2 pb = ld_p2(pin, (P::P1 * 3 + c) * n);
        h0[c] = p2add(p0, p2f<F0>(pa));
        h1[c] = p2add(p1, p2f<F1>(pb));
    }
    if (flip) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h0[c] = p2f<FM>(h0[c]);
            h1[c] = p2f<FM>(h1[c]);
        }
    }
    const float2 *Ul = AOS ? U + ((int64_t)link_site * 4 + MU) * 9 : U + (int64_t)MU * 9 * a.V + link_site;
    const int64_t ust = AOS ? 1 : a.V;
#pragma unroll
    for (int row = 0; row < 3; ++row) {
        P2 s0 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, s1 = s0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (FWD) {
                const float2 u = __ldg(Ul + (row * 3 + b) * ust);
                p2mac(s0, u, h0[b]);
                p2mac(s1, u, h1[b]);
            } else {
                const float2 u = __ldg(Ul + (b * 3 + row) * ust);
                p2mac_conj(s0, u, h0[b]);
                p2mac_conj(s1, u, h1[b]);
            }
        }
        acc[0 * 3 + row] = p2add(acc[0 * 3 + row], s0);
        acc[1 * 3 + row] = p2add(acc[1 * 3 + row], s1);
        acc[2 * 3 + row] = p2add(acc[2 * 3 + row], p2f<G2>(P::Q2 == 0 ? s0 : s1));
        acc[3 * 3 + row] = p2add(acc[3 * 3 + row], p2f<G3>(P::Q3 == 0 ? s0 : s1));
    }
}

template <int MU, int N, bool AOS>
__device__ __forceinline__ void hop_pair_x2(P2 (&acc)[12], const float2 *__restrict__ U,
                                           const float2 *__restrict__ in, const KArgs32 &a, int site,
                                           const int c[4], int r0) {
    const int L = a.L[MU];
    const int st = a.stride[MU];
    const bool wrapF = (c[MU] == L - 1), wrapB = (c[MU] == 0);
    const int sf = wrapF ? site - st * (L - 1) : site + st;
    const int sb = wrapB ? site + st * (L - 1) : site - st;
    const bool flipF = MU == 3 && wrapF && a.tb < 0;
    const bool flipB = MU == 3 && wrapB && a.tb < 0;
    hop_x2<MU, true, N, AOS>(acc, U, in, a, sf, site, flipF, r0);
    hop_x2<MU, false, N, AOS>(acc, U, in, a, sb, sb, flipB, r0);
}

// 128 threads, at most 168 registers (3 CTAs per SM): measured on GB300 (24^3 x
// 64) 8 % faster than 128 registers (4 CTAs), which left the compiler too few
// registers to issue the loads of one hop ahead of the previous hop's arithmetic
template <bool RESID, int N, bool AOS>
__global__ void __launch_bounds__(128, 3) k_dslash_x2(const float2 *__restrict__ U, const float2 *__restrict__ C,
                                                       const float2 *__restrict__ in, float2 *__restrict__ out,
                                                       const float2 *__restrict__ y, KArgs32 a) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    int c[4], r0;
    if (!visit_coords(a, item, a.V, false, c, r0)) return;
    const int site = c[0] + a.L[0] * (c[1] + a.L[1] * (c[2] + a.L[2] * c[3]));
    P2 acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    hop_pair_x2<0, N, AOS>(acc, U, in, a, site, c, r0);
    hop_pair_x2<1, N, AOS>(acc, U, in, a, site, c, r0);
    hop_pair_x2<2, N, AOS>(acc, U, in, a, site, c, r0);
    hop_pair_x2<3, N, AOS>(acc, U, in, a, site, c, r0);

    const int V = a.V;
    const int n = rhs_count<N>(a);
    const int64_t base = (int64_t)site * 12 * n + r0;
    const float2 *pin = in + base;
    const float2 mhalf = make_float2(-0.5f, -0.5f);
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        P2 v[6], o[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = ld_p2(pin, (6 * chi + i) * n);
        site_mat_x2<AOS>(C, V, site, chi, v, o);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const P2 acc_i = acc[6 * chi + i];
            P2 res = {__ffma2_rn(mhalf, acc_i.re, o[i].re), __ffma2_rn(mhalf, acc_i.im, o[i].im)};
            if constexpr (RESID) {
                const P2 yy = ld_p2(y + base, (6 * chi + i) * n);
                res = {__fadd2_rn(yy.re, neg2(res.re)), __fadd2_rn(yy.im, neg2(res.im))};
            }
            st_p2(out + base, (6 * chi + i) * n, res);
        }
    }
}

// ------------------------------------------------ one RHS per thread (FP32)
// The same arithmetic as the paired kernels, one RHS per thread in scalar FMA:
// every multiply-add, add and rounding happens in the order of the paired
// code (p2mac = cmac, p2mac_conj = cmac_conj, p2add = add), so each output is
// bitwise that of k_dslash_x2 / k_eo_x2.  No register pairs have to be built
// (the paired code spends about a third of its instructions forming pairs
// for FFMA2), and at half the registers twice the warps are resident to hide
// the neighbour-load latency.  Links and site matrices from the site-major
// copies; N: the RHS count compiled in.
__device__ __forceinline__ cplx<float> ld_c1(const float2 *__restrict__ p, int64_t off) {
    const float2 v = __ldg(p + off);
    return {v.x, v.y};
}
__device__ __forceinline__ cplx<float> cadd_rn(cplx<float> a, cplx<float> b) {
    return {__fadd_rn(a.re, b.re), __fadd_rn(a.im, b.im)};
}

// one complex value of a neighbour spinor: from global memory (read-only path)
// or from a shared-memory copy
template <bool SMEM> __device__ __forceinline__ cplx<float> ld_src(const float2 *__restrict__ p, int off) {
    if constexpr (SMEM) {
        const float2 v = p[off];
        return {v.x, v.y};
    } else {
        return ld_c1(p, off);
    }
}

// one hop for one RHS: pin points at the neighbour's first spin-colour
// component of this RHS, components n apart
template <int MU, bool FWD, bool SMEM>
__device__ __forceinline__ void hop_r1_at(cplx<float> (&acc)[12], const float2 *__restrict__ U,
                                         const float2 *__restrict__ pin, int n, int link_site, bool flip) {
    using P = Proj<MU>;
    constexpr int F0 = FWD ? P::F0 : neg_f<P::F0>::v;
    constexpr int F1 = FWD ? P::F1 : neg_f<P::F1>::v;
    constexpr int G2 = FWD ? P::G2 : neg_f<P::G2>::v;
    constexpr int G3 = FWD ? P::G3 : neg_f<P::G3>::v;
    cplx<float> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<float> p0 = ld_src<SMEM>(pin, (0 * 3 + c) * n);
        const cplx<float> p1 = ld_src<SMEM>(pin, (1 * 3 + c) * n);
        const cplx<float> pa = ld_src<SMEM>(pin, (P::P0 * 3 + c) * n);
        const cplx<float> pb = ld_src<SMEM>(pin, (P::P1 * 3 + c) * n);
        h0[c] = cadd_rn(p0, fmul<F0>(pa));
        h1[c] = cadd_rn(p1, fmul<F1>(pb));
    }
    if (flip) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h0[c] = fmul<FM>(h0[c]);
            h1[c] = fmul<FM>(h1[c]);
        }
    }
    const float2 *Ul = U + ((int64_t)link_site * 4 + MU) * 9;
#pragma unroll
    for (int row = 0; row < 3; ++row) {
        cplx<float> s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (FWD) {
                const cplx<float> u = ld_c1(Ul, row * 3 + b);
                cmac(s0, u, h0[b]);
                cmac(s1, u, h1[b]);
            } else {
                const cplx<float> u = ld_c1(Ul, b * 3 + row);
                cmac_conj(s0, u, h0[b]);
                cmac_conj(s1, u, h1[b]);
            }
        }
        acc[0 * 3 + row] = cadd_rn(acc[0 * 3 + row], s0);
        acc[1 * 3 + row] = cadd_rn(acc[1 * 3 + row], s1);
        acc[2 * 3 + row] = cadd_rn(acc[2 * 3 + row], fmul<G2>(P::Q2 == 0 ? s0 : s1));
        acc[3 * 3 + row] = cadd_rn(acc[3 * 3 + row], fmul<G3>(P::Q3 == 0 ? s0 : s1));
    }
}

template <int MU, bool FWD, int N>
__device__ __forceinline__ void hop_r1(cplx<float> (&acc)[12], const float2 *__restrict__ U,
                                      const float2 *__restrict__ in, int nb, int link_site, bool flip, int r,
                                      int n_rt = 0) {
    const int n = N ? N : n_rt;  // RHS count: compiled in, or at run time (N = 0)
    hop_r1_at<MU, FWD, false>(acc, U, in + ((int64_t)nb * 12 * n + r), n, link_site, flip);
}

// o = M v for chirality block chi of a site-major compact Hermitian site matrix (one RHS)
__device__ __forceinline__ void site_mat_r1(const float2 *__restrict__ M, int site, int chi, const cplx<float> (&v)[6],
                                            cplx<float> (&o)[6]) {
    const float2 *Mp = M + (int64_t)site * 36 + chi * 18;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float2 d = __ldg(Mp + q);
        o[2 * q] = {__fmul_rn(d.x, v[2 * q].re), __fmul_rn(d.x, v[2 * q].im)};
        o[2 * q + 1] = {__fmul_rn(d.y, v[2 * q + 1].re), __fmul_rn(d.y, v[2 * q + 1].im)};
    }
    int q = 3;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j, ++q) {
            const cplx<float> l = ld_c1(Mp, q);
            cmac(o[i], l, v[j]);
            cmac_conj(o[j], l, v[i]);
        }
    }
}

template <int MU, int N>
__device__ __forceinline__ void hop_pair_r1(cplx<float> (&acc)[12], const float2 *__restrict__ U,
                                           const float2 *__restrict__ in, const KArgs32 &a, int site, const int c[4],
                                           int r) {
    const int L = a.L[MU];
    const int st = a.stride[MU];
    const bool wrapF = (c[MU] == L - 1), wrapB = (c[MU] == 0);
    const int sf = wrapF ? site - st * (L - 1) : site + st;
    const int sb = wrapB ? site + st * (L - 1) : site - st;
    const bool flipF = MU == 3 && wrapF && a.tb < 0;
    const bool flipB = MU == 3 && wrapB && a.tb < 0;
    hop_r1<MU, true, N>(acc, U, in, sf, site, flipF, r, a.n);
    hop_r1<MU, false, N>(acc, U, in, sb, sb, flipB, r, a.n);
}

// out(x) = (D in)(x) (RESID: y(x) - (D in)(x)) for RHS r of the site at coordinates c:
// the hop, the clover term and the axpy of one thread (one RHS).  SPLIT (even-odd
// smoother): the result goes to half fields instead, out (even sites) or ro (odd sites)
// at index site / 2, and at the even sites also te = Cinv out.
template <bool RESID, int N, bool SPLIT = false>
__device__ __forceinline__ void dslash_r1_site(const float2 *__restrict__ U, const float2 *__restrict__ C,
                                               const float2 *__restrict__ in, float2 *__restrict__ out,
                                               const float2 *__restrict__ y, const KArgs32 &a, const int c[4],
                                               int r, float2 *__restrict__ ro = nullptr,
                                               float2 *__restrict__ te = nullptr,
                                               const float2 *__restrict__ Cinv = nullptr) {
    const int n = N ? N : a.n;
    const int site = c[0] + a.L[0] * (c[1] + a.L[1] * (c[2] + a.L[2] * c[3]));
    cplx<float> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
    hop_pair_r1<0, N>(acc, U, in, a, site, c, r);
    hop_pair_r1<1, N>(acc, U, in, a, site, c, r);
    hop_pair_r1<2, N>(acc, U, in, a, site, c, r);
    hop_pair_r1<3, N>(acc, U, in, a, site, c, r);
    const int64_t base = (int64_t)site * 12 * n + r;
    const int64_t hbase = (int64_t)(site >> 1) * 12 * n + r;  // SPLIT: the half-field index
    const bool odd = ((c[0] + c[1] + c[2] + c[3]) & 1) != 0;
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        cplx<float> v[6], o[6], res6[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = ld_c1(in, base + (6 * chi + i) * n);
        site_mat_r1(C, site, chi, v, o);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const cplx<float> ai = acc[6 * chi + i];
            cplx<float> res = {__fmaf_rn(-0.5f, ai.re, o[i].re), __fmaf_rn(-0.5f, ai.im, o[i].im)};
            const int64_t off = base + (6 * chi + i) * n;
            if constexpr (RESID) {
                const cplx<float> yy = ld_c1(y, off);
                res = {__fadd_rn(yy.re, -res.re), __fadd_rn(yy.im, -res.im)};
            }
            if constexpr (SPLIT) {
                res6[i] = res;
                __stcs((odd ? ro : out) + hbase + (6 * chi + i) * n, make_float2(res.re, res.im));
            } else {
                __stcs(out + off, make_float2(res.re, res.im));
            }
        }
        if constexpr (SPLIT) {
            if (!odd) {
                cplx<float> t[6];
                site_mat_r1(Cinv, site, chi, res6, t);
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    __stcs(te + hbase + (6 * chi + i) * n, make_float2(t[i].re, t[i].im));
            }
        }
    }
}

template <bool RESID, int N, int MINB = 6>
__global__ void __launch_bounds__(128, MINB) k_dslash_r1(const float2 *__restrict__ U, const float2 *__restrict__ C,
                                                       const float2 *__restrict__ in, float2 *__restrict__ out,
                                                       const float2 *__restrict__ y, KArgs32 a) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    int c[4], r;
    if (!visit_coords(a, item, a.V, false, c, r, 1)) return;
    dslash_r1_site<RESID, N>(U, C, in, out, y, a, c, r);
}

// the even-odd smoother's residual r = y - D x written as r_e, r_o and te = C_ee^-1 r_e
template <int N, int MINB = 6>
__global__ void __launch_bounds__(128, MINB) k_dslash_r1_split(const float2 *__restrict__ U, const float2 *__restrict__ C,
                                                             const float2 *__restrict__ Cinv,
                                                             const float2 *__restrict__ in,
                                                             const float2 *__restrict__ y, float2 *__restrict__ re,
                                                             float2 *__restrict__ ro, float2 *__restrict__ te,
                                                             KArgs32 a) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    int c[4], r;
    if (!visit_coords(a, item, a.V, false, c, r, 1)) return;
    dslash_r1_site<true, N, true>(U, C, in, re, y, a, c, r, ro, te, Cinv);
}

// ------------------------------------- fused batch of uneven problems
// One persistent launch applies D (or y - D x) to up to kMaxBatch problems of
// different lattice volumes and RHS counts: the problems' work blocks (128
// threads of one RHS each) are concatenated, and a grid of one occupancy wave
// walks them grid-stride, so small problems share the GPU instead of each
// paying a launch and a partial wave.  Per thread the arithmetic is that of
// k_dslash_r1 (bitwise equal to the single-problem stencil).
constexpr int kMaxBatch = 8;
struct BatchItem {
    const float2 *U, *C, *in;
    float2 *out;
    const float2 *y;  // nullptr: out = D in
    KArgs32 a;        // one RHS per thread (G = n), site tiles
    int first_block;  // first work block of this problem
};
struct BatchArgs {
    BatchItem it[kMaxBatch];
    int count;
    int total_blocks;
};

template <bool RESID>
__device__ __forceinline__ void batch_site(const BatchItem &w, const int c[4], int r) {
    switch (w.a.n) {
        case 2: dslash_r1_site<RESID, 2>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 4: dslash_r1_site<RESID, 4>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 6: dslash_r1_site<RESID, 6>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 8: dslash_r1_site<RESID, 8>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 12: dslash_r1_site<RESID, 12>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 16: dslash_r1_site<RESID, 16>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 24: dslash_r1_site<RESID, 24>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 32: dslash_r1_site<RESID, 32>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 48: dslash_r1_site<RESID, 48>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        case 64: dslash_r1_site<RESID, 64>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
        default: dslash_r1_site<RESID, 0>(w.U, w.C, w.in, w.out, w.y, w.a, c, r); break;
    }
}

__global__ void __launch_bounds__(128, 6) k_dslash_batch(const __grid_constant__ BatchArgs b) {
    for (int blk = blockIdx.x; blk < b.total_blocks; blk += gridDim.x) {
        int p = 0;
        while (p + 1 < b.count && blk >= b.it[p + 1].first_block) ++p;
        const BatchItem &w = b.it[p];
        const int item = (blk - w.first_block) * blockDim.x + threadIdx.x;
        int c[4], r;
        if (!visit_coords(w.a, item, w.a.V, false, c, r, 1)) continue;
        if (w.y) batch_site<true>(w, c, r);
        else batch_site<false>(w, c, r);
    }
}

// geometry of the paired stencil with tiles of the largest powers of two up to
// pref[mu] that divide L[mu] (pref[0] may be L[0]: whole x rows)
static KArgs32 x2_args(const mrhs_lattice &lat, int n, const int pref[4]) {
    KArgs32 a{};
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = lat.g.L[mu];
    a.V = (int)lat.g.V;
    a.n = n;
    a.G = n / 2;
    a.stride[0] = 1;
    a.stride[1] = a.L[0];
    a.stride[2] = a.L[0] * a.L[1];
    a.stride[3] = a.L[0] * a.L[1] * a.L[2];
    a.tb = lat.g.tb;
    a.tsites = 1;
    for (int mu = 0; mu < 4; ++mu) {
        int t = pref[mu];
        while (t > 1 && a.L[mu] % t) t /= 2;
        a.T[mu] = t;
        a.tsites *= t;
    }
    for (int mu = 0; mu < 3; ++mu) a.NT[mu] = a.L[mu] / a.T[mu];
    a.mode = 0;
    a.RX = a.L[0];
    a.GS = a.G;
    return a;
}

// the traversal variants beyond the tiles: x-regions (nr regions, nr dividing
// L[0]; `xstep` 2 for the even-odd kernels, whose regions hold whole x pairs)
// and RHS slabs (ns slabs of G / ns pairs).  `base` is taken by value: it may
// be an element of `v`, which the push_back below can reallocate.
static void add_order_variants(std::vector<KArgs32> &v, const KArgs32 base, int xstep) {
    for (int nr : {1, 2, 3}) {
        if (base.L[0] % (nr * xstep)) continue;
        KArgs32 a = base;
        a.mode = 1;
        a.RX = a.L[0] / nr;
        a.tsites = (a.RX / xstep) * a.L[1] * a.L[2] * a.L[3];
        v.push_back(a);
    }
    for (int ns : {2, 3}) {
        if (base.G % ns) continue;
        KArgs32 a = base;
        a.mode = 2;
        a.GS = a.G / ns;
        v.push_back(a);
    }
}

static bool launch_dslash_x2(const mrhs_lattice &lat, const void *in, void *out, const void *y, int n,
                             cudaStream_t s) {
    if (n % 2 || lat.g.V * 12LL * n >= (1LL << 31) || lat.g.V * (int64_t)(n / 2) >= (1LL << 31)) return false;
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!al(in) || !al(out) || (y && !al(y))) return false;
    // tile extents: the largest powers of two up to the preferred extents that
    // divide L; with fewer than 16 RHS a warp spans several sites, which must
    // then be consecutive in x for coalesced loads: whole x rows.  Variant 0 is
    // 1 x 4 x 8 x 8 (measured best at 24^3 x 64, 48 RHS); the autotuner also
    // tries the others per (lattice, n).
    const int X = n < 16 ? lat.g.L[0] : 1;
    const int prefs[][4] = {{X, 4, 8, 8}, {X, 4, 4, 8}, {X, 2, 8, 8}, {X, 8, 8, 8}, {X, 4, 8, 4}};
    std::vector<KArgs32> args;
    for (const auto &pref : prefs) {
        const KArgs32 a = x2_args(lat, n, pref);
        bool dup = false;
        for (const KArgs32 &b : args) dup = dup || (b.T[0] == a.T[0] && b.T[1] == a.T[1] && b.T[2] == a.T[2] && b.T[3] == a.T[3]);
        if (!dup) args.push_back(a);
    }
    add_order_variants(args, args[0], 1);
    // one-RHS-per-thread variants (compiled RHS counts only) on the first two tile
    // shapes, placed first: measured 1-4 % faster than the paired kernel on GB300
    // (24^4 and 24^3 x 64, 16 to 64 RHS), so the first of them is the default
    const bool r1 = n == 16 || n == 24 || n == 32 || n == 48 || n == 64;
    int nr1 = 0;
    if (r1) {
        std::vector<KArgs32> one;
        for (int i = 0; i < 2 && i < (int)args.size(); ++i) {
            KArgs32 b = args[(size_t)i];
            b.G = n;
            b.GS = n;
            one.push_back(b);
        }
        {
            // the first tile shape built for 8 CTAs per SM (64 registers, a few bytes of spills),
            // placed first: measured on GB300 (24^3 x 64, 48 RHS) 3.6 % faster than 6 CTAs per SM
            KArgs32 b = one[0];
            b.occ8 = 1;
            one.insert(one.begin(), b);
        }
        nr1 = (int)one.size();
        args.insert(args.begin(), one.begin(), one.end());
    }
    const int64_t items = (int64_t)args[nr1].V * args[nr1].G;
    const int threads = 128;
    const unsigned blocks = (unsigned)((items + threads - 1) / threads);
    const unsigned blocks_r1 = (unsigned)(((int64_t)args[0].V * n + threads - 1) / threads);
    const int nx2 = nr1;  // variants below nr1 are one RHS per thread
    const float2 *yy = static_cast<const float2 *>(y);
    const float2 *ii = static_cast<const float2 *>(in);
    float2 *oo = static_cast<float2 *>(out);
    // 16, 24, 32, 48, 64 RHS: compile-time RHS count and site-major links / clover;
    // fewer: a warp spans several sites, whose link-major loads coalesce
    auto launch = [&](int v) {
        const KArgs32 &a = args[(size_t)v];
        const bool one = v < nx2;
        auto go = [&](auto resid, auto nc, auto aos) {
            constexpr bool R = decltype(resid)::value;
            constexpr int NC = decltype(nc)::value;
            constexpr bool AO = decltype(aos)::value;
            const float2 *U = AO ? lat.U32a.as<float2>() : lat.U32.as<float2>();
            const float2 *C = AO ? lat.C32a.as<float2>() : lat.C32.as<float2>();
            if constexpr (NC > 0 && AO) {
                if (one) {
                    if (a.occ8) k_dslash_r1<R, NC, 8><<<blocks_r1, threads, 0, s>>>(U, C, ii, oo, yy, a);
                    else k_dslash_r1<R, NC><<<blocks_r1, threads, 0, s>>>(U, C, ii, oo, yy, a);
                    return;
                }
            }
            k_dslash_x2<R, NC, AO><<<blocks, threads, 0, s>>>(U, C, ii, oo, yy, a);
        };
        auto pick = [&](auto resid) {
            using T = std::true_type;
            using F = std::false_type;
            switch (n) {
                case 16: go(resid, std::integral_constant<int, 16>{}, T{}); break;
                case 24: go(resid, std::integral_constant<int, 24>{}, T{}); break;
                case 32: go(resid, std::integral_constant<int, 32>{}, T{}); break;
                case 48: go(resid, std::integral_constant<int, 48>{}, T{}); break;
                case 64: go(resid, std::integral_constant<int, 64>{}, T{}); break;
                default: go(resid, std::integral_constant<int, 0>{}, F{}); break;
            }
        };
        if (y) pick(std::true_type{});
        else pick(std::false_type{});
        MRHS_CUDA(cudaGetLastError());
    };
    // y == out (an in-place residual) would not survive repeated launches: no tuning then
    const int v = y == out ? 0 : tune_pick(y ? "k_dslash_x2_resid" : "k_dslash_x2", lat.g.L, n, (int)args.size(),
                                           launch, s);
    MRHS_TIMED("k_dslash_x2", s);
    launch(v);
    MRHS_LAUNCHED("k_dslash_x2");
    return true;
}

void dslash_batch(const BatchItemHost *items, int count, cudaStream_t s) {
    if (count < 1 || count > kMaxBatch) fail(MRHS_ERR_INVALID, "batch holds 1..8 problems");
    BatchArgs b{};
    b.count = count;
    int blocks = 0, dev = -1;
    for (int i = 0; i < count; ++i) {
        const BatchItemHost &h = items[i];
        const mrhs_lattice *lat = h.lat;
        if (!lat || !lat->has_clover) fail(MRHS_ERR_INVALID, "every batch item needs a lattice with its clover term");
        if (dev >= 0 && lat->device != dev) fail(MRHS_ERR_INVALID, "batch items must share one device");
        dev = lat->device;
        if (h.n < 1 || h.n > 256) fail(MRHS_ERR_INVALID, "batch item nrhs must be in 1..256");
        if (!h.in || !h.out || h.in == h.out) fail(MRHS_ERR_INVALID, "batch item needs distinct non-null in and out");
        if (lat->g.V * 12LL * h.n >= (1LL << 31) || lat->g.V * (int64_t)h.n >= (1LL << 31))
            fail(MRHS_ERR_INVALID, "batch item too large for 32-bit indexing");
        static const int pref[4] = {1, 4, 8, 8};
        KArgs32 a = x2_args(*lat, h.n, pref);
        a.G = h.n;
        a.GS = h.n;
        BatchItem &w = b.it[i];
        w.U = lat->U32a.as<float2>();
        w.C = lat->C32a.as<float2>();
        w.in = static_cast<const float2 *>(h.in);
        w.out = static_cast<float2 *>(h.out);
        w.y = static_cast<const float2 *>(h.y);
        w.a = a;
        w.first_block = blocks;
        blocks += (int)ceil_div((int64_t)lat->g.V * h.n, 128);
    }
    b.total_blocks = blocks;
    int per_sm = 0;
    MRHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash_batch, 128, 0));
    int devc = 0;
    MRHS_CUDA(cudaGetDevice(&devc));
    const int grid = std::max(1, std::min(blocks, std::max(1, per_sm) * sm_count(devc)));
    MRHS_TIMED("k_dslash_batch", s);
    k_dslash_batch<<<grid, 128, 0, s>>>(b);
    MRHS_CUDA(cudaGetLastError());
    MRHS_LAUNCHED("k_dslash_batch");
}

// ------------------------------------------------ even-odd (M_eooe) kernels
// Half-lattice fields [V/2][12][n] hold the sites of one parity
// ((x + y + z + t) mod 2) in increasing lexicographic order: with an even x
// extent, site s sits at index s / 2.  The hopping term only connects sites
// of opposite parity (H_eo, H_oe: the paper's M_eooe, Sec. 4), so every
// neighbour of an output site is read from the other parity's half field at
// index neighbour / 2.  One thread per (output site, RHS pair), FFMA2 as in
// k_dslash_x2; modes:
//   EO_HOP      out = H in
//   EO_CINV_HOP out = C^-1 H in                 (C = clover + mass of the output site)
//   EO_SCHUR    out = C self - 1/4 H in         (self: the output parity's own field)
//   EO_AXPY_HOP      out = self + 1/2 H in
//   EO_CINV_AXPY_HOP out = C^-1 (self + 1/2 H in)
// so that D_hat = C_oo - 1/4 H_oe C_ee^-1 H_eo is EO_CINV_HOP onto the even
// sites followed by EO_SCHUR onto the odd ones, and the even-odd solution of
// D x = b takes b_hat = b_o + 1/2 H_oe C_ee^-1 b_e (EO_AXPY_HOP onto the odd
// sites) and x_e = C_ee^-1 (b_e + 1/2 H_eo x_o) (EO_CINV_AXPY_HOP).
//   EO_CINV_AXPY_HOP_MERGE: the even-odd smoother's last step in one pass,
//        z_e += C^-1 (self + 1/2 H in) at the output sites and z_o += in at
//        their x-pair partners, with z the full-lattice field `out`
enum { EO_HOP = 0, EO_CINV_HOP = 1, EO_SCHUR = 2, EO_AXPY_HOP = 3, EO_CINV_AXPY_HOP = 4, EO_CINV_AXPY_HOP_MERGE = 5 };

struct KArgsEO {
    KArgs32 k;   // full-lattice geometry (k.V is the full volume), n, RHS pairs
    int parity;  // parity of the output sites
    int V2;      // V / 2
    int ts;      // host side: > 0 selects the half-line ring kernel with ts time slices per CTA
};

template <int MODE, int N, bool AOS>
__global__ void __launch_bounds__(128, 3) k_eo_x2(const float2 *__restrict__ U, const float2 *__restrict__ M,
                                                   const float2 *__restrict__ in, const float2 *__restrict__ self,
                                                   float2 *__restrict__ out, KArgsEO e) {
    const KArgs32 &a = e.k;
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    // visit order over x pairs (one output site per pair) as the full stencil's
    // orders; x = 2k or 2k + 1 is the member of the pair with the output parity
    int c[4], r0;
    if (!visit_coords(a, item, e.V2, true, c, r0)) return;
    c[0] *= 2;
    if (((c[0] + c[1] + c[2] + c[3]) & 1) != e.parity) ++c[0];
    const int site = c[0] + a.L[0] * (c[1] + a.L[1] * (c[2] + a.L[2] * c[3]));
    const int cb = site >> 1;
    P2 acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int L = a.L[mu], st = a.stride[mu];
        const bool wrapF = (c[mu] == L - 1), wrapB = (c[mu] == 0);
        const int sf = wrapF ? site - st * (L - 1) : site + st;
        const int sb = wrapB ? site + st * (L - 1) : site - st;
        const bool flipF = mu == 3 && wrapF && a.tb < 0;
        const bool flipB = mu == 3 && wrapB && a.tb < 0;
        // neighbours live in the other parity's half field, at index site / 2
        if (mu == 0) {
            hop_x2<0, true, N, AOS>(acc, U, in, a, sf >> 1, site, flipF, r0);
            hop_x2<0, false, N, AOS>(acc, U, in, a, sb >> 1, sb, flipB, r0);
        } else if (mu == 1) {
            hop_x2<1, true, N, AOS>(acc, U, in, a, sf >> 1, site, flipF, r0);
            hop_x2<1, false, N, AOS>(acc, U, in, a, sb >> 1, sb, flipB, r0);
        } else if (mu == 2) {
            hop_x2<2, true, N, AOS>(acc, U, in, a, sf >> 1, site, flipF, r0);
            hop_x2<2, false, N, AOS>(acc, U, in, a, sb >> 1, sb, flipB, r0);
        } else {
            hop_x2<3, true, N, AOS>(acc, U, in, a, sf >> 1, site, flipF, r0);
            hop_x2<3, false, N, AOS>(acc, U, in, a, sb >> 1, sb, flipB, r0);
        }
    }
    const int n = rhs_count<N>(a);
    const int64_t base = (int64_t)cb * 12 * n + r0;
    if constexpr (MODE == EO_HOP) {
#pragma unroll
        for (int i = 0; i < 12; ++i) st_p2(out, base + i * n, acc[i]);
    } else if constexpr (MODE == EO_AXPY_HOP || MODE == EO_CINV_AXPY_HOP || MODE == EO_CINV_AXPY_HOP_MERGE) {
        const float2 half = make_float2(0.5f, 0.5f);
        const int64_t zbase = (int64_t)site * 12 * n + r0;  // MERGE: z at the output site
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
            P2 v[6], o[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const P2 y = ld_p2(self, base + (6 * chi + i) * n);
                const P2 ai = acc[6 * chi + i];
                v[i] = {__ffma2_rn(half, ai.re, y.re), __ffma2_rn(half, ai.im, y.im)};
            }
            if constexpr (MODE != EO_AXPY_HOP) site_mat_x2<AOS>(M, a.V, site, chi, v, o);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if constexpr (MODE == EO_CINV_AXPY_HOP_MERGE)
                    st_p2(out, zbase + (6 * chi + i) * n, p2add(ld_p2(out, zbase + (6 * chi + i) * n), o[i]));
                else
                    st_p2(out, base + (6 * chi + i) * n, MODE == EO_CINV_AXPY_HOP ? o[i] : v[i]);
            }
        }
        if constexpr (MODE == EO_CINV_AXPY_HOP_MERGE) {
            // the x-pair partner (the other parity, same half-field index): z_o += in
            const int64_t pbase = (int64_t)(site ^ 1) * 12 * n + r0;
#pragma unroll
            for (int i = 0; i < 12; ++i) st_p2(out, pbase + i * n, p2add(ld_p2(out, pbase + i * n), ld_p2(in, base + i * n)));
        }
    } else {
        const float2 quarter = make_float2(-0.25f, -0.25f);
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
            P2 v[6], o[6];
#pragma unroll
            for (int i = 0; i < 6; ++i)
                v[i] = MODE == EO_CINV_HOP ? acc[6 * chi + i] : ld_p2(self, base + (6 * chi + i) * n);
            site_mat_x2<AOS>(M, a.V, site, chi, v, o);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                P2 res = o[i];
                if constexpr (MODE == EO_SCHUR) {
                    const P2 ai = acc[6 * chi + i];
                    res = {__ffma2_rn(quarter, ai.re, o[i].re), __ffma2_rn(quarter, ai.im, o[i].im)};
                }
                st_p2(out, base + (6 * chi + i) * n, res);
            }
        }
    }
}

// k_eo_x2 with one RHS per thread (scalar FMA in the paired code's order: bitwise equal results).
// eo_r1_finish: the mode's epilogue at the output site (site, half-field index cb) for RHS r,
// shared with the ring kernel below.
template <int MODE, int N>
__device__ __forceinline__ void eo_r1_finish(const cplx<float> (&acc)[12], const float2 *__restrict__ M,
                                             const float2 *__restrict__ in, const float2 *__restrict__ self,
                                             float2 *__restrict__ out, int site, int cb, int r) {
    const int64_t base = (int64_t)cb * 12 * N + r;
    auto st1 = [&](int i, cplx<float> v) { __stcs(out + base + i * N, make_float2(v.re, v.im)); };
    if constexpr (MODE == EO_HOP) {
#pragma unroll
        for (int i = 0; i < 12; ++i) st1(i, acc[i]);
    } else if constexpr (MODE == EO_AXPY_HOP || MODE == EO_CINV_AXPY_HOP || MODE == EO_CINV_AXPY_HOP_MERGE) {
        const int64_t zbase = (int64_t)site * 12 * N + r;  // MERGE: z at the output site
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
            cplx<float> v[6], o[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const cplx<float> yv = ld_c1(self, base + (6 * chi + i) * N);
                const cplx<float> ai = acc[6 * chi + i];
                v[i] = {__fmaf_rn(0.5f, ai.re, yv.re), __fmaf_rn(0.5f, ai.im, yv.im)};
            }
            if constexpr (MODE != EO_AXPY_HOP) site_mat_r1(M, site, chi, v, o);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if constexpr (MODE == EO_CINV_AXPY_HOP_MERGE) {
                    const int64_t zi = zbase + (6 * chi + i) * N;
                    const float2 zv = out[zi];
                    out[zi] = make_float2(__fadd_rn(zv.x, o[i].re), __fadd_rn(zv.y, o[i].im));
                } else {
                    st1(6 * chi + i, MODE == EO_CINV_AXPY_HOP ? o[i] : v[i]);
                }
            }
        }
        if constexpr (MODE == EO_CINV_AXPY_HOP_MERGE) {
            // the x-pair partner (the other parity, same half-field index): z_o += in
            const int64_t pbase = (int64_t)(site ^ 1) * 12 * N + r;
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const float2 zv = out[pbase + i * N], d = __ldg(in + base + i * N);
                out[pbase + i * N] = make_float2(__fadd_rn(zv.x, d.x), __fadd_rn(zv.y, d.y));
            }
        }
    } else {
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
            cplx<float> v[6], o[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = MODE == EO_CINV_HOP ? acc[6 * chi + i] : ld_c1(self, base + (6 * chi + i) * N);
            site_mat_r1(M, site, chi, v, o);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                cplx<float> res = o[i];
                if constexpr (MODE == EO_SCHUR) {
                    const cplx<float> ai = acc[6 * chi + i];
                    res = {__fmaf_rn(-0.25f, ai.re, o[i].re), __fmaf_rn(-0.25f, ai.im, o[i].im)};
                }
                st1(6 * chi + i, res);
            }
        }
    }
}

// the hops of direction mu at output site `site` (coordinates c) from the other
// parity's half field in global memory
template <int MU, int N>
__device__ __forceinline__ void eo_r1_hops_global(cplx<float> (&acc)[12], const float2 *__restrict__ U,
                                                  const float2 *__restrict__ in, const KArgs32 &a, int site,
                                                  const int c[4], int r) {
    const int L = a.L[MU], st = a.stride[MU];
    const bool wrapF = (c[MU] == L - 1), wrapB = (c[MU] == 0);
    const int sf = wrapF ? site - st * (L - 1) : site + st;
    const int sb = wrapB ? site + st * (L - 1) : site - st;
    const bool flipF = MU == 3 && wrapF && a.tb < 0;
    const bool flipB = MU == 3 && wrapB && a.tb < 0;
    // neighbours live in the other parity's half field, at index site / 2
    hop_r1<MU, true, N>(acc, U, in, sf >> 1, site, flipF, r);
    hop_r1<MU, false, N>(acc, U, in, sb >> 1, sb, flipB, r);
}

template <int MODE, int N>
__device__ __forceinline__ void eo_r1_site(const float2 *__restrict__ U, const float2 *__restrict__ M,
                                           const float2 *__restrict__ in, const float2 *__restrict__ self,
                                           float2 *__restrict__ out, const KArgs32 &a, const int c[4], int r) {
    const int site = c[0] + a.L[0] * (c[1] + a.L[1] * (c[2] + a.L[2] * c[3]));
    cplx<float> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
    eo_r1_hops_global<0, N>(acc, U, in, a, site, c, r);
    eo_r1_hops_global<1, N>(acc, U, in, a, site, c, r);
    eo_r1_hops_global<2, N>(acc, U, in, a, site, c, r);
    eo_r1_hops_global<3, N>(acc, U, in, a, site, c, r);
    eo_r1_finish<MODE, N>(acc, M, in, self, out, site, site >> 1, r);
}

template <int MODE, int N, int MINB = 6>
__global__ void __launch_bounds__(128, MINB) k_eo_r1(const float2 *__restrict__ U, const float2 *__restrict__ M,
                                                   const float2 *__restrict__ in, const float2 *__restrict__ self,
                                                   float2 *__restrict__ out, KArgsEO e) {
    const KArgs32 &a = e.k;
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    int c[4], r;
    if (!visit_coords(a, item, e.V2, true, c, r, 1)) return;
    c[0] *= 2;
    if (((c[0] + c[1] + c[2] + c[3]) & 1) != e.parity) ++c[0];
    eo_r1_site<MODE, N>(U, M, in, self, out, a, c, r);
}

// ----------------------------------- even-odd hop with a ring of half lines
// One CTA per (y, z) column and segment of `ts` time slices.  The other
// parity's half line at (y, z, t) -- Lx / 2 sites x 12 x N, contiguous in the
// half field -- is bulk-copied into a ring of RING_SLOTS shared-memory slots,
// one copy per site, by a producer warp; the compute threads (one per output
// site of the line and RHS) read the x neighbours (same half line) and the t
// neighbours (the lines of t - 1 and t + 1) from the ring and only the y and
// z neighbours from global memory.  Each half line crosses L2 -> SM once per
// column instead of once per consumer, and the staged half of the neighbour
// reads no longer waits on L2.  Line j of the segment is t = t0 - 1 + j; step
// i computes t0 + i from lines i, i + 1, i + 2 while line i + 3 lands; a
// compute warp releases line i's slot (empty barrier) after step i and the
// producer then copies line i + 4 into it.  Every hop is the one-RHS hop of
// k_eo_r1 in the same order, so outputs are bitwise those of k_eo_r1.
// Every wait is bounded: a compute warp whose wait gives up (or that finds the
// abort flag set) computes from global memory from then on (the same values),
// and the producer stops copying and waits, bounded, for the copies it issued.
constexpr int RING_SLOTS = 4;
constexpr int RING_MAX_COMPUTE = 576;  // compute threads per CTA (Lx / 2 x N)

mrhs_status api_record(mrhs_status code, const std::string &msg);

// eager ring launches whose compute warps are to give up their first wait at once (test hook)
std::atomic<int> g_expire_ring{0};

static uint32_t ring_first_wait_limit(cudaStream_t s) {
    if (g_expire_ring.load() <= 0) return tc::SPIN_LIMIT;
    // a launch recorded into a graph would keep the expired limit for every replay: only eager launches
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MRHS_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return tc::SPIN_LIMIT;
    int left = g_expire_ring.load();
    while (left > 0 && !g_expire_ring.compare_exchange_weak(left, left - 1)) {
    }
    return left > 0 ? 0u : tc::SPIN_LIMIT;
}

struct RingArgs {
    int H;                 // sites per half line (L[0] / 2)
    int ts;                // time slices per CTA
    uint32_t first_limit;  // try_wait rounds of a compute warp's first wait (SPIN_LIMIT; 0 expires it)
};

__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int MODE, int N>
__global__ void __launch_bounds__(RING_MAX_COMPUTE + 32, 1)
    k_eo_ring(const float2 *__restrict__ U, const float2 *__restrict__ M, const float2 *__restrict__ in,
              const float2 *__restrict__ self, float2 *__restrict__ out, KArgsEO e, RingArgs g) {
    extern __shared__ __align__(16) float2 ring_raw[];
    __shared__ __align__(8) uint64_t bars[2 * RING_SLOTS];
    // [RING_SLOTS][H][12][N], 16-byte aligned for the bulk copies
    float2 *const ring = ring_raw + ((16u - (tc::smem_u32(ring_raw) & 15u)) & 15u) / 8u;
    __shared__ int abort_sh;
    const KArgs32 &a = e.k;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = g.H, NCT = H * N, ncw = NCT / 32;
    int u = blockIdx.x;
    const int y = u % a.L[1];
    u /= a.L[1];
    const int z = u % a.L[2];
    const int t0 = (u / a.L[2]) * g.ts;
    const int nlines = g.ts + 2;
    const int slot_elems = H * 12 * N;
    const uint32_t site_bytes = 12u * N * 8u, slot_bytes = (uint32_t)H * site_bytes;
    const uint32_t full0 = tc::smem_u32(&bars[0]), empty0 = tc::smem_u32(&bars[RING_SLOTS]);
    if (tid == 0) {
        for (int s = 0; s < RING_SLOTS; ++s) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, ncw);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // first half-field index of the half line of line j (t periodic)
    auto line_base = [&](int j) -> int64_t {
        int t = t0 - 1 + j;
        t = t < 0 ? t + a.L[3] : (t >= a.L[3] ? t - a.L[3] : t);
        return (int64_t)(y + a.L[1] * (z + a.L[2] * t)) * H;
    };
    if (warp == ncw) {
        // producer: lane 0 copies line j into slot j % RING_SLOTS once the compute
        // warps have released line j - RING_SLOTS
        if (lane != 0) return;
        const uint32_t ring0 = tc::smem_u32(ring);
        int issued = 0;
        for (int j = 0; j < nlines; ++j) {
            const int s = j % RING_SLOTS;
            if (j >= RING_SLOTS) {
                if (!tc::mbar_wait(empty0 + 8 * s, ((j / RING_SLOTS) - 1) & 1)) {
                    abort_sh = 1;
                    break;
                }
                if (*(volatile int *)&abort_sh) break;
                tc::fence_async_smem();
            }
            tc::mbar_expect_tx(full0 + 8 * s, slot_bytes);
            const float2 *src = in + line_base(j) * 12 * N;
            for (int q = 0; q < H; ++q)
                tc::bulk_g2s(ring0 + s * slot_bytes + q * site_bytes, src + (int64_t)q * 12 * N, site_bytes,
                             full0 + 8 * s);
            issued = j + 1;
        }
        // the last copies issued into each slot land before the CTA exits
        for (int s = 0; s < RING_SLOTS && s < issued; ++s) {
            const int jl = s + ((issued - 1 - s) / RING_SLOTS) * RING_SLOTS;
            tc::mbar_wait(full0 + 8 * s, (jl / RING_SLOTS) & 1);
        }
        return;
    }
    const int k = tid / N, r = tid - k * N;
    bool fb = false;  // this warp computes from global memory (a wait gave up)
    int waited = 0;   // lines this warp has waited for
    for (int i = 0; i < g.ts; ++i) {
        const int t = t0 + i;
        for (; waited <= i + 2; ++waited) {
            if (fb) continue;
            const uint32_t bar = full0 + 8 * (waited % RING_SLOTS), par = (waited / RING_SLOTS) & 1;
            const uint32_t lim = waited == 0 ? g.first_limit : tc::SPIN_LIMIT;
            bool ok = false;
            for (uint32_t it = 0; it < lim; ++it) {
                if (tc::mbar_try_wait(bar, par)) {
                    ok = true;
                    break;
                }
                if (*(volatile int *)&abort_sh) break;
            }
            if (!__all_sync(0xffffffffu, ok)) {
                fb = true;
                if (lane == 0) *(volatile int *)&abort_sh = 1;
            }
        }
        const int off = (e.parity ^ (y + z + t)) & 1;
        const int x = 2 * k + off;
        const int c[4] = {x, y, z, t};
        if (fb) {
            eo_r1_site<MODE, N>(U, M, in, self, out, a, c, r);
        } else {
            const int site = x + a.L[0] * (y + a.L[1] * (z + a.L[2] * t));
            const float2 *lm = ring + ((i + 0) % RING_SLOTS) * slot_elems;  // t - 1
            const float2 *l0 = ring + ((i + 1) % RING_SLOTS) * slot_elems;  // t
            const float2 *lp = ring + ((i + 2) % RING_SLOTS) * slot_elems;  // t + 1
            cplx<float> acc[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) acc[q] = {0.f, 0.f};
            {
                // x: the neighbours x +- 1 are entries (x +- 1) / 2 of the current half line
                const int L = a.L[0];
                const int xf = x == L - 1 ? 0 : x + 1, xb = x == 0 ? L - 1 : x - 1;
                const int sb = x == 0 ? site + (L - 1) : site - 1;
                hop_r1_at<0, true, true>(acc, U, l0 + (xf >> 1) * 12 * N + r, N, site, false);
                hop_r1_at<0, false, true>(acc, U, l0 + (xb >> 1) * 12 * N + r, N, sb, false);
            }
            eo_r1_hops_global<1, N>(acc, U, in, a, site, c, r);
            eo_r1_hops_global<2, N>(acc, U, in, a, site, c, r);
            {
                // t: entry x / 2 = k of the half lines of t + 1 and t - 1
                const int L = a.L[3], st = a.stride[3];
                const bool wrapF = t == L - 1, wrapB = t == 0;
                const int sb = wrapB ? site + st * (L - 1) : site - st;
                hop_r1_at<3, true, true>(acc, U, lp + k * 12 * N + r, N, site, wrapF && a.tb < 0);
                hop_r1_at<3, false, true>(acc, U, lm + k * 12 * N + r, N, sb, wrapB && a.tb < 0);
            }
            eo_r1_finish<MODE, N>(acc, M, in, self, out, site, site >> 1, r);
        }
        // line i is no longer read by this warp
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(empty0 + 8 * (i % RING_SLOTS));
    }
}

static KArgsEO eo_args(const mrhs_lattice &lat, int n, int parity, const int pref[4] = nullptr) {
    KArgsEO e{};
    KArgs32 &a = e.k;
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = lat.g.L[mu];
    a.V = (int)lat.g.V;
    a.n = n;
    a.G = n / 2;
    a.stride[0] = 1;
    a.stride[1] = a.L[0];
    a.stride[2] = a.L[0] * a.L[1];
    a.stride[3] = a.L[0] * a.L[1] * a.L[2];
    a.tb = lat.g.tb;
    // tiles: one x pair times the largest powers of two up to 4 x 8 x 8 (or `pref`)
    // that divide L (tsites counts output sites: one per x pair)
    static const int pref0[4] = {2, 4, 8, 8};
    if (!pref) pref = pref0;
    a.T[0] = 2;
    a.tsites = 1;
    for (int mu = 1; mu < 4; ++mu) {
        int t = pref[mu];
        while (t > 1 && a.L[mu] % t) t /= 2;
        a.T[mu] = t;
        a.tsites *= t;
    }
    for (int mu = 0; mu < 3; ++mu) a.NT[mu] = a.L[mu] / a.T[mu];
    a.NT[0] = a.L[0] / 2;
    a.mode = 0;
    a.RX = a.L[0];
    a.GS = a.G;
    e.parity = parity;
    e.V2 = a.V / 2;
    return e;
}

static void check_eo(const mrhs_lattice &lat, int n) {
    for (int mu = 0; mu < 4; ++mu)
        if (lat.g.L[mu] % 2) fail(MRHS_ERR_INVALID, "even-odd decomposition needs even lattice extents");
    if (n < 2 || n % 2) fail(MRHS_ERR_INVALID, "even-odd operators take an even RHS count");
    if (lat.g.V * 6LL * n >= (1LL << 31)) fail(MRHS_ERR_INVALID, "half-lattice field too large for 32-bit indexing");
}

enum { EO_NOMAT = 0, EO_MAT_C = 1, EO_MAT_CINV = 2 };

// dynamic shared memory of the ring kernel: RING_SLOTS half lines of H sites (+ 16 B of alignment slack)
static size_t ring_smem_bytes(int H, int n) { return (size_t)RING_SLOTS * H * 12 * n * 8 + 16; }

static size_t ring_smem_limit() {
    static int cached[64] = {};
    int dev = 0, v = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && cached[dev] > 0) return (size_t)cached[dev];
    MRHS_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (dev >= 0 && dev < 64) cached[dev] = v;
    return (size_t)v;
}

// raise the dynamic shared-memory limit of k_eo_ring<MD, NC> once per device and size
template <int MD, int NC, typename K> static void ring_set_smem(K kernel, size_t bytes) {
    static size_t done[64] = {};
    int dev = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev] >= bytes) return;
    MRHS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (dev >= 0 && dev < 64) done[dev] = bytes;
}

// tune_scratch (EO_CINV_AXPY_HOP_MERGE only): a half field the tuner may write; the merge
// accumulates into z, so it takes the variant tuned for EO_CINV_AXPY_HOP, timed into the scratch
template <int MODE>
static void launch_eo(const mrhs_lattice &lat, int mat, const float2 *in, const float2 *self, float2 *out, int n,
                      int parity, cudaStream_t s, float2 *tune_scratch = nullptr) {
    // tile variants for the autotuner (variant 0: one x pair x 4 x 8 x 8)
    const int prefs[][4] = {{2, 4, 8, 8}, {2, 4, 4, 8}, {2, 2, 8, 8}, {2, 8, 8, 8}, {2, 4, 8, 4}};
    std::vector<KArgsEO> args;
    for (const auto &pref : prefs) {
        const KArgsEO e = eo_args(lat, n, parity, pref);
        bool dup = false;
        for (const KArgsEO &b : args) dup = dup || (b.k.T[1] == e.k.T[1] && b.k.T[2] == e.k.T[2] && b.k.T[3] == e.k.T[3]);
        if (!dup) args.push_back(e);
    }
    {
        std::vector<KArgs32> orders;
        add_order_variants(orders, args[0].k, 2);
        for (const KArgs32 &k : orders) {
            KArgsEO e = args[0];
            e.k = k;
            args.push_back(e);
        }
    }
    // one-RHS-per-thread variants (compiled RHS counts) on the first two tile shapes,
    // placed first (measured 2-4 % faster than the paired kernel for D_hat on GB300)
    int nx2 = 0;
    if (n == 16 || n == 24 || n == 32 || n == 48 || n == 64) {
        std::vector<KArgsEO> one;
        for (int i = 0; i < 2 && i < (int)args.size(); ++i) {
            KArgsEO b = args[(size_t)i];
            b.k.G = n;
            b.k.GS = n;
            one.push_back(b);
        }
        {
            // the first tile shape built for 8 CTAs per SM (64 registers), placed first:
            // measured on GB300 (24^3 x 64, 48 RHS) 3.2 % faster for D_hat than 6 CTAs per SM
            KArgsEO b = one[0];
            b.k.occ8 = 1;
            one.insert(one.begin(), b);
        }
        nx2 = (int)one.size();
        args.insert(args.begin(), one.begin(), one.end());
    }
    const int64_t items = (int64_t)args[nx2].V2 * args[nx2].k.G;
    const unsigned blocks = (unsigned)((items + 127) / 128);
    const unsigned blocks_r1 = (unsigned)(((int64_t)args[0].V2 * n + 127) / 128);
    // half-line ring variants of the two Schur-operator launches (compiled RHS counts
    // below 64; Lx / 2 x n compute threads, whole warps, four slots of Lx / 2 x 12 x n
    // values in shared memory): one CTA per (y, z) column and segment of L[3] or
    // L[3] / 2 time slices.  Measured on GB300 (24^3 x 64, 48 RHS) 44 % slower for
    // D_hat than the default (18 resident warps per SM against 32); kept as autotuner
    // candidates for other shapes
    const int H = lat.g.L[0] / 2;
    const size_t ring_smem = ring_smem_bytes(H, n);
    constexpr bool RING_MODE = MODE == EO_CINV_HOP || MODE == EO_SCHUR;
    if (RING_MODE && nx2 > 0 && n != 64 && H <= 32 && H * n <= RING_MAX_COMPUTE && (H * n) % 32 == 0 && ring_smem <= ring_smem_limit() &&
        (reinterpret_cast<uintptr_t>(in) & 15u) == 0) {
        for (int seg : {1, 2}) {
            if (lat.g.L[3] % seg || lat.g.L[3] / seg < 2) continue;
            KArgsEO b = args[0];
            b.ts = lat.g.L[3] / seg;
            args.push_back(b);
        }
    }
    // as the full-lattice stencil: compile-time RHS count and site-major links /
    // site matrices for 16, 24, 32, 48, 64 RHS
    auto launch_m = [&](auto modec, int v, float2 *dst) {
        constexpr int MD = decltype(modec)::value;
        const KArgsEO &e = args[(size_t)v];
        const bool one = v < nx2;
        auto go = [&](auto nc, auto aos) {
            constexpr int NC = decltype(nc)::value;
            constexpr bool AO = decltype(aos)::value;
            const float2 *U = AO ? lat.U32a.as<float2>() : lat.U32.as<float2>();
            const float2 *M = mat == EO_MAT_C      ? (AO ? lat.C32a.as<float2>() : lat.C32.as<float2>())
                              : mat == EO_MAT_CINV ? (AO ? lat.Cinv32a.as<float2>() : lat.Cinv32.as<float2>())
                                                   : nullptr;
            if constexpr (NC > 0 && NC != 64 && AO && (MD == EO_CINV_HOP || MD == EO_SCHUR)) {
                if (e.ts > 0) {
                    const RingArgs g{H, e.ts, ring_first_wait_limit(s)};
                    const unsigned grid = (unsigned)(lat.g.L[1] * lat.g.L[2] * (lat.g.L[3] / e.ts));
                    ring_set_smem<MD, NC>(k_eo_ring<MD, NC>, ring_smem);
                    k_eo_ring<MD, NC><<<grid, H * NC + 32, ring_smem, s>>>(U, M, in, self, dst, e, g);
                    return;
                }
            }
            if constexpr (NC > 0 && AO) {
                if (one) {
                    if (e.k.occ8) k_eo_r1<MD, NC, 8><<<blocks_r1, 128, 0, s>>>(U, M, in, self, dst, e);
                    else k_eo_r1<MD, NC><<<blocks_r1, 128, 0, s>>>(U, M, in, self, dst, e);
                    return;
                }
            }
            k_eo_x2<MD, NC, AO><<<blocks, 128, 0, s>>>(U, M, in, self, dst, e);
        };
        switch (n) {
            case 16: go(std::integral_constant<int, 16>{}, std::true_type{}); break;
            case 24: go(std::integral_constant<int, 24>{}, std::true_type{}); break;
            case 32: go(std::integral_constant<int, 32>{}, std::true_type{}); break;
            case 48: go(std::integral_constant<int, 48>{}, std::true_type{}); break;
            case 64: go(std::integral_constant<int, 64>{}, std::true_type{}); break;
            default: go(std::integral_constant<int, 0>{}, std::false_type{}); break;
        }
        MRHS_CUDA(cudaGetLastError());
    };
    auto launch = [&](int v) { launch_m(std::integral_constant<int, MODE>{}, v, out); };
    static const char *names[] = {"k_eo_x2_hop", "k_eo_x2_cinv_hop", "k_eo_x2_schur", "k_eo_x2_axpy_hop",
                                  "k_eo_x2_cinv_axpy_hop"};
    int v = 0;
    if constexpr (MODE == EO_CINV_AXPY_HOP_MERGE) {
        auto tune_launch = [&](int vv) {
            launch_m(std::integral_constant<int, EO_CINV_AXPY_HOP>{}, vv, tune_scratch);
        };
        if (tune_scratch) v = tune_pick(names[EO_CINV_AXPY_HOP], lat.g.L, n, (int)args.size(), tune_launch, s);
    } else {
        // an output that aliases an input would not survive repeated launches: no tuning then
        const bool alias = out == in || (self && out == self);
        v = alias ? 0 : tune_pick(names[MODE], lat.g.L, n, (int)args.size(), launch, s);
    }
    MRHS_TIMED("k_eo_x2", s);
    launch(v);
    MRHS_LAUNCHED("k_eo_x2");
}

void hop_eo(const mrhs_lattice &lat, int out_parity, const void *in, void *out, int n, cudaStream_t s) {
    check_eo(lat, n);
    launch_eo<EO_HOP>(lat, EO_NOMAT, static_cast<const float2 *>(in), nullptr, static_cast<float2 *>(out), n,
                      out_parity, s);
}

void schur_apply(const mrhs_lattice &lat, const void *in_odd, void *out_odd, int n, void *tmp_even, cudaStream_t s) {
    check_eo(lat, n);
    if (!lat.has_clover) fail(MRHS_ERR_INVALID, "clover term not built");
    if (lat.cinv_singular) fail(MRHS_ERR_INVALID, "a block of the clover term is singular: no even-odd inverse");
    float2 *t_e = static_cast<float2 *>(tmp_even);
    // t_e = C_ee^-1 H_eo psi_o, then out_o = C_oo psi_o - 1/4 H_oe t_e
    launch_eo<EO_CINV_HOP>(lat, EO_MAT_CINV, static_cast<const float2 *>(in_odd), nullptr, t_e, n, 0, s);
    launch_eo<EO_SCHUR>(lat, EO_MAT_C, t_e, static_cast<const float2 *>(in_odd),
                        static_cast<float2 *>(out_odd), n, 1, s);
}

// the even and the odd site of the pair (2 cb, 2 cb + 1)
__device__ __forceinline__ void eo_pair_sites(const KArgs32 &a, int cb, int &even, int &odd) {
    int q = 2 * cb;
    const int x = q % a.L[0];
    q /= a.L[0];
    const int y = q % a.L[1];
    q /= a.L[1];
    const int z = q % a.L[2];
    const int t = q / a.L[2];
    const bool first_even = ((x + y + z + t) & 1) == 0;
    even = first_even ? 2 * cb : 2 * cb + 1;
    odd = first_even ? 2 * cb + 1 : 2 * cb;
}

// full field r -> r_e, r_o and t_e = C_ee^-1 r_e (half fields)
__global__ void __launch_bounds__(128) k_eo_split(const float2 *__restrict__ r, const float2 *__restrict__ Cinv,
                                                   float2 *__restrict__ re, float2 *__restrict__ ro,
                                                   float2 *__restrict__ te, KArgsEO e) {
    const KArgs32 &a = e.k;
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    const int cb = item / a.G;
    if (cb >= e.V2) return;
    const int r0 = (item - cb * a.G) * 2;
    int se, so;
    eo_pair_sites(a, cb, se, so);
    const int64_t hb = (int64_t)cb * 12 * a.n + r0;
    const int64_t fe = (int64_t)se * 12 * a.n + r0, fo = (int64_t)so * 12 * a.n + r0;
#pragma unroll
    for (int i = 0; i < 12; ++i) st_p2(ro, hb + (int64_t)i * a.n, ld_p2(r, fo + (int64_t)i * a.n));
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        P2 v[6], o[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            v[i] = ld_p2(r, fe + (int64_t)(6 * chi + i) * a.n);
            st_p2(re, hb + (int64_t)(6 * chi + i) * a.n, v[i]);
        }
        site_mat_x2(Cinv, a.V, se, chi, v, o);
#pragma unroll
        for (int i = 0; i < 6; ++i) st_p2(te, hb + (int64_t)(6 * chi + i) * a.n, o[i]);
    }
}

bool eo_supported(const mrhs_lattice &lat, int n) {
    for (int mu = 0; mu < 4; ++mu)
        if (lat.g.L[mu] % 2) return false;
    return n >= 2 && n % 2 == 0 && !lat.cinv_singular && lat.g.V * 6LL * n < (1LL << 31);
}

bool residual_eo_split(const mrhs_lattice &lat, const void *x, const void *y, void *re, void *ro, void *te, int n,
                       cudaStream_t s) {
    if (!(n == 16 || n == 24 || n == 32 || n == 48 || n == 64) || !eo_supported(lat, n)) return false;
    if (lat.g.V * 12LL * n >= (1LL << 31)) return false;
    // the one-RHS-per-thread stencil's tile shapes (its first two variants); every variant
    // computes the same values, the autotuner picks between them per (lattice, n)
    const int prefs[][4] = {{1, 4, 8, 8}, {1, 4, 4, 8}};
    std::vector<KArgs32> args;
    for (const auto &pref : prefs) {
        KArgs32 a = x2_args(lat, n, pref);
        a.G = n;
        a.GS = n;
        bool dup = false;
        for (const KArgs32 &b : args) dup = dup || (b.T[1] == a.T[1] && b.T[2] == a.T[2] && b.T[3] == a.T[3]);
        if (!dup) args.push_back(a);
    }
    {
        // the first tile shape built for 8 CTAs per SM (64 registers; this kernel spills more there
        // than the plain stencil, so it is a candidate, not the default)
        KArgs32 b = args[0];
        b.occ8 = 1;
        args.push_back(b);
    }
    const unsigned blocks = (unsigned)(((int64_t)lat.g.V * n + 127) / 128);
    const float2 *U = lat.U32a.as<float2>(), *C = lat.C32a.as<float2>(), *Ci = lat.Cinv32a.as<float2>();
    const float2 *xi = static_cast<const float2 *>(x), *yi = static_cast<const float2 *>(y);
    float2 *e = static_cast<float2 *>(re), *o = static_cast<float2 *>(ro), *t = static_cast<float2 *>(te);
    auto launch = [&](int v) {
        const KArgs32 &a = args[(size_t)v];
        auto go = [&](auto nc) {
            constexpr int NC = decltype(nc)::value;
            if (a.occ8) k_dslash_r1_split<NC, 8><<<blocks, 128, 0, s>>>(U, C, Ci, xi, yi, e, o, t, a);
            else k_dslash_r1_split<NC><<<blocks, 128, 0, s>>>(U, C, Ci, xi, yi, e, o, t, a);
        };
        switch (n) {
            case 16: go(std::integral_constant<int, 16>{}); break;
            case 24: go(std::integral_constant<int, 24>{}); break;
            case 32: go(std::integral_constant<int, 32>{}); break;
            case 48: go(std::integral_constant<int, 48>{}); break;
            default: go(std::integral_constant<int, 64>{}); break;
        }
        MRHS_CUDA(cudaGetLastError());
    };
    const int v = tune_pick("k_dslash_r1_split", lat.g.L, n, (int)args.size(), launch, s);
    MRHS_TIMED("k_dslash_r1_split", s);
    launch(v);
    MRHS_LAUNCHED("k_dslash_r1_split");
    return true;
}

void eo_split(const mrhs_lattice &lat, const void *r, void *re, void *ro, void *te, int n, cudaStream_t s) {
    check_eo(lat, n);
    const KArgsEO e = eo_args(lat, n, 0);
    const int64_t items = (int64_t)e.V2 * e.k.G;
    k_eo_split<<<(unsigned)((items + 127) / 128), 128, 0, s>>>(
        static_cast<const float2 *>(r), lat.Cinv32.as<float2>(), static_cast<float2 *>(re),
        static_cast<float2 *>(ro), static_cast<float2 *>(te), e);
    MRHS_LAUNCHED("k_eo_split");
}

void eo_axpy_hop(const mrhs_lattice &lat, int out_parity, const void *self, const void *in, void *out, bool cinv,
                 int n, cudaStream_t s) {
    check_eo(lat, n);
    if (cinv)
        launch_eo<EO_CINV_AXPY_HOP>(lat, EO_MAT_CINV, static_cast<const float2 *>(in),
                                    static_cast<const float2 *>(self), static_cast<float2 *>(out), n, out_parity, s);
    else
        launch_eo<EO_AXPY_HOP>(lat, EO_NOMAT, static_cast<const float2 *>(in), static_cast<const float2 *>(self),
                               static_cast<float2 *>(out), n, out_parity, s);
}

void eo_cinv_axpy_hop_merge(const mrhs_lattice &lat, const void *r_e, const void *d_o, void *z, void *scratch_half,
                            int n, cudaStream_t s) {
    check_eo(lat, n);
    launch_eo<EO_CINV_AXPY_HOP_MERGE>(lat, EO_MAT_CINV, static_cast<const float2 *>(d_o),
                                      static_cast<const float2 *>(r_e), static_cast<float2 *>(z), n, 0, s,
                                      static_cast<float2 *>(scratch_half));
}

int clover_inverse_error(const mrhs_lattice &lat) {
    int e = 0;
    MRHS_CUDA(cudaMemcpy(&e, lat.CinvErr.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    return e;
}

template <typename Real, typename TIn, int R, bool RESID, bool GENERAL>
static void launch_dslash(const mrhs_lattice &lat, const void *in, void *out, const void *y, int n,
                          cudaStream_t s, const HopMask &mask) {
    KArgs a;
    a.g = lat.g;
    a.n = n;
    a.G = n / R;
    a.stride[0] = 1;
    a.stride[1] = lat.g.L[0];
    a.stride[2] = (int64_t)lat.g.L[0] * lat.g.L[1];
    a.stride[3] = (int64_t)lat.g.L[0] * lat.g.L[1] * lat.g.L[2];
    const int64_t items = lat.g.V * a.G;
    const int threads = 128;
    const int64_t blocks = (items + threads - 1) / threads;
    const cplx<Real> *U = sizeof(Real) == 4 ? lat.U32.as<cplx<Real>>() : lat.U64.as<cplx<Real>>();
    const cplx<Real> *C = sizeof(Real) == 4 ? lat.C32.as<cplx<Real>>() : lat.C64.as<cplx<Real>>();
    MRHS_TIMED("k_dslash", s);
    k_dslash<Real, TIn, R, RESID, GENERAL><<<(unsigned)blocks, threads, 0, s>>>(
        U, C, static_cast<const TIn *>(in), static_cast<Real *>(out), static_cast<const Real *>(y), a, mask);
    MRHS_LAUNCHED("k_dslash");
}

void dslash(const mrhs_lattice &lat, mrhs_precision compute, mrhs_precision in_prec, const void *in,
            void *out, const void *y, int n, cudaStream_t s, const HopMask *mask) {
    if (!lat.has_clover) fail(MRHS_ERR_INVALID, "clover term not built (call mrhs_build_clover)");
    HopMask m{1, -1, 0, {1, 1, 1, 1}};
    const bool general = mask != nullptr;
    if (general) m = *mask;
    const bool resid = y != nullptr;
    if (general && resid) fail(MRHS_ERR_INVALID, "masked operator has no residual form");
    if (compute == MRHS_FP32) {
        if (in_prec != MRHS_FP32) fail(MRHS_ERR_INVALID, "FP32 operator needs FP32 input");
        const bool r2 = (n % 2) == 0;
        if (!general && launch_dslash_x2(lat, in, out, y, n, s)) return;
        if (general) {
            if (r2) launch_dslash<float, float, 2, false, true>(lat, in, out, y, n, s, m);
            else launch_dslash<float, float, 1, false, true>(lat, in, out, y, n, s, m);
        } else if (resid) {
            if (r2) launch_dslash<float, float, 2, true, false>(lat, in, out, y, n, s, m);
            else launch_dslash<float, float, 1, true, false>(lat, in, out, y, n, s, m);
        } else {
            if (r2) launch_dslash<float, float, 2, false, false>(lat, in, out, y, n, s, m);
            else launch_dslash<float, float, 1, false, false>(lat, in, out, y, n, s, m);
        }
    } else if (compute == MRHS_FP64) {
        if (general) {
            if (in_prec != MRHS_FP64) fail(MRHS_ERR_INVALID, "masked FP64 operator needs FP64 input");
            launch_dslash<double, double, 1, false, true>(lat, in, out, y, n, s, m);
        } else if (in_prec == MRHS_FP64) {
            if (resid) launch_dslash<double, double, 1, true, false>(lat, in, out, y, n, s, m);
            else launch_dslash<double, double, 1, false, false>(lat, in, out, y, n, s, m);
        } else if (in_prec == MRHS_FP32) {
            if (resid) launch_dslash<double, float, 1, true, false>(lat, in, out, y, n, s, m);
            else launch_dslash<double, float, 1, false, false>(lat, in, out, y, n, s, m);
        } else {
            fail(MRHS_ERR_INVALID, "unsupported input precision");
        }
    } else if (compute == MRHS_DF64) {
        if (general) fail(MRHS_ERR_INVALID, "masked operator has no float-float form");
        if (in_prec != MRHS_FP32) fail(MRHS_ERR_INVALID, "float-float operator takes an FP32 input");
        dslash_df(lat, in, out, y, n, s);
    } else {
        fail(MRHS_ERR_INVALID, "fine operator computes in FP32, FP64 or float-float");
    }
}

// ------------------------------------------------------------ gauge layout
__global__ void k_gauge_to_soa(const double2 *__restrict__ aos, double2 *__restrict__ u64,
                               float2 *__restrict__ u32, int64_t V) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V * 36) return;
    const int64_t site = i / 36;
    const int e = (int)(i - site * 36);  // mu*9 + a*3 + b
    const double2 v = aos[i];
    u64[(int64_t)e * V + site] = v;
    u32[(int64_t)e * V + site] = make_float2((float)v.x, (float)v.y);
}

// site-major copy of an entry-major FP32 array: aos[x * E + e] = soa[e * V + x]
__global__ void k_site_major32(const float2 *__restrict__ soa, float2 *__restrict__ aos, int64_t V, int E) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V * E) return;
    const int64_t x = i / E;
    const int e = (int)(i - x * E);
    aos[i] = soa[(int64_t)e * V + x];
}

static void site_major32(const DeviceBuffer &soa, DeviceBuffer &aos, int64_t V, cudaStream_t s) {
    k_site_major32<<<ceil_div(V * 36, 256), 256, 0, s>>>(soa.as<float2>(), aos.as<float2>(), V, 36);
    MRHS_LAUNCHED("k_site_major32");
}

void gauge_to_soa(mrhs_lattice &lat, const double *aos_dev, cudaStream_t s) {
    const int64_t V = lat.g.V;
    const int64_t n = V * 36;
    k_gauge_to_soa<<<ceil_div(n, 256), 256, 0, s>>>(reinterpret_cast<const double2 *>(aos_dev),
                                                     lat.U64.as<double2>(), lat.U32.as<float2>(), V);
    MRHS_LAUNCHED("k_gauge_to_soa");
    split_df(lat.U64.ptr, lat.Udf.ptr, n, s);
    site_major32(lat.U32, lat.U32a, V, s);
}

// ------------------------------------------------------------ clover build
// 3x3 complex matrices in registers
struct M3 { cplx<double> a[3][3]; };

__device__ __forceinline__ M3 mat_mul(const M3 &x, const M3 &y) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cplx<double> s = {0, 0};
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(s, x.a[i][k], y.a[k][j]);
            r.a[i][j] = s;
        }
    return r;
}
__device__ __forceinline__ M3 mat_dag(const M3 &x) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.a[i][j] = conj(x.a[j][i]);
    return r;
}
__device__ __forceinline__ M3 load_link(const double2 *U, int64_t V, int mu, int64_t site) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double2 v = U[(int64_t)(mu * 9 + i * 3 + j) * V + site];
            r.a[i][j] = {v.x, v.y};
        }
    return r;
}

__device__ __forceinline__ int64_t nbr(const int c[4], const int L[4], int mu, int step) {
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + step + L[mu]) % L[mu];
    return coords_to_site(d, L);
}

// G_{mu nu} = i F_{mu nu} = i (Q - Q^+)/8 (Hermitian), Q the clover-leaf sum at x
__device__ M3 clover_G(const double2 *U, const Geom &g, const int c[4], int64_t site, int mu, int nu) {
    const int64_t V = g.V;
    int cm[4] = {c[0], c[1], c[2], c[3]};
    cm[mu] = (cm[mu] - 1 + g.L[mu]) % g.L[mu];          // x - mu
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[nu] = (cn[nu] - 1 + g.L[nu]) % g.L[nu];          // x - nu
    int cmn[4] = {cm[0], cm[1], cm[2], cm[3]};
    cmn[nu] = (cmn[nu] - 1 + g.L[nu]) % g.L[nu];        // x - mu - nu
    const int64_t s_pm = nbr(c, g.L, mu, 1), s_pn = nbr(c, g.L, nu, 1);
    const int64_t s_m = coords_to_site(cm, g.L), s_n = coords_to_site(cn, g.L), s_mn = coords_to_site(cmn, g.L);
    const int64_t s_m_pn = nbr(cm, g.L, nu, 1), s_n_pm = nbr(cn, g.L, mu, 1);
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    M3 Q = mat_mul(mat_mul(load_link(U, V, mu, site), load_link(U, V, nu, s_pm)),
                   mat_mul(mat_dag(load_link(U, V, mu, s_pn)), mat_dag(load_link(U, V, nu, site))));
    // leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    M3 t = mat_mul(mat_mul(load_link(U, V, nu, site), mat_dag(load_link(U, V, mu, s_m_pn))),
                   mat_mul(mat_dag(load_link(U, V, nu, s_m)), load_link(U, V, mu, s_m)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.a[i][j] = Q.a[i][j] + t.a[i][j];
    // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    t = mat_mul(mat_mul(mat_dag(load_link(U, V, mu, s_m)), mat_dag(load_link(U, V, nu, s_mn))),
                mat_mul(load_link(U, V, mu, s_mn), load_link(U, V, nu, s_n)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.a[i][j] = Q.a[i][j] + t.a[i][j];
    // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    t = mat_mul(mat_mul(mat_dag(load_link(U, V, nu, s_n)), load_link(U, V, mu, s_n)),
                mat_mul(load_link(U, V, nu, s_n_pm), mat_dag(load_link(U, V, mu, site))));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.a[i][j] = Q.a[i][j] + t.a[i][j];
    M3 G;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const cplx<double> d = Q.a[i][j] - conj(Q.a[j][i]);  // Q - Q^+
            G.a[i][j] = ti(d);                                  // times i
            G.a[i][j].re *= 0.125;
            G.a[i][j].im *= 0.125;
        }
    return G;
}

// In the chiral basis sigma_{mu nu} is block diagonal; per chirality block
// (c_sw/2) sum_{mu<nu} sigma^chi_{mu nu} (x) G_{mu nu}
//   = (c_sw/2) (sigma_x (x) X + sigma_y (x) Y + sigma_z (x) Z)
// with, for the upper block,  X = G03 - G12, Y = G02 + G13, Z = G23 - G01,
// and for the lower block     X = -G03 - G12, Y = G02 - G13, Z = -G23 - G01.
// As a 6x6 matrix (index s*3 + c): [[Z, X - iY], [X + iY, -Z]].
__global__ void k_build_clover(const double2 *__restrict__ U, Geom g, double mass, double csw,
                               double2 *__restrict__ C64, float2 *__restrict__ C32) {
    const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.V) return;
    int c[4];
    site_to_coords(site, g.L, c);
    const M3 G01 = clover_G(U, g, c, site, 0, 1), G02 = clover_G(U, g, c, site, 0, 2),
             G03 = clover_G(U, g, c, site, 0, 3), G12 = clover_G(U, g, c, site, 1, 2),
             G13 = clover_G(U, g, c, site, 1, 3), G23 = clover_G(U, g, c, site, 2, 3);
    const double h = 0.5 * csw;
    for (int chi = 0; chi < 2; ++chi) {
        const double s = chi == 0 ? 1.0 : -1.0;
        cplx<double> B[6][6];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cplx<double> X = s * G03.a[a][b] - G12.a[a][b];
                const cplx<double> Y = G02.a[a][b] + s * G13.a[a][b];
                const cplx<double> Z = s * G23.a[a][b] - G01.a[a][b];
                B[a][b] = h * Z;
                B[3 + a][3 + b] = (-h) * Z;
                B[a][3 + b] = h * (X - ti(Y));
                B[3 + a][b] = h * (X + ti(Y));
            }
        for (int i = 0; i < 6; ++i) B[i][i].re += 4.0 + mass;
        const int64_t V = g.V;
        for (int q = 0; q < 3; ++q) {
            const double2 d = make_double2(B[2 * q][2 * q].re, B[2 * q + 1][2 * q + 1].re);
            C64[(int64_t)(chi * 18 + q) * V + site] = d;
            C32[(int64_t)(chi * 18 + q) * V + site] = make_float2((float)d.x, (float)d.y);
        }
        int q = 3;
        for (int i = 1; i < 6; ++i)
            for (int j = 0; j < i; ++j, ++q) {
                const double2 l = make_double2(B[i][j].re, B[i][j].im);
                C64[(int64_t)(chi * 18 + q) * V + site] = l;
                C32[(int64_t)(chi * 18 + q) * V + site] = make_float2((float)l.x, (float)l.y);
            }
    }
}

// Inverse of the site matrix C (clover + mass) per site and chirality block:
// Gauss-Jordan elimination with partial pivoting in FP64 on the 6 x 6
// Hermitian block, written back in the compact Hermitian layout of C.  A
// pivot below 1e-300 (a singular block) sets *singular.
__global__ void k_clover_inverse(const double2 *__restrict__ C64, int64_t V, double2 *__restrict__ I64,
                                 float2 *__restrict__ I32, int *__restrict__ singular) {
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= 2 * V) return;
    const int chi = (int)(item / V);
    const int64_t site = item - chi * V;
    cplx<double> A[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) A[i][j] = {0.0, 0.0};
    for (int q = 0; q < 3; ++q) {
        const double2 d = C64[(int64_t)(chi * 18 + q) * V + site];
        A[2 * q][2 * q] = {d.x, 0.0};
        A[2 * q + 1][2 * q + 1] = {d.y, 0.0};
    }
    int q = 3;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j, ++q) {
            const double2 l = C64[(int64_t)(chi * 18 + q) * V + site];
            A[i][j] = {l.x, l.y};
            A[j][i] = {l.x, -l.y};
        }
    for (int i = 0; i < 6; ++i) A[i][6 + i] = {1.0, 0.0};
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        double best = A[col][col].re * A[col][col].re + A[col][col].im * A[col][col].im;
        for (int r = col + 1; r < 6; ++r) {
            const double m = A[r][col].re * A[r][col].re + A[r][col].im * A[r][col].im;
            if (m > best) {
                best = m;
                piv = r;
            }
        }
        if (!(best > 1e-300)) {
            atomicExch(singular, 1);
            return;
        }
        if (piv != col)
            for (int j = 0; j < 12; ++j) {
                const cplx<double> t = A[col][j];
                A[col][j] = A[piv][j];
                A[piv][j] = t;
            }
        const cplx<double> p = A[col][col];
        const cplx<double> pinv = {p.re / best, -p.im / best};
        for (int j = 0; j < 12; ++j) A[col][j] = A[col][j] * pinv;
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            const cplx<double> f = A[r][col];
            for (int j = 0; j < 12; ++j) A[r][j] = A[r][j] - f * A[col][j];
        }
    }
    for (int k = 0; k < 3; ++k) {
        const double2 d = make_double2(A[2 * k][6 + 2 * k].re, A[2 * k + 1][6 + 2 * k + 1].re);
        I64[(int64_t)(chi * 18 + k) * V + site] = d;
        I32[(int64_t)(chi * 18 + k) * V + site] = make_float2((float)d.x, (float)d.y);
    }
    q = 3;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j, ++q) {
            const double2 l = make_double2(A[i][6 + j].re, A[i][6 + j].im);
            I64[(int64_t)(chi * 18 + q) * V + site] = l;
            I32[(int64_t)(chi * 18 + q) * V + site] = make_float2((float)l.x, (float)l.y);
        }
}

void build_clover(mrhs_lattice &lat, double mass, double csw, cudaStream_t s) {
    const int64_t V = lat.g.V;
    k_build_clover<<<ceil_div(V, 128), 128, 0, s>>>(lat.U64.as<double2>(), lat.g, mass, csw,
                                                     lat.C64.as<double2>(), lat.C32.as<float2>());
    MRHS_LAUNCHED("k_build_clover");
    split_df(lat.C64.ptr, lat.Cdf.ptr, V * 36, s);
    MRHS_CUDA(cudaMemsetAsync(lat.CinvErr.ptr, 0, sizeof(int), s));
    k_clover_inverse<<<ceil_div(2 * V, 128), 128, 0, s>>>(lat.C64.as<double2>(), V, lat.Cinv64.as<double2>(),
                                                          lat.Cinv32.as<float2>(), lat.CinvErr.as<int>());
    MRHS_LAUNCHED("k_clover_inverse");
    site_major32(lat.C32, lat.C32a, V, s);
    site_major32(lat.Cinv32, lat.Cinv32a, V, s);
}

}  // namespace mrhs

extern "C" mrhs_status mrhs_debug_expire_ring_waits(int launches) {
    if (launches < 0) return mrhs::api_record(MRHS_ERR_INVALID, "launches must be >= 0");
    mrhs::g_expire_ring.store(launches);
    return mrhs::api_record(MRHS_OK, "");
}
