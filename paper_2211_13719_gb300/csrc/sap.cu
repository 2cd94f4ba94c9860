// SAP smoother on the fine level: the Schwarz alternating procedure the
// paper's outlook (Sec. 9) names as the next smoother for the MRHS solver.
//
// The lattice is cut into blocks of extents B with an even number of blocks
// in every direction and coloured by block parity c = (sum_mu x_mu / B_mu)
// mod 2, so blocks of one colour never touch and D restricted to one colour
// is block diagonal.  One SAP cycle for D z = v:
//     for c = 0, 1:  r = v - D z;  z += e,  e_B ~= D_BB^{-1} r_B on every
//                    block B of colour c,
// each block system approximated by `mr_steps` minimal-residual iterations
// from zero with inner products over the block alone:
//     rho = r_B;  q = D_BB rho;  alpha = <q, rho> / <q, q>;
//     e_B += alpha rho;  rho -= alpha q.
//
// GB300 design: one CTA per (block of colour c, group of RHS pairs) runs all
// MR steps of its block systems on chip.  The block's forward links and clover
// matrices (2 x 72 KB for a 4^4 block) are staged in shared memory once and
// serve every RHS pair and step of the CTA; per pair, rho (48 KB) lives in
// shared memory and e in registers.  A step is one in-block stencil pass
// (neighbours and links from shared memory, paired-FP32 arithmetic as in the
// fine stencil) and one block reduction of <q, rho> and <q, q> for the two RHS
// of the pair.  A hop that leaves the block is dropped (D_BB), so no
// antiperiodic sign ever applies inside a block: block boundaries sit on
// multiples of B and the time wrap is one; the backward hop inside the block
// uses the forward link of the in-block neighbour.
#include <algorithm>

#include "internal.cuh"
#include "pair.cuh"
#include "spin.cuh"

namespace mrhs {

namespace {

constexpr int SAP_MAX_BVOL = 256;
constexpr int SAP_THREADS = 256;

struct SapArgs {
    int L[4];
    int V;
    int n;
    int B[4];
    int NB[4];
    int bvol;
    int color;
    int steps;
    int pair0;          // first RHS pair of the launch (0)
    int pairs_per_cta;  // RHS pairs each CTA runs one after the other
};

// shared-memory field [12][bvol] of RHS pairs stored as (re r0, re r1, im r0, im r1)
__device__ __forceinline__ P2 sm_ld(const float4 *f, int bvol, int k, int t) {
    const float4 v = f[k * bvol + t];
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void sm_st(float4 *f, int bvol, int k, int t, P2 v) {
    f[k * bvol + t] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
}

// acc += (1 -+ gamma_mu) U h for the in-block neighbour at local index nb; the
// block's forward links are staged in shared memory as Us[(mu * 9 + e) * bvol + s]
// (the backward hop from t uses the forward link of its in-block neighbour nb)
template <int MU, bool FWD>
__device__ __forceinline__ void sap_hop(P2 (&acc)[12], const float2 *Us, const float4 *rho, int bvol, int nb,
                                        int link_s) {
    using P = Proj<MU>;
    constexpr int F0 = FWD ? P::F0 : neg_f<P::F0>::v;
    constexpr int F1 = FWD ? P::F1 : neg_f<P::F1>::v;
    constexpr int G2 = FWD ? P::G2 : neg_f<P::G2>::v;
    constexpr int G3 = FWD ? P::G3 : neg_f<P::G3>::v;
    P2 h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const P2 p0 = sm_ld(rho, bvol, 0 * 3 + c, nb);
        const P2 p1 = sm_ld(rho, bvol, 1 * 3 + c, nb);
        const P2 pa = sm_ld(rho, bvol, P::P0 * 3 + c, nb);
        const P2 pb = sm_ld(rho, bvol, P::P1 * 3 + c, nb);
        h0[c] = p2add(p0, p2f<F0>(pa));
        h1[c] = p2add(p1, p2f<F1>(pb));
    }
    const float2 *Ul = Us + MU * 9 * bvol + link_s;
#pragma unroll
    for (int row = 0; row < 3; ++row) {
        P2 s0 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, s1 = s0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (FWD) {
                const float2 u = Ul[(row * 3 + b) * bvol];
                p2mac(s0, u, h0[b]);
                p2mac(s1, u, h1[b]);
            } else {
                const float2 u = Ul[(b * 3 + row) * bvol];
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

template <int MU>
__device__ __forceinline__ void sap_hop_pair(P2 (&acc)[12], const float2 *Us, const SapArgs &a, const float4 *rho,
                                             int t, const int lc[4], int lstride) {
    if (lc[MU] < a.B[MU] - 1) sap_hop<MU, true>(acc, Us, rho, a.bvol, t + lstride, t);
    if (lc[MU] > 0) sap_hop<MU, false>(acc, Us, rho, a.bvol, t - lstride, t - lstride);
}

// o = C v for chirality block chi of the site matrix staged in shared memory as
// Cs[(chi * 18 + q) * bvol + s] (3 diagonal pairs, then the 15 lower entries)
__device__ __forceinline__ void sap_site_mat(const float2 *Cs, int bvol, int t, int chi, const P2 (&v)[6],
                                             P2 (&o)[6]) {
    const float2 *Mp = Cs + chi * 18 * bvol + t;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float2 d = Mp[q * bvol];
        const float2 d0 = make_float2(d.x, d.x), d1 = make_float2(d.y, d.y);
        o[2 * q] = {__fmul2_rn(d0, v[2 * q].re), __fmul2_rn(d0, v[2 * q].im)};
        o[2 * q + 1] = {__fmul2_rn(d1, v[2 * q + 1].re), __fmul2_rn(d1, v[2 * q + 1].im)};
    }
    int q = 3;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j, ++q) {
            const float2 l = Mp[q * bvol];
            p2mac(o[i], l, v[j]);
            p2mac_conj(o[j], l, v[i]);
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per (block of colour a.color, group of RHS pairs).  The block's
// forward links and clover matrices are staged in shared memory once and serve
// every RHS pair and MR step of the CTA; per pair, rho lives in shared memory,
// e in registers.
__global__ void __launch_bounds__(SAP_THREADS, 1) k_sap_mr(const float2 *__restrict__ U, const float2 *__restrict__ C,
                                                             const float2 *__restrict__ r, float2 *__restrict__ z,
                                                             SapArgs a) {
    extern __shared__ float4 sap_sm[];
    float4 *rho = sap_sm;                                         // [12][bvol]
    float2 *Us = reinterpret_cast<float2 *>(sap_sm + 12 * a.bvol);  // [36][bvol]
    float2 *Cs = Us + 36 * a.bvol;                                // [36][bvol]
    __shared__ float red[SAP_THREADS / 32][6];
    __shared__ float2 alpha_sm[2];

    // the blockIdx.x-th block of colour a.color, blocks ordered (bx / 2, by, bz, bt)
    int q = blockIdx.x;
    const int hx = a.NB[0] / 2;
    const int j = q % hx;
    q /= hx;
    const int by = q % a.NB[1];
    q /= a.NB[1];
    const int bz = q % a.NB[2];
    const int bt = q / a.NB[2];
    const int bx = 2 * j + ((by + bz + bt + a.color) & 1);

    const int t = threadIdx.x;
    const bool active = t < a.bvol;
    int lc[4];
    {
        int u = active ? t : 0;
        lc[0] = u % a.B[0];
        u /= a.B[0];
        lc[1] = u % a.B[1];
        u /= a.B[1];
        lc[2] = u % a.B[2];
        lc[3] = u / a.B[2];
    }
    const int x = bx * a.B[0] + lc[0], y = by * a.B[1] + lc[1], zc = bz * a.B[2] + lc[2], tc = bt * a.B[3] + lc[3];
    const int site = x + a.L[0] * (y + a.L[1] * (zc + a.L[2] * tc));
    const int ls1 = a.B[0], ls2 = a.B[0] * a.B[1], ls3 = a.B[0] * a.B[1] * a.B[2];
    const P2 zero = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};

    if (active) {
#pragma unroll 4
        for (int e = 0; e < 36; ++e) {
            Us[e * a.bvol + t] = __ldg(U + (int64_t)e * a.V + site);
            Cs[e * a.bvol + t] = __ldg(C + (int64_t)e * a.V + site);
        }
    }

    const float2 mhalf = make_float2(-0.5f, -0.5f);
    for (int pair = a.pair0 + blockIdx.y * a.pairs_per_cta; pair < min(a.pair0 + (int)(blockIdx.y + 1) * a.pairs_per_cta, a.n / 2);
         ++pair) {
        const int64_t base = (int64_t)site * 12 * a.n + 2 * pair;
        P2 e[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) e[k] = zero;
        if (active) {
#pragma unroll
            for (int k = 0; k < 12; ++k) sm_st(rho, a.bvol, k, t, ld_p2(r, base + (int64_t)k * a.n));
        }
        __syncthreads();  // rho of this pair (and, on the first pair, the staged links / clover) complete

        for (int step = 0; step < a.steps; ++step) {
            P2 qv[12];
            float part[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (active) {
                P2 acc[12];
#pragma unroll
                for (int i = 0; i < 12; ++i) acc[i] = zero;
                sap_hop_pair<0>(acc, Us, a, rho, t, lc, 1);
                sap_hop_pair<1>(acc, Us, a, rho, t, lc, ls1);
                sap_hop_pair<2>(acc, Us, a, rho, t, lc, ls2);
                sap_hop_pair<3>(acc, Us, a, rho, t, lc, ls3);
#pragma unroll
                for (int chi = 0; chi < 2; ++chi) {
                    P2 v[6], o[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i) v[i] = sm_ld(rho, a.bvol, 6 * chi + i, t);
                    sap_site_mat(Cs, a.bvol, t, chi, v, o);
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        const P2 ai = acc[6 * chi + i];
                        const P2 qi = {__ffma2_rn(mhalf, ai.re, o[i].re), __ffma2_rn(mhalf, ai.im, o[i].im)};
                        qv[6 * chi + i] = qi;
                        // <q, rho> = sum conj(q) rho, and |q|^2, for both RHS of the pair
                        part[0] += qi.re.x * v[i].re.x + qi.im.x * v[i].im.x;
                        part[1] += qi.re.x * v[i].im.x - qi.im.x * v[i].re.x;
                        part[2] += qi.re.y * v[i].re.y + qi.im.y * v[i].im.y;
                        part[3] += qi.re.y * v[i].im.y - qi.im.y * v[i].re.y;
                        part[4] += qi.re.x * qi.re.x + qi.im.x * qi.im.x;
                        part[5] += qi.re.y * qi.re.y + qi.im.y * qi.im.y;
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) part[i] = warp_sum(part[i]);
            if ((t & 31) == 0) {
#pragma unroll
                for (int i = 0; i < 6; ++i) red[t >> 5][i] = part[i];
            }
            __syncthreads();  // every read of rho for this step is done
            if (t == 0) {
                float sm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < SAP_THREADS / 32; ++w)
#pragma unroll
                    for (int i = 0; i < 6; ++i) sm[i] += red[w][i];
                // a block that has converged to zero keeps alpha = 0
                const float tiny = 1.17549435e-38f;
                alpha_sm[0] = sm[4] > tiny ? make_float2(sm[0] / sm[4], sm[1] / sm[4]) : make_float2(0.f, 0.f);
                alpha_sm[1] = sm[5] > tiny ? make_float2(sm[2] / sm[5], sm[3] / sm[5]) : make_float2(0.f, 0.f);
            }
            __syncthreads();
            if (active) {
                const float2 al0 = alpha_sm[0], al1 = alpha_sm[1];
                const float2 ar = make_float2(al0.x, al1.x), ai = make_float2(al0.y, al1.y);
                const float2 nai = make_float2(-al0.y, -al1.y);
                const float2 nar = make_float2(-al0.x, -al1.x);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    P2 rk = sm_ld(rho, a.bvol, k, t);
                    // e += alpha rho
                    e[k].re = __ffma2_rn(ar, rk.re, e[k].re);
                    e[k].re = __ffma2_rn(nai, rk.im, e[k].re);
                    e[k].im = __ffma2_rn(ar, rk.im, e[k].im);
                    e[k].im = __ffma2_rn(ai, rk.re, e[k].im);
                    // rho -= alpha q
                    const P2 qk = qv[k];
                    rk.re = __ffma2_rn(nar, qk.re, rk.re);
                    rk.re = __ffma2_rn(ai, qk.im, rk.re);
                    rk.im = __ffma2_rn(nar, qk.im, rk.im);
                    rk.im = __ffma2_rn(nai, qk.re, rk.im);
                    sm_st(rho, a.bvol, k, t, rk);
                }
            }
            __syncthreads();
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const int64_t off = base + (int64_t)k * a.n;
                const P2 zk = ld_p2(z, off);
                const float4 o = make_float4(zk.re.x + e[k].re.x, zk.im.x + e[k].im.x, zk.re.y + e[k].re.y,
                                             zk.im.y + e[k].im.y);
                *reinterpret_cast<float4 *>(z + off) = o;
            }
        }
        __syncthreads();  // the next pair overwrites rho
    }
}

}  // namespace

static int current_sm_count_sap() {
    int dev = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    return sm_count(dev);
}

bool sap_supported(const mrhs_lattice &lat, const int B[4], int n) {
    if (n < 2 || n % 2) return false;
    int64_t bvol = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (B[mu] < 1 || lat.g.L[mu] % B[mu] || (lat.g.L[mu] / B[mu]) % 2) return false;
        bvol *= B[mu];
    }
    if (bvol > SAP_MAX_BVOL) return false;
    if (lat.g.V * 12LL * n >= (1LL << 31)) return false;
    return true;
}

void sap_smooth(const mrhs_lattice &lat, const void *v, void *z, int n, const int B[4], int cycles, int mr_steps,
                void *r_tmp, cudaStream_t s) {
    if (!lat.has_clover) fail(MRHS_ERR_INVALID, "clover term not built");
    if (!sap_supported(lat, B, n))
        fail(MRHS_ERR_INVALID, "SAP needs an even nrhs, block extents dividing the lattice into an even number of "
                               "blocks per direction, at most 256 sites per block and 32-bit field indexing");
    if (cycles < 0 || mr_steps < 0) fail(MRHS_ERR_INVALID, "SAP cycles and MR steps must be >= 0");
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!al(v) || !al(z) || !al(r_tmp)) fail(MRHS_ERR_INVALID, "SAP fields must be 16-byte aligned");
    SapArgs a;
    a.V = (int)lat.g.V;
    a.n = n;
    a.bvol = 1;
    for (int mu = 0; mu < 4; ++mu) {
        a.L[mu] = lat.g.L[mu];
        a.B[mu] = B[mu];
        a.NB[mu] = a.L[mu] / B[mu];
        a.bvol *= B[mu];
    }
    a.steps = mr_steps;
    a.pair0 = 0;
    // per site: 12 RHS-pair entries of rho (16 B), 36 link and 36 clover entries (8 B)
    const size_t smem = (sizeof(float4) * 12 + sizeof(float2) * 72) * (size_t)a.bvol;
    static thread_local int configured_dev = -1;
    int dev = 0;
    MRHS_CUDA(cudaGetDevice(&dev));
    if (configured_dev != dev) {
        MRHS_CUDA(cudaFuncSetAttribute(k_sap_mr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((sizeof(float4) * 12 + sizeof(float2) * 72) * SAP_MAX_BVOL)));
        configured_dev = dev;
    }
    // one CTA per SM (192 KB of shared memory for a 4^4 block): split the RHS pairs
    // of a block over CTAs so that the grid covers the SMs several times over
    const int nblk = a.NB[0] * a.NB[1] * a.NB[2] * a.NB[3] / 2;
    const int npairs = n / 2;
    int groups = 1;
    while (groups < npairs && (int64_t)nblk * groups < 16LL * current_sm_count_sap()) groups *= 2;
    groups = std::min(groups, npairs);
    a.pairs_per_cta = (npairs + groups - 1) / groups;
    const dim3 grid((unsigned)nblk, (unsigned)((npairs + a.pairs_per_cta - 1) / a.pairs_per_cta));
    const float2 *vv = static_cast<const float2 *>(v);
    float2 *zz = static_cast<float2 *>(z);
    float2 *rr = static_cast<float2 *>(r_tmp);
    for (int cyc = 0; cyc < cycles; ++cyc) {
        for (int c = 0; c < 2; ++c) {
            dslash(lat, MRHS_FP32, MRHS_FP32, zz, rr, vv, n, s);  // r = v - D z
            a.color = c;
            MRHS_TIMED("k_sap_mr", s);
            k_sap_mr<<<grid, SAP_THREADS, smem, s>>>(lat.U32.as<float2>(), lat.C32.as<float2>(), rr, zz, a);
            MRHS_LAUNCHED("k_sap_mr");
        }
    }
}

}  // namespace mrhs
