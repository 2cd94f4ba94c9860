// Spin projection tables of the fine operator (paper Sec. 4), shared by the
// stencil kernels.  Chiral basis, gamma_mu = [[0, A_mu], [A_mu^+, 0]] with
// A_k = -i sigma_k, A_t = 1: (1 -+ gamma_mu) psi has rank 2, so each hop forms
// a 2-spin half spinor h = psi_up -+ A psi_dn, multiplies it by the link, and
// rebuilds the lower spins from the two products.
#pragma once

#include "common.cuh"

namespace mrhs {

// ---------------------------------------------------------------- factors
// multiply by one of +1, -1, +i, -i
enum { FP = 0, FM = 1, FI = 2, FMI = 3 };
template <int F, typename T> __device__ __forceinline__ cplx<T> fmul(cplx<T> a) {
    if constexpr (F == FP) return a;
    else if constexpr (F == FM) return {-a.re, -a.im};
    else if constexpr (F == FI) return ti(a);
    else return tmi(a);
}
template <int F> struct neg_f { static constexpr int v = F == FP ? FM : F == FM ? FP : F == FI ? FMI : FI; };

// Half-spinor rule of direction MU for the forward hop (1 - gamma_mu):
//   h0 = psi0 + F0 psi_{P0},  h1 = psi1 + F1 psi_{P1}
//   acc2 += G2 (U h)_{Q2},    acc3 += G3 (U h)_{Q3},  acc0 += (U h)_0, acc1 += (U h)_1
// The backward hop (1 + gamma_mu) negates F0, F1, G2, G3.
template <int MU> struct Proj;
template <> struct Proj<0> { static constexpr int P0 = 3, F0 = FI, P1 = 2, F1 = FI, Q2 = 1, G2 = FMI, Q3 = 0, G3 = FMI; };
template <> struct Proj<1> { static constexpr int P0 = 3, F0 = FP, P1 = 2, F1 = FM, Q2 = 1, G2 = FM, Q3 = 0, G3 = FP; };
template <> struct Proj<2> { static constexpr int P0 = 2, F0 = FI, P1 = 3, F1 = FMI, Q2 = 0, G2 = FMI, Q3 = 1, G3 = FI; };
template <> struct Proj<3> { static constexpr int P0 = 2, F0 = FM, P1 = 3, F1 = FM, Q2 = 0, G2 = FM, Q3 = 1, G3 = FM; };

}  // namespace mrhs
