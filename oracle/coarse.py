"""Aggregation, intergrid operators and the Galerkin coarse operator in FP64.

Sec. 5 of the paper: "nbasis" is twice the number of basis vectors, so each
basis vector v_k is split into its two chiral halves; on an aggregate A the
prolongator has the columns

    P_{(chi, k)} = Pi_chi v_k  restricted to A,   chi in {+, -},  k < N,

orthonormalised per aggregate and chirality.  Projection (restriction) is
R = P^dagger, promotion (prolongation) is P, and the coarse-grid operator is
the Galerkin product D_c = R D P.  Because D couples nearest neighbours, D_c
couples each aggregate only to itself and to its eight neighbour aggregates:
the 9-point coarse stencil of Sec. 6,

    (D_c phi)(xh) = A_0(xh) phi(xh) + sum_mu [ A_{+mu}(xh) phi(xh + mu)
                                              + A_{-mu}(xh) phi(xh - mu) ],

each A an nc x nc dense complex matrix (nc = 2N), coarse lattice periodic.

Stencil direction index d: 0 = self, 1 + mu = +mu, 5 + mu = -mu.

A fine hop x -> x + s*mu contributes to A_{s mu}(xh) when it leaves the
aggregate of x through its face in direction s*mu, i.e. when x_mu mod b_mu is
b_mu - 1 (s = +1) or 0 (s = -1); otherwise it stays inside and contributes to
A_0.  This holds for any coarse extent, including 2 (xh + mu = xh - mu: the two
blocks then act on the same neighbour and add) and 1 (every face hop returns
to xh itself).

Coarse dof index K = chi * N + k (chi = 0 for +), so the coarse gamma_5 is
diag(+1_N, -1_N).  Coarse fields are (Vc, nc, n), RHS innermost.
"""
from __future__ import annotations

import numpy as np

from . import wilson
from .conventions import FINE_CHIRALITY


def coarse_dims(dims, block):
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError(f"block {block} does not divide lattice {dims}")
    return tuple(int(L) // int(b) for L, b in zip(dims, block))


def aggregate_of_site(dims, block) -> np.ndarray:
    """Coarse site index of the aggregate containing each fine site, (V,)."""
    V = wilson.volume(dims)
    Lx, Ly, Lz, _ = dims
    i = np.arange(V)
    c = [i % Lx, (i // Lx) % Ly, (i // (Lx * Ly)) % Lz, i // (Lx * Ly * Lz)]
    cd = coarse_dims(dims, block)
    h = [c[m] // block[m] for m in range(4)]
    return h[0] + cd[0] * (h[1] + cd[1] * (h[2] + cd[2] * h[3]))


def aggregate_sites(dims, block) -> np.ndarray:
    """(Vc, |A|) fine site indices of each aggregate, increasing within a row."""
    agg = aggregate_of_site(dims, block)
    order = np.argsort(agg, kind="stable")
    Vc = wilson.volume(coarse_dims(dims, block))
    return order.reshape(Vc, -1)


def coarse_chirality(nc: int) -> np.ndarray:
    return np.array([0] * (nc // 2) + [1] * (nc // 2))


def _orthonormal_columns(M: np.ndarray) -> np.ndarray:
    """Q of M = Q R with diag(R) real and positive (= Gram-Schmidt on the columns)."""
    Q, R = np.linalg.qr(M)
    d = np.diagonal(R)
    ph = d / np.abs(d)
    return Q * ph[None, :]


def build_prolongator(vecs: np.ndarray, dims, block, chirality) -> np.ndarray:
    """P of shape (V, dof, 2N) from N basis vectors `vecs` (V, dof, N).

    `chirality[d]` is 0 or 1 for each site component d (spin halves on the fine
    level, first / second half of the coarse dof on coarser levels).
    Column K = chi*N + k holds Pi_chi v_k, orthonormalised over each aggregate
    separately for each chirality (QR with positive diagonal, i.e. the result
    of Gram-Schmidt on k = 0, 1, ..., N-1 in order).
    """
    V, dof, N = vecs.shape
    chirality = np.asarray(chirality)
    P = np.zeros((V, dof, 2 * N), dtype=np.complex128)
    sites = aggregate_sites(dims, block)
    for chi in (0, 1):
        comp = np.nonzero(chirality == chi)[0]
        for a in range(sites.shape[0]):
            s = sites[a]
            M = vecs[s][:, comp, :].reshape(len(s) * len(comp), N)
            Q = _orthonormal_columns(M).reshape(len(s), len(comp), N)
            P[np.ix_(s, comp, np.arange(chi * N, chi * N + N))] = Q
    return P


def restrict(P: np.ndarray, psi: np.ndarray, dims, block) -> np.ndarray:
    """R psi = P^dagger psi: c(xh)[K, r] = sum_{x in A(xh)} sum_d conj(P[x,d,K]) psi[x,d,r]."""
    sites = aggregate_sites(dims, block)
    return np.einsum("vadk,vadr->vkr", np.conj(P[sites]), psi[sites])


def prolong(P: np.ndarray, c: np.ndarray, dims, block) -> np.ndarray:
    """P c: psi[x, d, r] = sum_K P[x, d, K] c(xh(x))[K, r]."""
    agg = aggregate_of_site(dims, block)
    return np.einsum("xdk,xkr->xdr", P, c[agg])


def _crossing(dims, block, mu: int, sign: int) -> np.ndarray:
    """True where the hop x -> x + sign*mu leaves the aggregate of x."""
    V = wilson.volume(dims)
    Lx, Ly, Lz, _ = dims
    i = np.arange(V)
    c = [i % Lx, (i // Lx) % Ly, (i // (Lx * Ly)) % Lz, i // (Lx * Ly * Lz)]
    loc = c[mu] % block[mu]
    return loc == (block[mu] - 1) if sign > 0 else loc == 0


def direction_of(d: int):
    """Stencil index d (1..8) -> (mu, sign)."""
    return (d - 1, +1) if d <= 4 else (d - 5, -1)


def galerkin(diag_apply, hop_apply, P: np.ndarray, dims, block) -> np.ndarray:
    """Coarse stencil blocks (Vc, 9, nc, nc) of R A P for a nearest-neighbour A.

    diag_apply(F): the site-local part of A applied to F (V, dof, m).
    hop_apply(mu, sign, F): the single hop x -> x + sign*mu of A applied to F
    (the value at x uses F(x + sign*mu)).
    """
    nc = P.shape[2]
    cd = coarse_dims(dims, block)
    Vc = wilson.volume(cd)
    A = np.zeros((Vc, 9, nc, nc), dtype=np.complex128)
    internal = diag_apply(P)
    for d in range(1, 9):
        mu, sgn = direction_of(d)
        H = hop_apply(mu, sgn, P)
        cross = _crossing(dims, block, mu, sgn)[:, None, None]
        A[:, d] = restrict(P, np.where(cross, H, 0), dims, block)
        internal = internal + np.where(cross, 0, H)
    A[:, 0] = restrict(P, internal, dims, block)
    return A


def galerkin_fine(U, clover, P, dims, block, mass, antiperiodic=True) -> np.ndarray:
    """D_c = R D P for the fine Wilson-clover operator."""
    def diag_apply(F):
        return (4.0 + mass) * F + np.einsum("vij,vjn->vin", clover, F)

    def hop_apply(mu, sgn, F):
        return -0.5 * wilson.hop_term(U, F, dims, antiperiodic, [(mu, sgn)])

    return galerkin(diag_apply, hop_apply, P, dims, block)


def apply_coarse(A: np.ndarray, phi: np.ndarray, cdims) -> np.ndarray:
    """9-point stencil: out(xh) = sum_d A_d(xh) phi(xh + delta_d), periodic."""
    out = np.einsum("vkl,vlr->vkr", A[:, 0], phi)
    g = wilson.to_grid(phi, cdims)
    for d in range(1, 9):
        mu, sgn = direction_of(d)
        nb = wilson.from_grid(wilson.shift(g, mu, sgn), cdims)
        out += np.einsum("vkl,vlr->vkr", A[:, d], nb)
    return out


def coarse_hop(A: np.ndarray, mu: int, sgn: int, phi: np.ndarray, cdims) -> np.ndarray:
    """The single stencil term A_{sgn mu}(xh) phi(xh + sgn*mu)."""
    d = 1 + mu if sgn > 0 else 5 + mu
    g = wilson.to_grid(phi, cdims)
    nb = wilson.from_grid(wilson.shift(g, mu, sgn), cdims)
    return np.einsum("vkl,vlr->vkr", A[:, d], nb)


def galerkin_coarse(A: np.ndarray, P: np.ndarray, cdims, block) -> np.ndarray:
    """R D_c P for a coarse stencil operator (next level of a 3-level MG)."""
    def diag_apply(F):
        return np.einsum("vkl,vlr->vkr", A[:, 0], F)

    def hop_apply(mu, sgn, F):
        return coarse_hop(A, mu, sgn, F, cdims)

    return galerkin(diag_apply, hop_apply, P, cdims, block)


def dense_prolongator(P: np.ndarray, dims, block) -> np.ndarray:
    """P as a (V*dof, Vc*nc) matrix."""
    V, dof, nc = P.shape
    Vc = wilson.volume(coarse_dims(dims, block))
    agg = aggregate_of_site(dims, block)
    M = np.zeros((V, dof, Vc, nc), dtype=np.complex128)
    M[np.arange(V), :, agg, :] = P
    return M.reshape(V * dof, Vc * nc)


def dense_coarse(A: np.ndarray, cdims) -> np.ndarray:
    Vc, _, nc, _ = A.shape
    E = np.eye(Vc * nc, dtype=np.complex128).reshape(Vc, nc, Vc * nc)
    return apply_coarse(A, E, cdims).reshape(Vc * nc, Vc * nc)


FINE_DOF_CHIRALITY = FINE_CHIRALITY
