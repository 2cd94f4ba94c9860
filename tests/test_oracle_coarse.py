"""Pins of the oracle's intergrid operators and Galerkin coarse operator (Sec. 5, 6).

The stencil assembly of D_c = R D P is checked against the brute-force dense
product P^dagger D P, including coarse extents 2 and 1 where the +mu and -mu
neighbour aggregates coincide; the prolongator against orthonormality and the
chiral split; the identity prolongator against D itself.
"""
import numpy as np
import pytest

import synth
from oracle import coarse, wilson
from oracle.conventions import FINE_CHIRALITY


def _fine_problem(dims, seed=21, csw=1.0, mass=-0.1):
    U = synth.gauge_exp(dims, 0.5, seed)
    C = wilson.clover_term(U, dims, csw)
    return U, C, mass


@pytest.mark.parametrize("dims,block,N", [
    ((4, 4, 4, 4), (2, 2, 2, 2), 3),     # coarse extent 2 everywhere (aliasing)
    ((4, 2, 2, 4), (2, 2, 1, 4), 2),     # coarse extents 2, 1, 2, 1
    ((2, 2, 2, 4), (1, 2, 2, 2), 2),     # block extent 1 (every x hop leaves)
])
def test_galerkin_stencil_equals_dense(dims, block, N):
    """P5: the 9-point stencil of R D P equals the dense P^dagger D P."""
    U, C, mass = _fine_problem(dims)
    V = wilson.volume(dims)
    vecs = synth.gaussian_field(V, 12, N, 31)
    P = coarse.build_prolongator(vecs, dims, block, FINE_CHIRALITY)
    A = coarse.galerkin_fine(U, C, P, dims, block, mass)
    cd = coarse.coarse_dims(dims, block)
    Dd = wilson.dense_D(U, C, dims, mass)
    Pd = coarse.dense_prolongator(P, dims, block)
    Dc_dense = Pd.conj().T @ Dd @ Pd
    Dc_stencil = coarse.dense_coarse(A, cd)
    assert np.abs(Dc_dense - Dc_stencil).max() < 1e-12 * np.abs(Dc_dense).max()
    # coarse gamma5-hermiticity: Dc^dagger = G5 Dc G5
    Vc = wilson.volume(cd)
    g5 = np.tile(np.r_[np.ones(N), -np.ones(N)], Vc)
    assert np.abs(Dc_dense.conj().T - g5[:, None] * Dc_dense * g5[None, :]).max() < 1e-12


def test_prolongator_orthonormal_and_chiral():
    dims, block, N = (4, 4, 2, 4), (2, 2, 2, 2), 4
    V = wilson.volume(dims)
    vecs = synth.gaussian_field(V, 12, N, 41)
    P = coarse.build_prolongator(vecs, dims, block, FINE_CHIRALITY)
    Pd = coarse.dense_prolongator(P, dims, block)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-13  # R P = 1
    # chirality: column K < N lives on spins 0,1 only; K >= N on spins 2,3
    assert np.abs(P[:, 6:, :N]).max() == 0 and np.abs(P[:, :6, N:]).max() == 0
    # Pi_chi v_k restricted to an aggregate lies in the span of that aggregate's columns
    sites = coarse.aggregate_sites(dims, block)
    for a in (0, sites.shape[0] - 1):
        s = sites[a]
        for chi, comp in ((0, slice(0, 6)), (1, slice(6, 12))):
            Q = P[s][:, comp, chi * N:(chi + 1) * N].reshape(-1, N)
            v = vecs[s][:, comp, :].reshape(-1, N)
            assert np.abs(Q @ (Q.conj().T @ v) - v).max() < 1e-12
            # Gram-Schmidt order: the first column is v_0 normalised
            assert np.allclose(Q[:, 0], v[:, 0] / np.linalg.norm(v[:, 0]), atol=1e-14)


def test_restrict_prolong_match_dense():
    dims, block, N = (4, 2, 2, 4), (2, 2, 2, 2), 3
    V = wilson.volume(dims)
    P = coarse.build_prolongator(synth.gaussian_field(V, 12, N, 5), dims, block, FINE_CHIRALITY)
    Pd = coarse.dense_prolongator(P, dims, block)
    psi = synth.gaussian_field(V, 12, 4, 6)
    c = coarse.restrict(P, psi, dims, block)
    assert np.abs(c.reshape(-1, 4) - Pd.conj().T @ psi.reshape(-1, 4)).max() < 1e-13
    f = coarse.prolong(P, c, dims, block)
    assert np.abs(f.reshape(-1, 4) - Pd @ c.reshape(-1, 4)).max() < 1e-13
    # P R is a projector
    assert np.abs(coarse.prolong(P, coarse.restrict(P, f, dims, block), dims, block) - f).max() < 1e-13


def test_identity_prolongator():
    """P6: 1^4 aggregates and N = 6 make P unitary, so P D_c P^dagger = D."""
    dims, block, N = (2, 2, 2, 4), (1, 1, 1, 1), 6
    U, C, mass = _fine_problem(dims, seed=3)
    V = wilson.volume(dims)
    P = coarse.build_prolongator(synth.gaussian_field(V, 12, N, 8), dims, block, FINE_CHIRALITY)
    A = coarse.galerkin_fine(U, C, P, dims, block, mass)
    Pd = coarse.dense_prolongator(P, dims, block)
    assert np.abs(Pd @ Pd.conj().T - np.eye(12 * V)).max() < 1e-13
    Dc = coarse.dense_coarse(A, dims)
    Dd = wilson.dense_D(U, C, dims, mass)
    assert np.abs(Pd @ Dc @ Pd.conj().T - Dd).max() < 1e-12
    ev1 = np.sort_complex(np.round(np.linalg.eigvals(Dc), 8))
    ev2 = np.sort_complex(np.round(np.linalg.eigvals(Dd), 8))
    assert np.abs(ev1 - ev2).max() < 1e-7


@pytest.mark.parametrize("cdims,block,N2", [((4, 2, 2, 4), (2, 1, 2, 2), 2),
                                            ((2, 2, 2, 2), (2, 2, 1, 1), 3)])
def test_second_level_galerkin_equals_dense(cdims, block, N2):
    """R2 D_c P2 of a random coarse stencil (3-level hierarchy) vs dense."""
    nc1 = 6
    Vc = wilson.volume(cdims)
    rng = np.random.default_rng(12)
    A = rng.standard_normal((Vc, 9, nc1, nc1)) + 1j * rng.standard_normal((Vc, 9, nc1, nc1))
    chir = coarse.coarse_chirality(nc1)
    P2 = coarse.build_prolongator(synth.gaussian_field(Vc, nc1, N2, 9), cdims, block, chir)
    A2 = coarse.galerkin_coarse(A, P2, cdims, block)
    Dd = coarse.dense_coarse(A, cdims)
    Pd = coarse.dense_prolongator(P2, cdims, block)
    dense = Pd.conj().T @ Dd @ Pd
    stencil = coarse.dense_coarse(A2, coarse.coarse_dims(cdims, block))
    assert np.abs(dense - stencil).max() < 1e-12 * np.abs(dense).max()


def test_coarse_apply_mrhs_and_aliasing():
    """The coarse stencil on extent-1/2 lattices adds both hops into one neighbour."""
    cdims = (2, 1, 2, 1)
    Vc, nc = wilson.volume(cdims), 4
    rng = np.random.default_rng(2)
    A = rng.standard_normal((Vc, 9, nc, nc)) + 1j * rng.standard_normal((Vc, 9, nc, nc))
    phi = synth.gaussian_field(Vc, nc, 3, 1)
    out = coarse.apply_coarse(A, phi, cdims)
    # brute force by coordinates
    ext = cdims
    for v in range(Vc):
        c = synth.site_coords(v, cdims)
        acc = A[v, 0] @ phi[v]
        for mu in range(4):
            for sgn, d in ((+1, 1 + mu), (-1, 5 + mu)):
                cc = c.copy()
                cc[mu] = (cc[mu] + sgn) % ext[mu]
                acc = acc + A[v, d] @ phi[synth.site_index(cc, cdims)]
        assert np.abs(acc - out[v]).max() < 1e-13
