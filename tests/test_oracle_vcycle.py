"""Pins of the oracle's V-cycle and null-vector setup against dense linear algebra.

The oracle's MG solve converges with almost any preconditioner, so a wrong
V-cycle would not show in the solve pins.  Here one V-cycle is compared with
the same cycle written out densely (paper Sec. 5, 6, 8: R = P^dagger,
D_c = R D P, prolongation P, then post-smoothing; readings 4-7, 14):

* GMRES(m) from x0 is written as x0 + Q y with Q an orthonormal basis of the
  explicit Krylov space span{r0, A r0, ..., A^{m-1} r0} (numpy QR) and y the
  least-squares minimiser of ||r0 - A Q y|| (numpy lstsq): the defining
  property of GMRES, computed without Arnoldi;
* FGMRES(m) from 0 is written with Z = [M(v_1) .. M(v_m)], v_1 = c / ||c||
  and v_{j+1} the next orthonormal direction of span{c, A z_1, .., A z_j}
  (QR), and y = argmin ||c - A Z y||;
* the coarsest solve uses a Krylov length equal to the coarse dimension, so
  it is the exact inverse (numpy.linalg.solve);
* the even-odd smoother is the block-LU (Schur) solve of the dense D with
  the rows and columns permuted to (even, odd).

Cases: the identity prolongator (1^4 aggregates, N = 6, P unitary), where a
V-cycle with an exact coarse solve is D^{-1} itself; a genuine 2^4
aggregation (coarse extent 2, aliased neighbours) with the GMRES and the
even-odd post-smoother; and a three-level cycle with an FGMRES(2)
intermediate solve preconditioned by the level-1 V-cycle.  The null-vector
relaxation is pinned the same way: one setup cycle is one GMRES(m) step on
A v = 0 from v, and the hierarchy's prolongator is built from exactly those
vectors (relaxed against the full Wilson-clover operator).
"""
import numpy as np

import synth
from oracle import coarse, evenodd, krylov, mg, wilson


def dense_gmres(A, b, x0, m):
    """x0 + argmin over the Krylov space K_m(A, r0) of ||b - A x||, per RHS column."""
    x = np.array(x0, dtype=np.complex128, copy=True)
    r0 = b - A @ x0
    for k in range(b.shape[1]):
        K = np.empty((b.shape[0], m), dtype=np.complex128)
        K[:, 0] = r0[:, k]
        for j in range(1, m):
            K[:, j] = A @ K[:, j - 1]
        Q, _ = np.linalg.qr(K)
        y = np.linalg.lstsq(A @ Q, r0[:, k], rcond=None)[0]
        x[:, k] += Q @ y
    return x


def dense_fgmres0(A, c, precond, m):
    """One FGMRES(m) cycle from 0 with a (possibly nonlinear) preconditioner, per RHS."""
    out = np.zeros_like(c)
    for k in range(c.shape[1]):
        ck = c[:, k:k + 1]
        dirs = [ck / np.linalg.norm(ck)]
        Z = []
        for j in range(m):
            Z.append(precond(dirs[j]))
            if j + 1 < m:
                Q, _ = np.linalg.qr(np.hstack([ck] + [A @ z for z in Z]))
                dirs.append(Q[:, j + 1:j + 2])
        Zm = np.hstack(Z)
        y = np.linalg.lstsq(A @ Zm, ck[:, 0], rcond=None)[0]
        out[:, k] = Zm @ y
    return out


def dense_vcycle(mats, Ps, l, v, p):
    """The V-cycle of level l on dense matrices: mats[l] the level operator,
    Ps[l] the dense prolongator l -> l + 1 (exact coarsest solve)."""
    A, P = mats[l], Ps[l]
    c = P.conj().T @ v
    if l + 1 == len(mats) - 1:
        e = np.linalg.solve(mats[l + 1], c)
    else:
        e = dense_fgmres0(mats[l + 1], c, lambda u: dense_vcycle(mats, Ps, l + 1, u, p), p.inter_m)
    z0 = P @ e
    return dense_gmres(A, v, z0, p.smooth_m)


def dense_evenodd_smooth(D, r, dims, m):
    """delta with D delta ~= r: m GMRES steps on the Schur complement of the dense D
    in (even, odd) order from 0, then the even sites by block back-substitution."""
    e_idx = (evenodd.cb_sites(dims, 0)[:, None] * 12 + np.arange(12)).ravel()
    o_idx = (evenodd.cb_sites(dims, 1)[:, None] * 12 + np.arange(12)).ravel()
    Dee, Deo = D[np.ix_(e_idx, e_idx)], D[np.ix_(e_idx, o_idx)]
    Doe, Doo = D[np.ix_(o_idx, e_idx)], D[np.ix_(o_idx, o_idx)]
    S = Doo - Doe @ np.linalg.solve(Dee, Deo)
    bh = r[o_idx] - Doe @ np.linalg.solve(Dee, r[e_idx])
    d_o = dense_gmres(S, bh, np.zeros_like(bh), m)
    d_e = np.linalg.solve(Dee, r[e_idx] - Deo @ d_o)
    delta = np.zeros_like(r)
    delta[e_idx], delta[o_idx] = d_e, d_o
    return delta


def _field_to_mat(f):
    return f.reshape(-1, f.shape[-1])


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def _problem(dims, seed=1001, eps=0.4, mass=-0.2, csw=1.0):
    U = synth.gauge_exp(dims, eps, seed)
    C = wilson.clover_term(U, dims, csw)
    return U, C, mass, csw


# Each pin below returns the largest relative deviation of the oracle (module
# `mgm`, the oracle's mg or a planted mutant of it) from the dense formula.

def identity_prolongator_error(mgm=mg):
    """1^4 aggregates with N = 6: P is unitary, the exact coarse solve is D^{-1}."""
    dims = (2, 2, 2, 4)
    U, C, mass, csw = _problem(dims)
    V = wilson.volume(dims)
    p = mgm.MGParams(blocks=[(1, 1, 1, 1)], nvec=[6], setup_sweeps=0, smooth_m=2, coarse_m=12 * V,
                     coarse_cycles=1)
    vecs = synth.gaussian_field(V, 12, 6, 11)
    levels = mgm.build_hierarchy(U, dims, mass, csw, p, None, nullvecs=[vecs])
    v = synth.gaussian_field(V, 12, 2, 12)
    z = mgm.vcycle(levels, 0, v, p)
    D = wilson.dense_D(U, C, dims, mass)
    return _rel(_field_to_mat(z), np.linalg.solve(D, _field_to_mat(v)))


def two_level_error(mgm=mg, evenodd_smoother=False):
    """z = S(v; z0), z0 = P (P^H D P)^{-1} P^H v, with S = smooth_m GMRES steps on D
    from z0, or (even-odd smoother) z = z0 + delta(v - D z0) from the dense Schur solve."""
    dims = (4, 4, 4, 4)
    U, C, mass, csw = _problem(dims)
    V = wilson.volume(dims)
    block, N = (2, 2, 2, 2), 4
    cd = coarse.coarse_dims(dims, block)
    p = mgm.MGParams(blocks=[block], nvec=[N], setup_sweeps=0, smooth_m=3,
                     coarse_m=wilson.volume(cd) * 2 * N, coarse_cycles=1, smoother_evenodd=evenodd_smoother)
    vecs = synth.gaussian_field(V, 12, N, 21)
    levels = mgm.build_hierarchy(U, dims, mass, csw, p, None, nullvecs=[vecs])
    D = wilson.dense_D(U, C, dims, mass)
    P = coarse.dense_prolongator(levels[0].P, dims, block)
    v = synth.gaussian_field(V, 12, 2, 41 if evenodd_smoother else 31)
    z = mgm.vcycle(levels, 0, v, p)
    vm = _field_to_mat(v)
    if evenodd_smoother:
        z0 = P @ np.linalg.solve(P.conj().T @ D @ P, P.conj().T @ vm)
        zd = z0 + dense_evenodd_smooth(D, vm - D @ z0, dims, p.smooth_m)
    else:
        zd = dense_vcycle([D, P.conj().T @ D @ P], [P], 0, vm, p)
    return _rel(_field_to_mat(z), zd)


def three_level_error(mgm=mg):
    """Intermediate level: one FGMRES(2) cycle preconditioned by the level-1 V-cycle."""
    dims = (4, 4, 4, 4)
    U, C, mass, csw = _problem(dims)
    V = wilson.volume(dims)
    blocks, nvec = [(2, 2, 2, 2), (2, 2, 2, 2)], [4, 3]
    d1 = coarse.coarse_dims(dims, blocks[0])
    d2 = coarse.coarse_dims(d1, blocks[1])
    p = mgm.MGParams(blocks=blocks, nvec=nvec, setup_sweeps=0, smooth_m=2, inter_m=2,
                     coarse_m=wilson.volume(d2) * 2 * nvec[1], coarse_cycles=1)
    v0 = synth.gaussian_field(V, 12, nvec[0], 51)
    v1 = synth.gaussian_field(wilson.volume(d1), 2 * nvec[0], nvec[1], 52)
    levels = mgm.build_hierarchy(U, dims, mass, csw, p, None, nullvecs=[v0, v1])
    D = wilson.dense_D(U, C, dims, mass)
    P0 = coarse.dense_prolongator(levels[0].P, dims, blocks[0])
    P1 = coarse.dense_prolongator(levels[1].P, d1, blocks[1])
    A1 = P0.conj().T @ D @ P0
    A2 = P1.conj().T @ A1 @ P1
    v = synth.gaussian_field(V, 12, 2, 53)
    z = mgm.vcycle(levels, 0, v, p)
    zd = dense_vcycle([D, A1, A2], [P0, P1], 0, _field_to_mat(v), p)
    return _rel(_field_to_mat(z), zd)


def setup_cycle_error(mgm=mg):
    """One setup cycle = one GMRES(m) step on D v = 0 from v, then unit norm."""
    dims = (4, 4, 2, 4)
    U, C, mass, csw = _problem(dims, seed=17)
    V = wilson.volume(dims)
    D = wilson.dense_D(U, C, dims, mass)
    v0 = synth.gaussian_field(V, 12, 3, 61)
    got = mgm.setup_nullvecs(lambda f: wilson.apply_D(U, C, f, dims, mass), v0, sweeps=1, m=5)
    x = dense_gmres(D, np.zeros((12 * V, 3), np.complex128), _field_to_mat(v0), 5)
    x = x / np.linalg.norm(x, axis=0)
    return _rel(_field_to_mat(got), x)


def hierarchy_setup_error(mgm=mg):
    """build_hierarchy relaxes its start vectors against the Wilson-clover D (two
    dense GMRES(4) steps each) and orthonormalises exactly those vectors."""
    dims = (4, 4, 2, 4)
    U, C, mass, csw = _problem(dims, seed=18)
    V = wilson.volume(dims)
    block, N = (2, 2, 2, 2), 3
    p = mgm.MGParams(blocks=[block], nvec=[N], setup_sweeps=2, setup_m=4)
    v0 = synth.gaussian_field(V, 12, N, 71)
    levels = mgm.build_hierarchy(U, dims, mass, csw, p, [v0])
    D = wilson.dense_D(U, C, dims, mass)
    x = _field_to_mat(v0)
    for _ in range(2):
        x = dense_gmres(D, np.zeros_like(x), x, 4)
        x = x / np.linalg.norm(x, axis=0)
    Pd = coarse.build_prolongator(x.reshape(V, 12, N), dims, block, levels[0].chirality)
    return float(np.abs(levels[0].P - Pd).max())


def test_identity_prolongator_vcycle_is_exact_inverse():
    assert identity_prolongator_error() < 1e-10


def test_two_level_vcycle_equals_dense_two_grid():
    assert two_level_error() < 1e-10


def test_two_level_vcycle_with_evenodd_smoother_equals_dense_schur():
    assert two_level_error(evenodd_smoother=True) < 1e-10


def test_three_level_vcycle_equals_dense_recursion():
    assert three_level_error() < 1e-10


def test_setup_cycle_is_one_dense_gmres_step_on_the_null_equation():
    assert setup_cycle_error() < 1e-10


def test_hierarchy_prolongator_comes_from_vectors_relaxed_against_D():
    assert hierarchy_setup_error() < 1e-9
