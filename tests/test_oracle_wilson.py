"""Pins of the FP64 oracle's fine Wilson-clover operator (Sec. 4 of the paper).

Each test checks the oracle against something other than itself: the Clifford
algebra, the closed-form free-field spectrum, the closed-form clover term of a
constant abelian field, gamma_5-hermiticity, gauge covariance, and a second
(site-by-site) evaluation of the operator.
"""
import numpy as np
import pytest

import synth
from oracle import conventions as cv
from oracle import wilson


def test_clifford_algebra_and_gamma5():
    G = cv.GAMMA
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T, atol=1e-15)
        for nu in range(4):
            ac = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    assert np.allclose(cv.GAMMA5, np.diag([1, 1, -1, -1]), atol=1e-15)
    for mu in range(4):
        for nu in range(4):
            s = cv.sigma_munu(mu, nu)
            assert np.allclose(s, s.conj().T, atol=1e-15)
            # sigma commutes with gamma_5: block diagonal in the chiral basis
            assert np.allclose(s @ cv.GAMMA5, cv.GAMMA5 @ s, atol=1e-15)


def _free_symbol(p, mass):
    """D(p) = (4+m) - sum cos p_mu + i sum gamma_mu sin p_mu (4x4 in spin)."""
    D = (4.0 + mass - np.sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        D = D + 1j * np.sin(p[mu]) * cv.GAMMA[mu]
    return D


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (3, 5, 2, 6)])
def test_free_field_plane_waves(dims):
    """P1: with U = 1, D e^{ipx} u = D(p) u e^{ipx}; antiperiodic p_t."""
    mass, csw = -0.3, 1.7
    U = synth.gauge_unit(dims)
    C = wilson.clover_term(U, dims, csw)
    assert np.abs(C).max() < 1e-15  # F = 0 for the unit field
    V = wilson.volume(dims)
    coords = synth.site_coords(np.arange(V), dims)
    rng = np.random.default_rng(7)
    for n_mom in [(0, 0, 0, 0), (1, 0, 2, 1), (2, 1, 1, 3), (1, 3, 1, 0)]:
        p = np.array([2 * np.pi * n_mom[k] / dims[k] for k in range(3)]
                     + [(2 * n_mom[3] + 1) * np.pi / dims[3]])
        u = rng.standard_normal((4, 3, 2)) + 1j * rng.standard_normal((4, 3, 2))
        phase = np.exp(1j * coords @ p)
        psi = (phase[:, None, None, None] * u[None]).reshape(V, 12, 2)
        out = wilson.apply_D(U, C, psi, dims, mass)
        expect = phase[:, None, None, None] * np.einsum("st,tan->san", _free_symbol(p, mass), u)[None]
        assert np.abs(out - expect.reshape(V, 12, 2)).max() < 1e-13


def test_free_field_spectrum_dense():
    """P1: spectrum of the dense free D = m + sum(1-cos p) +- i |sin p|, 6-fold each."""
    dims = (2, 2, 4, 4)
    mass = 0.1
    U = synth.gauge_unit(dims)
    C = wilson.clover_term(U, dims, 1.0)
    D = wilson.dense_D(U, C, dims, mass)
    ev = np.sort_complex(np.round(np.linalg.eigvals(D), 10))
    expect = []
    for nx in range(dims[0]):
        for ny in range(dims[1]):
            for nz in range(dims[2]):
                for nt in range(dims[3]):
                    p = np.array([2 * np.pi * nx / dims[0], 2 * np.pi * ny / dims[1],
                                  2 * np.pi * nz / dims[2], (2 * nt + 1) * np.pi / dims[3]])
                    re = mass + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.sort_complex(np.round(np.array(expect), 10))
    assert np.abs(ev - expect).max() < 1e-8


def test_abelian_lambda3_clover_closed_form():
    """P2: U_x(x) = diag(e^{-i phi y}, e^{i phi y}, 1), phi = 2 pi / Ly.

    Every xy plaquette is diag(e^{i phi}, e^{-i phi}, 1), so F_xy = i sin(phi)
    diag(1, -1, 0), all other F vanish, and the clover term is
    -(c_sw/2) sin(phi) sigma_xy (x) diag(1, -1, 0).
    """
    dims = (3, 5, 2, 4)
    csw = 1.3
    U = synth.gauge_unit(dims)
    V = wilson.volume(dims)
    y = synth.site_coords(np.arange(V), dims)[:, 1]
    phi = 2 * np.pi / dims[1]
    U[:, 0, 0, 0] = np.exp(-1j * phi * y)
    U[:, 0, 1, 1] = np.exp(1j * phi * y)
    F = wilson.field_strength(U, dims)
    for key, Fmn in F.items():
        if key == (0, 1):
            assert np.abs(Fmn - 1j * np.sin(phi) * np.diag([1, -1, 0])).max() < 1e-14
        else:
            assert np.abs(Fmn).max() < 1e-14
    C = wilson.clover_term(U, dims, csw).reshape(V, 4, 3, 4, 3)
    expect = -(csw / 2) * np.sin(phi) * np.einsum("st,ab->satb", cv.sigma_munu(0, 1),
                                                   np.diag([1.0, -1.0, 0.0]))
    assert np.abs(C - expect[None]).max() < 1e-14
    ev = np.linalg.eigvalsh(C[0].reshape(12, 12))
    amp = csw / 2 * np.sin(phi)
    assert np.allclose(np.sort(ev), np.sort([-amp] * 4 + [amp] * 4 + [0] * 4), atol=1e-14)


def _random_setup(dims, seed=11, eps=None):
    U = synth.gauge_haar(dims, seed) if eps is None else synth.gauge_exp(dims, eps, seed)
    return U


def test_clover_hermitian_and_chiral():
    dims = (4, 2, 3, 4)
    U = _random_setup(dims)
    C = wilson.clover_term(U, dims, 1.0)
    assert np.abs(C - np.conj(np.swapaxes(C, 1, 2))).max() < 1e-14
    g5 = np.kron(cv.GAMMA5, np.eye(3))
    assert np.abs(C @ g5 - g5 @ C).max() < 1e-14
    assert np.abs(C).max() > 0.1


def test_gamma5_hermiticity():
    """P3: <x, D y> = <gamma5 D gamma5 x, y> for random fields."""
    dims = (4, 4, 2, 4)
    U = _random_setup(dims, eps=0.7)
    C = wilson.clover_term(U, dims, 1.0)
    V = wilson.volume(dims)
    x = synth.gaussian_field(V, 12, 3, 1)
    y = synth.gaussian_field(V, 12, 3, 2)
    lhs = np.einsum("vdr,vdr->r", x.conj(), wilson.apply_D(U, C, y, dims, -0.2))
    g5Dg5x = wilson.gamma5_field(wilson.apply_D(U, C, wilson.gamma5_field(x), dims, -0.2))
    rhs = np.einsum("vdr,vdr->r", g5Dg5x.conj(), y)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def test_gauge_covariance():
    """P4: U'_mu(x) = g(x) U_mu(x) g(x+mu)^dagger gives D[U'](g psi) = g D[U] psi."""
    dims = (4, 3, 2, 4)
    U = _random_setup(dims, seed=5)
    g = synth.gauge_transform_haar(dims, 6)
    V = wilson.volume(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = wilson.from_grid(wilson.shift(wilson.to_grid(g, dims), mu, +1), dims)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(gp, 1, 2))
    psi = synth.gaussian_field(V, 12, 2, 3)

    def gmul(f):
        return np.einsum("vab,vsbn->vsan", g, f.reshape(V, 4, 3, 2)).reshape(V, 12, 2)

    C = wilson.clover_term(U, dims, 1.1)
    Cg = wilson.clover_term(Ug, dims, 1.1)
    lhs = wilson.apply_D(Ug, Cg, gmul(psi), dims, 0.05)
    rhs = gmul(wilson.apply_D(U, C, psi, dims, 0.05))
    assert np.abs(lhs - rhs).max() < 1e-12


def test_sitewise_matches_whole_lattice():
    dims = (3, 4, 2, 5)
    U = _random_setup(dims, seed=9)
    C = wilson.clover_term(U, dims, 0.9)
    V = wilson.volume(dims)
    psi = synth.gaussian_field(V, 12, 3, 4)
    full = wilson.apply_D(U, C, psi, dims, -0.1)
    sites = [0, 1, V - 1, 17, 33, 59, V // 2]
    part = wilson.apply_D_sites(U, psi, dims, -0.1, 0.9, sites)
    assert np.abs(part - full[sites]).max() < 1e-13


def test_mrhs_equals_per_rhs():
    """P9 for the operator: applying to n RHS = n single-RHS applications."""
    dims = (4, 2, 2, 4)
    U = _random_setup(dims, seed=3)
    C = wilson.clover_term(U, dims, 1.0)
    V = wilson.volume(dims)
    psi = synth.gaussian_field(V, 12, 5, 8)
    full = wilson.apply_D(U, C, psi, dims, -0.2)
    for r in range(5):
        single = wilson.apply_D(U, C, psi[:, :, r:r + 1], dims, -0.2)
        assert np.array_equal(single[:, :, 0], full[:, :, r]) or \
            np.abs(single[:, :, 0] - full[:, :, r]).max() < 1e-14
