"""Pins of the oracle's Krylov solvers and MG solve (Sec. 7, 8 of the paper).

Checks: GMRES with a full Krylov space is an exact solve; the MG-preconditioned
FGMRES solution equals numpy.linalg.solve of the dense D (P7); on a unit gauge
field it equals the closed-form momentum-space inverse (P8); solving n RHS
together equals solving them one at a time (P9); the true residual reaches
1e-10 (P10); the null-vector relaxation lowers ||D v|| / ||v||.
"""
import numpy as np
import pytest

import synth
from oracle import coarse, krylov, mg, wilson
from oracle import conventions as cv


def test_gmres_full_space_is_exact():
    rng = np.random.default_rng(0)
    n, N = 3, 12
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)) + 5 * np.eye(N)
    b = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n))
    x = krylov.gmres(lambda v: A @ v, b, np.zeros_like(b), m=N, cycles=1)
    assert np.abs(A @ x - b).max() < 1e-10
    # each RHS is its own problem: a zero RHS stays exactly zero
    b[:, 1] = 0
    x = krylov.gmres(lambda v: A @ v, b, np.zeros_like(b), m=N, cycles=1)
    assert np.all(x[:, 1] == 0)


def _problem(dims, seed, eps=0.4, mass=-0.2, csw=1.0):
    U = synth.gauge_exp(dims, eps, seed)
    return U, mass, csw


def _init_vecs(levels_dims, dofs, nvec, seed):
    return [synth.gaussian_field(wilson.volume(d), dof, N, seed + l)
            for l, (d, dof, N) in enumerate(zip(levels_dims, dofs, nvec))]


def test_mg_solve_matches_dense_solve():
    """P7 + P10: 2-level MG-FGMRES x equals the dense solve; residual <= 1e-10."""
    dims = (4, 4, 4, 4)
    U, mass, csw = _problem(dims, 1001)
    params = mg.MGParams(blocks=[(2, 2, 2, 2)], nvec=[4], setup_sweeps=3, setup_m=6,
                         smooth_m=4, coarse_m=12, coarse_cycles=2, outer_m=8, tol=1e-10)
    V = wilson.volume(dims)
    levels = mg.build_hierarchy(U, dims, mass, csw, params,
                                _init_vecs([dims], [12], [4], 77))
    b = synth.gaussian_field(V, 12, 3, 2001)
    x, hist = mg.solve(levels, b, params)
    r = b - levels[0].apply(x)
    assert np.all(krylov.norms(r) / krylov.norms(b) <= 1e-10)
    C = wilson.clover_term(U, dims, csw)
    Dd = wilson.dense_D(U, C, dims, mass)
    xd = np.linalg.solve(Dd, b.reshape(-1, 3)).reshape(V, 12, 3)
    cond = np.linalg.cond(Dd)
    err = krylov.norms(x - xd) / krylov.norms(xd)
    assert np.all(err <= cond * 1e-10)


def test_free_field_solve_by_fft():
    """P8: on U = 1, D^{-1} b is diagonal in momentum space (4x4 D(p)^{-1})."""
    dims = (8, 8, 8, 8)
    mass, csw = 0.05, 1.0
    U = synth.gauge_unit(dims)
    V = wilson.volume(dims)
    params = mg.MGParams(blocks=[(4, 4, 4, 4)], nvec=[6], setup_sweeps=3, setup_m=8,
                         smooth_m=4, coarse_m=16, coarse_cycles=2, outer_m=8, tol=1e-10)
    levels = mg.build_hierarchy(U, dims, mass, csw, params,
                                _init_vecs([dims], [12], [6], 5))
    b = synth.gaussian_field(V, 12, 2, 9)
    x, _ = mg.solve(levels, b, params)
    # closed form: twist the antiperiodic time direction, FFT, invert D(p), back
    Lx, Ly, Lz, Lt = dims
    t = synth.site_coords(np.arange(V), dims)[:, 3]
    tw = np.exp(1j * np.pi * t / Lt)
    bg = (b / tw[:, None, None]).reshape(Lt, Lz, Ly, Lx, 4, 3, 2)
    bk = np.fft.fftn(bg, axes=(0, 1, 2, 3))
    kt = 2 * np.pi * np.fft.fftfreq(Lt) + np.pi / Lt
    kz = 2 * np.pi * np.fft.fftfreq(Lz)
    ky = 2 * np.pi * np.fft.fftfreq(Ly)
    kx = 2 * np.pi * np.fft.fftfreq(Lx)
    P = np.stack(np.meshgrid(kt, kz, ky, kx, indexing="ij"), axis=-1)  # (.., [t,z,y,x])
    p = P[..., ::-1]  # -> (px, py, pz, pt)
    Dp = (4 + mass - np.cos(p).sum(-1))[..., None, None] * np.eye(4)
    for mu in range(4):
        Dp = Dp + 1j * np.sin(p[..., mu])[..., None, None] * cv.GAMMA[mu]
    xk = np.einsum("...st,...tan->...san", np.linalg.inv(Dp), bk)
    xg = np.fft.ifftn(xk, axes=(0, 1, 2, 3)).reshape(V, 12, 2) * tw[:, None, None]
    err = krylov.norms(x - xg) / krylov.norms(xg)
    assert np.all(err < 1e-8)


def test_mrhs_solve_equals_per_rhs():
    """P9: the n-RHS solve is n independent solves."""
    dims = (4, 4, 4, 4)
    U, mass, csw = _problem(dims, 1001)
    params = mg.MGParams(blocks=[(2, 2, 2, 2)], nvec=[4], setup_sweeps=2, setup_m=6,
                         smooth_m=3, coarse_m=8, coarse_cycles=1, outer_m=6, tol=1e-10)
    V = wilson.volume(dims)
    levels = mg.build_hierarchy(U, dims, mass, csw, params, _init_vecs([dims], [12], [4], 3))
    b = synth.gaussian_field(V, 12, 3, 4)
    pre = lambda v: mg.vcycle(levels, 0, v, params)  # noqa: E731
    # a fixed number of cycles so both runs do identical work
    r = b.copy()
    x_all = krylov.arnoldi_correction(levels[0].apply, r, 6, pre)
    for k in range(3):
        xk = krylov.arnoldi_correction(levels[0].apply, r[:, :, k:k + 1], 6, pre)
        assert np.abs(xk[:, :, 0] - x_all[:, :, k]).max() < 1e-12 * np.abs(xk).max()


def test_setup_relaxation_lowers_rayleigh_quotient():
    dims = (4, 4, 4, 4)
    U, mass, csw = _problem(dims, 17)
    C = wilson.clover_term(U, dims, csw)
    A = lambda v: wilson.apply_D(U, C, v, dims, mass)  # noqa: E731
    V = wilson.volume(dims)
    v0 = synth.gaussian_field(V, 12, 4, 1)
    v = mg.setup_nullvecs(A, v0, sweeps=4, m=8)
    q0 = krylov.norms(A(v0)) / krylov.norms(v0)
    q1 = krylov.norms(A(v)) / krylov.norms(v)
    assert np.all(q1 < 0.3 * q0)
    assert np.allclose(krylov.norms(v), 1.0)


def test_three_level_solve():
    """3-level MG-FGMRES reaches 1e-10 (intermediate FGMRES + coarsest GMRES)."""
    dims = (8, 4, 4, 8)
    U, mass, csw = _problem(dims, 1301, eps=0.3, mass=-0.1)
    params = mg.MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[4, 4], setup_sweeps=3,
                         setup_m=6, smooth_m=4, coarse_m=10, coarse_cycles=2, inter_m=4,
                         outer_m=8, tol=1e-10)
    V = wilson.volume(dims)
    d1 = coarse.coarse_dims(dims, (2, 2, 2, 2))
    levels = mg.build_hierarchy(U, dims, mass, csw, params,
                                _init_vecs([dims, d1], [12, 8], [4, 4], 50))
    assert len(levels) == 3 and levels[2].dims == (2, 1, 1, 2)
    b = synth.gaussian_field(V, 12, 2, 2301)
    x, hist = mg.solve(levels, b, params)
    r = b - levels[0].apply(x)
    assert np.all(krylov.norms(r) / krylov.norms(b) <= 1e-10)
