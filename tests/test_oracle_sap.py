"""Pins of the SAP oracle (oracle/sap.py) against dense linear algebra.

The block systems D_BB are cut out of the full matrix of D (wilson.dense_D)
by row and column index, an independent path from the oracle's masked
whole-lattice applications; planted mistakes (a site checkerboard instead of
the block one, one MR step size for all blocks, a missing residual update
between the colours) must fail them.
"""
import importlib.util
import os

import numpy as np
import pytest

import synth
from oracle import sap, wilson

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
DIMS, BLOCK = (4, 4, 2, 4), (2, 2, 1, 2)


def _problem(dims=DIMS, mass=-0.2, csw=1.0, seed=31):
    U = synth.gauge_haar(dims, seed)
    clover = wilson.clover_term(U, dims, csw)
    D = wilson.dense_D(U, clover, dims, mass)

    def apply_D(psi):
        return wilson.apply_D(U, clover, psi, dims, mass)

    return apply_D, D


def _block_sites(dims, B):
    """Site lists of every block, from explicit coordinates."""
    Lx, Ly, Lz, Lt = dims
    out = {}
    for s in range(wilson.volume(dims)):
        x, y, z, t = s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)
        key = (x // B[0], y // B[1], z // B[2], t // B[3])
        out.setdefault(key, []).append(s)
    return out


def _rows(sites):
    return (12 * np.asarray(sites)[:, None] + np.arange(12)[None, :]).reshape(-1)


def test_blocks_of_one_colour_never_touch():
    """Every hop between two different blocks joins blocks of opposite colour."""
    for dims, B in ((DIMS, BLOCK), ((4, 4, 4, 8), (2, 2, 2, 4)), ((8, 4, 4, 4), (4, 2, 1, 2))):
        color = sap.block_color(dims, B)
        bid = sap.block_index(dims, B)
        Lx, Ly, Lz, Lt = dims
        stride = (1, Lx, Lx * Ly, Lx * Ly * Lz)
        for s in range(wilson.volume(dims)):
            c = (s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz))
            for mu in range(4):
                nb = s + stride[mu] if c[mu] < dims[mu] - 1 else s - stride[mu] * (dims[mu] - 1)
                if bid[nb] != bid[s]:
                    assert color[nb] != color[s]
                else:
                    assert color[nb] == color[s]
    with pytest.raises(ValueError):
        sap.block_color((6, 4, 4, 4), (2, 2, 2, 2))   # three blocks along x


def test_block_index_matches_coordinates():
    bid = sap.block_index(DIMS, BLOCK)
    for sites in _block_sites(DIMS, BLOCK).values():
        assert len(set(bid[sites])) == 1
    assert len(set(bid)) == len(_block_sites(DIMS, BLOCK))


def _one_mr_step_error(mod):
    """One MR step on every colour-0 block against the closed form
    e_B = alpha_B r_B, alpha_B = <D_BB r_B, r_B> / |D_BB r_B|^2 (dense blocks)."""
    apply_D, D = _problem()
    V = wilson.volume(DIMS)
    r = synth.gaussian_field(V, 12, 3, 32)
    color = mod.block_color(DIMS, BLOCK)
    bid = mod.block_index(DIMS, BLOCK)
    e = mod.block_mr(apply_D, r, (color == 0).astype(float), bid, int(bid.max()) + 1, 1)
    ref = np.zeros_like(r)
    for sites in _block_sites(DIMS, BLOCK).values():
        if sap.block_color(DIMS, BLOCK)[sites[0]] != 0:
            continue
        rows = _rows(sites)
        DBB = D[np.ix_(rows, rows)]
        rB = r[sites].reshape(-1, 3)
        qB = DBB @ rB
        alpha = np.einsum("ir,ir->r", np.conj(qB), rB) / np.einsum("ir,ir->r", np.conj(qB), qB).real
        ref[sites] = (alpha[None, :] * rB).reshape(len(sites), 12, 3)
    return np.abs(e - ref).max() / np.abs(ref).max()


def _block_solve_error(mod, steps=60):
    """Many MR steps converge to the exact block solves D_BB^{-1} r_B on the
    colour-1 blocks and leave the colour-0 sites untouched."""
    apply_D, D = _problem(mass=0.6)
    V = wilson.volume(DIMS)
    r = synth.gaussian_field(V, 12, 2, 33)
    color = mod.block_color(DIMS, BLOCK)
    bid = mod.block_index(DIMS, BLOCK)
    e = mod.block_mr(apply_D, r, (color == 1).astype(float), bid, int(bid.max()) + 1, steps)
    ref = np.zeros_like(r)
    for sites in _block_sites(DIMS, BLOCK).values():
        if sap.block_color(DIMS, BLOCK)[sites[0]] != 1:
            continue
        rows = _rows(sites)
        ref[sites] = np.linalg.solve(D[np.ix_(rows, rows)], r[sites].reshape(-1, 2)).reshape(len(sites), 12, 2)
    return np.abs(e - ref).max() / np.abs(ref).max()


def _sap_solve_error(mod, cycles=40):
    """SAP as a stationary iteration converges to D^{-1} v (dense solve)."""
    apply_D, D = _problem(mass=0.6)
    V = wilson.volume(DIMS)
    v = synth.gaussian_field(V, 12, 2, 34)
    z = mod.sap_smooth(apply_D, v, np.zeros_like(v), DIMS, BLOCK, cycles, 6)
    ref = np.linalg.solve(D, v.reshape(-1, 2)).reshape(v.shape)
    return np.abs(z - ref).max() / np.abs(ref).max()


def test_one_mr_step_is_the_closed_form():
    assert _one_mr_step_error(sap) < 1e-13


def test_mr_converges_to_the_dense_block_solves():
    assert _block_solve_error(sap) < 1e-10


def test_sap_iteration_converges_to_the_dense_solution():
    assert _sap_solve_error(sap) < 1e-9


def test_exact_block_solves_zero_the_residual_on_that_colour():
    """Multiplicative Schwarz: after the colour-c half sweep with exact block
    solves, b - D z vanishes on every colour-c site."""
    apply_D, D = _problem(mass=0.6)
    V = wilson.volume(DIMS)
    v = synth.gaussian_field(V, 12, 2, 35)
    color = sap.block_color(DIMS, BLOCK)
    bid = sap.block_index(DIMS, BLOCK)
    z = synth.gaussian_field(V, 12, 2, 36)
    for c in (0, 1):
        mask = (color == c).astype(float)
        z = z + sap.block_mr(apply_D, v - apply_D(z), mask, bid, int(bid.max()) + 1, 60)
        res = v - apply_D(z)
        assert np.abs(res[color == c]).max() < 1e-9 * np.abs(v).max()
        assert np.abs(res[color != c]).max() > 1e-3


def test_mrhs_equals_per_rhs():
    apply_D, _ = _problem()
    V = wilson.volume(DIMS)
    v = synth.gaussian_field(V, 12, 3, 37)
    z0 = synth.gaussian_field(V, 12, 3, 38)
    z = sap.sap_smooth(apply_D, v, z0, DIMS, BLOCK, 2, 3)
    for r in range(3):
        zr = sap.sap_smooth(apply_D, v[..., r:r + 1], z0[..., r:r + 1], DIMS, BLOCK, 2, 3)
        assert np.abs(z[..., r:r + 1] - zr).max() < 1e-13 * np.abs(z).max()


def _mutant(old, new):
    path = os.path.join(ORACLE, "sap.py")
    src = open(path).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    spec = importlib.util.spec_from_loader("oracle._mutant_sap", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), path, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new,pin", [
    # site checkerboard instead of block colours
    ("return (site_coords(dims) // np.asarray(B)).sum(axis=1) % 2", "return site_coords(dims).sum(axis=1) % 2",
     "solve"),
    # one step size for all blocks (global instead of block-local inner products)
    ("a_site = alpha[bid][:, None, :]", "a_site = (qr.sum(0) / qq.sum(0))[None, None, :]", "one_step"),
    # residual not refreshed between the two colours
    ("            r = v - apply_D(z)\n", "            r = v - apply_D(z) if c == 0 else r\n", "sap"),
    # conjugate on the wrong side of the MR step size
    ('per_site = np.einsum("vir,vir->vr", np.conj(a), b)', 'per_site = np.einsum("vir,vir->vr", a, np.conj(b))',
     "one_step"),
])
def test_planted_mistakes_are_caught(old, new, pin):
    mod = _mutant(old, new)
    if pin == "one_step":
        assert _one_mr_step_error(mod) > 1e-6
    elif pin == "solve":
        assert _block_solve_error(mod) > 1e-6
    else:
        assert _sap_solve_error(mod, 6) > 10 * _sap_solve_error(sap, 6)


def test_mg_solve_with_sap_smoother_matches_dense_solve():
    """The 2-level MG-FGMRES with SAP post-smoothing reaches 1e-10 and equals
    the dense solve (within the condition number times the tolerance)."""
    from oracle import krylov, mg

    dims = (4, 4, 4, 4)
    U = synth.gauge_exp(dims, 0.4, 1001)
    mass, csw = -0.2, 1.0
    params = mg.MGParams(blocks=[(2, 2, 2, 2)], nvec=[4], setup_sweeps=3, setup_m=6, coarse_m=12,
                         coarse_cycles=2, outer_m=8, tol=1e-10, smoother_sap=True, sap_block=(2, 2, 2, 2),
                         sap_cycles=1, sap_mr=3)
    V = wilson.volume(dims)
    levels = mg.build_hierarchy(U, dims, mass, csw, params, [synth.gaussian_field(V, 12, 4, 77)])
    b = synth.gaussian_field(V, 12, 2, 2001)
    x, hist = mg.solve(levels, b, params)
    assert np.all(krylov.norms(b - levels[0].apply(x)) / krylov.norms(b) <= 1e-10)
    Dd = wilson.dense_D(U, wilson.clover_term(U, dims, csw), dims, mass)
    xd = np.linalg.solve(Dd, b.reshape(-1, 2)).reshape(V, 12, 2)
    assert np.all(krylov.norms(x - xd) / krylov.norms(xd) <= np.linalg.cond(Dd) * 1e-10)
