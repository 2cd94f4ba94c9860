"""Pins of the even-odd oracle (oracle/evenodd.py) against the dense full operator.

The Schur complement, its right-hand side and the reconstruction are checked
against dense linear algebra on the full matrix of D (wilson.dense_D, permuted
into even/odd blocks), an independent path; planted mistakes (a wrong factor
or sign in D_hat, the right-hand side or the reconstruction) must fail them.
"""
import importlib.util
import os

import numpy as np
import pytest

import synth
from oracle import evenodd as eo
from oracle import wilson

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
CASES = [((2, 2, 2, 4), True, True), ((4, 2, 2, 2), False, True), ((2, 4, 2, 2), True, False)]


def _problem(dims, hot, seed=11):
    U = synth.gauge_haar(dims, seed) if hot else synth.gauge_exp(dims, 0.5, seed)
    return U, wilson.clover_term(U, dims, 1.3)


def _dense_blocks(U, clover, dims, mass, antiperiodic):
    D = wilson.dense_D(U, clover, dims, mass, antiperiodic)
    idx = lambda p: (12 * eo.cb_sites(dims, p)[:, None] + np.arange(12)[None, :]).reshape(-1)
    e, o = idx(0), idx(1)
    return D[np.ix_(e, e)], D[np.ix_(e, o)], D[np.ix_(o, e)], D[np.ix_(o, o)], D


def _schur_error(mod, dims, hot, antiperiodic, mass=-0.4):
    U, clover = _problem(dims, hot)
    Dee, Deo, Doe, Doo, _ = _dense_blocks(U, clover, dims, mass, antiperiodic)
    Dhat = Doo - Doe @ np.linalg.solve(Dee, Deo)
    V2 = wilson.volume(dims) // 2
    psi = synth.gaussian_field(V2, 12, 3, 77)
    got = mod.schur_apply(U, mod.site_matrix(clover, mass), psi, dims, antiperiodic)
    ref = (Dhat @ psi.reshape(-1, 3)).reshape(psi.shape)
    return np.abs(got - ref).max() / np.abs(ref).max()


def _solve_error(mod, dims, hot, antiperiodic, mass=-0.4):
    U, clover = _problem(dims, hot)
    Dee, Deo, Doe, Doo, D = _dense_blocks(U, clover, dims, mass, antiperiodic)
    V = wilson.volume(dims)
    b = synth.gaussian_field(V, 12, 2, 78)
    x_ref = np.linalg.solve(D, b.reshape(-1, 2)).reshape(b.shape)
    C = mod.site_matrix(clover, mass)
    bhat = mod.schur_rhs(U, C, b, dims, antiperiodic)
    Dhat = Doo - Doe @ np.linalg.solve(Dee, Deo)
    x_o = np.linalg.solve(Dhat, bhat.reshape(-1, 2)).reshape(bhat.shape)
    x = mod.schur_reconstruct(U, C, b, x_o, dims, antiperiodic)
    return np.abs(x - x_ref).max() / np.abs(x_ref).max()


@pytest.mark.parametrize("dims,hot,antiperiodic", CASES)
def test_schur_operator_is_the_dense_schur_complement(dims, hot, antiperiodic):
    assert _schur_error(eo, dims, hot, antiperiodic) < 1e-12


@pytest.mark.parametrize("dims,hot,antiperiodic", CASES)
def test_schur_solve_reproduces_the_full_solution(dims, hot, antiperiodic):
    assert _solve_error(eo, dims, hot, antiperiodic) < 1e-11


def test_hopping_term_connects_opposite_parities_only():
    dims = (4, 2, 2, 4)
    U, _ = _problem(dims, True)
    V = wilson.volume(dims)
    for p in (0, 1):
        psi = eo.from_half(synth.gaussian_field(V // 2, 12, 2, 80 + p), dims, p)
        h = wilson.hop_term(U, psi, dims)
        assert np.abs(h[eo.cb_sites(dims, p)]).max() == 0.0
        assert np.abs(h[eo.cb_sites(dims, 1 - p)]).max() > 0.0


def test_checkerboard_numbering_is_half_the_site_index():
    for dims in ((2, 2, 2, 2), (4, 3, 5, 2), (6, 2, 3, 4)):
        V = wilson.volume(dims)
        for p in (0, 1):
            s = eo.cb_sites(dims, p)
            assert np.array_equal(s // 2, np.arange(V // 2))
    with pytest.raises(ValueError):
        eo.cb_sites((3, 2, 2, 2), 0)


def _mutant(old, new):
    path = os.path.join(ORACLE, "evenodd.py")
    src = open(path).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    spec = importlib.util.spec_from_loader("oracle._mutant_evenodd", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), path, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new,pin", [
    ("- 0.25 * hop_between(U, t_e, dims, 1, antiperiodic)", "- 0.5 * hop_between(U, t_e, dims, 1, antiperiodic)",
     "schur"),
    ("- 0.25 * hop_between(U, t_e, dims, 1, antiperiodic)", "+ 0.25 * hop_between(U, t_e, dims, 1, antiperiodic)",
     "schur"),
    ("return to_half(b, dims, 1) + 0.5 * hop_between", "return to_half(b, dims, 1) - 0.5 * hop_between", "solve"),
    ("to_half(b, dims, 0) + 0.5 * hop_between(U, x_o, dims, 0, antiperiodic)",
     "to_half(b, dims, 0) - 0.5 * hop_between(U, x_o, dims, 0, antiperiodic)", "solve"),
    ("return clover + (4.0 + mass) * np.eye(12)", "return clover + (4.0 - mass) * np.eye(12)", "schur"),
])
def test_planted_mistakes_are_caught(old, new, pin):
    mod = _mutant(old, new)
    dims, hot, antiperiodic = CASES[0]
    err = _schur_error(mod, dims, hot, antiperiodic) if pin == "schur" else _solve_error(mod, dims, hot, antiperiodic)
    assert err > 1e-6


def test_evenodd_smoother_in_the_full_krylov_limit_solves_exactly():
    """With as many GMRES steps as odd-site unknowns, the even-odd smoother
    returns delta = D^-1 r (dense solve), so z0 + delta solves D z = v."""
    from oracle import mg as omg

    dims, mass, csw = (2, 2, 2, 4), -0.3, 1.1
    U = synth.gauge_haar(dims, 21)
    clover = wilson.clover_term(U, dims, csw)
    lev = omg.Level(dims, 12, None, None, eo=(U, eo.site_matrix(clover, mass), dims, True))
    V = wilson.volume(dims)
    r = synth.gaussian_field(V, 12, 2, 22)
    delta = omg.evenodd_smooth(lev, r, 12 * V // 2)
    D = wilson.dense_D(U, clover, dims, mass)
    ref = np.linalg.solve(D, r.reshape(-1, 2)).reshape(r.shape)
    assert np.abs(delta - ref).max() / np.abs(ref).max() < 1e-9
