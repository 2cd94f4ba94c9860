"""Planted mistakes in the oracle must be caught by its pins.

Each case rewrites one line of an oracle module in memory (a dropped sign, a
missing dagger, a wrong factor, an off-by-one aggregate face, a transposed
operand), loads the mutant, and checks that the pin it targets now fails.
Nothing on disk changes.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

import synth
from oracle import conventions as cv

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def _mutant(modname, old, new):
    path = os.path.join(ORACLE, modname + ".py")
    src = open(path).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    src = src.replace(old, new, 1)
    name = f"oracle._mutant_{modname}"
    spec = importlib.util.spec_from_loader(name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    # registered so that dataclasses defined in the mutant can resolve their module
    sys.modules[name] = mod
    exec(compile(src, path, "exec"), mod.__dict__)
    return mod


def _plane_wave_error(wilson):
    dims, mass = (4, 4, 2, 4), -0.3
    U = synth.gauge_unit(dims)
    C = wilson.clover_term(U, dims, 1.0)
    V = wilson.volume(dims)
    coords = synth.site_coords(np.arange(V), dims)
    p = np.array([2 * np.pi / 4, 0, 2 * np.pi / 2, 3 * np.pi / 4])
    u = np.random.default_rng(1).standard_normal((4, 3, 1)) + 0j
    phase = np.exp(1j * coords @ p)
    psi = (phase[:, None, None, None] * u[None]).reshape(V, 12, 1)
    Dp = (4 + mass - np.cos(p).sum()) * np.eye(4) + sum(1j * np.sin(p[m]) * cv.GAMMA[m] for m in range(4))
    expect = (phase[:, None, None, None] * np.einsum("st,tan->san", Dp, u)[None]).reshape(V, 12, 1)
    return np.abs(wilson.apply_D(U, C, psi, dims, mass) - expect).max()


def _abelian_error(wilson):
    dims, csw = (3, 4, 2, 2), 1.0
    U = synth.gauge_unit(dims)
    V = wilson.volume(dims)
    y = synth.site_coords(np.arange(V), dims)[:, 1]
    phi = 2 * np.pi / dims[1]
    U[:, 0, 0, 0] = np.exp(-1j * phi * y)
    U[:, 0, 1, 1] = np.exp(1j * phi * y)
    C = wilson.clover_term(U, dims, csw).reshape(V, 4, 3, 4, 3)
    expect = -(csw / 2) * np.sin(phi) * np.einsum("st,ab->satb", cv.sigma_munu(0, 1),
                                                   np.diag([1.0, -1.0, 0.0]))
    return np.abs(C - expect[None]).max()


def _covariance_error(wilson):
    dims = (4, 2, 2, 4)
    U = synth.gauge_haar(dims, 5)
    g = synth.gauge_transform_haar(dims, 6)
    V = wilson.volume(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = wilson.from_grid(wilson.shift(wilson.to_grid(g, dims), mu, +1), dims)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(gp, 1, 2))
    psi = synth.gaussian_field(V, 12, 1, 3)

    def gmul(f):
        return np.einsum("vab,vsbn->vsan", g, f.reshape(V, 4, 3, 1)).reshape(V, 12, 1)

    lhs = wilson.apply_D(Ug, wilson.clover_term(Ug, dims, 1.0), gmul(psi), dims, 0.0)
    rhs = gmul(wilson.apply_D(U, wilson.clover_term(U, dims, 1.0), psi, dims, 0.0))
    return np.abs(lhs - rhs).max()


def _galerkin_error(coarse_mod, wilson):
    dims, block, N = (4, 2, 2, 4), (2, 1, 2, 2), 2
    U = synth.gauge_exp(dims, 0.5, 21)
    C = wilson.clover_term(U, dims, 1.0)
    V = wilson.volume(dims)
    P = coarse_mod.build_prolongator(synth.gaussian_field(V, 12, N, 31), dims, block, cv.FINE_CHIRALITY)
    A = coarse_mod.galerkin_fine(U, C, P, dims, block, -0.1)
    Dd = wilson.dense_D(U, C, dims, -0.1)
    Pd = coarse_mod.dense_prolongator(P, dims, block)
    return np.abs(Pd.conj().T @ Dd @ Pd - coarse_mod.dense_coarse(A, coarse_mod.coarse_dims(dims, block))).max()


WILSON_MUTANTS = [
    # (old, new, pin)
    ("nb[Lt - 1] *= -1.0", "nb[Lt - 1] *= 1.0", _plane_wave_error),           # lost antiperiodic sign
    ("out += t - np.einsum", "out += t + np.einsum", _plane_wave_error),       # (1+gamma) on the forward hop
    ('np.einsum("...ba,...sbn->...san", np.conj(link), nb)',
     'np.einsum("...ab,...sbn->...san", link, nb)', _covariance_error),         # missing dagger
    ("out -= 0.5 * hop_term", "out -= 0.25 * hop_term", _plane_wave_error),    # wrong hop factor
    ("(4.0 + mass) * psi + np", "(4.0 - mass) * psi + np", _plane_wave_error),  # mass sign
    ("(csw * 0.5j * C)", "(csw * 0.25j * C)", _abelian_error),                 # clover normalisation
    ("(Q - dag(Q)) / 8.0, dims)", "(Q + dag(Q)) / 8.0, dims)", _abelian_error),  # F not anti-Hermitian
    ("leaf2 = Un @ dag(Um_xmmpn)", "leaf2 = Un @ (Um_xmmpn)", _covariance_error),  # leaf orientation
]


@pytest.mark.parametrize("old,new,pin", WILSON_MUTANTS)
def test_wilson_pins_catch_planted_mistakes(old, new, pin):
    from oracle import wilson
    assert pin(wilson) < 1e-12
    mutant = _mutant("wilson", old, new)
    assert pin(mutant) > 1e-6


COARSE_MUTANTS = [
    ('np.einsum("vadk,vadr->vkr", np.conj(P[sites]), psi[sites])',
     'np.einsum("vadk,vadr->vkr", P[sites], psi[sites])'),                     # R without conj
    ("return loc == (block[mu] - 1) if sign > 0 else loc == 0",
     "return loc == 0 if sign > 0 else loc == (block[mu] - 1)"),               # wrong face
    ("A[:, d] = restrict(P, np.where(cross, H, 0), dims, block)",
     "A[:, 9 - d if d > 0 else 0] = restrict(P, np.where(cross, H, 0), dims, block)"),  # +mu/-mu swap
    ('out = np.einsum("vkl,vlr->vkr", A[:, 0], phi)',
     'out = np.einsum("vlk,vlr->vkr", A[:, 0], phi)'),                         # transposed block
]


@pytest.mark.parametrize("old,new", COARSE_MUTANTS)
def test_coarse_pins_catch_planted_mistakes(old, new):
    from oracle import coarse, wilson
    assert _galerkin_error(coarse, wilson) < 1e-11
    mutant = _mutant("coarse", old, new)
    assert _galerkin_error(mutant, wilson) > 1e-6


def _pin_or_inf(fn, mod):
    """A mutant that makes the oracle raise (e.g. a shape mismatch) is caught too."""
    try:
        return fn(mod)
    except (ValueError, IndexError):
        return float("inf")


def _mg_pins():
    from tests import test_oracle_vcycle as tv
    return {
        "two_level": tv.two_level_error,
        "evenodd": lambda m: tv.two_level_error(m, evenodd_smoother=True),
        "three_level": tv.three_level_error,
        "identity": tv.identity_prolongator_error,
        "setup_cycle": tv.setup_cycle_error,
        "hierarchy_setup": tv.hierarchy_setup_error,
    }


MG_MUTANTS = [
    # (old, new, pin): the V-cycle and the setup of oracle/mg.py
    ("z0 = coarse.prolong(lev.P, e, lev.dims, lev.block)",
     "z0 = 0 * coarse.prolong(lev.P, e, lev.dims, lev.block)", "two_level"),          # dropped coarse correction
    ("return krylov.gmres(lev.apply, v, z0, params.smooth_m, 1)",
     "return z0 + krylov.gmres(lev.apply, v, 0 * z0, params.smooth_m, 1)", "two_level"),  # smoothing from 0
    ("z0 = coarse.prolong(lev.P, e, lev.dims, lev.block)",
     "z0 = coarse.prolong(np.conj(lev.P), e, lev.dims, lev.block)", "identity"),     # prolongation with conj(P)
    ("c = coarse.restrict(lev.P, v, lev.dims, lev.block)",
     "c = coarse.restrict(levels[0].P, v, levels[0].dims, levels[0].block)", "three_level"),  # wrong level's P
    ("lambda u: vcycle(levels, l + 1, u, params)", "lambda u: u", "three_level"),    # no intermediate V-cycle
    ("return z0 + evenodd_smooth(lev, v - lev.apply(z0), params.smooth_m)",
     "return z0 + evenodd_smooth(lev, v, params.smooth_m)", "evenodd"),              # stale residual
    ("v = krylov.gmres(apply_A, zero, v, m, 1)",
     "v = krylov.gmres(apply_A, v, v, m, 1)", "setup_cycle"),                        # relaxes A v = v
    ("vecs = setup_nullvecs(lev.apply, init_vecs[l]",
     "vecs = setup_nullvecs(lambda f: lev.apply(f) - np.einsum('vij,vjn->vin', clover, f), init_vecs[l]",
     "hierarchy_setup"),                                                             # D without the clover
]


@pytest.mark.parametrize("old,new,pin", MG_MUTANTS)
def test_mg_pins_catch_planted_mistakes(old, new, pin):
    from oracle import mg
    fn = _mg_pins()[pin]
    assert fn(mg) < 1e-9
    mutant = _mutant("mg", old, new)
    assert _pin_or_inf(fn, mutant) > 1e-6
