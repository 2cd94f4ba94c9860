"""Pins of the coarse even-odd oracle (Sec. 6, coarse M_eooe) against dense
linear algebra on a Galerkin coarse operator with coarse extent 2 (the +mu and
-mu neighbours coincide, and both have the other parity).

* The Schur complement applied column by column equals
  D_oo - D_oe D_ee^{-1} D_eo of the dense D_c permuted to (even, odd) order.
* Solving D_hat x_o = b_hat densely and reconstructing x_e gives
  numpy.linalg.solve(D_c, b).
* D_hat inherits the coarse gamma_5-hermiticity: G5 D_hat G5 = D_hat^H with
  G5 = diag(1_N, -1_N) per site.
* Planted mistakes (sign of the hop term, transposed self-block inverse,
  swapped parities in the reconstruction) fail these pins.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

import synth
from oracle import coarse, coarse_evenodd as ceo, evenodd, wilson
from oracle.conventions import FINE_CHIRALITY


def _operator():
    dims, block, N = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = synth.gauge_exp(dims, 0.4, 8101)
    V = wilson.volume(dims)
    P = coarse.build_prolongator(synth.gaussian_field(V, 12, N, 8102), dims, block, FINE_CHIRALITY)
    A = coarse.galerkin_fine(U, wilson.clover_term(U, dims, 1.0), P, dims, block, -0.2)
    return A, coarse.coarse_dims(dims, block), 2 * N


def _blocks(A, cd, nc):
    D = coarse.dense_coarse(A, cd)
    e = (evenodd.cb_sites(cd, 0)[:, None] * nc + np.arange(nc)).ravel()
    o = (evenodd.cb_sites(cd, 1)[:, None] * nc + np.arange(nc)).ravel()
    return D, e, o


def schur_error(mod=ceo):
    A, cd, nc = _operator()
    D, e, o = _blocks(A, cd, nc)
    S = D[np.ix_(o, o)] - D[np.ix_(o, e)] @ np.linalg.solve(D[np.ix_(e, e)], D[np.ix_(e, o)])
    V2 = wilson.volume(cd) // 2
    cols = np.eye(V2 * nc, dtype=np.complex128).reshape(V2, nc, V2 * nc)
    got = mod.schur_apply(A, cols, cd).reshape(V2 * nc, V2 * nc)
    return float(np.abs(got - S).max() / np.abs(S).max())


def solve_error(mod=ceo):
    A, cd, nc = _operator()
    D, e, o = _blocks(A, cd, nc)
    Vc = wilson.volume(cd)
    b = synth.gaussian_field(Vc, nc, 2, 8103)
    V2 = Vc // 2
    cols = np.eye(V2 * nc, dtype=np.complex128).reshape(V2, nc, V2 * nc)
    S = mod.schur_apply(A, cols, cd).reshape(V2 * nc, V2 * nc)
    xo = np.linalg.solve(S, mod.schur_rhs(A, b, cd).reshape(V2 * nc, 2)).reshape(V2, nc, 2)
    x = mod.schur_reconstruct(A, b, xo, cd)
    xd = np.linalg.solve(D, b.reshape(-1, 2)).reshape(x.shape)
    return float(np.abs(x - xd).max() / np.abs(xd).max())


def test_schur_complement_equals_dense():
    assert schur_error() < 1e-12


def test_schur_solve_and_reconstruction_equal_dense_solve():
    assert solve_error() < 1e-10


def test_schur_complement_is_gamma5_hermitian():
    A, cd, nc = _operator()
    V2 = wilson.volume(cd) // 2
    cols = np.eye(V2 * nc, dtype=np.complex128).reshape(V2, nc, V2 * nc)
    S = ceo.schur_apply(A, cols, cd).reshape(V2 * nc, V2 * nc)
    g5 = np.tile(np.concatenate([np.ones(nc // 2), -np.ones(nc // 2)]), V2)
    assert np.abs(g5[:, None] * S * g5[None, :] - S.conj().T).max() < 1e-12 * np.abs(S).max()


def test_rejects_odd_coarse_extents():
    with pytest.raises(ValueError):
        ceo.check_dims((3, 2, 2, 2))


ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def _mutant(old, new):
    path = os.path.join(ORACLE, "coarse_evenodd.py")
    src = open(path).read()
    assert src.count(old) >= 1, old
    name = "oracle._mutant_coarse_evenodd"
    spec = importlib.util.spec_from_loader(name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    sys.modules[name] = mod
    exec(compile(src.replace(old, new, 1), path, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new,pin", [
    ("return apply_blocks(A_oo, phi_o) - hop_between(A, t_e, cdims, 1)",
     "return apply_blocks(A_oo, phi_o) + hop_between(A, t_e, cdims, 1)", schur_error),     # hop sign
    ("return np.linalg.inv(A[evenodd.cb_sites(cdims, p), 0])",
     "return np.linalg.inv(np.swapaxes(A[evenodd.cb_sites(cdims, p), 0], 1, 2))", schur_error),  # transposed
    ("x_e = apply_blocks(self_block_inverse(A, cdims, 0),",
     "x_e = apply_blocks(self_block_inverse(A, cdims, 1),", solve_error),                 # wrong parity
    ("return evenodd.to_half(b, cdims, 1) - hop_between(A, t_e, cdims, 1)",
     "return evenodd.to_half(b, cdims, 1) + hop_between(A, t_e, cdims, 1)", solve_error),  # rhs sign
])
def test_pins_catch_planted_mistakes(old, new, pin):
    assert pin() < 1e-10
    assert pin(_mutant(old, new)) > 1e-6
