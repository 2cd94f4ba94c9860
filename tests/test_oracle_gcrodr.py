"""Pins of the GCRO-DR oracle (oracle/gcrodr.py).

Checked against independent facts: with no recycle space (k = 0) it is
restarted GMRES(m) (the oracle's GMRES, itself pinned by a dense solve); it
converges to numpy.linalg.solve; its residual never grows from cycle to
cycle; on a diagonal matrix its recycle space converges to the eigenvectors
of the k smallest eigenvalues (closed form: unit vectors); recycling across
a sequence of right-hand sides with one matrix cuts the cycles; an MG solve
with a GCRO-DR coarsest level reaches 1e-10 and the dense solution.  Planted
mistakes (largest instead of smallest harmonic Ritz values, no projection
against C in the Arnoldi steps, no column scaling of U in G) must fail a pin;
one cycle entered with a recycle space must reach the least-squares optimum
over the augmented space, computed here from explicit bases.
"""
import importlib.util
import os

import numpy as np
import pytest

import synth
from oracle import gcrodr, krylov, wilson

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
N = 120


def _matrix(seed=0):
    """Six small outlying eigenvalues (1e-3 .. 1e-2), the rest in [1, 3], complex phases,
    in a random unitary basis."""
    rng = np.random.default_rng(seed)
    lam = np.concatenate([[1e-3, 2e-3, 4e-3, 6e-3, 8e-3, 1e-2], rng.uniform(1, 3, N - 6)])
    lam = lam * np.exp(1j * rng.uniform(-0.3, 0.3, N))
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    bs = [rng.standard_normal(N) + 1j * rng.standard_normal(N) for _ in range(3)]
    return Q @ np.diag(lam) @ Q.conj().T, bs


def test_without_recycling_it_is_restarted_gmres():
    A, bs = _matrix()
    x1, U, h = gcrodr.solve_one(lambda v: A @ v, bs[0], np.zeros(N), 10, 0, 0.0, 3)
    x2 = krylov.gmres(lambda v: A @ v, bs[0][:, None], np.zeros((N, 1)), 10, 3)[:, 0]
    assert U is None and len(h) == 4
    assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x2).max()


def _sequence(mod, k=6, m=20):
    """Solve three RHS with one matrix, recycling; returns cycles per solve and the
    largest error against the dense solution."""
    A, bs = _matrix()
    U, cycles, err = None, [], 0.0
    for b in bs:
        x, U, h = mod.solve_one(lambda v: A @ v, b, np.zeros(N), m, k, 1e-10, 200, U)
        xd = np.linalg.solve(A, b)
        cycles.append(len(h) - 1)
        err = max(err, np.linalg.norm(x - xd) / np.linalg.norm(xd))
        assert all(h[i + 1] <= h[i] * (1 + 1e-9) for i in range(len(h) - 1)), h
    return cycles, err


def test_converges_to_the_dense_solution_with_monotone_residuals():
    cycles, err = _sequence(gcrodr)
    # condition number ~ 3e3: the 1e-10 residual bounds the error by ~3e-7
    assert err <= 3e3 * 1e-10
    assert max(cycles) < 200


def test_recycling_cuts_the_cycles():
    A, bs = _matrix()
    plain = [len(gcrodr.solve_one(lambda v: A @ v, b, np.zeros(N), 20, 0, 1e-10, 200)[2]) - 1 for b in bs]
    cycles, _ = _sequence(gcrodr)
    # deflating the six small eigenvalues: far fewer cycles than GMRES(20), and the
    # recycled space makes every later solve cheaper than the first
    assert max(cycles) * 4 <= min(plain)
    assert cycles[1] < cycles[0] and cycles[2] < cycles[0]


def _ritz_angle(mod):
    """sin of the largest principal angle between the recycle space and the
    eigenvectors of the 4 smallest eigenvalues of a diagonal matrix."""
    d = np.concatenate([[0.01, 0.02, 0.03, 0.04], np.linspace(1, 2, N - 4)])
    rng = np.random.default_rng(5)
    x, U, h = mod.solve_one(lambda v: d * v, rng.standard_normal(N) + 0j, np.zeros(N), 15, 4, 1e-12, 200)
    Qu, _ = np.linalg.qr(U)
    E = np.eye(N)[:, :4]
    return np.linalg.norm(Qu - E @ (E.T @ Qu), 2)


def test_recycle_space_converges_to_the_smallest_eigenvectors():
    assert _ritz_angle(gcrodr) <= 1e-8


def _one_cycle_excess(mod, m=12, k=4):
    """One GCRO-DR cycle entered with a recycle space U must reach the smallest residual
    over x' + span(U, K), K the Krylov space of (I - C C^H) A of dimension m - k from the
    projected residual r' (C = orth(A U)); the optimum is computed here by dense least
    squares on explicit bases.  Returns |r_cycle| / |r_opt| - 1."""
    A, bs = _matrix(7)
    _, U0, _ = mod.solve_one(lambda v: A @ v, bs[0], np.zeros(N), m, k, 1e-6, 100)
    b = bs[1]
    x1, _, h = mod.solve_one(lambda v: A @ v, b, np.zeros(N), m, k, 0.0, 1, U0)
    r_cycle = np.linalg.norm(b - A @ x1)
    C, _ = np.linalg.qr(A @ U0)
    Pc = np.eye(N) - C @ C.conj().T
    rp = Pc @ b                                    # residual after the projection onto C
    K = [rp / np.linalg.norm(rp)]
    for _ in range(m - k - 1):
        K.append(Pc @ (A @ K[-1]))
    Kb, _ = np.linalg.qr(np.stack(K, axis=1))
    S = np.concatenate([U0, Kb], axis=1)
    y = np.linalg.lstsq(A @ S, rp, rcond=None)[0]
    r_opt = np.linalg.norm(rp - A @ S @ y)
    return r_cycle / r_opt - 1.0


def test_one_cycle_minimises_over_the_augmented_space():
    assert abs(_one_cycle_excess(gcrodr)) <= 1e-8


def test_mrhs_equals_per_rhs_and_recycle_spaces_are_per_rhs():
    A, bs = _matrix(3)
    B = np.stack(bs, axis=1)
    apply = lambda f: A @ f
    x, rec, hists = gcrodr.solve(apply, B, np.zeros_like(B), 12, 4, 1e-9, 100)
    assert len(rec) == 3
    for r in range(3):
        xr, Ur, _ = gcrodr.solve_one(lambda v: A @ v, B[:, r], np.zeros(N), 12, 4, 1e-9, 100)
        assert np.abs(x[:, r] - xr).max() <= 1e-13 * np.abs(xr).max()
        assert np.abs(rec[r] - Ur).max() <= 1e-12 * np.abs(Ur).max()


def test_mg_solve_with_gcrodr_coarsest_level_matches_dense_solve():
    from oracle import mg

    dims = (4, 4, 4, 4)
    U = synth.gauge_exp(dims, 0.4, 1001)
    mass, csw = -0.2, 1.0
    params = mg.MGParams(blocks=[(2, 2, 2, 2)], nvec=[4], setup_sweeps=3, setup_m=6, smooth_m=4, coarse_m=8,
                         coarse_cycles=1, outer_m=8, tol=1e-10, coarse_solver="gcrodr", coarse_recycle=3)
    V = wilson.volume(dims)
    levels = mg.build_hierarchy(U, dims, mass, csw, params, [synth.gaussian_field(V, 12, 4, 77)])
    b = synth.gaussian_field(V, 12, 2, 2001)
    x, hist = mg.solve(levels, b, params)
    assert np.all(krylov.norms(b - levels[0].apply(x)) / krylov.norms(b) <= 1e-10)
    assert levels[1].recycle is not None and all(u is not None for u in levels[1].recycle)
    Dd = wilson.dense_D(U, wilson.clover_term(U, dims, csw), dims, mass)
    xd = np.linalg.solve(Dd, b.reshape(-1, 2)).reshape(V, 12, 2)
    assert np.all(krylov.norms(x - xd) / krylov.norms(xd) <= np.linalg.cond(Dd) * 1e-10)


def _mutant(old, new):
    path = os.path.join(ORACLE, "gcrodr.py")
    src = open(path).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    spec = importlib.util.spec_from_loader("oracle._mutant_gcrodr", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new,pin", [
    # largest harmonic Ritz values kept instead of the smallest
    ("return np.argsort(mod, kind=\"stable\")[:k]", "return np.argsort(-np.where(np.isfinite(mod), mod, 0), "
     "kind=\"stable\")[:k]", "ritz"),
    # Arnoldi steps not projected against C
    ("            w = w - C @ B[:, j]\n", "", "cycle"),
    # U columns not scaled in G (identity instead of D)
    ("G[:k, :k] = np.diag(dn)", "G[:k, :k] = np.eye(k)", "cycle"),
])
def test_planted_mistakes_are_caught(old, new, pin):
    mod = _mutant(old, new)
    if pin == "ritz":
        assert _ritz_angle(mod) > 1e-3
    else:
        assert _one_cycle_excess(mod) > 1e-6
