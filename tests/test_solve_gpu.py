"""GPU solve: MG-preconditioned mixed-precision FGMRES (Sec. 8) to a true
FP64 relative residual of 1e-10, checked with the oracle's own D.

The solution is unique, so it is compared with the oracle's FP64 MG-FGMRES
solution within the accuracy both residuals allow; the n-RHS solve is
compared with n single-RHS solves (MRHS = per-RHS).
"""
import numpy as np
import pytest

import synth
from oracle import krylov, mg as omg, wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, to_dev, to_host

pytestmark = pytest.mark.gpu

# 8^4 lattice, antiperiodic t, exp(i 0.4 H), m = -0.2, c_sw = 1, 2 levels with
# 4^4 aggregates and 8 chirally split null vectors, 4 Gaussian sources.
DIMS, MASS, CSW, NRHS = (8, 8, 8, 8), -0.2, 1.0, 4
BLOCKS, NVEC = [(4, 4, 4, 4)], [8]


@pytest.fixture(scope="module")
def problem():
    U = synth.gauge_exp(DIMS, 0.4, 1001)
    V = wilson.volume(DIMS)
    b = synth.gaussian_field(V, 12, NRHS, 2001)
    v0 = synth.gaussian_field(V, 12, NVEC[0], 3001)
    return U, b, v0


def _gpu_solve(U, b, v0, nrhs_list, **over):
    params = dict(n_levels=2, blocks=BLOCKS, nvec=NVEC, setup_sweeps=4, setup_m=8, smooth_m=4,
                  coarse_m=16, coarse_cycles=2, inner_m=8, inner_tol=1e-5, outer_m=4, max_outer_iters=30,
                  max_rhs=NRHS, coarse_precision=mrhs.MRHS_FP32)
    params.update(over)
    lat = make_lattice(U, DIMS, MASS, CSW)
    mg = make_mg(lat, params, [v0])
    outs = []
    try:
        for cols in nrhs_list:
            bb = np.ascontiguousarray(b[:, :, cols])
            d_b = to_dev(bb)
            d_x = to_dev(np.zeros_like(bb))
            rel = np.zeros(len(cols))
            status, st = mrhs.mrhs_solve(mg, d_b, d_x, len(cols), 1e-10, rel)
            outs.append((to_host(d_x), rel, st))
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
    return outs


def test_solve_true_residual_and_oracle_solution(problem):
    U, b, v0 = problem
    (x, rel, st), = _gpu_solve(U, b, v0, [list(range(NRHS))])
    C = wilson.clover_term(U, DIMS, CSW)
    r = b - wilson.apply_D(U, C, x, DIMS, MASS)
    true_rel = krylov.norms(r) / krylov.norms(b)
    assert np.all(true_rel <= 1e-10), true_rel
    assert np.allclose(rel, true_rel, rtol=1e-3, atol=1e-13)
    assert st.outer_iters >= 1 and st.vcycles >= 1
    # the oracle's own FP64 MG-FGMRES solution of the same system
    op = omg.MGParams(blocks=BLOCKS, nvec=NVEC, setup_sweeps=2, setup_m=8, smooth_m=4, coarse_m=16,
                      coarse_cycles=2, outer_m=8, tol=1e-11)
    levels = omg.build_hierarchy(U, DIMS, MASS, CSW, op, [v0])
    xo, _ = omg.solve(levels, b, op)
    err = krylov.norms(x - xo) / krylov.norms(xo)
    assert np.all(err <= 1e-6), err


def test_outer_operator_precisions_agree(problem):
    """Outer Arnoldi applies in float-float (default) or FP64: both reach the
    FP64 true residual, and their solutions agree within what it allows."""
    U, b, v0 = problem
    C = wilson.clover_term(U, DIMS, CSW)
    xs = []
    for prec in (mrhs.MRHS_DF64, mrhs.MRHS_FP64):
        (x, rel, st), = _gpu_solve(U, b, v0, [list(range(NRHS))], outer_op_precision=prec)
        r = b - wilson.apply_D(U, C, x, DIMS, MASS)
        assert np.all(krylov.norms(r) / krylov.norms(b) <= 1e-10)
        xs.append(x)
    err = krylov.norms(xs[0] - xs[1]) / krylov.norms(xs[1])
    assert np.all(err <= 1e-7), err


def test_evenodd_smoother_solve(problem):
    """With the even-odd post-smoother the solve still reaches the FP64 true
    residual, and its solution agrees with the default smoother's."""
    U, b, v0 = problem
    C = wilson.clover_term(U, DIMS, CSW)
    xs = []
    for eo in (1, 0):
        (x, rel, st), = _gpu_solve(U, b, v0, [list(range(NRHS))], smoother_evenodd=eo)
        r = b - wilson.apply_D(U, C, x, DIMS, MASS)
        assert np.all(krylov.norms(r) / krylov.norms(b) <= 1e-10)
        xs.append(x)
    err = krylov.norms(xs[0] - xs[1]) / krylov.norms(xs[1])
    assert np.all(err <= 1e-7), err


def test_nonzero_start_vector(problem):
    """A nonzero initial x takes the FP64 residual path (no zero-start shortcut)."""
    U, b, v0 = problem
    params = dict(n_levels=2, blocks=BLOCKS, nvec=NVEC, setup_sweeps=4, max_rhs=NRHS,
                  coarse_precision=mrhs.MRHS_FP32)
    lat = make_lattice(U, DIMS, MASS, CSW)
    mg = make_mg(lat, params, [v0])
    try:
        d_b = to_dev(b)
        x0 = np.zeros_like(b)
        x0[5, 3, 1] = 1e-3   # a single nonzero entry in one RHS column
        d_x = to_dev(x0)
        rel = np.zeros(NRHS)
        mrhs.mrhs_solve(mg, d_b, d_x, NRHS, 1e-10, rel)
        x = to_host(d_x)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
    C = wilson.clover_term(U, DIMS, CSW)
    r = b - wilson.apply_D(U, C, x, DIMS, MASS)
    assert np.all(krylov.norms(r) / krylov.norms(b) <= 1e-10)


def test_mrhs_equals_single_rhs(problem):
    U, b, v0 = problem
    outs = _gpu_solve(U, b, v0, [list(range(NRHS)), [0], [3]])
    x_all = outs[0][0]
    for (x1, rel, _), col in zip(outs[1:], (0, 3)):
        assert rel[0] <= 1e-10
        err = np.linalg.norm(x1[:, :, 0] - x_all[:, :, col]) / np.linalg.norm(x_all[:, :, col])
        assert err <= 1e-7, err


def test_solve_rejects_bad_arguments(problem):
    U, b, v0 = problem
    lat = make_lattice(U, DIMS, MASS, CSW)
    mg = make_mg(lat, dict(n_levels=2, blocks=BLOCKS, nvec=NVEC, setup_sweeps=0, max_rhs=2,
                           coarse_precision=mrhs.MRHS_FP32), [v0])
    try:
        d_b = to_dev(np.ascontiguousarray(b[:, :, :3]))
        d_x = to_dev(np.zeros((b.shape[0], 12, 3)))
        with pytest.raises(mrhs.MrhsError) as e:
            mrhs.mrhs_solve(mg, d_b, d_x, 3, 1e-10)
        assert e.value.status == mrhs.MRHS_ERR_INVALID
        with pytest.raises(mrhs.MrhsError):
            mrhs.mrhs_solve(mg, d_b, d_x, 1, 0.0)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)


def test_repeated_solve_is_deterministic(problem):
    """Solving the same system twice with one hierarchy gives the identical x
    (no workspace state leaks from one solve into the next)."""
    U, b, v0 = problem
    outs = _gpu_solve(U, b, v0, [list(range(NRHS)), list(range(NRHS))])
    (x1, r1, s1), (x2, r2, s2) = outs
    assert s1.inner_iters == s2.inner_iters and s1.outer_iters == s2.outer_iters
    assert np.array_equal(x1, x2)


def test_not_converged_returns_the_partial_solution(problem):
    """An outer iteration cap below what the tolerance needs: the solve returns
    MRHS_ERR_NOT_CONVERGED with x holding the iterate reached and rel its true
    FP64 relative residual (failure detection by status, not by abort)."""
    U, b, v0 = problem
    params = dict(n_levels=2, blocks=BLOCKS, nvec=NVEC, setup_sweeps=4, setup_m=8, smooth_m=4, coarse_m=16,
                  coarse_cycles=2, inner_m=8, inner_tol=1e-5, outer_m=4, max_outer_iters=1, max_rhs=NRHS,
                  coarse_precision=mrhs.MRHS_FP32)
    lat = make_lattice(U, DIMS, MASS, CSW)
    mg = make_mg(lat, params, [v0])
    try:
        d_b, d_x = to_dev(b), to_dev(np.zeros_like(b))
        rel = np.zeros(NRHS)
        status, st = mrhs.mrhs_solve(mg, d_b, d_x, NRHS, 1e-14, rel, allow_not_converged=True)
        x = to_host(d_x)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
    assert status == mrhs.MRHS_ERR_NOT_CONVERGED
    assert np.all(np.isfinite(x))
    C = wilson.clover_term(U, DIMS, CSW)
    true_rel = krylov.norms(b - wilson.apply_D(U, C, x, DIMS, MASS)) / krylov.norms(b)
    assert np.all(rel > 1e-14)
    assert np.all(true_rel < 1e-2)     # one outer step, preconditioned by an inner solve to 1e-5
    assert np.allclose(rel, true_rel, rtol=1e-3, atol=1e-13)
