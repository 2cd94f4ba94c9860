"""GPU parity of the SAP smoother (mrhs_sap_smooth) against the FP64 oracle
(oracle/sap.py), and an MG solve that uses it as the fine post-smoother.

Bar: the smoother runs in FP32 (stencil in paired FP32, the MR step sizes
from FP32 block sums of 12 |B| terms per RHS).  Each step size carries a
relative error of a few 1e-6 (sqrt(3072) * 6e-8 for a 4^4 block) and every
MR step and SAP half-sweep passes the previous rounding on; the bar is
max|z_gpu - z_oracle| <= 2e-5 max|z_oracle| for one cycle of one MR step and
1e-4 for two cycles of four MR steps (16 step sizes in a row).
"""
import numpy as np
import pytest

import synth
from oracle import krylov, sap, wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [
    # dims, block, n, t boundary, hot gauge, cycles, MR steps, bar
    ((8, 8, 8, 8), (4, 4, 4, 4), 4, -1, True, 1, 1, 2e-5),
    ((8, 8, 8, 8), (4, 4, 4, 4), 6, -1, True, 2, 4, 1e-4),
    ((8, 8, 4, 8), (2, 4, 2, 4), 2, 1, False, 2, 4, 1e-4),
    ((4, 4, 4, 8), (2, 2, 2, 2), 48, -1, True, 1, 3, 1e-4),
    ((8, 4, 4, 4), (4, 2, 2, 2), 2, -1, True, 1, 0, 0.0),   # no MR step: z unchanged
]


@pytest.mark.parametrize("dims,block,n,tb,hot,cycles,mr,bar", CASES)
def test_sap_smoother_matches_oracle(dims, block, n, tb, hot, cycles, mr, bar):
    mass, csw = -0.2, 1.0
    U = synth.gauge_haar(dims, 5101) if hot else synth.gauge_exp(dims, 0.4, 5101)
    V = wilson.volume(dims)
    v = synth.gaussian_field(V, 12, n, 5201, np.complex64)
    z0 = synth.gaussian_field(V, 12, n, 5202, np.complex64) * 0.1
    lat = make_lattice(U, dims, mass, csw, tb)
    try:
        d_z = to_dev(z0)
        mrhs.mrhs_sap_smooth(lat, to_dev(v), d_z, n, block, cycles, mr)
        got = to_host(d_z).astype(np.complex128)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    clover = wilson.clover_term(U, dims, csw)

    def apply_D(psi):
        return wilson.apply_D(U, clover, psi, dims, mass, antiperiodic=(tb == -1))

    ref = sap.sap_smooth(apply_D, v.astype(np.complex128), z0.astype(np.complex128), dims, block, cycles, mr)
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref).max() / np.abs(ref).max()
    if bar == 0.0:
        assert np.array_equal(got, z0.astype(np.complex128))
    else:
        assert err <= bar, err


def test_sap_rejects_unsupported_arguments():
    dims = (8, 8, 8, 8)
    U = synth.gauge_haar(dims, 5301)
    V = wilson.volume(dims)
    lat = make_lattice(U, dims, -0.2, 1.0)
    try:
        v = to_dev(synth.gaussian_field(V, 12, 4, 5302, np.complex64))
        z = to_dev(np.zeros((V, 12, 4), np.complex64))
        v3 = to_dev(synth.gaussian_field(V, 12, 3, 5303, np.complex64))
        z3 = to_dev(np.zeros((V, 12, 3), np.complex64))
        for args in [(v3, z3, 3, (4, 4, 4, 4)),      # odd RHS count
                     (v, z, 4, (8, 4, 4, 4)),        # one block along x: colours would touch
                     (v, z, 4, (4, 4, 4, 3)),        # extent does not divide
                     (v, z, 4, (4, 4, 8, 8))]:       # 1024 sites per block
            with pytest.raises(mrhs.MrhsError) as e:
                mrhs.mrhs_sap_smooth(lat, args[0], args[1], args[2], args[3], 1, 2)
            assert e.value.status == mrhs.MRHS_ERR_INVALID
    finally:
        mrhs.mrhs_destroy_lattice(lat)


def test_mg_solve_with_sap_smoother():
    """2-level MG-FGMRES with SAP post-smoothing: true FP64 residual <= 1e-10."""
    dims, mass, csw, n = (8, 8, 8, 8), -0.2, 1.0, 4
    U = synth.gauge_exp(dims, 0.4, 1001)
    V = wilson.volume(dims)
    b = synth.gaussian_field(V, 12, n, 2001)
    v0 = synth.gaussian_field(V, 12, 8, 3001)
    lat = make_lattice(U, dims, mass, csw)
    params = dict(n_levels=2, blocks=[(4, 4, 4, 4)], nvec=[8], setup_sweeps=4, setup_m=8, coarse_m=16,
                  coarse_cycles=2, inner_m=8, inner_tol=1e-5, outer_m=4, max_outer_iters=30, max_rhs=n,
                  coarse_precision=mrhs.MRHS_FP32, smoother_sap=1, sap_cycles=1, sap_mr=4)
    mg = make_mg(lat, params, [v0])
    for mu in range(4):
        assert mrhs.mrhs_mg_default_params().sap_block[mu] == 4
    try:
        d_b, d_x = to_dev(b), to_dev(np.zeros_like(b))
        rel = np.zeros(n)
        status, st = mrhs.mrhs_solve(mg, d_b, d_x, n, 1e-10, rel)
        x = to_host(d_x)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
    r = b - wilson.apply_D(U, wilson.clover_term(U, dims, csw), x, dims, mass)
    true_rel = krylov.norms(r) / krylov.norms(b)
    assert np.all(true_rel <= 1e-10), true_rel
    assert st.vcycles >= 1
