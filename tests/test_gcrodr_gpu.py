"""GPU GCRO-DR on the coarsest level (Sec. 9 outlook) against the oracle's
GCRO-DR (oracle/gcrodr.py) on the GPU's own coarse operator.

A 2-level hierarchy with FP32 coarse links (the CUDA-core stencil, accurate to
FP32 rounding) runs the coarsest solve with coarse_solver = 1:
* a first solve from no recycle space (a GMRES(m) cycle that seeds the space,
  then cycles with it) equals oracle.gcrodr.solve for the same number of
  cycles;
* a second solve that enters with the recycled space (A U = Q R, x = U C^H b)
  equals the oracle's second solve with the oracle's recycled space;
both within 1e-4 relative per RHS (FP32 fields against FP64: the Krylov
recurrences amplify FP32 rounding over 3 cycles of 8 steps);
* an MG solve with the GCRO-DR coarsest solver reaches the 1e-10 true
  residual (oracle D).
"""
import numpy as np
import pytest

import synth
from oracle import coarse, gcrodr, krylov, wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, to_dev, to_host

pytestmark = pytest.mark.gpu

DIMS, MASS, CSW = (8, 8, 8, 8), -0.2, 1.0
BLOCK, N = (4, 4, 4, 4), 8
M, K, CYCLES = 8, 3, 3


def _setup(**over):
    U = synth.gauge_exp(DIMS, 0.4, 9101)
    V = wilson.volume(DIMS)
    lat = make_lattice(U, DIMS, MASS, CSW)
    params = dict(n_levels=2, blocks=[BLOCK], nvec=[N], setup_sweeps=2, max_rhs=4, coarse_precision=mrhs.MRHS_FP32,
                  coarse_solver=1, coarse_m=M, coarse_recycle=K, coarse_cycles=CYCLES)
    params.update(over)
    mg = make_mg(lat, params, [synth.gaussian_field(V, 12, N, 9102)])
    return U, lat, mg


def test_gcrodr_matches_oracle_with_and_without_recycle_space():
    U, lat, mg = _setup()
    try:
        cd = coarse.coarse_dims(DIMS, BLOCK)
        Vc, nc, n = wilson.volume(cd), 2 * N, 3
        Ag = np.zeros((Vc, 9, nc, nc), np.complex128)
        mrhs.mrhs_mg_get_coarse_links(mg, 1, Ag)

        def A(phi):
            return coarse.apply_coarse(Ag, phi, cd)

        recycle = None
        mrhs.mrhs_coarsest_reset(mg)
        for solve in range(2):
            b = synth.gaussian_field(Vc, nc, n, 9200 + solve, np.complex64)
            xd = to_dev(np.full((Vc, nc, n), np.nan, np.complex64))
            mrhs.mrhs_coarsest_solve(mg, to_dev(b), xd, n)
            x = to_host(xd).astype(np.complex128)
            assert np.all(np.isfinite(x))
            x_or, recycle, hist = gcrodr.solve(A, b.astype(np.complex128), np.zeros((Vc, nc, n), np.complex128),
                                               M, K, 0.0, CYCLES, recycle)
            err = krylov.norms(x - x_or) / krylov.norms(x_or)
            assert np.all(err < 1e-4), (solve, err)
            # the residual it reaches is the oracle's
            res = krylov.norms(b.astype(np.complex128) - A(x)) / krylov.norms(b.astype(np.complex128))
            res_or = np.array([h[-1] for h in hist])
            assert np.all(res <= 1.2 * res_or + 1e-6), (res, res_or)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)


def test_mg_solve_with_gcrodr_coarsest_reaches_1e10():
    U, lat, mg = _setup(coarse_cycles=1, coarse_m=10, coarse_recycle=4, smooth_m=4, outer_m=4,
                        coarse_precision=mrhs.MRHS_FP32)
    try:
        V = wilson.volume(DIMS)
        b = synth.gaussian_field(V, 12, 4, 9301)
        xd = to_dev(np.zeros_like(b))
        rel = np.zeros(4)
        status, st = mrhs.mrhs_solve(mg, to_dev(b), xd, 4, 1e-10, rel)
        assert status == mrhs.MRHS_OK
        x = to_host(xd)
        r = b - wilson.apply_D(U, wilson.clover_term(U, DIMS, CSW), x, DIMS, MASS)
        assert np.all(krylov.norms(r) / krylov.norms(b) <= 1e-10)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
