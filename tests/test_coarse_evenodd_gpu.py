"""GPU parity of the coarse even-odd decomposition (Sec. 6, coarse M_eooe).

A three-level hierarchy with FP16 tensor-core coarse levels and
coarse_smoother_evenodd = 1 prepares the inverse self blocks A_0(x)^-1 of its
intermediate level (coarse extents 2 x 2 x 2 x 4: every hop joins opposite
parities, +mu and -mu neighbours coincide).  Checked:
* the Schur complement D_hat = A_oo - H_oe A_ee^-1 H_eo on the tensor cores
  against the oracle's FP64 Schur complement on the GPU's own coarse links,
  within the 2e-3 bar of the 16-bit coarse path (relative per site);
* an MG solve whose intermediate level post-smooths with GMRES on D_hat
  reaches a true residual of 1e-10 with the oracle's D.
"""
import numpy as np
import pytest

import synth
from oracle import coarse, coarse_evenodd as ceo, evenodd, krylov, wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

DIMS, MASS, CSW = (8, 8, 8, 16), -0.2, 1.0
BLOCKS, NVEC = [(4, 4, 4, 4), (2, 2, 2, 2)], [32, 32]


def _hierarchy(n_max=8, **over):
    U = synth.gauge_exp(DIMS, 0.4, 8201)
    V = wilson.volume(DIMS)
    d1 = coarse.coarse_dims(DIMS, BLOCKS[0])
    v0 = synth.gaussian_field(V, 12, NVEC[0], 8202)
    v1 = synth.gaussian_field(wilson.volume(d1), 2 * NVEC[0], NVEC[1], 8203)
    lat = make_lattice(U, DIMS, MASS, CSW)
    params = dict(n_levels=3, blocks=BLOCKS, nvec=NVEC, setup_sweeps=0, max_rhs=n_max,
                  coarse_precision=mrhs.MRHS_FP16, coarse_smoother_evenodd=1)
    params.update(over)
    mg = make_mg(lat, params, [v0, v1])
    return U, lat, mg, d1


def test_coarse_schur_complement_matches_oracle():
    U, lat, mg, cd = _hierarchy()
    try:
        Vc = wilson.volume(cd)
        Ag = np.zeros((Vc, 9, 64, 64), np.complex128)
        mrhs.mrhs_mg_get_coarse_links(mg, 1, Ag)
        for n in (2, 8):
            phi = synth.gaussian_field(Vc // 2, 64, n, 8300 + n, np.complex64)
            d_o = to_dev(np.full((Vc // 2, 64, n), np.nan, np.complex64))
            mrhs.mrhs_coarse_apply_schur(mg, 1, to_dev(phi), d_o, n)
            got = to_host(d_o).astype(np.complex128)
            assert np.all(np.isfinite(got))
            ref = ceo.schur_apply(Ag, phi.astype(np.complex128), cd)
            err = site_rel_err(got, ref)
            assert err < 2e-3, (n, err)
        with pytest.raises(mrhs.MrhsError):
            mrhs.mrhs_coarse_apply_schur(mg, 2, to_dev(phi), d_o, 2)  # the coarsest level has no smoother
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)


def test_solve_with_coarse_evenodd_smoother_reaches_1e10():
    U, lat, mg, _ = _hierarchy(n_max=4, smooth_m=3, coarse_m=8, inter_m=3, inner_m=8)
    try:
        V = wilson.volume(DIMS)
        b = synth.gaussian_field(V, 12, 4, 8401)
        xd = to_dev(np.zeros_like(b))
        rel = np.zeros(4)
        status, st = mrhs.mrhs_solve(mg, to_dev(b), xd, 4, 1e-10, rel)
        assert status == mrhs.MRHS_OK
        x = to_host(xd)
        r = b - wilson.apply_D(U, wilson.clover_term(U, DIMS, CSW), x, DIMS, MASS)
        true_rel = krylov.norms(r) / krylov.norms(b)
        assert np.all(true_rel <= 1e-10), true_rel
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
