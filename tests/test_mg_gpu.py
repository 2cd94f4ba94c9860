"""GPU parity of the multigrid rows (Sec. 5, 6, 8) against the FP64 oracle.

Start vectors come from the seeded generator and are given to both sides, with
no setup relaxation, so both build the prolongator from the same vectors:
* prolongator (FP64 block Gram-Schmidt) to 1e-12,
* Galerkin links (FP32 on the GPU) to 2e-6 relative per stencil block with
  the restriction of the build on the CUDA cores in FP32, and to 2e-5 with it
  on the tensor cores in split FP16 (hi + lo operands, 22 significant bits,
  three MMA terms; the remaining error, about 1e-5, is the tensor cores' FP32
  accumulation over the aggregate's rows; the kernel timer shows which ran),
* restriction / prolongation (FP32) to 2e-6 relative per site,
* coarse stencil (FP32 links, FP32 fields) to 1e-6 relative per site
  against the oracle's FP64 stencil on the same (GPU-built FP32) links, so
  that only the stencil's own rounding is measured, on coarse extents 2 and
  1 where +mu and -mu neighbours coincide,
* the second-level Galerkin of a three-level hierarchy,
* the V-cycle (fixed-iteration Krylov pieces) against the oracle's V-cycle.
"""
import numpy as np
import pytest

import synth
from oracle import coarse, mg as omg, wilson
from oracle.conventions import FINE_CHIRALITY
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def _block_rel_err(a, b):
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=(-1, -2)))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=(-1, -2)))
    return float(np.max(num / np.maximum(den, 1e-300)))


CASES = [
    # dims, blocks, nvec
    ((8, 8, 8, 8), [(4, 4, 4, 4)], [8]),              # coarse extent 2 (aliasing)
    ((4, 4, 4, 8), [(4, 4, 2, 4)], [6]),              # coarse extents 1, 1, 2, 2
    ((6, 4, 4, 8), [(3, 2, 2, 4)], [4]),              # odd aggregate extent
]


@pytest.mark.parametrize("galerkin_tc", [2, 0])
@pytest.mark.parametrize("dims,blocks,nvec", CASES)
def test_two_level_rows(dims, blocks, nvec, galerkin_tc):
    mass, csw, n = -0.2, 1.0, 5
    U = synth.gauge_exp(dims, 0.4, 1001)
    V = wilson.volume(dims)
    v0 = synth.gaussian_field(V, 12, nvec[0], 3001)
    lat = make_lattice(U, dims, mass, csw)
    mrhs.mrhs_kernel_timer_start("k_restrict_tc")
    mg = make_mg(lat, dict(n_levels=2, blocks=blocks, nvec=nvec, setup_sweeps=0, max_rhs=8,
                           coarse_precision=mrhs.MRHS_FP32, galerkin_tc=galerkin_tc), [v0])
    _, tc_launches, _ = mrhs.mrhs_kernel_timer_stop()
    assert tc_launches == (9 if galerkin_tc else 0)
    try:
        # prolongator
        Pg = np.zeros((V, 12, nvec[0]), np.complex128)
        mrhs.mrhs_mg_get_prolongator(mg, 0, Pg)
        Po = coarse.build_prolongator(v0, dims, blocks[0], FINE_CHIRALITY)
        N = nvec[0]
        Pcompact = np.where(FINE_CHIRALITY[None, :, None] == 0, Po[:, :, :N], Po[:, :, N:])
        assert np.abs(Pg - Pcompact).max() < 1e-12
        # Galerkin links
        cd = coarse.coarse_dims(dims, blocks[0])
        Vc, nc = wilson.volume(cd), 2 * N
        C = wilson.clover_term(U, dims, csw)
        Ao = coarse.galerkin_fine(U, C, Po, dims, blocks[0], mass)
        Ag = np.zeros((Vc, 9, nc, nc), np.complex128)
        mrhs.mrhs_mg_get_coarse_links(mg, 1, Ag)
        gal_err = _block_rel_err(Ag.reshape(-1, nc, nc), Ao.reshape(-1, nc, nc))
        print(f"galerkin_tc={galerkin_tc} dims={dims} nvec={nvec}: Galerkin block error {gal_err:.2e}")
        assert gal_err < (2e-5 if galerkin_tc else 2e-6)
        # restriction and prolongation
        psi = synth.gaussian_field(V, 12, n, 4001, np.complex64)
        d_psi = to_dev(psi)
        d_c = to_dev(np.full((Vc, nc, n), np.nan, np.complex64))
        mrhs.mrhs_restrict(mg, 0, d_psi, d_c, n)
        c_gpu = to_host(d_c).astype(np.complex128)
        c_ref = coarse.restrict(Po, psi.astype(np.complex128), dims, blocks[0])
        assert site_rel_err(c_gpu, c_ref) < 2e-6
        d_f = to_dev(np.full((V, 12, n), np.nan, np.complex64))
        cin = synth.gaussian_field(Vc, nc, n, 4002, np.complex64)
        mrhs.mrhs_prolong(mg, 0, to_dev(cin), d_f, n)
        f_ref = coarse.prolong(Po, cin.astype(np.complex128), dims, blocks[0])
        assert site_rel_err(to_host(d_f).astype(np.complex128), f_ref) < 2e-6
        # coarse stencil: the oracle's stencil on the GPU's own FP32 links
        d_o = to_dev(np.full((Vc, nc, n), np.nan, np.complex64))
        mrhs.mrhs_coarse_apply(mg, 1, to_dev(cin), d_o, n, mrhs.MRHS_FP32)
        o_ref = coarse.apply_coarse(Ag, cin.astype(np.complex128), cd)
        assert site_rel_err(to_host(d_o).astype(np.complex128), o_ref) < 1e-6
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)


@pytest.mark.parametrize("evenodd", [False, True])
def test_three_level_second_galerkin_and_vcycle(evenodd):
    dims, mass, csw = (8, 8, 8, 8), -0.2, 1.0
    n = 4 if evenodd else 3      # the even-odd smoother takes an even RHS count
    blocks, nvec = [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 4]
    U = synth.gauge_exp(dims, 0.4, 1001)
    V = wilson.volume(dims)
    d1 = coarse.coarse_dims(dims, blocks[0])
    d2 = coarse.coarse_dims(d1, blocks[1])
    v0 = synth.gaussian_field(V, 12, nvec[0], 3101)
    v1 = synth.gaussian_field(wilson.volume(d1), 2 * nvec[0], nvec[1], 3102)
    params = dict(n_levels=3, blocks=blocks, nvec=nvec, setup_sweeps=0, max_rhs=4, smooth_m=3,
                  coarse_m=5, coarse_cycles=1, inter_m=2, coarse_precision=mrhs.MRHS_FP32, use_graph=0,
                  smoother_evenodd=int(evenodd))
    lat = make_lattice(U, dims, mass, csw)
    mg = make_mg(lat, params, [v0, v1])
    try:
        op = omg.MGParams(blocks=blocks, nvec=nvec, smooth_m=3, coarse_m=5, coarse_cycles=1, inter_m=2,
                          smoother_evenodd=evenodd)
        levels = omg.build_hierarchy(U, dims, mass, csw, op, None, nullvecs=[v0, v1])
        nc2 = 2 * nvec[1]
        Ag = np.zeros((wilson.volume(d2), 9, nc2, nc2), np.complex128)
        mrhs.mrhs_mg_get_coarse_links(mg, 2, Ag)
        assert _block_rel_err(Ag.reshape(-1, nc2, nc2), levels[2].stencil.reshape(-1, nc2, nc2)) < 1e-5
        # one V-cycle on the same residual
        v = synth.gaussian_field(V, 12, n, 5001, np.complex64)
        d_z = to_dev(np.full((V, 12, n), np.nan, np.complex64))
        mrhs.mrhs_vcycle(mg, to_dev(v), d_z, n)
        z = to_host(d_z).astype(np.complex128)
        zr = omg.vcycle(levels, 0, v.astype(np.complex128), op)
        err = np.sqrt(np.sum(np.abs(z - zr) ** 2, axis=(0, 1)) / np.sum(np.abs(zr) ** 2, axis=(0, 1)))
        assert np.all(err < 1e-3), err
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
