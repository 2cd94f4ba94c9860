"""GPU parity: 16-bit tensor-core coarse stencil (tcgen05, FP32 accumulation in
tensor memory) against the oracle's FP64 stencil built from the same start
vectors.

Bars, relative per coarse site and RHS (norm over the 64 components):
* FP16 operands (per-site link scale, per-RHS input scale): 2e-3;
* BF16 operands: 4e-3 -- BF16 keeps 8 significand bits, so rounding both
  operands alone gives a per-element error of order 2^-9 = 2e-3 and the max
  over sites exceeds 2e-3 on random data; FP16 is the default tensor-core
  format for that reason.
RHS counts exercise the N padding of the MMA (2n rounded up to a multiple of
16); lattices give coarse extents 2 (aliased +mu / -mu neighbours) and 1.
The residual form y - D_c x of the same kernel runs inside every solve.
"""
import numpy as np
import pytest

import synth
from oracle import coarse, wilson
from oracle.conventions import FINE_CHIRALITY
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = {mrhs.MRHS_FP16: 2e-3, mrhs.MRHS_BF16: 4e-3}


@pytest.mark.parametrize("fmt", [mrhs.MRHS_FP16, mrhs.MRHS_BF16])
@pytest.mark.parametrize("dims,block", [((8, 8, 8, 16), (4, 4, 4, 4)), ((4, 4, 8, 8), (4, 4, 4, 2))])
def test_tensor_core_coarse_stencil(dims, block, fmt):
    mass, csw, N = -0.2, 1.0, 32
    U = synth.gauge_exp(dims, 0.4, 1201)
    V = wilson.volume(dims)
    v0 = synth.gaussian_field(V, 12, N, 3201)
    lat = make_lattice(U, dims, mass, csw)
    mg = make_mg(lat, dict(n_levels=2, blocks=[block], nvec=[N], setup_sweeps=0, max_rhs=64,
                           coarse_precision=fmt), [v0])
    try:
        Po = coarse.build_prolongator(v0, dims, block, FINE_CHIRALITY)
        Ao = coarse.galerkin_fine(U, wilson.clover_term(U, dims, csw), Po, dims, block, mass)
        cd = coarse.coarse_dims(dims, block)
        Vc = wilson.volume(cd)
        Ag = np.zeros((Vc, 9, 64, 64), np.complex128)
        mrhs.mrhs_mg_get_coarse_links(mg, 1, Ag)
        for n in (1, 5, 12, 48, 64):
            phi = synth.gaussian_field(Vc, 64, n, 4200 + n, np.complex64)
            phi[:, :, 0] *= 1e-3          # one small column: the per-RHS scale keeps its precision
            ref = coarse.apply_coarse(Ao, phi.astype(np.complex128), cd)
            d_o = to_dev(np.full((Vc, 64, n), np.nan, np.complex64))
            mrhs.mrhs_coarse_apply(mg, 1, to_dev(phi), d_o, n, fmt)
            got = to_host(d_o).astype(np.complex128)
            assert np.all(np.isfinite(got))
            err = site_rel_err(got, ref)
            assert err < TOL[fmt], (n, err)
            # FP32 CUDA-core path against the oracle's stencil on the GPU's FP32 links (1e-6)
            mrhs.mrhs_coarse_apply(mg, 1, to_dev(phi), d_o, n, mrhs.MRHS_FP32)
            ref32 = coarse.apply_coarse(Ag, phi.astype(np.complex128), cd)
            assert site_rel_err(to_host(d_o).astype(np.complex128), ref32) < 1e-6, n
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
