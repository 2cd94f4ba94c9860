"""GPU parity: fused fine hopping + clover operator (Sec. 4) vs the FP64 oracle.

Bars: FP32 <= 1e-6 relative per site and RHS (norm over the 12 components),
FP64 <= 1e-12, float-float (FP32 input, FP64 output) <= 1e-12.  Lattices span several thread blocks with a ragged tail, odd
and even RHS counts (scalar and vector load paths), both time boundaries, and
the full 24^4 x 64-RHS workload on sampled sites.
"""
import numpy as np
import pytest

import synth
from oracle import wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-6
FP64_TOL = 1e-12


def _problem(dims, seed, hot=True):
    U = synth.gauge_haar(dims, seed) if hot else synth.gauge_exp(dims, 0.4, seed)
    return U


@pytest.mark.parametrize("dims,nrhs,tb,hot", [
    ((4, 4, 4, 4), 1, -1, True),
    ((4, 4, 4, 4), 2, -1, True),
    ((6, 4, 2, 8), 3, -1, False),
    ((8, 4, 4, 6), 4, 1, True),
    ((3, 5, 2, 7), 5, -1, True),     # odd extents, odd RHS count, ragged block tail
    ((8, 8, 4, 4), 12, -1, False),
    ((4, 4, 2, 4), 64, -1, True),
    ((1, 2, 1, 4), 2, -1, True),     # extent 1: the +-mu neighbours are the site itself
    # RHS counts with a compile-time kernel and site-major links / clover
    ((4, 4, 4, 4), 16, -1, True),
    ((6, 4, 2, 8), 24, 1, False),
    ((4, 4, 2, 4), 32, -1, True),
    ((4, 2, 6, 4), 48, -1, True),
])
def test_apply_D_fp32_fp64_parity(dims, nrhs, tb, hot):
    mass, csw = -0.2, 1.0
    U = _problem(dims, 1101 + nrhs, hot)
    V = wilson.volume(dims)
    C = wilson.clover_term(U, dims, csw)
    psi32 = synth.gaussian_field(V, 12, nrhs, 2101 + nrhs, np.complex64)
    psi64 = synth.gaussian_field(V, 12, nrhs, 2201 + nrhs)
    lat = make_lattice(U, dims, mass, csw, tb)
    try:
        for psi, prec, tol in ((psi32, mrhs.MRHS_FP32, FP32_TOL), (psi64, mrhs.MRHS_FP64, FP64_TOL)):
            expect = wilson.apply_D(U, C, psi.astype(np.complex128), dims, mass, antiperiodic=(tb == -1))
            d_in = to_dev(psi)
            d_out = to_dev(np.full_like(psi, np.nan))
            mrhs.mrhs_apply_D(lat, d_in, d_out, nrhs, prec)
            got = to_host(d_out).astype(np.complex128)
            assert np.all(np.isfinite(got)), "unwritten output sites"
            assert site_rel_err(got, expect) <= tol
            # fused residual y - D psi
            y = psi[::-1].copy()
            d_y = to_dev(y)
            mrhs.mrhs_residual_D(lat, d_in, d_y, d_out, nrhs, prec)
            got = to_host(d_out).astype(np.complex128)
            ref = y.astype(np.complex128) - expect
            assert site_rel_err(got, ref) <= 10 * tol
    finally:
        mrhs.mrhs_destroy_lattice(lat)


DF64_TOL = 1e-12


@pytest.mark.parametrize("dims,nrhs,tb,hot", [
    ((4, 4, 4, 4), 1, -1, True),
    ((6, 4, 2, 8), 3, -1, False),
    ((8, 4, 4, 6), 4, 1, True),
    ((3, 5, 2, 7), 48, -1, True),    # odd extents, the workload's RHS count, ragged block tail
    ((1, 2, 1, 4), 2, -1, True),
])
def test_apply_D_float_float_parity(dims, nrhs, tb, hot):
    """MRHS_DF64: FP32 input, FP64 output, float-float arithmetic, against the FP64
    oracle on the same (exactly representable) input, and against the FP64 kernel."""
    mass, csw = -0.2, 1.0
    U = _problem(dims, 1301 + nrhs, hot)
    V = wilson.volume(dims)
    C = wilson.clover_term(U, dims, csw)
    psi = synth.gaussian_field(V, 12, nrhs, 2301 + nrhs, np.complex64)
    lat = make_lattice(U, dims, mass, csw, tb)
    try:
        expect = wilson.apply_D(U, C, psi.astype(np.complex128), dims, mass, antiperiodic=(tb == -1))
        d_in = to_dev(psi)
        d_out = to_dev(np.full(psi.shape, np.nan, np.complex128))
        mrhs.mrhs_apply_D(lat, d_in, d_out, nrhs, mrhs.MRHS_DF64)
        got = to_host(d_out)
        assert got.dtype == np.complex128 and np.all(np.isfinite(got))
        assert site_rel_err(got, expect) <= DF64_TOL
        d_in64 = to_dev(psi.astype(np.complex128))
        d_out64 = to_dev(np.full(psi.shape, np.nan, np.complex128))
        mrhs.mrhs_apply_D(lat, d_in64, d_out64, nrhs, mrhs.MRHS_FP64)
        assert site_rel_err(got, to_host(d_out64)) <= DF64_TOL
        # fused residual y - D psi with FP64 y
        y = synth.gaussian_field(V, 12, nrhs, 2401 + nrhs)
        mrhs.mrhs_residual_D(lat, d_in, to_dev(y), d_out, nrhs, mrhs.MRHS_DF64)
        assert site_rel_err(to_host(d_out), y - expect) <= 10 * DF64_TOL
    finally:
        mrhs.mrhs_destroy_lattice(lat)


def test_clover_build_matches_oracle():
    dims, mass, csw = (4, 6, 2, 4), 0.13, 1.7
    U = _problem(dims, 77, hot=False)
    V = wilson.volume(dims)
    lat = make_lattice(U, dims, mass, csw)
    try:
        packed = np.zeros((V, 2, 36))
        mrhs.mrhs_get_clover(lat, packed)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    full = wilson.clover_term(U, dims, csw) + (4 + mass) * np.eye(12)
    for chi in range(2):
        blk = full[:, 6 * chi:6 * chi + 6, 6 * chi:6 * chi + 6]
        assert np.abs(packed[:, chi, :6] - np.real(np.diagonal(blk, axis1=1, axis2=2))).max() < 1e-13
        low = packed[:, chi, 6:].reshape(V, 15, 2)
        q = 0
        for i in range(1, 6):
            for j in range(i):
                v = low[:, q, 0] + 1j * low[:, q, 1]
                assert np.abs(v - blk[:, i, j]).max() < 1e-13
                q += 1
    # off-chirality blocks of the oracle's clover vanish (what makes the compact form exact)
    assert np.abs(full[:, :6, 6:]).max() < 1e-14


def test_full_size_24x4_64rhs_sampled_sites():
    """The 24^4 hot-start workload with 64 RHS, on sampled sites (incl. all boundaries)."""
    dims, mass, csw, nrhs = (24, 24, 24, 24), -0.2, 1.0, 64
    U = synth.gauge_haar(dims, 1101)
    V = wilson.volume(dims)
    psi = synth.gaussian_field(V, 12, nrhs, 2101, np.complex64)
    lat = make_lattice(U, dims, mass, csw, -1)
    try:
        d_in = to_dev(psi)
        d_out = to_dev(np.full_like(psi, np.nan))
        mrhs.mrhs_apply_D(lat, d_in, d_out, nrhs, mrhs.MRHS_FP32)
        got = to_host(d_out)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    assert np.all(np.isfinite(got))
    rng = np.random.default_rng(5)
    corners = [0, V - 1, 23, 24 * 23, 24 ** 3 * 23, 24 ** 3 - 1, 24 ** 3 * 23 + 24 * 24 - 1]
    sites = np.unique(np.r_[corners, rng.integers(0, V, 40)])
    ref = wilson.apply_D_sites(U, psi, dims, mass, csw, sites)
    assert site_rel_err(got[sites].astype(np.complex128), ref) <= FP32_TOL


def test_apply_D_rejects_bad_arguments():
    dims = (2, 2, 2, 2)
    lat = make_lattice(synth.gauge_unit(dims), dims, 0.0, 1.0)
    try:
        import torch
        a = torch.zeros(16 * 12 * 2, dtype=torch.complex64, device="cuda")
        with pytest.raises(mrhs.MrhsError) as e:
            mrhs.mrhs_apply_D(lat, a, a, 2, mrhs.MRHS_FP32)
        assert e.value.status == mrhs.MRHS_ERR_INVALID
        with pytest.raises(mrhs.MrhsError):
            mrhs.mrhs_apply_D(lat, a, a[1:], 0, mrhs.MRHS_FP32)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
