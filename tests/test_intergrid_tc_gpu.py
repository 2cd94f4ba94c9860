"""GPU parity: tensor-core restriction and prolongation (FP16 operands with one
scale per RHS column, FP32 accumulation) against the oracle's FP64 R = P^dagger
and P built from the same start vectors.

Bar: 2e-3 relative per site and RHS (norm over the site's components), the
same as the 16-bit coarse stencil.  Aggregate row counts that are not a
multiple of the 128-row / 64-row MMA tiles, 1..64 RHS, the level-1 -> level-2
transfer of a three-level hierarchy, and an RHS column a thousand times
smaller than the others are covered.
"""
import numpy as np
import pytest

import synth
from oracle import coarse, wilson
from oracle.conventions import FINE_CHIRALITY
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu
TOL = 2e-3


def _check_level(mg, level, P, dims, block, dof, nc):
    V = wilson.volume(dims)
    cd = coarse.coarse_dims(dims, block)
    Vc = wilson.volume(cd)
    for n in (1, 5, 12, 48, 64):
        psi = synth.gaussian_field(V, dof, n, 6100 + n, np.complex64)
        psi[:, :, 0] *= 1e-3
        d_c = to_dev(np.full((Vc, nc, n), np.nan, np.complex64))
        mrhs.mrhs_restrict(mg, level, to_dev(psi), d_c, n)
        ref = coarse.restrict(P, psi.astype(np.complex128), dims, block)
        got = to_host(d_c).astype(np.complex128)
        assert np.all(np.isfinite(got))
        assert site_rel_err(got, ref) < TOL, ("restrict", n, site_rel_err(got, ref))
        cin = synth.gaussian_field(Vc, nc, n, 6200 + n, np.complex64)
        cin[:, :, -1] *= 1e-3
        d_f = to_dev(np.full((V, dof, n), np.nan, np.complex64))
        mrhs.mrhs_prolong(mg, level, to_dev(cin), d_f, n)
        ref = coarse.prolong(P, cin.astype(np.complex128), dims, block)
        got = to_host(d_f).astype(np.complex128)
        assert np.all(np.isfinite(got))
        assert site_rel_err(got, ref) < TOL, ("prolong", n, site_rel_err(got, ref))


@pytest.mark.parametrize("dims,block,N", [((8, 8, 8, 16), (4, 4, 4, 4), 32),   # 1536 rows: full tiles
                                          ((4, 4, 8, 8), (4, 4, 4, 2), 8),      # 768 rows
                                          ((6, 4, 4, 8), (3, 2, 2, 4), 4)])     # 288 rows: partial tiles
def test_tensor_core_transfer_fine_level(dims, block, N):
    U = synth.gauge_exp(dims, 0.4, 1201)
    V = wilson.volume(dims)
    v0 = synth.gaussian_field(V, 12, N, 3301)
    lat = make_lattice(U, dims, -0.2, 1.0)
    mg = make_mg(lat, dict(n_levels=2, blocks=[block], nvec=[N], setup_sweeps=0, max_rhs=64,
                           coarse_precision=mrhs.MRHS_FP16), [v0])
    try:
        P = coarse.build_prolongator(v0, dims, block, FINE_CHIRALITY)
        _check_level(mg, 0, P, dims, block, 12, 2 * N)
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)


def test_tensor_core_transfer_second_level():
    dims, blocks, nvec = (8, 8, 8, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 4]
    U = synth.gauge_exp(dims, 0.4, 1201)
    V = wilson.volume(dims)
    d1 = coarse.coarse_dims(dims, blocks[0])
    v0 = synth.gaussian_field(V, 12, nvec[0], 3401)
    v1 = synth.gaussian_field(wilson.volume(d1), 2 * nvec[0], nvec[1], 3402)
    lat = make_lattice(U, dims, -0.2, 1.0)
    mg = make_mg(lat, dict(n_levels=3, blocks=blocks, nvec=nvec, setup_sweeps=0, max_rhs=64,
                           coarse_precision=mrhs.MRHS_FP16), [v0, v1])
    try:
        P1 = coarse.build_prolongator(v1, d1, blocks[1], coarse.coarse_chirality(2 * nvec[0]))
        _check_level(mg, 1, P1, d1, blocks[1], 2 * nvec[0], 2 * nvec[1])
    finally:
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)


@pytest.mark.parametrize("n", [5, 48])
def test_prolongation_variants_are_bitwise_equal(tmp_path, n):
    """The autotuner's prolongation variants (128 and 256 threads: the same MMAs, the epilogue's
    columns split over more warps) write the same field, bit for bit, and pass the oracle's bar."""
    dims, block, N = (8, 8, 8, 16), (4, 4, 4, 4), 32
    U = synth.gauge_exp(dims, 0.4, 1201)
    V = wilson.volume(dims)
    v0 = synth.gaussian_field(V, 12, N, 3301)
    lat = make_lattice(U, dims, -0.2, 1.0)
    mg = make_mg(lat, dict(n_levels=2, blocks=[block], nvec=[N], setup_sweeps=0, max_rhs=64,
                           coarse_precision=mrhs.MRHS_FP16), [v0])
    try:
        cd = coarse.coarse_dims(dims, block)
        Vc = wilson.volume(cd)
        cin = synth.gaussian_field(Vc, 2 * N, n, 6300 + n, np.complex64)
        outs = []
        for variant in (0, 1):
            path = tmp_path / f"tune{variant}.txt"
            path.write_text(f"k_prolong_tc {cd[0]} {cd[1]} {cd[2]} {cd[3]} {n} {variant} 2 1.0 1.0\n")
            mrhs.mrhs_tune_clear()
            mrhs.mrhs_tune_load(str(path))
            d_f = to_dev(np.full((V, 12, n), np.nan, np.complex64))
            mrhs.mrhs_prolong(mg, 0, to_dev(cin), d_f, n)
            outs.append(to_host(d_f))
        assert np.array_equal(outs[0], outs[1])
        P = coarse.build_prolongator(v0, dims, block, FINE_CHIRALITY)
        ref = coarse.prolong(P, cin.astype(np.complex128), dims, block)
        assert site_rel_err(outs[1].astype(np.complex128), ref) < TOL
    finally:
        mrhs.mrhs_tune_clear()
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
