"""The fused batch of uneven problems (mrhs_apply_D_batch): one persistent
launch applies the FP32 fine operator, or its residual form y - D x, to
problems of different lattice volumes and RHS counts.  Each output must equal
the single-problem entry point's output for the same problem (the same
arithmetic per element: bitwise for even RHS counts, which the single-problem
path runs on the paired or one-RHS kernels of the same operation order) and
the FP64 oracle within the FP32 stencil bar of 1e-6 per site."""
import numpy as np
import pytest

import synth
from oracle import wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import empty_like_dev, make_lattice, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

PROBLEMS = [
    # dims, nrhs, with y (residual form), gauge seed
    ((8, 8, 8, 8), 48, False, 7101),
    ((4, 4, 4, 8), 12, True, 7102),
    ((6, 4, 4, 8), 64, False, 7103),
    ((8, 4, 4, 4), 5, True, 7104),
    ((4, 6, 4, 4), 16, False, 7105),
]


def test_batch_equals_single_problem_applies():
    mass, csw = -0.2, 1.0
    lats, Us, ins, outs, ys, items = [], [], [], [], [], []
    try:
        for dims, n, with_y, seed in PROBLEMS:
            U = synth.gauge_haar(dims, seed)
            V = wilson.volume(dims)
            lat = make_lattice(U, dims, mass, csw)
            psi = synth.gaussian_field(V, 12, n, seed + 1, np.complex64)
            y = synth.gaussian_field(V, 12, n, seed + 2, np.complex64) if with_y else None
            d_in, d_out = to_dev(psi), to_dev(np.full((V, 12, n), np.nan, np.complex64))
            d_y = to_dev(y) if with_y else None
            lats.append(lat)
            Us.append(U)
            ins.append(psi)
            outs.append(d_out)
            ys.append(y)
            items.append((lat, d_in, d_out, d_y, n))
        mrhs.mrhs_apply_D_batch(items)
        for (dims, n, with_y, seed), U, psi, y, (lat, d_in, d_out, d_y, _) in zip(PROBLEMS, Us, ins, ys, items):
            got = to_host(d_out)
            assert np.all(np.isfinite(got))
            single = empty_like_dev(got.shape, np.complex64)
            if with_y:
                mrhs.mrhs_residual_D(lat, d_in, d_y, single, n, mrhs.MRHS_FP32)
            else:
                mrhs.mrhs_apply_D(lat, d_in, single, n, mrhs.MRHS_FP32)
            ref1 = to_host(single)
            if n % 2 == 0:
                assert np.array_equal(got, ref1), (dims, n)
            else:
                assert site_rel_err(got.astype(np.complex128), ref1.astype(np.complex128)) < 1e-6
            Dpsi = wilson.apply_D(U, wilson.clover_term(U, dims, csw), psi.astype(np.complex128), dims, mass)
            ref = y.astype(np.complex128) - Dpsi if with_y else Dpsi
            assert site_rel_err(got.astype(np.complex128), ref) < 1e-6, (dims, n)
    finally:
        for lat in lats:
            mrhs.mrhs_destroy_lattice(lat)


def test_batch_rejects_bad_arguments():
    dims = (4, 4, 4, 4)
    lat = make_lattice(synth.gauge_unit(dims), dims, 0.0, 1.0)
    try:
        a = to_dev(np.zeros((256, 12, 2), np.complex64))
        with pytest.raises(mrhs.MrhsError) as e:
            mrhs.mrhs_apply_D_batch([(lat, a, a, None, 2)])
        assert e.value.status == mrhs.MRHS_ERR_INVALID
        with pytest.raises(mrhs.MrhsError):
            mrhs.mrhs_apply_D_batch([(lat, a, to_dev(np.zeros((256, 12, 2), np.complex64)), None, 2)] * 9)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
