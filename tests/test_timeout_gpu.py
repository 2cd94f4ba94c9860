"""The bounded-wait path of the tensor-core coarse stencil, forced safely.

Every mbarrier wait in the tcgen05 kernels gives up after a bounded number
of try_wait rounds, sets a flag and lets the call return MRHS_ERR_TIMEOUT.
mrhs_debug_expire_waits(k) makes the first operand wait of the next k eager
launches give up at once; the kernel still waits for the copies it issued
before freeing its tensor memory, so no copy is left in flight and the GPU
context stays usable.  Checked: a standalone apply and a solve both return
MRHS_ERR_TIMEOUT, the flag is cleared, and the next call on the same
hierarchy succeeds (the apply bitwise equal to the one before, the solve to
a true residual of 1e-10).
"""
import numpy as np
import pytest

import synth
from oracle import wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, to_dev, to_host

pytestmark = pytest.mark.gpu


def _setup():
    dims, block, N, mass, csw = (8, 8, 8, 16), (4, 4, 4, 4), 32, -0.2, 1.0
    U = synth.gauge_exp(dims, 0.4, 1201)
    V = wilson.volume(dims)
    v0 = synth.gaussian_field(V, 12, N, 3201)
    lat = make_lattice(U, dims, mass, csw)
    mg = make_mg(lat, dict(n_levels=2, blocks=[block], nvec=[N], setup_sweeps=2, max_rhs=4,
                           coarse_precision=mrhs.MRHS_FP16, smooth_m=3, coarse_m=12, inner_m=8),
                 [v0])
    return U, dims, mass, csw, lat, mg


def test_expired_wait_gives_timeout_then_recovers():
    U, dims, mass, csw, lat, mg = _setup()
    try:
        cd = (2, 2, 2, 4)
        Vc, n = wilson.volume(cd), 6
        phi = to_dev(synth.gaussian_field(Vc, 64, n, 77, np.complex64))
        out = to_dev(np.zeros((Vc, 64, n), np.complex64))
        mrhs.mrhs_coarse_apply(mg, 1, phi, out, n, mrhs.MRHS_FP16)
        ref = to_host(out).copy()
        # one launch whose first operand wait expires
        mrhs.mrhs_debug_expire_waits(1)
        with pytest.raises(mrhs.MrhsError) as e:
            mrhs.mrhs_coarse_apply(mg, 1, phi, out, n, mrhs.MRHS_FP16)
        assert e.value.status == mrhs.MRHS_ERR_TIMEOUT
        # the flag was cleared: the next apply succeeds and is the same computation
        out2 = to_dev(np.full((Vc, 64, n), np.nan, np.complex64))
        mrhs.mrhs_coarse_apply(mg, 1, phi, out2, n, mrhs.MRHS_FP16)
        assert np.array_equal(to_host(out2), ref)

        # a solve whose first coarse stencil launch gives up
        V = wilson.volume(dims)
        b = synth.gaussian_field(V, 12, 2, 2001)
        bd = to_dev(b)
        xd = to_dev(np.zeros_like(b))
        mrhs.mrhs_debug_expire_waits(1)
        with pytest.raises(mrhs.MrhsError) as e:
            mrhs.mrhs_solve(mg, bd, xd, 2, 1e-10)
        assert e.value.status == mrhs.MRHS_ERR_TIMEOUT
        mrhs.mrhs_debug_expire_waits(0)
        xd.zero_()
        rel = np.zeros(2)
        status, st = mrhs.mrhs_solve(mg, bd, xd, 2, 1e-10, rel)
        assert status == mrhs.MRHS_OK
        x = to_host(xd)
        C = wilson.clover_term(U, dims, csw)
        r = b - wilson.apply_D(U, C, x, dims, mass)
        true_rel = np.sqrt(np.sum(np.abs(r) ** 2, axis=(0, 1)) / np.sum(np.abs(b) ** 2, axis=(0, 1)))
        assert np.all(true_rel <= 1e-10), true_rel
    finally:
        mrhs.mrhs_debug_expire_waits(0)
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
