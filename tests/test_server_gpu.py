"""Continuous-batching server: two resident configurations of different volume,
requests of 1-3 sources arriving while others run, more sources than slots so
later requests are admitted only as earlier columns retire.  Every result must
reach the 1e-10 true residual (oracle D) and equal the same sources solved
alone through mrhs_solve within the accuracy both residuals allow."""
import time

import numpy as np
import pytest

import synth
from oracle import krylov, wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, to_dev, to_host

pytestmark = pytest.mark.gpu

CONFIGS = [
    # dims, blocks, nvec, slots, seed
    ((8, 8, 8, 8), [(4, 4, 4, 4)], [8], 4, 1401),
    ((4, 4, 4, 8), [(2, 2, 2, 4)], [6], 2, 1402),
]
MASS, CSW, TOL = -0.2, 1.0, 1e-10


def _params(blocks, nvec, slots):
    return dict(n_levels=2, blocks=blocks, nvec=nvec, setup_sweeps=3, setup_m=8, smooth_m=4, coarse_m=12,
                coarse_cycles=2, inner_m=8, inner_tol=1e-5, outer_m=3, max_outer_iters=40, max_rhs=slots,
                coarse_precision=mrhs.MRHS_FP32)


def test_server_mix_equals_alone():
    lats, mgs, Us = [], [], []
    srv = None
    try:
        for dims, blocks, nvec, slots, seed in CONFIGS:
            U = synth.gauge_exp(dims, 0.4, seed)
            lat = make_lattice(U, dims, MASS, CSW)
            V = wilson.volume(dims)
            mg = make_mg(lat, _params(blocks, nvec, slots), [synth.gaussian_field(V, 12, nvec[0], seed + 7)])
            lats.append(lat)
            mgs.append(mg)
            Us.append(U)
        srv = mrhs.mrhs_server_create(max_queue=64, hbm_reserve_gb=0.0)
        cids = [mrhs.mrhs_server_add_config(srv, mg, cfg[3]) for mg, cfg in zip(mgs, CONFIGS)]
        plan = [(0, 2), (1, 1), (0, 3), (1, 2), (0, 1), (0, 4), (1, 1)]
        reqs = []
        for i, (c, nr) in enumerate(plan):
            V = wilson.volume(CONFIGS[c][0])
            b = synth.gaussian_field(V, 12, nr, 2401 + i)
            x = np.zeros_like(b)
            rid = mrhs.mrhs_submit(srv, cids[c], b, x, nr, TOL)
            reqs.append((rid, c, b, x))
            time.sleep(0.01)
        mrhs.mrhs_server_drain(srv)
        for rid, c, b, x in reqs:
            status, st = mrhs.mrhs_poll(srv, rid)
            assert status == mrhs.MRHS_OK, mrhs.lib().mrhs_last_error()
            assert st.latency_s >= st.queue_s >= 0
            dims = CONFIGS[c][0]
            C = wilson.clover_term(Us[c], dims, CSW)
            rel = krylov.norms(b - wilson.apply_D(Us[c], C, x, dims, MASS)) / krylov.norms(b)
            assert np.all(rel <= TOL), rel
            # the same sources solved alone
            d_b = to_dev(b)
            d_x = to_dev(np.zeros_like(b))
            mrhs.mrhs_solve(mgs[c], d_b, d_x, b.shape[2], TOL)
            xa = to_host(d_x)
            err = krylov.norms(x - xa) / krylov.norms(xa)
            assert np.all(err <= 1e-7), err
        status, _ = mrhs.mrhs_poll(srv, 10 ** 9)
        assert status == mrhs.MRHS_ERR_NOT_FOUND
    finally:
        if srv is not None:
            mrhs.mrhs_server_destroy(srv)
        for mg in mgs:
            mrhs.mrhs_destroy_mg(mg)
        for lat in lats:
            mrhs.mrhs_destroy_lattice(lat)


def test_admission_waits_for_free_hbm():
    """With the reserve set so that free HBM above it holds one request's staging
    and not two, requests are staged one at a time (admissions deferred for
    memory), and every one still completes to 1e-10; a request whose staging
    exceeds the whole device above the reserve is refused at submit."""
    import torch
    dims, blocks, nvec, slots, seed = CONFIGS[0]
    U = synth.gauge_exp(dims, 0.4, seed)
    lat = make_lattice(U, dims, MASS, CSW)
    V = wilson.volume(dims)
    mg = make_mg(lat, _params(blocks, nvec, slots), [synth.gaussian_field(V, 12, nvec[0], seed + 7)])
    srv = None
    try:
        srv = mrhs.mrhs_server_create(max_queue=64, hbm_reserve_gb=0.0)
        cid = mrhs.mrhs_server_add_config(srv, mg, slots)
        # warm the hierarchy's lazily sized buffers with one request at no reserve
        b0 = synth.gaussian_field(V, 12, 1, 2500)
        x0 = np.zeros_like(b0)
        mrhs.mrhs_submit(srv, cid, b0, x0, 1, TOL)
        mrhs.mrhs_server_drain(srv)
        free_b, total_b = torch.cuda.mem_get_info()
        need = V * 12 * 2 * 16  # staging of a 2-source request
        mrhs.mrhs_server_set_reserve(srv, (free_b - 1.5 * need) / 1e9)
        with pytest.raises(mrhs.MrhsError) as e:
            big = np.zeros((V, 12, 1), np.complex128)
            mrhs.mrhs_server_set_reserve(srv, total_b / 1e9)
            mrhs.mrhs_submit(srv, cid, big, big.copy(), 1, TOL)
        assert e.value.status == mrhs.MRHS_ERR_OOM
        mrhs.mrhs_server_set_reserve(srv, (free_b - 1.5 * need) / 1e9)
        w0 = mrhs.mrhs_server_memory_waits(srv)
        reqs = []
        for i in range(3):
            b = synth.gaussian_field(V, 12, 2, 2510 + i)
            x = np.zeros_like(b)
            reqs.append((mrhs.mrhs_submit(srv, cid, b, x, 2, TOL), b, x))
        mrhs.mrhs_server_drain(srv)
        assert mrhs.mrhs_server_memory_waits(srv) > w0
        C = wilson.clover_term(U, dims, CSW)
        for rid, b, x in reqs:
            status, _ = mrhs.mrhs_poll(srv, rid)
            assert status == mrhs.MRHS_OK
            rel = krylov.norms(b - wilson.apply_D(U, C, x, dims, MASS)) / krylov.norms(b)
            assert np.all(rel <= TOL), rel
    finally:
        if srv is not None:
            mrhs.mrhs_server_destroy(srv)
        mrhs.mrhs_destroy_mg(mg)
        mrhs.mrhs_destroy_lattice(lat)
