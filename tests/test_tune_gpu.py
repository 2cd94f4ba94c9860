"""GPU checks of the autotuner: it times every tile-shape variant of the FP32
stencils at the first eager launch of a (kernel, lattice, nrhs) key, caches
the fastest, and never changes a result (the variants differ only in which
thread computes which site), so the tuned output equals the untuned one bit
for bit and still matches the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import evenodd as eo
from oracle import wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture
def tuner_state():
    mrhs.mrhs_tune_clear()
    yield
    mrhs.mrhs_tune_clear()
    mrhs.mrhs_tune_set_enabled(True)


@pytest.mark.parametrize("dims,n", [((8, 8, 8, 8), 48), ((8, 8, 4, 8), 4)])
def test_tuned_fine_stencil_is_bitwise_the_default(tuner_state, dims, n):
    mass, csw = -0.2, 1.0
    U = synth.gauge_haar(dims, 6101)
    V = wilson.volume(dims)
    psi = synth.gaussian_field(V, 12, n, 6102, np.complex64)
    lat = make_lattice(U, dims, mass, csw)
    try:
        d_in = to_dev(psi)
        d_out = to_dev(np.zeros_like(psi))
        mrhs.mrhs_tune_set_enabled(False)
        mrhs.mrhs_apply_D(lat, d_in, d_out, n, mrhs.MRHS_FP32)
        untuned = to_host(d_out)
        assert mrhs.mrhs_tune_entries() == []
        mrhs.mrhs_tune_set_enabled(True)
        mrhs.mrhs_apply_D(lat, d_in, d_out, n, mrhs.MRHS_FP32)
        tuned = to_host(d_out)
        ents = [e for e in mrhs.mrhs_tune_entries() if e["kernel"] == "k_dslash_x2"]
        assert len(ents) == 1
        e = ents[0]
        assert e["dims"] == tuple(dims) and e["nrhs"] == n
        assert e["nvariants"] >= 2 and 0 <= e["variant"] < e["nvariants"]
        assert 0 < e["best_ms"] <= e["default_ms"]
        # a second call reuses the cached choice
        mrhs.mrhs_apply_D(lat, d_in, d_out, n, mrhs.MRHS_FP32)
        assert len(mrhs.mrhs_tune_entries()) == 1
        again = to_host(d_out)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    assert np.array_equal(tuned, untuned)
    assert np.array_equal(again, untuned)
    ref = wilson.apply_D(U, wilson.clover_term(U, dims, csw), psi.astype(np.complex128), dims, mass)
    assert site_rel_err(tuned.astype(np.complex128), ref) <= 1e-6


def test_tuned_schur_operator_is_bitwise_the_default(tuner_state):
    dims, n, mass, csw = (8, 8, 8, 8), 48, -0.2, 1.0
    U = synth.gauge_haar(dims, 6201)
    V2 = wilson.volume(dims) // 2
    psi = synth.gaussian_field(V2, 12, n, 6202, np.complex64)
    lat = make_lattice(U, dims, mass, csw)
    try:
        d_in = to_dev(psi)
        d_out = to_dev(np.zeros_like(psi))
        mrhs.mrhs_tune_set_enabled(False)
        mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
        untuned = to_host(d_out)
        mrhs.mrhs_tune_set_enabled(True)
        mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
        tuned = to_host(d_out)
        names = {e["kernel"] for e in mrhs.mrhs_tune_entries()}
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    assert {"k_eo_x2_cinv_hop", "k_eo_x2_schur"} <= names
    assert np.array_equal(tuned, untuned)
    C = eo.site_matrix(wilson.clover_term(U, dims, csw), mass)
    ref = eo.schur_apply(U, C, psi.astype(np.complex128), dims)
    assert site_rel_err(tuned.astype(np.complex128), ref) <= 2e-6


def _force(tmp_path, entries):
    """Load a tuner cache that pins the given (kernel, dims, n, variant, nvariants) choices."""
    path = tmp_path / "tune.txt"
    with open(path, "w") as f:
        for k, d, n, v, nv in entries:
            f.write(f"{k} {d[0]} {d[1]} {d[2]} {d[3]} {n} {v} {nv} 1.0 1.0\n")
    mrhs.mrhs_tune_clear()
    mrhs.mrhs_tune_load(str(path))


@pytest.mark.parametrize("dims,n", [((8, 8, 8, 8), 48), ((8, 8, 4, 8), 4), ((12, 4, 4, 8), 24)])
def test_every_visit_order_of_the_fine_stencil_is_bitwise_the_default(tuner_state, tmp_path, dims, n):
    """Each variant (site tiles, x-regions, RHS slabs) computes every output
    element with the same arithmetic: all are bitwise equal to variant 0."""
    U = synth.gauge_haar(dims, 6301)
    V = wilson.volume(dims)
    psi = synth.gaussian_field(V, 12, n, 6302, np.complex64)
    lat = make_lattice(U, dims, -0.2, 1.0)
    try:
        d_in = to_dev(psi)
        d_out = to_dev(np.zeros_like(psi))
        mrhs.mrhs_apply_D(lat, d_in, d_out, n, mrhs.MRHS_FP32)
        nv = [e for e in mrhs.mrhs_tune_entries() if e["kernel"] == "k_dslash_x2"][0]["nvariants"]
        assert nv >= 6
        outs = []
        for v in range(nv):
            _force(tmp_path, [("k_dslash_x2", dims, n, v, nv)])
            d_out.fill_(float("nan"))
            mrhs.mrhs_apply_D(lat, d_in, d_out, n, mrhs.MRHS_FP32)
            outs.append(to_host(d_out))
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    for v in range(1, nv):
        assert np.array_equal(outs[v], outs[0]), v
    assert np.all(np.isfinite(outs[0]))


def test_every_visit_order_of_the_schur_operator_is_bitwise_the_default(tuner_state, tmp_path):
    dims, n = (8, 8, 8, 8), 48
    U = synth.gauge_haar(dims, 6401)
    V2 = wilson.volume(dims) // 2
    psi = synth.gaussian_field(V2, 12, n, 6402, np.complex64)
    lat = make_lattice(U, dims, -0.2, 1.0)
    try:
        d_in = to_dev(psi)
        d_out = to_dev(np.zeros_like(psi))
        mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
        ents = {e["kernel"]: e["nvariants"] for e in mrhs.mrhs_tune_entries()}
        nv = ents["k_eo_x2_schur"]
        assert nv >= 6 and ents["k_eo_x2_cinv_hop"] == nv
        outs = []
        for v in range(nv):
            _force(tmp_path, [("k_eo_x2_cinv_hop", dims, n, v, nv), ("k_eo_x2_schur", dims, n, v, nv)])
            d_out.fill_(float("nan"))
            mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
            outs.append(to_host(d_out))
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    for v in range(1, nv):
        assert np.array_equal(outs[v], outs[0]), v
    assert np.all(np.isfinite(outs[0]))
