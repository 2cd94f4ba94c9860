"""GPU checks of the half-line ring form of the even-odd hop (Sec. 4, M_eooe).

The ring kernel stages the other parity's x half lines of one (y, z) column
in shared memory and marches along t; every output element is computed with
the arithmetic of the one-RHS-per-thread kernel in the same order, so each
ring variant must be bitwise equal to the default variant in both modes the
Schur operator D_hat = C_oo - 1/4 H_oe C_ee^-1 H_eo is built from (its two
launches, C^-1 H onto the even sites and C - 1/4 H onto the odd ones), and a
whole MG solve with the ring variants forced must return the identical x.
The variants are forced through a tuner cache file.
"""
import numpy as np
import pytest

import synth
from oracle import evenodd as eo
from oracle import wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, make_mg, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

# the two launches of the Schur operator D_hat, the kernels with ring variants
EO_KERNELS = ("k_eo_x2_cinv_hop", "k_eo_x2_schur")


@pytest.fixture
def tuner_state():
    mrhs.mrhs_tune_clear()
    yield
    mrhs.mrhs_tune_clear()
    mrhs.mrhs_tune_set_enabled(True)


def _force(tmp_path, dims, n, variant, nv, kernels=EO_KERNELS):
    path = tmp_path / "tune.txt"
    with open(path, "w") as f:
        for k in kernels:
            f.write(f"{k} {dims[0]} {dims[1]} {dims[2]} {dims[3]} {n} {variant} {nv} 1.0 1.0\n")
    mrhs.mrhs_tune_clear()
    mrhs.mrhs_tune_load(str(path))


def _nvariants(lat, dims, n):
    """Variant count of the even-odd kernels for (dims, n), read from one tuned Schur apply."""
    V2 = wilson.volume(dims) // 2
    d = to_dev(np.zeros((V2, 12, n), np.complex64))
    o = to_dev(np.zeros((V2, 12, n), np.complex64))
    mrhs.mrhs_tune_set_enabled(True)
    mrhs.mrhs_apply_schur(lat, d, o, n)
    ents = {e["kernel"]: e["nvariants"] for e in mrhs.mrhs_tune_entries()}
    return ents["k_eo_x2_schur"]


def _ring_variants(dims, n, nv):
    """Indices of the ring variants: the last one or two (time slices L_t and L_t / 2)."""
    nseg = [s for s in (1, 2) if dims[3] % s == 0 and dims[3] // s >= 2]
    return list(range(nv - len(nseg), nv))


# (dims, n, t boundary): Lx / 2 x n a multiple of 32
SHAPES = [((8, 8, 8, 8), 48, -1), ((4, 2, 6, 4), 48, 1), ((12, 4, 6, 2), 16, -1), ((4, 4, 2, 4), 32, -1),
          ((16, 4, 4, 4), 24, -1)]


@pytest.mark.parametrize("dims,n,tb", SHAPES)
def test_ring_variants_are_bitwise_the_default(tuner_state, tmp_path, dims, n, tb):
    mass, csw = -0.2, 1.0
    U = synth.gauge_haar(dims, 7101)
    V2 = wilson.volume(dims) // 2
    psi = synth.gaussian_field(V2, 12, n, 7102, np.complex64)
    lat = make_lattice(U, dims, mass, csw, tb)
    try:
        nv = _nvariants(lat, dims, n)
        rings = _ring_variants(dims, n, nv)
        d_in = to_dev(psi)
        d_out = to_dev(np.zeros_like(psi))
        res = {}
        for v in [0] + rings:
            _force(tmp_path, dims, n, v, nv)
            mrhs.mrhs_tune_set_enabled(False)
            d_out.fill_(float("nan"))
            mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
            res[v] = to_host(d_out)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    assert np.all(np.isfinite(res[0]))
    for v in rings:
        assert np.array_equal(res[v], res[0]), v
    C = eo.site_matrix(wilson.clover_term(U, dims, csw), mass)
    ref = eo.schur_apply(U, C, psi.astype(np.complex128), dims, antiperiodic=(tb == -1))
    for v in rings:
        assert site_rel_err(res[v].astype(np.complex128), ref) <= 2e-6


def test_ring_at_the_benchmark_size(tuner_state, tmp_path):
    """24^3x64 with 48 RHS (one CTA per SM, 576 compute threads): D_hat through the
    ring variants equals the default bitwise (the default is held to the oracle by
    the even-odd parity tests)."""
    dims, n = (24, 24, 24, 64), 48
    U = synth.gauge_exp(dims, 0.25, 7201)
    V2 = wilson.volume(dims) // 2
    lat = make_lattice(U, dims, -0.13, 1.0)
    try:
        import torch
        g = torch.Generator(device="cuda").manual_seed(7202)
        d_in = torch.randn((V2, 12, n), dtype=torch.complex64, device="cuda", generator=g)
        d_out = torch.empty_like(d_in)
        nv = _nvariants(lat, dims, n)
        outs = {}
        for v in [0] + _ring_variants(dims, n, nv):
            _force(tmp_path, dims, n, v, nv)
            mrhs.mrhs_tune_set_enabled(False)
            d_out.fill_(float("nan"))
            mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
            torch.cuda.synchronize()
            outs[v] = d_out.clone()
        for v, o in outs.items():
            assert torch.equal(o, outs[0]), v
        assert bool(torch.isfinite(torch.view_as_real(outs[0])).all())
    finally:
        mrhs.mrhs_destroy_lattice(lat)


def test_solve_with_ring_variants_is_bitwise_the_default(tuner_state, tmp_path):
    """A 2-level MG solve with the even-odd smoother (8^4, 16 RHS): both launches of
    the smoother's Schur operator forced to a ring variant give the identical x."""
    dims, n = (8, 8, 8, 8), 16
    U = synth.gauge_exp(dims, 0.4, 7301)
    V = wilson.volume(dims)
    b = synth.gaussian_field(V, 12, n, 7302)
    v0 = synth.gaussian_field(V, 12, 8, 7303)
    params = dict(n_levels=2, blocks=[(4, 4, 4, 4)], nvec=[8], setup_sweeps=4, setup_m=8, smooth_m=3,
                  coarse_m=16, coarse_cycles=2, inner_m=8, inner_tol=1e-5, outer_m=4, max_outer_iters=30,
                  max_rhs=n, coarse_precision=mrhs.MRHS_FP32, smoother_evenodd=1)
    lat = make_lattice(U, dims, -0.2, 1.0)
    try:
        nv = _nvariants(lat, dims, n)
        rings = _ring_variants(dims, n, nv)
        _force(tmp_path, dims, n, 0, nv)
        mrhs.mrhs_tune_set_enabled(False)
        mg = make_mg(lat, params, [v0])
        xs = {}
        try:
            for v in [0] + rings:
                _force(tmp_path, dims, n, v, nv)
                mrhs.mrhs_tune_set_enabled(False)
                d_b = to_dev(b)
                d_x = to_dev(np.zeros_like(b))
                rel = np.zeros(n)
                mrhs.mrhs_solve(mg, d_b, d_x, n, 1e-10, rel)
                assert np.all(rel <= 1e-10)
                xs[v] = to_host(d_x)
        finally:
            mrhs.mrhs_destroy_mg(mg)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    for v in rings:
        assert np.array_equal(xs[v], xs[0]), v


def test_expired_ring_waits_fall_back_to_global_memory(tuner_state, tmp_path):
    """mrhs_debug_expire_ring_waits(k): the next k eager ring launches give up their
    first wait at once, every compute warp reads its neighbours from global memory
    and the producer drains the copies it issued; D_hat stays bitwise the default's,
    and the launches after it run the ring again with the same result."""
    dims, n = (8, 8, 8, 8), 48
    U = synth.gauge_haar(dims, 7401)
    V2 = wilson.volume(dims) // 2
    psi = synth.gaussian_field(V2, 12, n, 7402, np.complex64)
    lat = make_lattice(U, dims, -0.2, 1.0)
    try:
        nv = _nvariants(lat, dims, n)
        d_in = to_dev(psi)
        d_out = to_dev(np.zeros_like(psi))
        _force(tmp_path, dims, n, 0, nv)
        mrhs.mrhs_tune_set_enabled(False)
        mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
        ref = to_host(d_out)
        for v in _ring_variants(dims, n, nv):
            _force(tmp_path, dims, n, v, nv)
            mrhs.mrhs_tune_set_enabled(False)
            mrhs.mrhs_debug_expire_ring_waits(2)   # both launches of one D_hat
            d_out.fill_(float("nan"))
            mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
            expired = to_host(d_out)
            d_out.fill_(float("nan"))
            mrhs.mrhs_apply_schur(lat, d_in, d_out, n)
            again = to_host(d_out)
            assert np.array_equal(expired, ref), v
            assert np.array_equal(again, ref), v
        with pytest.raises(mrhs.MrhsError):
            mrhs.mrhs_debug_expire_ring_waits(-1)
    finally:
        mrhs.mrhs_debug_expire_ring_waits(0)
        mrhs.mrhs_destroy_lattice(lat)
