"""GPU parity of the even-odd kernels (Sec. 4, M_eooe) against the FP64 oracle.

Bars (FP32, relative per site and RHS): 1e-6 for the hop between the
checkerboards, 2e-6 for the Schur operator D_hat = C_oo - 1/4 H_oe C_ee^-1 H_eo
(two hops and the FP64-built, FP32-stored clover inverse).  At the 24^3x64
bench size with 48 RHS the hop is checked against the full-lattice stencil:
on a field that vanishes on the even sites, (D psi)_e = -1/2 H_eo psi_o.
"""
import numpy as np
import pytest

import synth
from oracle import evenodd as eo
from oracle import wilson
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import make_lattice, site_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [
    ((4, 4, 4, 4), 2, -1, True),
    ((6, 4, 2, 8), 4, -1, False),
    ((8, 4, 4, 6), 12, 1, True),
    ((2, 2, 2, 2), 2, -1, True),     # extent 2: the +-mu neighbours coincide
    ((4, 2, 6, 4), 48, -1, True),
    ((4, 4, 4, 4), 16, -1, True),
    ((6, 4, 2, 8), 24, 1, False),
    ((4, 4, 2, 4), 32, -1, True),
    ((2, 4, 2, 4), 64, -1, True),
]


@pytest.mark.parametrize("dims,n,tb,hot", CASES)
def test_hop_between_checkerboards(dims, n, tb, hot):
    U = synth.gauge_haar(dims, 4101) if hot else synth.gauge_exp(dims, 0.4, 4101)
    V2 = wilson.volume(dims) // 2
    lat = make_lattice(U, dims, -0.2, 1.0, tb)
    try:
        for out_p in (0, 1):
            psi = synth.gaussian_field(V2, 12, n, 4200 + out_p, np.complex64)
            d_out = to_dev(np.full_like(psi, np.nan))
            mrhs.mrhs_apply_hop_eo(lat, out_p, to_dev(psi), d_out, n)
            got = to_host(d_out).astype(np.complex128)
            ref = eo.hop_between(U, psi.astype(np.complex128), dims, out_p, antiperiodic=(tb == -1))
            assert np.all(np.isfinite(got))
            assert site_rel_err(got, ref) <= 1e-6
    finally:
        mrhs.mrhs_destroy_lattice(lat)


@pytest.mark.parametrize("dims,n,tb,hot", CASES)
def test_schur_operator(dims, n, tb, hot):
    mass, csw = -0.2, 1.0
    U = synth.gauge_haar(dims, 4301) if hot else synth.gauge_exp(dims, 0.4, 4301)
    V2 = wilson.volume(dims) // 2
    C = eo.site_matrix(wilson.clover_term(U, dims, csw), mass)
    lat = make_lattice(U, dims, mass, csw, tb)
    try:
        psi = synth.gaussian_field(V2, 12, n, 4400, np.complex64)
        d_out = to_dev(np.full_like(psi, np.nan))
        mrhs.mrhs_apply_schur(lat, to_dev(psi), d_out, n)
        got = to_host(d_out).astype(np.complex128)
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    ref = eo.schur_apply(U, C, psi.astype(np.complex128), dims, antiperiodic=(tb == -1))
    assert np.all(np.isfinite(got))
    assert site_rel_err(got, ref) <= 2e-6


def test_full_size_hop_matches_the_full_stencil():
    """24^3x64, 48 RHS: -1/2 H_eo psi_o from the even-odd kernel equals the even
    half of the full-lattice FP32 stencil applied to psi embedded on the odd sites."""
    import torch

    dims, n = (24, 24, 24, 64), 48
    V = wilson.volume(dims)
    U = synth.gauge_exp(dims, 0.25, 1301)
    lat = make_lattice(U, dims, -0.13, 1.0, -1)
    try:
        g = torch.Generator(device="cuda").manual_seed(44)
        psi_o = torch.randn((V // 2, 12, n), dtype=torch.complex64, device="cuda", generator=g)
        full = torch.zeros((V, 12, n), dtype=torch.complex64, device="cuda")
        odd = torch.from_numpy(eo.cb_sites(dims, 1)).cuda()
        even = torch.from_numpy(eo.cb_sites(dims, 0)).cuda()
        full[odd] = psi_o
        d_full = torch.empty_like(full)
        mrhs.mrhs_apply_D(lat, full, d_full, n, mrhs.MRHS_FP32)
        h_e = torch.empty_like(psi_o)
        mrhs.mrhs_apply_hop_eo(lat, 0, psi_o, h_e, n)
        torch.cuda.synchronize()
        ref = d_full[even].to(torch.complex128)
        got = (-0.5 * h_e).to(torch.complex128)
        err = ((got - ref).abs().pow(2).sum(dim=1) / ref.abs().pow(2).sum(dim=1)).sqrt().max().item()
    finally:
        mrhs.mrhs_destroy_lattice(lat)
    assert err <= 1e-6, err


def test_even_odd_rejects_bad_shapes():
    import torch

    for dims, n in (((3, 2, 2, 2), 2), ((4, 4, 4, 4), 3), ((4, 3, 4, 4), 2)):
        lat = make_lattice(synth.gauge_unit(dims), dims, 0.0, 1.0)
        try:
            V2 = max(1, wilson.volume(dims) // 2)
            a = torch.zeros((V2, 12, n), dtype=torch.complex64, device="cuda")
            b = torch.zeros_like(a)
            with pytest.raises(mrhs.MrhsError) as e:
                mrhs.mrhs_apply_schur(lat, a, b, n)
            assert e.value.status == mrhs.MRHS_ERR_INVALID
            with pytest.raises(mrhs.MrhsError):
                mrhs.mrhs_apply_hop_eo(lat, 0, a, b, n)
        finally:
            mrhs.mrhs_destroy_lattice(lat)
