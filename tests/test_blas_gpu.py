"""GPU parity: batched inner products, norms and linear combinations (Sec. 7).

Compared with the oracle's per-RHS dots/norms in FP64.  FP32 fields: relative
error of each result <= 1e-5 of the sum of magnitudes (FP32 products,
FP64 accumulation across blocks); FP64 fields: <= 1e-13.
"""
import numpy as np
import pytest

import synth
from oracle import krylov
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import empty_like_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rows,nrhs,k", [(1, 1, 1), (37, 3, 2), (12 * 4096 + 7, 12, 9),
                                         (5000, 48, 3), (777, 64, 17), (3000, 256, 1), (20000, 5, 8)])
@pytest.mark.parametrize("prec", [mrhs.MRHS_FP32, mrhs.MRHS_FP64])
def test_multi_dot_norm_lincomb(rows, nrhs, k, prec):
    cdt = np.complex64 if prec == mrhs.MRHS_FP32 else np.complex128
    tol = 1e-5 if prec == mrhs.MRHS_FP32 else 1e-13
    basis = synth.gaussian_field(k * rows, 1, nrhs, 11 + k, cdt).reshape(k, rows, nrhs)
    w = synth.gaussian_field(rows, 1, nrhs, 12, cdt).reshape(rows, nrhs)
    bd, wd = to_dev(basis), to_dev(w)
    out = empty_like_dev((k, nrhs), np.complex128)
    mrhs.mrhs_blas_multi_dot(bd, k, wd, rows, nrhs, prec, out)
    got = to_host(out)
    b64, w64 = basis.astype(np.complex128), w.astype(np.complex128)
    for j in range(k):
        ref = krylov.dots(b64[j], w64)
        scale = np.einsum("ir,ir->r", np.abs(b64[j]), np.abs(w64))
        assert np.all(np.abs(got[j] - ref) <= tol * scale)
    # twice in a row: the completion counter resets itself
    mrhs.mrhs_blas_multi_dot(bd, k, wd, rows, nrhs, prec, out)
    assert np.array_equal(to_host(out), got)

    nrm = empty_like_dev((nrhs,), np.float64)
    mrhs.mrhs_blas_norm2(wd, rows, nrhs, prec, nrm)
    ref = krylov.norms(w64) ** 2
    assert np.all(np.abs(to_host(nrm) - ref) <= tol * ref)

    coef = (synth.gaussian_field(k, 1, nrhs, 13)).reshape(k, nrhs)
    cd = to_dev(coef)
    mrhs.mrhs_blas_lincomb(wd, bd, k, cd, -0.5, rows, nrhs, prec)
    ref = w64 - 0.5 * np.einsum("jr,jir->ir", coef, b64)
    scale = np.abs(w64) + 0.5 * np.einsum("jr,jir->ir", np.abs(coef), np.abs(b64))
    assert np.all(np.abs(to_host(wd) - ref) <= 4 * tol * scale + 1e-30)


def test_batching_invariance_of_dots():
    """A column's result does not depend on the values in the other columns."""
    rows, nrhs = 4099, 12
    a = synth.gaussian_field(rows, 1, nrhs, 1, np.complex64).reshape(rows, nrhs)
    b = synth.gaussian_field(rows, 1, nrhs, 2, np.complex64).reshape(rows, nrhs)
    out1 = empty_like_dev((1, nrhs), np.complex128)
    mrhs.mrhs_blas_multi_dot(to_dev(a), 1, to_dev(b), rows, nrhs, mrhs.MRHS_FP32, out1)
    a2, b2 = a.copy(), b.copy()
    a2[:, 1:] = 0
    b2[:, 1:] = 7
    out2 = empty_like_dev((1, nrhs), np.complex128)
    mrhs.mrhs_blas_multi_dot(to_dev(a2), 1, to_dev(b2), rows, nrhs, mrhs.MRHS_FP32, out2)
    assert to_host(out1)[0, 0] == to_host(out2)[0, 0]
