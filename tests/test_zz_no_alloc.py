"""The no-allocation multi-dot (mrhs_blas_multi_dot_noalloc) against the
regular entry point, through the C ABI, on two calls in a row.

It exists for callers that may not allocate device memory while they run
(e.g. while recording a CUDA graph); its scratch is a static device array.
Same tolerance as the other BLAS tests: the two entry points sum in a
different block order, so results agree to rounding, not bit for bit.
This file is collected last so a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

import synth
from paper_2211_13719_gb300 import mrhs
from tests.gpu_util import empty_like_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,rows,nrhs,k", [(mrhs.MRHS_FP32, 12 * 4096 + 7, 12, 9),
                                              (mrhs.MRHS_FP64, 20011, 64, 3),
                                              (mrhs.MRHS_FP32, 3 * 10 ** 6, 48, 1)])
def test_noalloc_multi_dot_matches_regular(prec, rows, nrhs, k):
    cdt = np.complex64 if prec == mrhs.MRHS_FP32 else np.complex128
    tol = 1e-5 if prec == mrhs.MRHS_FP32 else 1e-13
    basis = synth.gaussian_field(k * rows, 1, nrhs, 51 + k, cdt).reshape(k, rows, nrhs)
    w = synth.gaussian_field(rows, 1, nrhs, 52, cdt).reshape(rows, nrhs)
    bd, wd = to_dev(basis), to_dev(w)
    ref = empty_like_dev((k, nrhs), np.complex128)
    mrhs.mrhs_blas_multi_dot(bd, k, wd, rows, nrhs, prec, ref)
    ref_h = to_host(ref)
    scale = np.stack([np.einsum("ir,ir->r", np.abs(basis[j]).astype(np.float64), np.abs(w).astype(np.float64))
                      for j in range(k)])
    for _ in range(2):
        out = empty_like_dev((k, nrhs), np.complex128)
        out.fill_(float("nan"))
        mrhs.mrhs_blas_multi_dot_noalloc(bd, k, wd, rows, nrhs, prec, out)
        got = to_host(out)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref_h) <= tol * scale)


def test_noalloc_multi_dot_rejects_too_many_rhs():
    rows, nrhs = 100, 65
    a = empty_like_dev((rows, nrhs), np.complex64)
    out = empty_like_dev((1, nrhs), np.complex128)
    with pytest.raises(mrhs.MrhsError) as e:
        mrhs.mrhs_blas_multi_dot_noalloc(a, 1, a, rows, nrhs, mrhs.MRHS_FP32, out)
    assert e.value.status == mrhs.MRHS_ERR_INVALID
