"""Per-RHS Krylov solvers in FP64 (Sec. 7 and 8 of the paper).

The n right-hand sides are n independent systems solved together: each RHS
keeps its own Krylov space, Hessenberg matrix and least-squares problem; only
the operator applications and the inner products are batched over the RHS
index ("simultaneous" rather than "sequential" inner products, Sec. 7).

Fields are arrays (..., n) with the RHS index last; inner products and norms
reduce over every other axis and return one value per RHS.
"""
from __future__ import annotations

import numpy as np


def dots(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """<a_r, b_r> = sum_i conj(a[i, r]) b[i, r] for every RHS r."""
    n = a.shape[-1]
    return np.einsum("ir,ir->r", np.conj(a.reshape(-1, n)), b.reshape(-1, n))


def norms(a: np.ndarray) -> np.ndarray:
    return np.sqrt(np.real(dots(a, a)))


def _safe_inverse(x: np.ndarray) -> np.ndarray:
    out = np.zeros_like(x)
    nz = x > 0
    out[nz] = 1.0 / x[nz]
    return out


def hessenberg_lstsq(H: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """y_r = argmin || beta_r e_1 - H_r y ||_2 for each RHS r; H is (n, m+1, m)."""
    n, m1, m = H.shape
    y = np.zeros((n, m), dtype=np.complex128)
    for r in range(n):
        rhs = np.zeros(m1, dtype=np.complex128)
        rhs[0] = beta[r]
        y[r] = np.linalg.lstsq(H[r], rhs, rcond=None)[0]
    return y


def arnoldi_correction(apply_A, r0: np.ndarray, m: int, precond=None) -> np.ndarray:
    """One GMRES(m) cycle (FGMRES(m) if `precond` is given) from residual r0.

    Arnoldi with modified Gram-Schmidt, per RHS.  Returns the correction
    V y (or Z y with Z_j = precond(V_j)) that minimises the residual norm of
    each RHS over its own Krylov space.
    """
    beta = norms(r0)
    basis = [r0 * _safe_inverse(beta)]
    Z = []
    n = r0.shape[-1]
    H = np.zeros((n, m + 1, m), dtype=np.complex128)
    for j in range(m):
        z = precond(basis[j]) if precond is not None else basis[j]
        Z.append(z)
        w = apply_A(z)
        for i in range(j + 1):
            h = dots(basis[i], w)
            H[:, i, j] = h
            w = w - basis[i] * h
        hn = norms(w)
        H[:, j + 1, j] = hn
        basis.append(w * _safe_inverse(hn))
    y = hessenberg_lstsq(H, beta)
    corr = np.zeros_like(r0)
    for j in range(m):
        corr = corr + Z[j] * y[:, j]
    return corr


def gmres(apply_A, b: np.ndarray, x0: np.ndarray, m: int, cycles: int = 1) -> np.ndarray:
    """Restarted GMRES(m) with a fixed number of cycles, per RHS."""
    x = np.array(x0, dtype=np.complex128, copy=True)
    for _ in range(cycles):
        r = b - apply_A(x)
        x = x + arnoldi_correction(apply_A, r, m)
    return x


def fgmres(apply_A, b: np.ndarray, precond, m: int, tol: float, max_cycles: int,
           x0=None):
    """Restarted flexible GMRES(m) to a relative true residual `tol`, per RHS.

    Each cycle starts from the true residual b - A x.  Returns (x, history)
    where history[c] holds ||b - A x|| / ||b|| per RHS before cycle c.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    bn = norms(b)
    hist = []
    for _ in range(max_cycles):
        r = b - apply_A(x)
        rel = norms(r) * _safe_inverse(bn)
        hist.append(rel)
        if np.all(rel <= tol):
            return x, hist
        x = x + arnoldi_correction(apply_A, r, m, precond)
    r = b - apply_A(x)
    hist.append(norms(r) * _safe_inverse(bn))
    return x, hist


def fgmres_fixed(apply_A, b: np.ndarray, precond, m: int) -> np.ndarray:
    """One FGMRES(m) cycle from x = 0 (the intermediate-level solve)."""
    return arnoldi_correction(apply_A, b, m, precond)
