"""GCRO-DR: GMRES with deflated restarting and subspace recycling, FP64.

Test infrastructure: the plain reference that a CUDA coarsest-level solver
would be checked against; nothing on the product path imports it.

The paper's outlook (Sec. 9) names a GCRO-DR coarsest-level solver that
recycles a deflation space across the many coarse solves of an MG solve.  The
method (GCRO with deflated restarting) is written here from its definition,
for one RHS at a time (every RHS keeps its own recycle space, as every RHS
keeps its own Krylov space elsewhere in this package):

* recycle space U (N x k) with C = A U orthonormal; entering a solve with a
  recycled U: A U = Q R (thin QR), C = Q, U = U R^{-1}, then
  x += U C^H r,  r -= C C^H r;
* a cycle with a recycle space: m - k Arnoldi steps of the projected operator
  (I - C C^H) A from v_1 = r / |r| give V_{m-k+1}, the Hessenberg H and
  B = C^H A V_{m-k}; with D = diag(1 / |u_i|), U^ = U D,
      G = [[D, B], [0, H]],   W^ = [C, V_{m-k+1}],   V^ = [U^, V_{m-k}],
  y minimises |W^H r - G y| (least squares), x += V^ y;
  the next recycle space comes from the k harmonic Ritz vectors of smallest
  |theta| of G^H G z = theta G^H W^H V^ z: with P = [z_1 .. z_k],
  G P = Q R, C = W^ Q, U = V^ P R^{-1};
* a cycle without one is GMRES(m); with k > 0 it seeds the recycle space from
  the k harmonic Ritz vectors of smallest |theta| of
  (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T) z = theta z, with U, C from
  H_{m+1,m} P = Q R, C = V_{m+1} Q, U = V_m P R^{-1}.
Every cycle restarts from the true residual b - A x.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def _cols(apply_A, M: np.ndarray) -> np.ndarray:
    return np.stack([apply_A(M[:, i]) for i in range(M.shape[1])], axis=1)


def _arnoldi(apply_A, r: np.ndarray, steps: int, C=None):
    """Arnoldi (modified Gram-Schmidt) on (I - C C^H) A from r / |r|: V (N x steps+1),
    H ((steps+1) x steps) and B = C^H A V_steps (None without C)."""
    N = r.shape[0]
    V = np.zeros((N, steps + 1), dtype=np.complex128)
    H = np.zeros((steps + 1, steps), dtype=np.complex128)
    B = None if C is None else np.zeros((C.shape[1], steps), dtype=np.complex128)
    V[:, 0] = r / np.linalg.norm(r)
    for j in range(steps):
        w = apply_A(V[:, j])
        if C is not None:
            B[:, j] = C.conj().T @ w
            w = w - C @ B[:, j]
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V[:, j + 1] = w / H[j + 1, j]
    return V, H, B


def _smallest(theta: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k eigenvalues of smallest modulus (infinite ones last)."""
    mod = np.where(np.isfinite(theta), np.abs(theta), np.inf)
    return np.argsort(mod, kind="stable")[:k]


def solve_one(apply_A, b: np.ndarray, x0: np.ndarray, m: int, k: int, tol: float, max_cycles: int,
              U=None):
    """GCRO-DR(m, k) for one RHS (1-D vectors).  Returns (x, U, history), history[c]
    = |b - A x| / |b| before cycle c and after the last one."""
    if not 0 <= k < m:
        raise ValueError("GCRO-DR needs 0 <= k < m")
    x = np.array(x0, dtype=np.complex128, copy=True)
    bn = np.linalg.norm(b)
    r = b - apply_A(x)
    hist = [np.linalg.norm(r) / bn if bn > 0 else 0.0]
    C = None
    if U is not None and k > 0:
        Q, R = np.linalg.qr(_cols(apply_A, U))
        C = Q
        U = scipy.linalg.solve_triangular(R, U.T, trans="T", lower=False).T  # U R^{-1}
        cr = C.conj().T @ r
        x = x + U @ cr
        r = b - apply_A(x)
    else:
        U = None
    cycles = 0
    while hist[-1] > tol and cycles < max_cycles and np.linalg.norm(r) > 0:
        if C is None:
            V, H, _ = _arnoldi(apply_A, r, m)
            rhs = np.zeros(m + 1, dtype=np.complex128)
            rhs[0] = np.linalg.norm(r)
            y = np.linalg.lstsq(H, rhs, rcond=None)[0]
            x = x + V[:, :m] @ y
            if k > 0:
                Hm = H[:m, :]
                em = np.zeros(m, dtype=np.complex128)
                em[-1] = 1.0
                F = Hm + abs(H[m, m - 1]) ** 2 * np.outer(np.linalg.solve(Hm.conj().T, em), em)
                theta, Z = np.linalg.eig(F)
                P = Z[:, _smallest(theta, k)]
                Q, R = np.linalg.qr(H @ P)
                C = V @ Q
                U = V[:, :m] @ P @ np.linalg.inv(R)
        else:
            mk = m - k
            V, H, B = _arnoldi(apply_A, r, mk, C)
            dn = 1.0 / np.linalg.norm(U, axis=0)
            G = np.zeros((m + 1, m), dtype=np.complex128)
            G[:k, :k] = np.diag(dn)
            G[:k, k:] = B
            G[k:, k:] = H
            W = np.concatenate([C, V], axis=1)
            Vh = np.concatenate([U * dn[None, :], V[:, :mk]], axis=1)
            y = np.linalg.lstsq(G, W.conj().T @ r, rcond=None)[0]
            x = x + Vh @ y
            theta, Z = scipy.linalg.eig(G.conj().T @ G, G.conj().T @ (W.conj().T @ Vh))
            P = Z[:, _smallest(theta, k)]
            Q, R = np.linalg.qr(G @ P)
            C = W @ Q
            U = Vh @ P @ np.linalg.inv(R)
        r = b - apply_A(x)
        cycles += 1
        hist.append(np.linalg.norm(r) / bn if bn > 0 else 0.0)
    return x, U, hist


def solve(apply_A, b: np.ndarray, x0: np.ndarray, m: int, k: int, tol: float, max_cycles: int,
          recycle=None):
    """GCRO-DR for fields (..., n): every RHS r on its own with its own recycle space
    recycle[r] (None: none yet).  Returns (x, recycle, histories)."""
    shape = b.shape
    n = shape[-1]
    flat = lambda f: f.reshape(-1, n)
    x = np.array(flat(x0), dtype=np.complex128, copy=True)
    bb = flat(b)
    recycle = list(recycle) if recycle is not None and len(recycle) == n else [None] * n
    hists = []
    for c in range(n):
        def A1(v):
            return apply_A(v.reshape(shape[:-1] + (1,))).reshape(-1)
        x[:, c], recycle[c], h = solve_one(A1, bb[:, c], x[:, c], m, k, tol, max_cycles, recycle[c])
        hists.append(h)
    return x.reshape(shape), recycle, hists
