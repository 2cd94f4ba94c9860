"""Seeded random inputs: SU(3) gauge fields, Gaussian sources, random vectors.

Conventions (shared by every consumer of these arrays):

* Lattice extents ``dims = (Lx, Ly, Lz, Lt)``; the lexicographic site index is
  ``x + Lx*(y + Ly*(z + Lz*t))`` (x fastest).
* Gauge field: complex128 array of shape ``(V, 4, 3, 3)``; ``U[x, mu]`` is the
  link from site x to x + mu_hat, mu = 0..3 for x, y, z, t.  In memory this is
  the interleaved (re, im) FP64 layout ``[V][4][3][3]``.
* Fields with several right-hand sides: shape ``(V, dof, n)`` with the RHS
  index innermost (``dof`` = 12 = 4 spins x 3 colours on the fine level).

Random numbers come from numpy's Philox-4x32-10 counter-based generator
(Salmon et al., SC'11), keyed by an integer seed, so the same seed gives the
same field on every machine.

The paper benchmarks its kernels on random ("hot") gauge fields with random
sources (Sec. 2); the full-solve workload uses smoother fields
U = exp(i*eps*H) with H a Gaussian traceless Hermitian 3x3 matrix.
"""
from __future__ import annotations

import numpy as np

_GELL_MANN = None


def lattice_volume(dims) -> int:
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return Lx * Ly * Lz * Lt


def site_index(coords, dims):
    """Lexicographic index of integer coordinates (..., 4) -> (...)."""
    c = np.asarray(coords)
    Lx, Ly, Lz, Lt = dims
    return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))


def site_coords(idx, dims):
    """Inverse of :func:`site_index`: (...) -> (..., 4)."""
    i = np.asarray(idx)
    Lx, Ly, Lz, Lt = dims
    x = i % Lx
    y = (i // Lx) % Ly
    z = (i // (Lx * Ly)) % Lz
    t = i // (Lx * Ly * Lz)
    return np.stack([x, y, z, t], axis=-1)


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    global _GELL_MANN
    if _GELL_MANN is None:
        g = np.zeros((8, 3, 3), dtype=np.complex128)
        g[0][0, 1] = g[0][1, 0] = 1
        g[1][0, 1] = -1j
        g[1][1, 0] = 1j
        g[2][0, 0] = 1
        g[2][1, 1] = -1
        g[3][0, 2] = g[3][2, 0] = 1
        g[4][0, 2] = -1j
        g[4][2, 0] = 1j
        g[5][1, 2] = g[5][2, 1] = 1
        g[6][1, 2] = -1j
        g[6][2, 1] = 1j
        g[7][0, 0] = g[7][1, 1] = 1 / np.sqrt(3)
        g[7][2, 2] = -2 / np.sqrt(3)
        _GELL_MANN = g
    return _GELL_MANN


def gauge_unit(dims) -> np.ndarray:
    V = lattice_volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def _haar_su3(rng: np.random.Generator, count: int) -> np.ndarray:
    """`count` Haar-distributed SU(3) matrices.

    QR of a complex Ginibre matrix with the phases of R's diagonal moved into
    Q gives a Haar U(3) matrix (Mezzadri, Notices AMS 54 (2007) 592); dividing
    by a cube root of its determinant maps it to SU(3) and keeps the measure
    invariant under left multiplication.
    """
    z = rng.standard_normal((count, 3, 3, 2))
    z = (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    ph = d / np.abs(d)
    q = q * ph[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q


def gauge_haar(dims, seed: int) -> np.ndarray:
    """Hot-start gauge field: every link Haar-random in SU(3)."""
    V = lattice_volume(dims)
    rng = make_rng(seed)
    out = np.empty((V * 4, 3, 3), dtype=np.complex128)
    chunk = 1 << 18
    for s in range(0, V * 4, chunk):
        e = min(V * 4, s + chunk)
        out[s:e] = _haar_su3(rng, e - s)
    return out.reshape(V, 4, 3, 3)


def gauge_exp(dims, eps: float, seed: int) -> np.ndarray:
    """U = exp(i*eps*H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1).

    exp is taken through the eigen-decomposition of the Hermitian H, which
    gives a unitary matrix of determinant exp(i*eps*tr H) = 1.
    """
    V = lattice_volume(dims)
    rng = make_rng(seed)
    lam = _gell_mann()
    out = np.empty((V * 4, 3, 3), dtype=np.complex128)
    chunk = 1 << 18
    for s in range(0, V * 4, chunk):
        e = min(V * 4, s + chunk)
        h = rng.standard_normal((e - s, 8))
        H = (h @ lam.reshape(8, 9)).reshape(e - s, 3, 3) * 0.5
        w, Q = np.linalg.eigh(H)
        out[s:e] = (Q * np.exp(1j * eps * w)[:, None, :]) @ np.swapaxes(Q.conj(), 1, 2)
    return out.reshape(V, 4, 3, 3)


def gauge_transform_haar(dims, seed: int) -> np.ndarray:
    """A random SU(3) gauge transformation g(x), shape (V, 3, 3)."""
    return _haar_su3(make_rng(seed), lattice_volume(dims))


def gaussian_field(nsites: int, dof: int, nrhs: int, seed: int,
                   dtype=np.complex128) -> np.ndarray:
    """Gaussian complex field (nsites, dof, nrhs): Re and Im iid N(0, 1)."""
    rng = make_rng(seed)
    real_dtype = np.float32 if dtype == np.complex64 else np.float64
    a = rng.standard_normal((nsites, dof, nrhs, 2), dtype=real_dtype)
    return a.view(dtype).reshape(nsites, dof, nrhs)
