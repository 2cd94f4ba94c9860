"""Even-odd (checkerboard) decomposition of the fine operator, FP64.

Test infrastructure: the plain reference that the CUDA path is checked
against; nothing on the product path imports it.

Sec. 4 of the paper benchmarks M_eooe, the hopping term between the two
checkerboarded lattices, next to the full-lattice hopping term.  Here:

* site parity p(x) = (x + y + z + t) mod 2; with an even x extent every x row
  holds half of its sites in each parity, and the sites of one parity in
  increasing lexicographic index s are numbered cb = s // 2 (half-lattice
  fields are (V/2, 12, n) arrays in that order);
* D = C - 1/2 H, C the site-diagonal clover + mass term (4 + m + clover),
  H the hopping term of `wilson.hop_term`.  H only connects sites of
  opposite parity, so in (even, odd) block form
      D = [[C_ee, -1/2 H_eo], [-1/2 H_oe, C_oo]],
  with H_eo the hops from odd to even sites (M_eooe applied to an odd field);
* the Schur complement on the odd sites is
      D_hat = C_oo - 1/4 H_oe C_ee^{-1} H_eo,
  and D x = b is solved by
      b_hat = b_o + 1/2 H_oe C_ee^{-1} b_e,   D_hat x_o = b_hat,
      x_e = C_ee^{-1} (b_e + 1/2 H_eo x_o).

Every function here is written from these definitions: the parity-restricted
hops embed the half field in a full one and call the full hopping term.
"""
from __future__ import annotations

import numpy as np

from . import wilson


def parity(dims) -> np.ndarray:
    """p[s] for the lexicographic site index s (x fastest)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


def cb_sites(dims, p: int) -> np.ndarray:
    """Full-lattice indices of the parity-p sites, increasing (cb order)."""
    if dims[0] % 2:
        raise ValueError("the checkerboard numbering needs an even x extent")
    return np.nonzero(parity(dims) == p)[0]


def to_half(psi: np.ndarray, dims, p: int) -> np.ndarray:
    return psi[cb_sites(dims, p)]


def from_half(half: np.ndarray, dims, p: int) -> np.ndarray:
    """A full field equal to `half` on the parity-p sites and zero elsewhere."""
    V = wilson.volume(dims)
    full = np.zeros((V,) + half.shape[1:], dtype=np.result_type(half, np.complex128))
    full[cb_sites(dims, p)] = half
    return full


def hop_between(U: np.ndarray, psi_half: np.ndarray, dims, out_parity: int,
                antiperiodic: bool = True) -> np.ndarray:
    """H_{p,1-p} psi: the hopping term (without -1/2) from the sites of parity
    1 - out_parity to those of parity out_parity (M_eooe).  Needs even extents
    in all four directions (else a periodic wrap joins equal parities)."""
    if any(int(L) % 2 for L in dims):
        raise ValueError("the even-odd decomposition needs even lattice extents")
    full = from_half(psi_half, dims, 1 - out_parity)
    return to_half(wilson.hop_term(U, full, dims, antiperiodic), dims, out_parity)


def site_matrix(clover: np.ndarray, mass: float) -> np.ndarray:
    """C = (4 + m) 1 + clover term, per site (V, 12, 12)."""
    return clover + (4.0 + mass) * np.eye(12)


def apply_sites(M: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return np.einsum("vij,vjn->vin", M, psi)


def schur_apply(U: np.ndarray, C: np.ndarray, psi_o: np.ndarray, dims,
                antiperiodic: bool = True) -> np.ndarray:
    """D_hat psi_o = C_oo psi_o - 1/4 H_oe C_ee^{-1} H_eo psi_o; C = site_matrix(...)."""
    Ce_inv = np.linalg.inv(C[cb_sites(dims, 0)])
    t_e = apply_sites(Ce_inv, hop_between(U, psi_o, dims, 0, antiperiodic))
    return apply_sites(C[cb_sites(dims, 1)], psi_o) - 0.25 * hop_between(U, t_e, dims, 1, antiperiodic)


def schur_rhs(U: np.ndarray, C: np.ndarray, b: np.ndarray, dims, antiperiodic: bool = True) -> np.ndarray:
    """b_hat = b_o + 1/2 H_oe C_ee^{-1} b_e."""
    Ce_inv = np.linalg.inv(C[cb_sites(dims, 0)])
    t_e = apply_sites(Ce_inv, to_half(b, dims, 0))
    return to_half(b, dims, 1) + 0.5 * hop_between(U, t_e, dims, 1, antiperiodic)


def schur_reconstruct(U: np.ndarray, C: np.ndarray, b: np.ndarray, x_o: np.ndarray, dims,
                      antiperiodic: bool = True) -> np.ndarray:
    """The full solution from x_o: x_e = C_ee^{-1} (b_e + 1/2 H_eo x_o)."""
    Ce_inv = np.linalg.inv(C[cb_sites(dims, 0)])
    x_e = apply_sites(Ce_inv, to_half(b, dims, 0) + 0.5 * hop_between(U, x_o, dims, 0, antiperiodic))
    return from_half(x_e, dims, 0) + from_half(x_o, dims, 1)
