"""Schwarz alternating procedure (SAP) smoother on the fine level, FP64.

Test infrastructure: the plain reference that the CUDA path is checked
against; nothing on the product path imports it.

The paper's outlook (Sec. 9) names SAP as the smoother to bring to the MRHS
solver next; the Krylov smoother is the one its measurements use.  SAP is a
multiplicative domain decomposition, written here from its definition:

* the lattice is cut into blocks of extents B (every B_mu divides L_mu, and
  L_mu / B_mu is even), coloured by block parity
      c(x) = (sum_mu floor(x_mu / B_mu)) mod 2;
  with an even number of blocks in every direction two blocks of one colour
  are never neighbours, not even across the periodic wrap, so the restriction
  D_cc of D to the sites of colour c is block diagonal: one independent
  system D_BB per block (the hops that leave a block are dropped);
* one SAP cycle for D z = v, starting from z:
      for c = 0, 1:   r = v - D z
                      e_B ~= D_BB^{-1} r_B on every block B of colour c
                      z = z + e
  where each block system is approximated by `mr_steps` minimal-residual
  (MR) iterations from zero with inner products over the block alone (one
  value per block and RHS):
      rho = r_B;  repeat:  q = D_BB rho,  alpha = <q, rho> / <q, q>,
                           e_B += alpha rho,  rho -= alpha q;
* the smoother applies `cycles` SAP cycles.

Fields are (V, 12, n) arrays with the RHS index last, as in `wilson`.
"""
from __future__ import annotations

import numpy as np


def site_coords(dims) -> np.ndarray:
    """(V, 4) coordinates (x, y, z, t) of the lexicographic sites (x fastest)."""
    Lx, Ly, Lz, Lt = dims
    s = np.arange(Lx * Ly * Lz * Lt)
    return np.stack([s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)], axis=1)


def check_blocks(dims, B) -> None:
    for L, b in zip(dims, B):
        if b <= 0 or L % b or (L // b) % 2:
            raise ValueError("SAP needs block extents that divide the lattice into an even number of blocks "
                             "in every direction")


def block_color(dims, B) -> np.ndarray:
    """c(x) = (sum_mu floor(x_mu / B_mu)) mod 2 for every site."""
    check_blocks(dims, B)
    return (site_coords(dims) // np.asarray(B)).sum(axis=1) % 2


def block_index(dims, B) -> np.ndarray:
    """Lexicographic index of the block that holds each site."""
    check_blocks(dims, B)
    nb = [L // b for L, b in zip(dims, B)]
    bc = site_coords(dims) // np.asarray(B)
    return bc[:, 0] + nb[0] * (bc[:, 1] + nb[1] * (bc[:, 2] + nb[2] * bc[:, 3]))


def block_dots(a: np.ndarray, b: np.ndarray, bid: np.ndarray, nblocks: int) -> np.ndarray:
    """<a, b> over each block and RHS: (nblocks, n)."""
    per_site = np.einsum("vir,vir->vr", np.conj(a), b)
    out = np.zeros((nblocks, a.shape[-1]), dtype=np.complex128)
    np.add.at(out, bid, per_site)
    return out


def restricted_apply(apply_D, rho: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """D_cc rho for rho living on the colour-c sites (mask): the hops from the
    other colour see zero, and the result is kept on colour c only."""
    m = mask[:, None, None]
    return m * apply_D(m * rho)


def block_mr(apply_D, r: np.ndarray, mask: np.ndarray, bid: np.ndarray, nblocks: int,
             steps: int) -> np.ndarray:
    """e ~= D_cc^{-1} r on the colour-c blocks by `steps` MR iterations per block."""
    m = mask[:, None, None]
    rho = m * r
    e = np.zeros_like(rho)
    for _ in range(steps):
        q = restricted_apply(apply_D, rho, mask)
        qr = block_dots(q, rho, bid, nblocks)
        qq = np.real(block_dots(q, q, bid, nblocks))
        alpha = np.zeros_like(qr)
        nz = qq > np.finfo(np.float64).tiny   # a block that has converged to zero keeps alpha = 0
        alpha[nz] = qr[nz] / qq[nz]
        a_site = alpha[bid][:, None, :]
        e = e + a_site * rho
        rho = rho - a_site * q
    return e


def sap_smooth(apply_D, v: np.ndarray, z0: np.ndarray, dims, B, cycles: int, mr_steps: int) -> np.ndarray:
    """`cycles` SAP cycles for D z = v from z0 (colour 0 first in every cycle)."""
    color = block_color(dims, B)
    bid = block_index(dims, B)
    nblocks = int(bid.max()) + 1
    z = np.array(z0, dtype=np.complex128, copy=True)
    for _ in range(cycles):
        for c in (0, 1):
            mask = (color == c).astype(np.float64)
            r = v - apply_D(z)
            z = z + block_mr(apply_D, r, mask, bid, nblocks, mr_steps)
    return z
