"""Even-odd (checkerboard) decomposition of the coarse 9-point operator, FP64.

Test infrastructure: the plain reference the coarse even-odd kernels are
checked against; nothing on the product path imports it.

Sec. 6 of the paper benchmarks the coarse-level M_eooe, the hop between the
two checkerboards of the coarse lattice.  The coarse operator is
    D_c = A_0 + H,   (H phi)(x) = sum_{d=1..8} A_d(x) phi(x + delta_d),
a site-local dense block A_0 (nc x nc) plus nearest-neighbour hops.  With all
coarse extents even, every hop joins sites of opposite parity
((x + y + z + t) mod 2), so in (even, odd) order
    D_c = [[A_ee, H_eo], [H_oe, A_oo]]
with A_ee, A_oo block diagonal.  Its Schur complement on the odd sites is
    D_hat = A_oo - H_oe A_ee^{-1} H_eo,
and D_c x = b is solved by
    b_hat = b_o - H_oe A_ee^{-1} b_e,   D_hat x_o = b_hat,
    x_e   = A_ee^{-1} (b_e - H_eo x_o).
Half fields hold the sites of one parity in increasing lexicographic order
(the numbering of the fine level's even-odd code).  The coarse operator has no
factor -1/2 on its hops (it is R D P, which already contains it), hence the
signs differ from the fine level's D = C - 1/2 H.
"""
from __future__ import annotations

import numpy as np

from . import coarse, evenodd


def check_dims(cdims) -> None:
    if any(int(L) % 2 for L in cdims):
        raise ValueError("the coarse even-odd decomposition needs even coarse extents")


def hop_between(A: np.ndarray, phi_half: np.ndarray, cdims, out_parity: int) -> np.ndarray:
    """H_{p,1-p} phi: the 8 hop terms of the stencil from the sites of parity
    1 - out_parity to those of parity out_parity (coarse M_eooe)."""
    check_dims(cdims)
    full = evenodd.from_half(phi_half, cdims, 1 - out_parity)
    hops = np.array(A, copy=True)
    hops[:, 0] = 0
    return evenodd.to_half(coarse.apply_coarse(hops, full, cdims), cdims, out_parity)


def self_block_inverse(A: np.ndarray, cdims, p: int) -> np.ndarray:
    """A_0(x)^{-1} on the sites of parity p, (V/2, nc, nc)."""
    return np.linalg.inv(A[evenodd.cb_sites(cdims, p), 0])


def apply_blocks(M: np.ndarray, phi: np.ndarray) -> np.ndarray:
    return np.einsum("vkl,vlr->vkr", M, phi)


def schur_apply(A: np.ndarray, phi_o: np.ndarray, cdims) -> np.ndarray:
    """D_hat phi_o = A_oo phi_o - H_oe A_ee^{-1} H_eo phi_o."""
    t_e = apply_blocks(self_block_inverse(A, cdims, 0), hop_between(A, phi_o, cdims, 0))
    A_oo = A[evenodd.cb_sites(cdims, 1), 0]
    return apply_blocks(A_oo, phi_o) - hop_between(A, t_e, cdims, 1)


def schur_rhs(A: np.ndarray, b: np.ndarray, cdims) -> np.ndarray:
    """b_hat = b_o - H_oe A_ee^{-1} b_e for a full coarse field b."""
    t_e = apply_blocks(self_block_inverse(A, cdims, 0), evenodd.to_half(b, cdims, 0))
    return evenodd.to_half(b, cdims, 1) - hop_between(A, t_e, cdims, 1)


def schur_reconstruct(A: np.ndarray, b: np.ndarray, x_o: np.ndarray, cdims) -> np.ndarray:
    """The full solution from x_o: x_e = A_ee^{-1} (b_e - H_eo x_o)."""
    x_e = apply_blocks(self_block_inverse(A, cdims, 0),
                       evenodd.to_half(b, cdims, 0) - hop_between(A, x_o, cdims, 0))
    return evenodd.from_half(x_e, cdims, 0) + evenodd.from_half(x_o, cdims, 1)
