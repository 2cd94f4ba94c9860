"""Multigrid hierarchy, V-cycle and MG-preconditioned FGMRES solve in FP64.

The paper's solver (Sec. 8) is FGMRES preconditioned by a two-level MG; its
kernel benchmarks use three levels (Sec. 5, 6).  The paper does not spell out
the setup or the cycle, so the oracle fixes these readings:

* null vectors: N random vectors per level, each relaxed by `setup_sweeps`
  cycles of GMRES(`setup_m`) on A v = 0 (starting from v itself, renormalised
  after every cycle), then chirally split and orthonormalised per aggregate;
* V-cycle on level l for a residual v:
    c = R_l v;
    e = approximate A_{l+1}^{-1} c: GMRES(`coarse_m`) for `coarse_cycles`
        cycles if l+1 is the coarsest level (with `coarse_solver` "gcrodr":
        GCRO-DR(`coarse_m`, `coarse_recycle`) cycles whose recycle space, one
        per RHS, carries over from one V-cycle's coarsest solve to the next),
        otherwise one FGMRES(`inter_m`) cycle preconditioned by the V-cycle of
        level l+1;
    z0 = P_l e;
    z = `smooth_m` iterations of GMRES on A_l v from z0 (post-smoothing only);
  with `smoother_evenodd` the fine level's post-smoothing is instead
    r = v - D z0;  z = z0 + delta,  delta the even-odd solution of D delta = r
    with `smooth_m` GMRES iterations (from 0) on the Schur complement D_hat
    (evenodd.py: right-hand side b_hat, D_hat delta_o = b_hat, reconstruction);
* outer solve: FGMRES(`outer_m`) on the fine operator, restarted from the
  true residual until ||b - D x|| / ||b|| <= tol for every RHS.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import coarse, evenodd, gcrodr, krylov, sap, wilson
from .conventions import FINE_CHIRALITY


@dataclass
class MGParams:
    blocks: list = field(default_factory=lambda: [(4, 4, 4, 4)])
    nvec: list = field(default_factory=lambda: [8])
    setup_sweeps: int = 4
    setup_m: int = 8
    smooth_m: int = 4
    coarse_m: int = 16
    coarse_cycles: int = 2
    inter_m: int = 8
    outer_m: int = 8
    tol: float = 1e-10
    max_outer_cycles: int = 100
    smoother_evenodd: bool = False
    smoother_sap: bool = False
    sap_block: tuple = (4, 4, 4, 4)
    sap_cycles: int = 1
    sap_mr: int = 4
    coarse_solver: str = "gmres"   # or "gcrodr": GCRO-DR(coarse_m, coarse_recycle) with a recycle space
    coarse_recycle: int = 0        # kept per RHS across the coarsest solves of all V-cycles


@dataclass
class Level:
    dims: tuple
    dof: int
    apply: object
    chirality: np.ndarray
    stencil: np.ndarray = None   # (V, 9, dof, dof) on coarse levels
    P: np.ndarray = None         # prolongator to the next level
    block: tuple = None
    eo: tuple = None             # fine level: (U, site matrix C, dims, antiperiodic) for the even-odd smoother
    recycle: list = None         # coarsest level with GCRO-DR: one recycle space per RHS


def setup_nullvecs(apply_A, v0: np.ndarray, sweeps: int, m: int) -> np.ndarray:
    """Relax random vectors towards the near-null space of A (one RHS each)."""
    v = np.array(v0, dtype=np.complex128, copy=True)
    zero = np.zeros_like(v)
    for _ in range(sweeps):
        v = krylov.gmres(apply_A, zero, v, m, 1)
        v = v / krylov.norms(v)
    return v


def build_hierarchy(U, dims, mass, csw, params: MGParams, init_vecs,
                    antiperiodic=True, nullvecs=None):
    """Levels 0 .. L-1; `init_vecs[l]` is the (V_l, dof_l, N_l) random start.

    If `nullvecs` is given it replaces the relaxed vectors (setup skipped).
    """
    clover = wilson.clover_term(U, dims, csw)

    def fine(psi):
        return wilson.apply_D(U, clover, psi, dims, mass, antiperiodic)

    levels = [Level(tuple(dims), 12, fine, FINE_CHIRALITY,
                    eo=(U, evenodd.site_matrix(clover, mass), tuple(dims), antiperiodic))]
    for l, (block, N) in enumerate(zip(params.blocks, params.nvec)):
        lev = levels[l]
        if nullvecs is not None:
            vecs = nullvecs[l]
        else:
            vecs = setup_nullvecs(lev.apply, init_vecs[l], params.setup_sweeps, params.setup_m)
        P = coarse.build_prolongator(vecs, lev.dims, block, lev.chirality)
        cd = coarse.coarse_dims(lev.dims, block)
        if l == 0:
            A = coarse.galerkin_fine(U, clover, P, lev.dims, block, mass, antiperiodic)
        else:
            A = coarse.galerkin_coarse(lev.stencil, P, lev.dims, block)
        lev.P = P
        lev.block = tuple(block)

        def capply(phi, A=A, cd=cd):
            return coarse.apply_coarse(A, phi, cd)

        levels.append(Level(cd, 2 * N, capply, coarse.coarse_chirality(2 * N), stencil=A))
    return levels


def vcycle(levels, l: int, v: np.ndarray, params: MGParams) -> np.ndarray:
    lev = levels[l]
    last = len(levels) - 1
    c = coarse.restrict(lev.P, v, lev.dims, lev.block)
    nxt = levels[l + 1]
    if l + 1 == last and params.coarse_solver == "gcrodr":
        e, nxt.recycle, _ = gcrodr.solve(nxt.apply, c, np.zeros_like(c), params.coarse_m, params.coarse_recycle,
                                         0.0, params.coarse_cycles, nxt.recycle)
    elif l + 1 == last:
        e = krylov.gmres(nxt.apply, c, np.zeros_like(c), params.coarse_m, params.coarse_cycles)
    else:
        e = krylov.fgmres_fixed(nxt.apply, c, lambda u: vcycle(levels, l + 1, u, params),
                                params.inter_m)
    z0 = coarse.prolong(lev.P, e, lev.dims, lev.block)
    if l == 0 and params.smoother_sap:
        return sap.sap_smooth(lev.apply, v, z0, lev.dims, params.sap_block, params.sap_cycles, params.sap_mr)
    if l == 0 and params.smoother_evenodd:
        return z0 + evenodd_smooth(lev, v - lev.apply(z0), params.smooth_m)
    return krylov.gmres(lev.apply, v, z0, params.smooth_m, 1)


def evenodd_smooth(lev, r: np.ndarray, m: int) -> np.ndarray:
    """delta with D delta ~= r: m GMRES iterations on D_hat delta_o = b_hat from 0,
    then delta_e from the reconstruction formula."""
    U, C, dims, ap = lev.eo
    bhat = evenodd.schur_rhs(U, C, r, dims, ap)
    d_o = krylov.gmres(lambda psi: evenodd.schur_apply(U, C, psi, dims, ap), bhat, np.zeros_like(bhat), m, 1)
    return evenodd.schur_reconstruct(U, C, r, d_o, dims, ap)


def solve(levels, b: np.ndarray, params: MGParams):
    """MG-preconditioned FGMRES on the fine level; returns (x, history)."""
    return krylov.fgmres(levels[0].apply, b, lambda v: vcycle(levels, 0, v, params),
                         params.outer_m, params.tol, params.max_outer_cycles)
