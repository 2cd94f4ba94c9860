"""Fine-level Wilson-clover operator in FP64 (Sec. 4 of the paper).

    D psi(x) = (4 + m) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]
               + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) psi(x)

with F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / 8 from the four clover-leaf
plaquettes Q_{mu nu}(x) in the mu-nu plane at x.  With an antiperiodic time
boundary every hop that crosses t = Lt-1 <-> t = 0 carries a factor -1; the
clover term uses the links as stored (each boundary-crossing plaquette holds
two crossing links, so the sign would cancel anyway).

Fields are (V, 12, n) complex arrays, component index s*3 + c, RHS innermost;
the lexicographic site index is x + Lx*(y + Ly*(z + Lz*t)).  Internally the
oracle reshapes them to the grid (Lt, Lz, Ly, Lx, ...) and shifts with np.roll.
"""
from __future__ import annotations

import numpy as np

from .conventions import GAMMA, GAMMA5, sigma_munu

# array axis of lattice direction mu in the grid view (Lt, Lz, Ly, Lx, ...)
AXIS = (3, 2, 1, 0)


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def to_grid(f: np.ndarray, dims) -> np.ndarray:
    Lx, Ly, Lz, Lt = dims
    return f.reshape((Lt, Lz, Ly, Lx) + f.shape[1:])


def from_grid(g: np.ndarray, dims) -> np.ndarray:
    return g.reshape((volume(dims),) + g.shape[4:])


def shift(g: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """Periodic shift on the grid view: result(x) = g(x + sign * mu_hat)."""
    return np.roll(g, -sign, axis=AXIS[mu])


def dag(a: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(a, -1, -2))


def field_strength(U: np.ndarray, dims) -> dict:
    """F_{mu nu}(x) for mu < nu, each of shape (V, 3, 3).

    Q_{mu nu}(x) is the sum of the four plaquettes that start and end at x and
    lie in the mu-nu plane, all with the same orientation (mu first, then nu).
    """
    Ug = to_grid(U, dims)
    F = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um = Ug[..., mu, :, :]
            Un = Ug[..., nu, :, :]
            Um_xpn = shift(Um, nu, +1)
            Un_xpm = shift(Un, mu, +1)
            Um_xmm = shift(Um, mu, -1)
            Un_xmm = shift(Un, mu, -1)
            Um_xmmpn = shift(Um_xmm, nu, +1)
            Un_xmn = shift(Un, nu, -1)
            Um_xmn = shift(Um, nu, -1)
            Um_xmmmn = shift(Um_xmm, nu, -1)
            Un_xmmmn = shift(Un_xmm, nu, -1)
            Un_xmnpm = shift(Un_xmn, mu, +1)
            leaf1 = Um @ Un_xpm @ dag(Um_xpn) @ dag(Un)
            leaf2 = Un @ dag(Um_xmmpn) @ dag(Un_xmm) @ Um_xmm
            leaf3 = dag(Um_xmm) @ dag(Un_xmmmn) @ Um_xmmmn @ Un_xmn
            leaf4 = dag(Un_xmn) @ Um_xmn @ Un_xmnpm @ dag(Um)
            Q = leaf1 + leaf2 + leaf3 + leaf4
            F[(mu, nu)] = from_grid((Q - dag(Q)) / 8.0, dims)
    return F


def clover_term(U: np.ndarray, dims, csw: float) -> np.ndarray:
    """c_sw (i/4) sum_{mu,nu} sigma_{mu nu} (x) F_{mu nu} as (V, 12, 12).

    The ordered sum over mu != nu equals twice the sum over mu < nu, because
    sigma and F are both antisymmetric in (mu, nu).
    """
    F = field_strength(U, dims)
    V = volume(dims)
    C = np.zeros((V, 4, 3, 4, 3), dtype=np.complex128)
    for (mu, nu), Fmn in F.items():
        C += np.einsum("st,vab->vsatb", sigma_munu(mu, nu), Fmn)
    return (csw * 0.5j * C).reshape(V, 12, 12)


def hop_term(U: np.ndarray, psi: np.ndarray, dims, antiperiodic: bool = True,
             directions=None) -> np.ndarray:
    """sum over the chosen hops of (1 -+ gamma_mu) U psi(x +- mu), without -1/2.

    `directions` is a list of (mu, sign) pairs; default: all eight.
    """
    Lt = dims[3]
    Ug = to_grid(U, dims)
    n = psi.shape[-1]
    pg = to_grid(psi.reshape(-1, 4, 3, n), dims)
    out = np.zeros_like(pg)
    if directions is None:
        directions = [(mu, s) for mu in range(4) for s in (+1, -1)]
    for mu, sgn in directions:
        if sgn > 0:
            nb = shift(pg, mu, +1).copy()
            if mu == 3 and antiperiodic and Lt > 0:
                nb[Lt - 1] *= -1.0
            link = Ug[..., mu, :, :]
            t = np.einsum("...ab,...sbn->...san", link, nb)
            out += t - np.einsum("st,...tan->...san", GAMMA[mu], t)
        else:
            nb = shift(pg, mu, -1).copy()
            if mu == 3 and antiperiodic:
                nb[0] *= -1.0
            link = shift(Ug[..., mu, :, :], mu, -1)
            t = np.einsum("...ba,...sbn->...san", np.conj(link), nb)
            out += t + np.einsum("st,...tan->...san", GAMMA[mu], t)
    return from_grid(out, dims).reshape(psi.shape)


def apply_D(U: np.ndarray, clover: np.ndarray, psi: np.ndarray, dims,
            mass: float, antiperiodic: bool = True) -> np.ndarray:
    """D psi for psi of shape (V, 12, n); `clover` is clover_term(...)."""
    out = (4.0 + mass) * psi + np.einsum("vij,vjn->vin", clover, psi)
    out -= 0.5 * hop_term(U, psi, dims, antiperiodic)
    return out


def apply_D_sites(U: np.ndarray, psi: np.ndarray, dims, mass: float, csw: float,
                  sites, antiperiodic: bool = True) -> np.ndarray:
    """(D psi)(x) at the listed sites only, evaluated site by site.

    An independent, loop-based statement of the same operator for large
    lattices: neighbours by coordinate arithmetic, the clover from the four
    leaves at x.  Returns (len(sites), 12, n).
    """
    Lx, Ly, Lz, Lt = dims
    ext = (Lx, Ly, Lz, Lt)

    def idx(c):
        return c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3]))

    def step(c, mu, s):
        d = list(c)
        d[mu] = (d[mu] + s) % ext[mu]
        return d

    def link(c, mu):
        return U[idx(c), mu]

    n = psi.shape[-1]
    res = np.zeros((len(sites), 12, n), dtype=np.complex128)
    for k, site in enumerate(sites):
        site = int(site)
        c = [site % Lx, (site // Lx) % Ly, (site // (Lx * Ly)) % Lz, site // (Lx * Ly * Lz)]
        # clover term at this site
        C = np.zeros((4, 3, 4, 3), dtype=np.complex128)
        for mu in range(4):
            for nu in range(mu + 1, 4):
                xm = step(c, mu, -1)
                xn = step(c, nu, -1)
                xmn = step(xm, nu, -1)
                l1 = link(c, mu) @ link(step(c, mu, 1), nu) @ dag(link(step(c, nu, 1), mu)) @ dag(link(c, nu))
                l2 = link(c, nu) @ dag(link(step(xm, nu, 1), mu)) @ dag(link(xm, nu)) @ link(xm, mu)
                l3 = dag(link(xm, mu)) @ dag(link(xmn, nu)) @ link(xmn, mu) @ link(xn, nu)
                l4 = dag(link(xn, nu)) @ link(xn, mu) @ link(step(xn, mu, 1), nu) @ dag(link(c, mu))
                Q = l1 + l2 + l3 + l4
                Fmn = (Q - dag(Q)) / 8.0
                C += np.einsum("st,ab->satb", sigma_munu(mu, nu), Fmn)
        C = (csw * 0.5j * C).reshape(12, 12)
        out = (4.0 + mass) * psi[site] + C @ psi[site]
        hop = np.zeros((4, 3, n), dtype=np.complex128)
        for mu in range(4):
            cf = step(c, mu, 1)
            sf = -1.0 if (mu == 3 and antiperiodic and c[3] == Lt - 1) else 1.0
            t = sf * np.einsum("ab,sbn->san", link(c, mu), psi[idx(cf)].reshape(4, 3, n))
            hop += t - np.einsum("st,tan->san", GAMMA[mu], t)
            cb = step(c, mu, -1)
            sb = -1.0 if (mu == 3 and antiperiodic and c[3] == 0) else 1.0
            t = sb * np.einsum("ab,sbn->san", dag(link(cb, mu)), psi[idx(cb)].reshape(4, 3, n))
            hop += t + np.einsum("st,tan->san", GAMMA[mu], t)
        res[k] = out - 0.5 * hop.reshape(12, n)
    return res


def dense_D(U: np.ndarray, clover: np.ndarray, dims, mass: float,
            antiperiodic: bool = True) -> np.ndarray:
    """The full (12V x 12V) matrix of D, column by column (small lattices)."""
    V = volume(dims)
    N = 12 * V
    E = np.eye(N, dtype=np.complex128).reshape(V, 12, N)
    return apply_D(U, clover, E, dims, mass, antiperiodic).reshape(N, N)


def gamma5_field(psi: np.ndarray) -> np.ndarray:
    """gamma_5 acting on the spin index of a (V, 12, n) field."""
    V, _, n = psi.shape
    return np.einsum("st,vtan->vsan", GAMMA5, psi.reshape(V, 4, 3, n)).reshape(psi.shape)
