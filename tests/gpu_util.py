"""Helpers shared by the GPU parity tests: upload / download through torch.

torch is used for device memory and streams only; every computation under
test runs in the CUDA library through its C ABI.
"""
import numpy as np

from paper_2211_13719_gb300 import mrhs


def torch_mod():
    import torch
    return torch


def to_dev(a: np.ndarray):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t) -> np.ndarray:
    torch = torch_mod()
    torch.cuda.synchronize()
    return t.cpu().numpy()


def empty_like_dev(shape, dtype):
    torch = torch_mod()
    tdt = {np.complex64: torch.complex64, np.complex128: torch.complex128,
           np.float64: torch.float64, np.float32: torch.float32}[dtype]
    return torch.empty(shape, dtype=tdt, device="cuda")


def make_lattice(U: np.ndarray, dims, mass, csw, t_boundary=-1):
    lat = mrhs.mrhs_create_lattice(dims, t_boundary, 0)
    mrhs.mrhs_load_gauge(lat, np.ascontiguousarray(U))
    mrhs.mrhs_build_clover(lat, mass, csw)
    return lat


def site_rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """max over sites and RHS of ||a - b|| / ||b|| (norm over the site's components)."""
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=1))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=1))
    return float(np.max(num / np.maximum(den, 1e-300)))


def make_mg(lat, params: dict, init_vecs=None):
    """mrhs_setup_mg with the defaults overridden by `params` (a dict of MgParams fields).

    `init_vecs[l]` (optional) are host FP64 start vectors (V_l, dof_l, N_l); the
    arrays must stay alive during the call."""
    p = mrhs.mrhs_mg_default_params()
    for k, v in params.items():
        if k == "blocks":
            for l, b in enumerate(v):
                for mu in range(4):
                    p.block[l][mu] = int(b[mu])
        elif k == "nvec":
            for l, nv in enumerate(v):
                p.n_vec[l] = int(nv)
        else:
            setattr(p, k, v)
    keep = []
    if init_vecs is not None:
        for l, a in enumerate(init_vecs):
            a = np.ascontiguousarray(a, dtype=np.complex128)
            keep.append(a)
            p.init_vecs[l] = a.ctypes.data
    mg = mrhs.mrhs_setup_mg(lat, p)
    del keep
    return mg
