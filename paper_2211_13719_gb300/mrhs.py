"""Thin ctypes binding of the C ABI in include/mrhs.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments and raise on a non-OK status.  All computation
runs in the CUDA library ``_build/libmrhs.so``; if that library is missing or
cannot load, importing this module raises: there is no fallback.

Device buffers are passed as integers (e.g. ``tensor.data_ptr()``), streams as
``torch.cuda.Stream.cuda_stream`` integers or None for the default stream.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmrhs.so")

MRHS_OK = 0
MRHS_PENDING = 1
MRHS_ERR_INVALID = -1
MRHS_ERR_OOM = -2
MRHS_ERR_CUDA = -3
MRHS_ERR_NOT_CONVERGED = -4
MRHS_ERR_TIMEOUT = -5
MRHS_ERR_BUSY = -6
MRHS_ERR_NOT_FOUND = -7

MRHS_FP32 = 0
MRHS_FP64 = 1
MRHS_BF16 = 2
MRHS_FP16 = 3
MRHS_DF64 = 4  # float-float fine operator: FP32 input, FP64 output

MAX_LEVELS = 3

_STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "INVALID", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED",
                 -5: "TIMEOUT", -6: "BUSY", -7: "NOT_FOUND"}


class MrhsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mrhs status {_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class MgParams(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int),
        ("block", (C.c_int * 4) * (MAX_LEVELS - 1)),
        ("n_vec", C.c_int * (MAX_LEVELS - 1)),
        ("setup_sweeps", C.c_int),
        ("setup_m", C.c_int),
        ("smooth_m", C.c_int),
        ("coarse_m", C.c_int),
        ("coarse_cycles", C.c_int),
        ("inter_m", C.c_int),
        ("inner_m", C.c_int),
        ("inner_max_iters", C.c_int),
        ("inner_tol", C.c_double),
        ("outer_m", C.c_int),
        ("max_outer_iters", C.c_int),
        ("coarse_precision", C.c_int),
        ("max_rhs", C.c_int),
        ("use_graph", C.c_int),
        ("outer_op_precision", C.c_int),
        ("smoother_evenodd", C.c_int),
        ("seed", C.c_uint64),
        ("init_vecs", C.c_void_p * (MAX_LEVELS - 1)),
        ("smoother_sap", C.c_int),
        ("sap_block", C.c_int * 4),
        ("sap_cycles", C.c_int),
        ("sap_mr", C.c_int),
        ("coarse_smoother_evenodd", C.c_int),
        ("coarse_solver", C.c_int),
        ("coarse_recycle", C.c_int),
        ("coarse_fused", C.c_int),
        ("galerkin_tc", C.c_int),
    ]


class SolveStats(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int),
        ("inner_iters", C.c_int),
        ("vcycles", C.c_int),
        ("seconds", C.c_double),
        ("t_fine", C.c_double),
        ("t_restrict", C.c_double),
        ("t_prolong", C.c_double),
        ("t_coarse", C.c_double),
        ("t_outer", C.c_double),
        ("max_rel_residual", C.c_double),
    ]


class ServerParams(C.Structure):
    _fields_ = [("max_queue", C.c_int), ("hbm_reserve_gb", C.c_double)]


class RequestStats(C.Structure):
    _fields_ = [
        ("state", C.c_int),
        ("latency_s", C.c_double),
        ("queue_s", C.c_double),
        ("outer_iters", C.c_int),
        ("max_rel_residual", C.c_double),
    ]


class ApplyItem(C.Structure):
    _fields_ = [
        ("lat", C.c_void_p),
        ("in_dev", C.c_void_p),
        ("out_dev", C.c_void_p),
        ("y_dev", C.c_void_p),
        ("nrhs", C.c_int),
    ]


class TuneEntry(C.Structure):
    _fields_ = [
        ("kernel", C.c_char * 32),
        ("dims", C.c_int * 4),
        ("nrhs", C.c_int),
        ("variant", C.c_int),
        ("nvariants", C.c_int),
        ("best_ms", C.c_float),
        ("default_ms", C.c_float),
    ]


_P = C.c_void_p
_I = C.c_int
_I64 = C.c_int64
_D = C.c_double

# name -> (restype, argtypes); restype None means a void function
PROTOTYPES = {
    "mrhs_last_error": (C.c_char_p, []),
    "mrhs_kernel_launch_count": (C.c_uint64, []),
    "mrhs_kernel_timer_start": (_I, [C.c_char_p]),
    "mrhs_apply_hop_eo": (_I, [_P, _I, _P, _P, _I, _P]),
    "mrhs_apply_schur": (_I, [_P, _P, _P, _I, _P]),
    "mrhs_sap_smooth": (_I, [_P, _P, _P, _I, C.POINTER(C.c_int), _I, _I, _P]),
    "mrhs_kernel_timer_stop": (_I, [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mrhs_create_lattice": (_I, [C.POINTER(C.c_int), _I, _I, C.POINTER(_P)]),
    "mrhs_destroy_lattice": (None, [_P]),
    "mrhs_load_gauge": (_I, [_P, _P]),
    "mrhs_build_clover": (_I, [_P, _D, _D]),
    "mrhs_get_clover": (_I, [_P, _P]),
    "mrhs_apply_D": (_I, [_P, _P, _P, _I, _I, _P]),
    "mrhs_residual_D": (_I, [_P, _P, _P, _P, _I, _I, _P]),
    "mrhs_apply_D_batch": (_I, [C.POINTER(ApplyItem), _I, _P]),
    "mrhs_blas_multi_dot": (_I, [_P, _I, _P, _I64, _I, _I, _P, _P]),
    "mrhs_blas_multi_dot_noalloc": (_I, [_P, _I, _P, _I64, _I, _I, _P, _P]),
    "mrhs_blas_norm2": (_I, [_P, _I64, _I, _I, _P, _P]),
    "mrhs_blas_lincomb": (_I, [_P, _P, _I, _P, _D, _I64, _I, _I, _P]),
    "mrhs_mg_default_params": (None, [C.POINTER(MgParams)]),
    "mrhs_setup_mg": (_I, [_P, C.POINTER(MgParams), C.POINTER(_P)]),
    "mrhs_destroy_mg": (None, [_P]),
    "mrhs_mg_level_info": (_I, [_P, _I, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mrhs_mg_get_prolongator": (_I, [_P, _I, _P]),
    "mrhs_mg_get_coarse_links": (_I, [_P, _I, _P]),
    "mrhs_restrict": (_I, [_P, _I, _P, _P, _I, _P]),
    "mrhs_prolong": (_I, [_P, _I, _P, _P, _I, _P]),
    "mrhs_coarse_apply": (_I, [_P, _I, _P, _P, _I, _I, _P]),
    "mrhs_vcycle": (_I, [_P, _P, _P, _I, _P]),
    "mrhs_coarse_apply_schur": (_I, [_P, _I, _P, _P, _I, _P]),
    "mrhs_coarsest_solve": (_I, [_P, _P, _P, _I, _P]),
    "mrhs_coarsest_reset": (_I, [_P]),
    "mrhs_coarsest_fused_info": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mrhs_mg_setup_times": (_I, [_P, _I, C.POINTER(C.c_double)]),
    "mrhs_debug_expire_waits": (_I, [_I]),
    "mrhs_debug_expire_ring_waits": (_I, [_I]),
    "mrhs_solve": (_I, [_P, _P, _P, _I, _D, _P, C.POINTER(SolveStats), _P]),
    "mrhs_server_create": (_I, [C.POINTER(ServerParams), C.POINTER(_P)]),
    "mrhs_server_add_config": (_I, [_P, _P, _I, C.POINTER(C.c_int)]),
    "mrhs_submit": (_I, [_P, _I, _P, _P, _I, _D, C.POINTER(C.c_uint64)]),
    "mrhs_poll": (_I, [_P, C.c_uint64, C.POINTER(RequestStats)]),
    "mrhs_server_drain": (_I, [_P]),
    "mrhs_server_set_reserve": (_I, [_P, _D]),
    "mrhs_server_memory_waits": (_I, [_P, C.POINTER(C.c_uint64)]),
    "mrhs_server_destroy": (None, [_P]),
    "mrhs_tune_set_enabled": (None, [_I]),
    "mrhs_tune_clear": (None, []),
    "mrhs_tune_count": (_I, []),
    "mrhs_tune_get": (_I, [_I, C.POINTER(TuneEntry)]),
    "mrhs_tune_save": (_I, [C.c_char_p]),
    "mrhs_tune_load": (_I, [C.c_char_p]),
}

_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2211_13719_gb300.build)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, ok=(MRHS_OK,)):
    if status not in ok:
        raise MrhsError(status, lib().mrhs_last_error().decode())
    return status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def mrhs_kernel_launch_count() -> int:
    return int(lib().mrhs_kernel_launch_count())


def mrhs_kernel_timer_start(kernel_name: str):
    _check(lib().mrhs_kernel_timer_start(kernel_name.encode()))


def mrhs_kernel_timer_stop():
    """(summed event milliseconds, timed launches, graph-captured launches)"""
    ms, timed, captured = C.c_double(), C.c_int64(), C.c_int64()
    _check(lib().mrhs_kernel_timer_stop(C.byref(ms), C.byref(timed), C.byref(captured)))
    return ms.value, timed.value, captured.value


# ------------------------------------------------------------------ lattice
def mrhs_create_lattice(dims, t_boundary=-1, device=0):
    d = (C.c_int * 4)(*[int(v) for v in dims])
    h = _P()
    _check(lib().mrhs_create_lattice(d, int(t_boundary), int(device), C.byref(h)))
    return h.value


def mrhs_destroy_lattice(lat):
    lib().mrhs_destroy_lattice(lat)


def mrhs_load_gauge(lat, U_host):
    _check(lib().mrhs_load_gauge(lat, _ptr(U_host)))


def mrhs_build_clover(lat, mass, csw):
    _check(lib().mrhs_build_clover(lat, float(mass), float(csw)))


def mrhs_get_clover(lat, out_host):
    _check(lib().mrhs_get_clover(lat, _ptr(out_host)))


def mrhs_apply_hop_eo(lat, out_parity, in_dev, out_dev, nrhs, stream=None):
    _check(lib().mrhs_apply_hop_eo(lat, int(out_parity), _ptr(in_dev), _ptr(out_dev), int(nrhs), _stream(stream)))


def mrhs_tune_set_enabled(enabled: bool):
    lib().mrhs_tune_set_enabled(1 if enabled else 0)


def mrhs_tune_clear():
    lib().mrhs_tune_clear()


def mrhs_tune_entries():
    """The autotuner's cached choices as dicts (kernel, dims, nrhs, variant, nvariants, best_ms, default_ms)."""
    out = []
    for i in range(lib().mrhs_tune_count()):
        e = TuneEntry()
        _check(lib().mrhs_tune_get(i, C.byref(e)))
        out.append({"kernel": e.kernel.decode(), "dims": tuple(e.dims), "nrhs": e.nrhs, "variant": e.variant,
                    "nvariants": e.nvariants, "best_ms": e.best_ms, "default_ms": e.default_ms})
    return out


def mrhs_tune_save(path: str):
    _check(lib().mrhs_tune_save(path.encode()))


def mrhs_tune_load(path: str):
    _check(lib().mrhs_tune_load(path.encode()))


def mrhs_apply_schur(lat, in_dev, out_dev, nrhs, stream=None):
    _check(lib().mrhs_apply_schur(lat, _ptr(in_dev), _ptr(out_dev), int(nrhs), _stream(stream)))


def mrhs_sap_smooth(lat, v_dev, z_dev, nrhs, block, cycles, mr_steps, stream=None):
    b = (C.c_int * 4)(*[int(x) for x in block])
    _check(lib().mrhs_sap_smooth(lat, _ptr(v_dev), _ptr(z_dev), int(nrhs), b, int(cycles), int(mr_steps),
                                 _stream(stream)))


def mrhs_apply_D(lat, in_dev, out_dev, nrhs, prec, stream=None):
    _check(lib().mrhs_apply_D(lat, _ptr(in_dev), _ptr(out_dev), int(nrhs), int(prec), _stream(stream)))


def mrhs_residual_D(lat, in_dev, y_dev, out_dev, nrhs, prec, stream=None):
    _check(lib().mrhs_residual_D(lat, _ptr(in_dev), _ptr(y_dev), _ptr(out_dev), int(nrhs), int(prec),
                                 _stream(stream)))


def mrhs_apply_D_batch(items, stream=None):
    """items: list of (lat, in_dev, out_dev, y_dev or None, nrhs)."""
    arr = (ApplyItem * len(items))(*[ApplyItem(lat, _ptr(i), _ptr(o), _ptr(y), int(n)) for lat, i, o, y, n in items])
    _check(lib().mrhs_apply_D_batch(arr, len(items), _stream(stream)))


# --------------------------------------------------------------------- BLAS
def mrhs_blas_multi_dot(basis_dev, k, w_dev, rows, nrhs, prec, out_dev, stream=None):
    _check(lib().mrhs_blas_multi_dot(_ptr(basis_dev), int(k), _ptr(w_dev), int(rows), int(nrhs), int(prec),
                                     _ptr(out_dev), _stream(stream)))


def mrhs_blas_multi_dot_noalloc(basis_dev, k, w_dev, rows, nrhs, prec, out_dev, stream=None):
    _check(lib().mrhs_blas_multi_dot_noalloc(_ptr(basis_dev), int(k), _ptr(w_dev), int(rows), int(nrhs), int(prec),
                                             _ptr(out_dev), _stream(stream)))


def mrhs_blas_norm2(w_dev, rows, nrhs, prec, out_dev, stream=None):
    _check(lib().mrhs_blas_norm2(_ptr(w_dev), int(rows), int(nrhs), int(prec), _ptr(out_dev), _stream(stream)))


def mrhs_blas_lincomb(w_dev, basis_dev, k, coef_dev, alpha, rows, nrhs, prec, stream=None):
    _check(lib().mrhs_blas_lincomb(_ptr(w_dev), _ptr(basis_dev), int(k), _ptr(coef_dev), float(alpha), int(rows),
                                   int(nrhs), int(prec), _stream(stream)))


# ----------------------------------------------------------------------- MG
def mrhs_mg_default_params():
    p = MgParams()
    lib().mrhs_mg_default_params(C.byref(p))
    return p


def mrhs_setup_mg(lat, params: MgParams):
    h = _P()
    _check(lib().mrhs_setup_mg(lat, C.byref(params), C.byref(h)))
    return h.value


def mrhs_destroy_mg(mg):
    lib().mrhs_destroy_mg(mg)


def mrhs_mg_level_info(mg, level):
    d = (C.c_int * 4)()
    dof = C.c_int()
    _check(lib().mrhs_mg_level_info(mg, int(level), d, C.byref(dof)))
    return tuple(d), dof.value


def mrhs_mg_get_prolongator(mg, level, out_host):
    _check(lib().mrhs_mg_get_prolongator(mg, int(level), _ptr(out_host)))


def mrhs_mg_get_coarse_links(mg, level, out_host):
    _check(lib().mrhs_mg_get_coarse_links(mg, int(level), _ptr(out_host)))


def mrhs_restrict(mg, level, fine_dev, coarse_dev, nrhs, stream=None):
    _check(lib().mrhs_restrict(mg, int(level), _ptr(fine_dev), _ptr(coarse_dev), int(nrhs), _stream(stream)))


def mrhs_prolong(mg, level, coarse_dev, fine_dev, nrhs, stream=None):
    _check(lib().mrhs_prolong(mg, int(level), _ptr(coarse_dev), _ptr(fine_dev), int(nrhs), _stream(stream)))


def mrhs_coarse_apply(mg, level, in_dev, out_dev, nrhs, links_prec=MRHS_FP32, stream=None):
    _check(lib().mrhs_coarse_apply(mg, int(level), _ptr(in_dev), _ptr(out_dev), int(nrhs), int(links_prec),
                                   _stream(stream)))


def mrhs_coarse_apply_schur(mg, level, in_dev, out_dev, nrhs, stream=None):
    _check(lib().mrhs_coarse_apply_schur(mg, int(level), _ptr(in_dev), _ptr(out_dev), int(nrhs), _stream(stream)))


def mrhs_coarsest_solve(mg, b_dev, x_dev, nrhs, stream=None):
    _check(lib().mrhs_coarsest_solve(mg, _ptr(b_dev), _ptr(x_dev), int(nrhs), _stream(stream)))


def mrhs_mg_setup_times(mg, level):
    """setup milliseconds of transfer level -> level + 1: null vectors, orthonormalisation, Galerkin, 16-bit prep"""
    out = (C.c_double * 4)()
    _check(lib().mrhs_mg_setup_times(mg, int(level), out))
    return list(out)


def mrhs_coarsest_fused_info(mg):
    """(in use, resident CTAs, coarsest sites) of the persistent coarsest kernel"""
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(lib().mrhs_coarsest_fused_info(mg, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def mrhs_coarsest_reset(mg):
    _check(lib().mrhs_coarsest_reset(mg))


def mrhs_vcycle(mg, v_dev, z_dev, nrhs, stream=None):
    _check(lib().mrhs_vcycle(mg, _ptr(v_dev), _ptr(z_dev), int(nrhs), _stream(stream)))


def mrhs_debug_expire_waits(launches):
    _check(lib().mrhs_debug_expire_waits(int(launches)))


def mrhs_debug_expire_ring_waits(launches):
    _check(lib().mrhs_debug_expire_ring_waits(int(launches)))


def mrhs_solve(mg, b_dev, x_dev, nrhs, tol, rel_res_host=None, stream=None, allow_not_converged=False):
    st = SolveStats()
    ok = (MRHS_OK, MRHS_ERR_NOT_CONVERGED) if allow_not_converged else (MRHS_OK,)
    status = _check(lib().mrhs_solve(mg, _ptr(b_dev), _ptr(x_dev), int(nrhs), float(tol), _ptr(rel_res_host),
                                     C.byref(st), _stream(stream)), ok)
    return status, st


# ------------------------------------------------------------------ serving
def mrhs_server_create(max_queue=4096, hbm_reserve_gb=4.0):
    p = ServerParams(int(max_queue), float(hbm_reserve_gb))
    h = _P()
    _check(lib().mrhs_server_create(C.byref(p), C.byref(h)))
    return h.value


def mrhs_server_add_config(srv, mg, slots):
    cid = C.c_int()
    _check(lib().mrhs_server_add_config(srv, mg, int(slots), C.byref(cid)))
    return cid.value


def mrhs_submit(srv, config_id, b_host, x_host, nrhs, tol):
    rid = C.c_uint64()
    _check(lib().mrhs_submit(srv, int(config_id), _ptr(b_host), _ptr(x_host), int(nrhs), float(tol), C.byref(rid)))
    return rid.value


def mrhs_poll(srv, req_id):
    st = RequestStats()
    status = lib().mrhs_poll(srv, C.c_uint64(req_id), C.byref(st))
    return status, st


def mrhs_server_drain(srv):
    _check(lib().mrhs_server_drain(srv))


def mrhs_server_set_reserve(srv, hbm_reserve_gb):
    _check(lib().mrhs_server_set_reserve(srv, float(hbm_reserve_gb)))


def mrhs_server_memory_waits(srv):
    c = C.c_uint64()
    _check(lib().mrhs_server_memory_waits(srv, C.byref(c)))
    return c.value


def mrhs_server_destroy(srv):
    lib().mrhs_server_destroy(srv)
