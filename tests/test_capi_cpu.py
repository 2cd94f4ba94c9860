"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol include/mrhs.h declares, and validates arguments before touching a GPU.
No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2211_13719_gb300 import build, mrhs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mrhs.lib()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mrhs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in mrhs.PROTOTYPES, f"binding lacks {name}"


def test_argument_validation_without_gpu(lib):
    out = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 0, 4, 4)
    assert lib.mrhs_create_lattice(bad, -1, 0, ctypes.byref(out)) == mrhs.MRHS_ERR_INVALID
    assert b"extents" in lib.mrhs_last_error()
    good = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.mrhs_create_lattice(good, 3, 0, ctypes.byref(out)) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_load_gauge(None, None) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_apply_D(None, None, None, 1, 0, None) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_blas_norm2(None, 10, 1, 0, None, None) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_setup_mg(None, None, ctypes.byref(out)) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_debug_expire_waits(-1) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_debug_expire_waits(0) == mrhs.MRHS_OK


def test_default_params_are_sane(lib):
    p = mrhs.mrhs_mg_default_params()
    assert p.n_levels in (2, 3)
    assert p.n_vec[0] >= 1 and p.outer_m >= 1 and p.max_rhs >= 1
    assert p.coarse_precision in (mrhs.MRHS_FP32, mrhs.MRHS_FP16, mrhs.MRHS_BF16)
    assert p.outer_op_precision in (mrhs.MRHS_DF64, mrhs.MRHS_FP64)
    assert p.smoother_evenodd in (0, 1)


def test_kernel_timer_state_without_gpu(lib):
    # start / stop with nothing launched needs no GPU; a second start is refused
    assert lib.mrhs_kernel_timer_stop(None, None, None) == mrhs.MRHS_ERR_INVALID
    assert lib.mrhs_kernel_timer_start(None) == mrhs.MRHS_ERR_INVALID
    mrhs.mrhs_kernel_timer_start("k_dslash_x2")
    assert lib.mrhs_kernel_timer_start(b"k_dots_norm") == mrhs.MRHS_ERR_INVALID
    assert mrhs.mrhs_kernel_timer_stop() == (0.0, 0, 0)


def test_tune_cache_file_roundtrip_without_gpu(lib, tmp_path):
    """The autotuner's cache file: load, list, save and reload (no kernel runs)."""
    mrhs.mrhs_tune_clear()
    assert mrhs.mrhs_tune_entries() == []
    src = tmp_path / "tune.txt"
    src.write_text("# kernel Lx Ly Lz Lt nrhs variant nvariants best_ms default_ms\n"
                   "k_dslash_x2 24 24 24 64 48 2 5 2.900000 3.000000\n"
                   "k_eo_x2_schur 24 24 24 64 48 0 5 1.600000 1.600000\n")
    mrhs.mrhs_tune_load(str(src))
    ents = mrhs.mrhs_tune_entries()
    assert [(e["kernel"], e["dims"], e["nrhs"], e["variant"], e["nvariants"]) for e in ents] == [
        ("k_dslash_x2", (24, 24, 24, 64), 48, 2, 5), ("k_eo_x2_schur", (24, 24, 24, 64), 48, 0, 5)]
    dst = tmp_path / "tune2.txt"
    mrhs.mrhs_tune_save(str(dst))
    mrhs.mrhs_tune_clear()
    mrhs.mrhs_tune_load(str(dst))
    assert [(e["kernel"], e["variant"], round(e["best_ms"], 3)) for e in mrhs.mrhs_tune_entries()] == [
        ("k_dslash_x2", 2, 2.9), ("k_eo_x2_schur", 0, 1.6)]
    bad = tmp_path / "bad.txt"
    bad.write_text("k_dslash_x2 24 24 24 64 48 7 5 1.0 1.0\n")   # variant beyond nvariants
    with pytest.raises(mrhs.MrhsError) as e:
        mrhs.mrhs_tune_load(str(bad))
    assert e.value.status == mrhs.MRHS_ERR_INVALID
    with pytest.raises(mrhs.MrhsError) as e:
        mrhs.mrhs_tune_load(str(tmp_path / "missing.txt"))
    assert e.value.status == mrhs.MRHS_ERR_NOT_FOUND
    mrhs.mrhs_tune_clear()
