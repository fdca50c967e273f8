"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/tg.h declares (no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_03070_gb300 import build, tg
    build.build()
    return tg.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tg_setup_operator", "tg_coarse_gmresdr", "tg_prolong", "tg_solve_proj",
                     "tg_adjoint_solve", "tg_destroy_op", "tg_destroy_defl", "tg_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2005_03070_gb300 import tg
    assert sorted(tg.EXPORTS) == _declared()


def test_status_strings(lib):
    assert lib.tg_status_string(0) == b"ok"
    assert lib.tg_status_string(4) == b"bad argument"
    assert lib.tg_status_string(99) == b"unknown status"


def test_bad_arguments_are_rejected_without_a_gpu(lib):
    import ctypes as C
    h = C.c_void_p()
    dims = (C.c_int64 * 1)(8)        # even N: rejected before any CUDA call
    beta = (C.c_double * 3)(1.0, 0.0, 0.0)
    st = lib.tg_setup_operator(C.byref(h), 0, dims, 1, beta, None, None, 2, None)
    assert st == 4 and not h.value
    assert b"odd" in lib.tg_last_error()
    st = lib.tg_setup_operator(C.byref(h), 7, dims, 1, beta, None, None, 2, None)
    assert st == 4
    st = lib.tg_setup_operator(C.byref(h), 0, dims, 1, beta, None, None, 3, None)
    assert st == 4
