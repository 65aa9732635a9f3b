"""The C ABI without a GPU: libabm.so builds (nvcc cross-compiles for
sm_103a), loads, and exports every function include/abm.h declares; the
ctypes binding names exactly those functions; the host-only calls work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abm.h")


def declared() -> set:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)  # comments
    names = re.findall(r"\b(abm_[a-z0-9_]+)\s*\(", text)
    # declarations only: a name followed by "(" that is preceded by a return type
    decl = set(re.findall(r"(?:abm_status|const char\s*\*|int32_t|void)\s+(abm_[a-z0-9_]+)\s*\(", text))
    assert decl, "no declarations found"
    assert decl <= set(names)
    return decl


@pytest.fixture(scope="module")
def lib_path():
    from paper_2508_16508_gb300 import build
    return build.build()


def test_every_declared_function_is_exported(lib_path):
    L = C.CDLL(lib_path)
    missing = sorted(n for n in declared() if not hasattr(L, n))
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_2508_16508_gb300 import abm
    abm.lib()
    assert set(abm.EXPORTED) == declared()


def test_host_only_calls(lib_path):
    from paper_2508_16508_gb300 import abm
    L = abm.lib()
    assert L.abm_version() >= 100
    assert L.abm_strerror(abm.OK) == b"ok"
    assert b"argument" in L.abm_strerror(abm.ERR_ARG)
    assert L.abm_strerror(12345) == b"unknown status"
    # argument checks happen before any CUDA call
    assert L.abm_select(None, None, None, None, None) == abm.ERR_ARG
    assert L.abm_step(None, 1, None, 0, None) == abm.ERR_ARG
    assert L.abm_resolve_static(None, None, -1, 1, None, None, None) == abm.ERR_ARG
    assert L.abm_resolve_static(None, None, 0, (1 << 18) + 1, C.c_void_p(16), None, None) == abm.ERR_TOO_LARGE
    assert L.abm_lob_match(-1, 8, None, None, None, None, None, None, None, None) == abm.ERR_ARG
    assert L.abm_lob_match(1, 0, None, None, None, None, None, None, None, None) == abm.ERR_ARG
    assert L.abm_lob_match(1, abm.LOB_MAX_CAP + 1, None, None, None, None, None, None, None, None) == abm.ERR_ARG
    assert L.abm_lob_match(0, 8, None, None, None, None, None, None, None, None) == abm.OK
    assert L.abm_lob_add(1, 8, None, None, None, None, None, None, None, -1, None, None) == abm.ERR_ARG
    assert L.abm_lob_add(1, 8, None, None, None, None, None, None, None, 0, None, None) == abm.ERR_ARG
    assert L.abm_lob_tune(3) == abm.ERR_ARG and L.abm_lob_tune(0) == abm.OK


def test_check_build_exports_the_same_functions():
    """The check build (-DABM_CHECK: index tests and canaries) compiles from the
    same sources and exports the same entry points; its version is negative."""
    from paper_2508_16508_gb300 import build
    path = build.build(check=True)
    assert path.endswith("libabm_check.so")
    L = C.CDLL(path)
    missing = sorted(n for n in declared() if not hasattr(L, n))
    assert not missing, missing
    L.abm_version.restype = C.c_int32
    assert L.abm_version() < 0
    L.abm_strerror.restype = C.c_char_p
    L.abm_strerror.argtypes = [C.c_int32]
    assert b"check build" in L.abm_strerror(8)
