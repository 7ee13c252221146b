"""The C ABI library builds, loads and exports every symbol declared in include/spm.h (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "spm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libspm():
    from paper_2605_09755_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["spm_sketch_create", "spm_sketch_destroy", "spm_sketch_apply", "spm_sketch_apply_t",
                 "spm_gaussian", "spm_range_finder", "spm_rsvd", "spm_lowrank", "spm_nystrom",
                 "spm_gemm_bf16"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libspm):
    missing = [s for s in declared_symbols() if not hasattr(libspm, s)]
    assert not missing, missing


def test_host_only_calls(libspm):
    libspm.spm_version.restype = ctypes.c_int
    assert libspm.spm_version() >= 100
    libspm.spm_status_string.restype = ctypes.c_char_p
    assert libspm.spm_status_string(1) == b"invalid argument"
    # argument checking happens before any device work
    h = ctypes.c_void_p()
    f = libspm.spm_sketch_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p]
    assert f(ctypes.byref(h), 100, 10, 11, 1, 0, None) == 1      # s > r1
    assert f(ctypes.byref(h), 0, 10, 1, 1, 0, None) == 1         # n < 1
    assert f(ctypes.byref(h), 100, 50, 1, 1, 1, None) == 1       # identity needs r1 == n
    assert f(None, 100, 10, 1, 1, 0, None) == 1
    # the dense families (Lemma 3.2 items 1 and 3)
    assert f(ctypes.byref(h), 100, 101, 1, 1, 3, None) == 1     # SRHT needs r1 <= n
    assert f(ctypes.byref(h), 40000, 100, 1, 1, 3, None) == 7   # n' = 2^16 > 2^15: unsupported
    assert f(ctypes.byref(h), 1 << 30, 1 << 10, 1, 1, 2, None) == 7   # n x r1 dense signs > 2^36
    assert f(ctypes.byref(h), 100, 10, 1, 1, 4, None) == 1      # unknown kind
    assert f(ctypes.byref(h), 100, 10, 0, 1, 2, None) == 1      # s < 1


def test_host_only_argument_checks_of_the_newer_entries(libspm):
    """Host-buffer, sparse and pool entries reject bad arguments before any device work."""
    vp = ctypes.c_void_p
    i64, i32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    f = libspm.spm_rsvd_host
    f.argtypes = [vp, vp, i32, i64, i64, i64, i32, u64, i64, vp, vp, i64, vp, vp, i64, vp, vp]
    assert f(None, None, 0, 10, 10, 5, 1, 1, 5, None, None, 5, None, None, 10, None, None) == 1
    f = libspm.spm_rsvd_csr
    f.argtypes = [vp, vp, i32, i64, i32, u64, i64, vp, vp, i64, vp, vp, i64, vp, vp]
    assert f(None, None, 0, 5, 1, 1, 5, None, None, 5, None, None, 10, None, None) == 1
    f = libspm.spm_sketch_apply_csr
    f.argtypes = [vp, vp, i32, vp, i64, vp]
    assert f(None, None, 0, None, 10, None) == 1
    libspm.spm_trim_memory.restype = ctypes.c_int
    assert libspm.spm_trim_memory() in (0, 3)   # SPM_ECUDA where no device is usable


def test_binding_has_no_cpu_path():
    src = open(os.path.join(ROOT, "paper_2605_09755_gb300", "spm.py")).read()
    assert "oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_2605_09755_gb300")):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(ROOT, "paper_2605_09755_gb300", f)).read()
