"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads
without a GPU, and exports every function that include/spfc.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spfc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_15133_gb300 import build
    path = build.build()
    return path


def test_library_exports_every_declared_symbol(lib):
    declared = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            declared += _declared(h)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (spfc_\w+)", out))
    missing = [s for s in declared if s not in exported]
    assert declared and not missing, missing


def test_library_loads_without_gpu_and_binding_covers_header(lib):
    from paper_2012_15133_gb300 import spfc
    L = spfc.load_library()
    declared = _declared("spfc.h")
    for name in declared:
        assert hasattr(L, name)
    assert set(spfc.EXPORTED_SYMBOLS) >= set(declared)


def test_create_rejects_invalid_arguments_before_touching_the_gpu(lib):
    import ctypes as ct
    from paper_2012_15133_gb300 import spfc
    L = spfc.load_library()
    h = ct.c_void_p()
    n = (ct.c_int * 2)(64, 64)
    Ls = (ct.c_double * 2)(32.0, 32.0)
    assert L.spfc_create(4, n, Ls, 0.1, 1.0, 0.01, 0, None, ct.byref(h)) == 1
    assert L.spfc_create(2, n, Ls, 1.5, 1.0, 0.01, 0, None, ct.byref(h)) == 1   # a = 1 - eps <= 0
    assert L.spfc_create(2, n, Ls, 0.1, -1.0, 0.01, 0, None, ct.byref(h)) == 1
    assert L.spfc_create(2, n, Ls, 0.1, 1.0, 0.0, 0, None, ct.byref(h)) == 1
    assert L.spfc_create(2, (ct.c_int * 2)(64, 32), Ls, 0.1, 1.0, 0.01, 0, None, ct.byref(h)) == 1
    assert b"same N" in L.spfc_last_error(None)


def test_other_entry_points_refuse_bad_arguments_before_touching_the_gpu(lib):
    """NULL handles and out-of-range arguments come back as SPFC_EINVAL (1),
    with a message, before any device work."""
    import ctypes as ct
    from paper_2012_15133_gb300 import spfc
    L = spfc.load_library()
    assert L.spfc_set_gamma3(None, 1.0) == 1
    assert L.spfc_set_stabilization(None, 1.0) == 1
    assert L.spfc_batch_set_gamma3(None, 0, 1.0) == 1
    assert L.spfc_batch_set_state(None, 0, None, None, 1.0, 1.0) == 1
    assert L.spfc_surrogate_advance(None, None, None, 1, 20, 1, 0, 1e-3, None, None, None) == 1
    assert b"bad argument" in L.spfc_surrogate_last_error()
    assert L.spfc_fno_save(None, b"w.fno") == 1 and L.spfc_fno_load(None, b"w.fno") == 1
    f = ct.c_void_p()
    assert L.spfc_fno_create(48, 32, 16, 16, 4, 64, 16, None, ct.byref(f)) == 1   # n not a power of two
    assert L.spfc_fno_create(256, 32, 200, 16, 4, 64, 16, None, ct.byref(f)) == 1  # modes beyond n/2
    assert b"invalid network size" in L.spfc_fno_last_error(None)
    b = ct.c_void_p()
    n1, L1 = (ct.c_int * 1)(64), (ct.c_double * 1)(32.0)
    assert L.spfc_batch_create(0, n1, L1, (ct.c_double * 1)(0.1), (ct.c_double * 1)(1.0), 0.02, 1, None,
                               ct.byref(b)) == 1
    assert L.spfc_batch_create(1, n1, L1, (ct.c_double * 1)(1.2), (ct.c_double * 1)(1.0), 0.02, 1, None,
                               ct.byref(b)) == 1                                  # a = 1 - eps <= 0
    assert b"1 - eps" in L.spfc_batch_last_error(None)
    # the tensor-core GEMM self-test: sizes, split count and flags are checked first
    buf = (ct.c_float * 64)()
    assert L.spfc_gemm_selftest(0, 4, 4, 1, 1, 0, buf, buf, buf, None) == 1       # M = 0
    assert L.spfc_gemm_selftest(4, 4, 4, 1, 2000, 0, buf, buf, buf, None) == 1    # splits > 1024
    assert L.spfc_gemm_selftest(4, 4, 4, 1, 1, 16, buf, buf, buf, None) == 1      # unknown flag
    assert L.spfc_gemm_selftest(4, 4, 4, 1, 1, 0, None, buf, buf, None) == 1      # NULL operand
    assert L.spfc_gemm_selftest(1 << 14, 1 << 13, 1, 1, 1, 0, buf, buf, buf, None) == 1  # C beyond 2^26


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2012_15133_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
