"""C ABI checks that need no GPU: the library builds, loads, exports every
symbol include/mwcg.h declares, and rejects malformed input on the host."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_13536_gb300 import _capi, build
    build.build()
    return _capi.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mwcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mwcg_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2510_13536_gb300 import _capi
    syms = declared_symbols()
    assert len(syms) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", _capi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mwcg_\w+)", out))
    assert set(syms) <= exported, set(syms) - exported
    assert set(syms) == set(_capi.EXPORTS)
    for s in syms:
        getattr(lib, s)


def test_words_and_error_string(lib):
    # 8-byte slots per element: the FP64 words; QQF and QF pack four FP32 words in 2.
    assert [lib.mwcg_words(a) for a in range(12)] == [1, 2, 2, 3, 3, 2, 3, 4, 4, 4, 2, 2]
    assert lib.mwcg_words(12) == -1 and lib.mwcg_words(-1) == -1
    assert isinstance(lib.mwcg_last_error(), bytes)


def _create(lib, n, rp, col, val):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    rc = lib.mwcg_create_csr(n, rp.ctypes.data_as(ctypes.c_void_p), col.ctypes.data_as(ctypes.c_void_p),
                             val.ctypes.data_as(ctypes.c_void_p), 0, None, ctypes.byref(h))
    return rc, lib.mwcg_last_error().decode()


def test_malformed_csr_rejected_on_host(lib):
    ok_rp, ok_col, ok_val = [0, 2, 3], [0, 1, 1], [2.0, -1.0, 2.0]
    cases = [
        ([1, 2, 3], ok_col, ok_val, "row_ptr[0]"),
        ([0, 3, 2], ok_col, ok_val, "decreases"),
        (ok_rp, [0, 2, 1], ok_val, "out of range"),
        (ok_rp, [0, -1, 1], ok_val, "out of range"),
        (ok_rp, ok_col, [2.0, np.nan, 2.0], "not finite"),
        (ok_rp, ok_col, [2.0, np.inf, 2.0], "not finite"),
    ]
    for rp, col, val, msg in cases:
        rc, err = _create(lib, 2, rp, col, val)
        assert rc == -1 and msg in err, (rp, col, val, rc, err)
    rc, err = _create(lib, -1, ok_rp, ok_col, ok_val)
    assert rc == -1


def test_null_arguments_rejected(lib):
    it, rr = ctypes.c_int32(), ctypes.c_double()
    assert lib.mwcg_solve(None, None, None, 4, 1e-10, 10, None, ctypes.byref(it), ctypes.byref(rr)) == -1
    assert lib.mwcg_create_csr(3, None, None, None, 0, None, None) == -1
    assert lib.mwcg_word_op(9, 4, 10, None, None, None, None) == -1
    assert lib.mwcg_dot(4, 10, None, None, 0, None, None) == -1
    assert lib.mwcg_collapse(None, 4, 10, None, None) == -1
    out = (ctypes.c_double * 4)()
    assert lib.mwcg_dot_noalloc(10, 10, None, None, 1, None, out) == -1      # QQF: null inputs
    assert b"null u or v" in lib.mwcg_last_error()
    assert lib.mwcg_dot_noalloc(12, 10, None, None, 1, None, out) == -1      # no arithmetic 12
    assert b"unknown arithmetic" in lib.mwcg_last_error()
