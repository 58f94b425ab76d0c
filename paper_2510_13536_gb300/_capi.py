"""ctypes declarations of ``libmwcg.so`` (the C ABI of include/mwcg.h).

There is no fallback: if the library is missing or fails to load, importing
the solver raises, so nothing can silently run elsewhere than the CUDA
kernels.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmwcg.so")

ARITH = {"fp64": 0, "dw": 1, "qdw": 2, "tw": 3, "qtw": 4, "qdw_nn": 5, "qtw_nn": 6, "qw": 7, "qqw": 8, "qqw_nn": 9,
         "qqf": 10, "qf": 11}
WORDS = {0: 1, 1: 2, 2: 2, 3: 3, 4: 3, 5: 2, 6: 3, 7: 4, 8: 4, 9: 4, 10: 4, 11: 4}
# 8-byte slots per element in the C ABI's vectors (mwcg_words): the four FP32
# words of QQF and QF are packed two to a slot; every other arithmetic has one
# FP64 word per slot.
SLOTS = {**WORDS, 10: 2, 11: 2}
FP32_WORDS = {10, 11}
STATUS = {0: "converged", 1: "not_converged", 2: "breakdown", 3: "bad_preconditioner", 4: "out_of_range"}
PRECOND = {"none": 0, "jacobi": 1}
ERRORS = {-1: "MWCG_ERR_ARG", -2: "MWCG_ERR_CUDA", -3: "MWCG_ERR_GUARD", -4: "MWCG_ERR_NOMEM"}

# Every symbol declared in include/mwcg.h.
EXPORTS = [
    "mwcg_words", "mwcg_last_error", "mwcg_create_csr", "mwcg_destroy_csr", "mwcg_update_values",
    "mwcg_n", "mwcg_nnz", "mwcg_get_plan", "mwcg_set_plan", "mwcg_get_plan_for", "mwcg_solve", "mwcg_solve_host",
    "mwcg_solve_history", "mwcg_solve_batched", "mwcg_adjoint", "mwcg_spmv", "mwcg_dot",
    "mwcg_word_op", "mwcg_collapse", "mwcg_profile_kernels", "mwcg_batched_cluster_size",
    "mwcg_dot_noalloc", "mwcg_probe_peak", "mwcg_set_normalization", "mwcg_get_normalization",
    "mwcg_set_preconditioner", "mwcg_get_preconditioner", "mwcg_solve_bicgstab",
]

# Normalisation places of the quasi arithmetics' policy (MWCG_NORM_* in mwcg.h).
NORM = {"r": 1, "x": 2, "p": 4, "q": 8, "sum": 16}


class Plan(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int32), ("T", ctypes.c_int32), ("G", ctypes.c_int32)]


class MWCGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libmwcg.so (built by ``paper_2510_13536_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2510_13536_gb300.build.build() "
                           "(the solver has no CPU fallback)")
    L = ctypes.CDLL(path)
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pi32, pd = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
    sig = {
        "mwcg_words": (ctypes.c_int, [ctypes.c_int]),
        "mwcg_last_error": (ctypes.c_char_p, []),
        "mwcg_create_csr": (ctypes.c_int, [i64, P, P, P, ctypes.c_int, P, ctypes.POINTER(P)]),
        "mwcg_destroy_csr": (None, [P]),
        "mwcg_update_values": (ctypes.c_int, [P, P, ctypes.c_int, P]),
        "mwcg_n": (i64, [P]),
        "mwcg_nnz": (i64, [P]),
        "mwcg_get_plan": (ctypes.c_int, [P, ctypes.POINTER(Plan)]),
        "mwcg_set_plan": (ctypes.c_int, [P, ctypes.POINTER(Plan)]),
        "mwcg_get_plan_for": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.POINTER(Plan), P]),
        "mwcg_set_normalization": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_uint32]),
        "mwcg_set_preconditioner": (ctypes.c_int, [P, ctypes.c_int]),
        "mwcg_get_preconditioner": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int)]),
        "mwcg_get_normalization": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_uint32)]),
        "mwcg_solve": (ctypes.c_int, [P, P, P, ctypes.c_int, d, i32, P, pi32, pd]),
        "mwcg_solve_host": (ctypes.c_int, [P, P, P, ctypes.c_int, d, i32, P, pi32, pd]),
        "mwcg_solve_history": (ctypes.c_int, [P, P, P, ctypes.c_int, d, i32, P, P, pi32, pd]),
        "mwcg_solve_bicgstab": (ctypes.c_int, [P, P, P, ctypes.c_int, d, i32, P, P, pi32, pd]),
        "mwcg_solve_batched": (ctypes.c_int, [i32, P, P, P, P, P, P, P, P, P, P]),
        "mwcg_adjoint": (ctypes.c_int, [P, P, P, ctypes.c_int, d, i32, P, P, P, pi32, pd]),
        "mwcg_spmv": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
        "mwcg_dot": (ctypes.c_int, [ctypes.c_int, i64, P, P, i32, P, P]),
        "mwcg_word_op": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, i64, P, P, P, P]),
        "mwcg_collapse": (ctypes.c_int, [P, i32, i64, P, P]),
        "mwcg_profile_kernels": (ctypes.c_int, [P, P, P, ctypes.c_int, i32, P, P]),
        "mwcg_batched_cluster_size": (ctypes.c_int, []),
        "mwcg_dot_noalloc": (ctypes.c_int, [ctypes.c_int, i64, P, P, i32, P, P]),
        "mwcg_probe_peak": (ctypes.c_int, [ctypes.c_int, P, i64, P, ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(rc: int) -> int:
    """Raise MWCGError for negative return codes; pass statuses through."""
    if rc < 0:
        raise MWCGError(rc, load().mwcg_last_error().decode(errors="replace"))
    return rc
