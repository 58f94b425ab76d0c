"""ctypes binding of the CPU oracle (``mwcg_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``; the solver package never imports
it.  Multi-word arrays are numpy float64 of shape ``(w, n)`` (structure of
arrays, word 0 leading).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mwcg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

ARITHS = {"fp64": 0, "dw": 1, "qdw": 2, "tw": 3, "qtw": 4, "qdw_nn": 5, "qtw_nn": 6, "qw": 7, "qqw": 8, "qqw_nn": 9,
          "qqf": 10, "qf": 11}
# Words per element; QQF's and QF's four words are FP32 values, held here as float64.
WORDS = {0: 1, 1: 2, 2: 2, 3: 3, 4: 3, 5: 2, 6: 3, 7: 4, 8: 4, 9: 4, 10: 4, 11: 4}
STATUS = {0: "converged", 1: "maxit", 2: "breakdown", 3: "bad_preconditioner", 4: "out_of_range"}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ at -O3 (strict IEEE: no contraction, no
    fast-math, so the optimiser may not reassociate or fuse any operation and
    the results are those of the source's operation order).  No -march flag:
    the same source builds on x86-64 and aarch64 hosts."""
    flags = ["-std=c++17", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    stamp = _LIB + ".cmd"                 # the flags the library was built with
    try:
        same_flags = open(stamp).read() == " ".join(flags)
    except OSError:
        same_flags = False
    if force or not same_flags or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["g++", *flags, "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(" ".join(flags))
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        L.orc_ops_reset.restype = None
        L.orc_ops_get.restype = ctypes.c_uint64
        for nm in ("orc_two_sum", "orc_quick_two_sum", "orc_two_prod"):
            getattr(L, nm).argtypes = [i64, P, P, P, P]
            getattr(L, nm).restype = None
        L.orc_vecsum3.argtypes = [i64, P, P]
        L.orc_vecsum3.restype = None
        for nm in ("orc_add", "orc_mul", "orc_div", "orc_dxmul"):
            getattr(L, nm).argtypes = [i32, i64, P, P, P]
            getattr(L, nm).restype = i32
        for nm in ("orc_normalize", "orc_collapse"):
            getattr(L, nm).argtypes = [i32, i64, P, P]
            getattr(L, nm).restype = i32
        L.orc_spmv.argtypes = [i32, i64, P, P, P, P, P, i32]
        L.orc_spmv.restype = i32
        L.orc_dot.argtypes = [i32, i64, P, P, P, i64, i32]
        L.orc_dot.restype = i32
        L.orc_cg.argtypes = [i32, i64, P, P, P, P, P, d, i32, i32, i32, i32, P, P, P]
        L.orc_cg.restype = i32
        L.orc_cg_norm.argtypes = [i32, i64, P, P, P, P, P, d, i32, i32, i32, i32, i32, ctypes.c_uint32, P, P, P]
        L.orc_cg_norm.restype = i32
        L.orc_pcg_jacobi.argtypes = [i32, i64, P, P, P, P, P, d, i32, i32, i32, i32, i32, ctypes.c_uint32, P, P, P]
        L.orc_pcg_jacobi.restype = i32
        L.orc_bicgstab.argtypes = [i32, i64, P, P, P, P, P, d, i32, i32, i32, i32, P, P, P]
        L.orc_bicgstab.restype = i32
        L.orc_grad_values.argtypes = [i32, i64, P, P, P, P, P]
        L.orc_grad_values.restype = i32
        L.orc_words.argtypes = [i32]
        L.orc_words.restype = i32
        _lib = L
    return _lib


def _a(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(x):
    return x.ctypes.data_as(ctypes.c_void_p)


def arith_id(arith) -> int:
    return ARITHS[arith] if isinstance(arith, str) else int(arith)


def ops_reset():
    lib().orc_ops_reset()


def ops_get() -> int:
    return int(lib().orc_ops_get())


def two_sum(a, b):
    a, b = _a(a), _a(b)
    x, y = np.empty_like(a), np.empty_like(a)
    lib().orc_two_sum(a.size, _p(a), _p(b), _p(x), _p(y))
    return x, y


def quick_two_sum(a, b):
    a, b = _a(a), _a(b)
    x, y = np.empty_like(a), np.empty_like(a)
    lib().orc_quick_two_sum(a.size, _p(a), _p(b), _p(x), _p(y))
    return x, y


def two_prod(a, b):
    a, b = _a(a), _a(b)
    x, y = np.empty_like(a), np.empty_like(a)
    lib().orc_two_prod(a.size, _p(a), _p(b), _p(x), _p(y))
    return x, y


def vecsum3(a):
    a = _a(a)
    c = np.empty_like(a)
    lib().orc_vecsum3(a.shape[-1], _p(a), _p(c))
    return c


def _binop(fn, arith, a, b):
    k = arith_id(arith)
    a, b = _a(a), _a(b)
    n = a.shape[-1]
    c = np.empty((WORDS[k], n))
    if getattr(lib(), fn)(k, n, _p(a), _p(b), _p(c)) != 0:
        raise ValueError(arith)
    return c


def add(arith, a, b):
    return _binop("orc_add", arith, a, b)


def mul(arith, a, b):
    return _binop("orc_mul", arith, a, b)


def div(arith, a, b):
    return _binop("orc_div", arith, a, b)


def dxmul(arith, a, b):
    """FP64 a[n] times multi-word b[w, n]."""
    return _binop("orc_dxmul", arith, a, b)


def normalize(arith, a):
    k = arith_id(arith)
    a = _a(a)
    c = np.empty_like(a)
    lib().orc_normalize(k, a.shape[-1], _p(a), _p(c))
    return c


def collapse(arith, a):
    k = arith_id(arith)
    a = _a(a)
    c = np.empty(a.shape[-1])
    lib().orc_collapse(k, a.shape[-1], _p(a), _p(c))
    return c


def _csr(A):
    return (np.ascontiguousarray(A.row_ptr, dtype=np.int64), np.ascontiguousarray(A.col, dtype=np.int32),
            np.ascontiguousarray(A.val, dtype=np.float64))


def spmv(arith, A, p, V: int = 0):
    """q = A p in the arithmetic; V = 0 plain order, V > 0 the V-lane order."""
    k = arith_id(arith)
    rp, col, val = _csr(A)
    p = _a(p).reshape(WORDS[k], A.n)
    q = np.empty_like(p)
    lib().orc_spmv(k, A.n, _p(rp), _p(col), _p(val), _p(p), _p(q), V)
    return q


def dot(arith, u, v, R: int = 0, G: int = 1):
    """u^T v; R = 0 plain order, else tiles of R rows over G blocks."""
    k = arith_id(arith)
    w = WORDS[k]
    u, v = _a(u).reshape(w, -1), _a(v).reshape(w, -1)
    out = np.empty(w)
    lib().orc_dot(k, u.shape[1], _p(u), _p(v), _p(out), R, G)
    return out


# Normalisation places of the policy (see NormPolicy in mwcg_oracle.cpp).
NORM_R, NORM_X, NORM_P, NORM_Q, NORM_SUM = 1, 2, 4, 8, 16


def cg(arith, A, b, x0=None, tol=1e-12, maxit=1000, plan=None, history=False, norm=None, precond=None):
    """Algorithm 1 in the given arithmetic.

    ``plan`` = (V, T, G) mirrors the CUDA summation order; None is the plain
    order.  ``norm`` = (every, mask) is the normalisation policy of the quasi
    arithmetics (None: Sec. IV-D's r after its AXPY, every iteration).
    ``precond`` = "jacobi" runs Jacobi-preconditioned CG (status 3: a
    diagonal entry missing or not positive).
    Returns (x[w, n], iters, relres, status[, history]).
    """
    k = arith_id(arith)
    w = WORDS[k]
    rp, col, val = _csr(A)
    b = _a(b)
    x = np.zeros((w, A.n)) if x0 is None else _a(x0).reshape(w, A.n).copy()
    V, T, G = plan if plan is not None else (0, 0, 0)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.full(max(maxit, 1), np.nan) if history else None
    if precond not in (None, "none", "jacobi"):
        raise ValueError(precond)
    if precond == "jacobi":
        every, mask = norm if norm is not None else (1, NORM_R)
        st = lib().orc_pcg_jacobi(k, A.n, _p(rp), _p(col), _p(val), _p(b), _p(x), float(tol), int(maxit),
                                  int(V), int(T), int(G), int(every), int(mask), ctypes.byref(it),
                                  ctypes.byref(rr), _p(hist) if history else None)
    elif norm is None:
        st = lib().orc_cg(k, A.n, _p(rp), _p(col), _p(val), _p(b), _p(x), float(tol), int(maxit),
                          int(V), int(T), int(G), ctypes.byref(it), ctypes.byref(rr),
                          _p(hist) if history else None)
    else:
        every, mask = norm
        st = lib().orc_cg_norm(k, A.n, _p(rp), _p(col), _p(val), _p(b), _p(x), float(tol), int(maxit),
                               int(V), int(T), int(G), int(every), int(mask), ctypes.byref(it),
                               ctypes.byref(rr), _p(hist) if history else None)
    if st < 0:
        raise ValueError(arith)
    if history:
        return x, it.value, rr.value, st, hist[: it.value]
    return x, it.value, rr.value, st


def bicgstab(arith, A, b, x0=None, tol=1e-12, maxit=1000, plan=None, history=False):
    """BiCGStab in the given arithmetic (nonsymmetric A); as cg()."""
    k = arith_id(arith)
    w = WORDS[k]
    rp, col, val = _csr(A)
    b = _a(b)
    x = np.zeros((w, A.n)) if x0 is None else _a(x0).reshape(w, A.n).copy()
    V, T, G = plan if plan is not None else (0, 0, 0)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.full(max(maxit, 1), np.nan) if history else None
    st = lib().orc_bicgstab(k, A.n, _p(rp), _p(col), _p(val), _p(b), _p(x), float(tol), int(maxit),
                            int(V), int(T), int(G), ctypes.byref(it), ctypes.byref(rr),
                            _p(hist) if history else None)
    if st < 0:
        raise ValueError(arith)
    if history:
        return x, it.value, rr.value, st, hist[: it.value]
    return x, it.value, rr.value, st


def grad_values(arith, A, lam, x):
    """g_k = -collapse(lambda_row(k) * x_col(k)) for every stored entry k."""
    k = arith_id(arith)
    w = WORDS[k]
    rp, col, _ = _csr(A)
    lam, x = _a(lam).reshape(w, A.n), _a(x).reshape(w, A.n)
    g = np.empty(A.nnz)
    lib().orc_grad_values(k, A.n, _p(rp), _p(col), _p(lam), _p(x), _p(g))
    return g


def adjoint(arith, A, x, gx, tol, maxit, plan=None, norm=None, precond=None):
    """Gradients of L with dL/dx = gx: (g_b = lambda collapsed, g_val, lambda, iters, relres, status)."""
    k = arith_id(arith)
    lam, it, rr, st = cg(k, A, gx, None, tol, maxit, plan, norm=norm, precond=precond)
    g_b = collapse(k, lam) if WORDS[k] > 1 else lam[0].copy()
    g_val = grad_values(k, A, lam, x)
    return g_b, g_val, lam, it, rr, st
