"""Python API over the C ABI: matrices, solves, adjoints, building blocks.

Argument marshalling only -- every arithmetic step runs in libmwcg.so.
Device arrays are torch CUDA tensors (float64, contiguous); multi-word
vectors have shape (w, n) with word 0 leading (the C ABI's structure of
arrays).  QQF vectors are float32 of shape (4, n) here; the C ABI packs their
words two to an 8-byte slot, and the binding converts between the layouts.
Work is issued on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _capi
from ._capi import ARITH, FP32_WORDS, SLOTS, WORDS, Plan, check

__all__ = ["CSRMatrix", "SolveResult", "solve", "solve_host", "solve_batched", "batched_cluster_size", "adjoint", "spmv", "dot",
           "word_op", "collapse", "words", "arith_id", "MWCGSolve", "solve_differentiable"]


def arith_id(arith) -> int:
    if isinstance(arith, str):
        return ARITH[arith.lower()]
    a = int(arith)
    if a not in WORDS:
        raise ValueError(f"unknown arithmetic {arith}")
    return a


def words(arith) -> int:
    return WORDS[arith_id(arith)]


def _pack(x: torch.Tensor, n: int) -> torch.Tensor:
    """(4, n) FP32 words -> the C ABI's (2, n) slots (words 2k, 2k+1 in slot k)."""
    if n == 0:
        return torch.empty((2, 0), dtype=torch.float64, device=x.device)
    f = x.to(torch.float32).reshape(2, 2, n).permute(0, 2, 1).reshape(2, 2 * n).contiguous()
    return f.view(torch.float64)             # (2, n); the flat last axis views at any n


def _unpack(x: torch.Tensor, n: int) -> torch.Tensor:
    """The C ABI's (2, n) slots -> (4, n) FP32 words."""
    if n == 0:
        return torch.empty((4, 0), dtype=torch.float32, device=x.device)
    return x.contiguous().view(torch.float32).reshape(2, n, 2).permute(0, 2, 1).reshape(4, n).contiguous()


def _pack_np(x: np.ndarray, n: int) -> np.ndarray:
    if n == 0:
        return np.empty((2, 0))
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(2, 2, n).transpose(0, 2, 1))
    return f.view(np.float64).reshape(2, n).copy()


def _unpack_np(x: np.ndarray, n: int) -> np.ndarray:
    if n == 0:
        return np.empty((4, 0), dtype=np.float32)
    return np.ascontiguousarray(x.view(np.float32).reshape(2, n, 2).transpose(0, 2, 1).reshape(4, n))


def _to_abi(a: int, x: torch.Tensor, n: int) -> torch.Tensor:
    if a in FP32_WORDS:
        return _pack(x, n)
    return x.to(torch.float64).reshape(WORDS[a], n).contiguous()


def _from_abi(a: int, x: torch.Tensor, n: int) -> torch.Tensor:
    return _unpack(x, n) if a in FP32_WORDS else x


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class CSRMatrix:
    """A CSR matrix copied to the device, with its solver workspace and plan."""

    def __init__(self, n: int, row_ptr, col, val):
        L = _capi.load()
        self._h = ctypes.c_void_p()
        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            rp = row_ptr.to(torch.int64).contiguous()
            cl = col.to(torch.int32).contiguous()
            vl = val.to(torch.float64).contiguous()
            self._keep = (rp, cl, vl)
            args = (ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(cl.data_ptr()), ctypes.c_void_p(vl.data_ptr()), 1)
        else:
            rp = np.ascontiguousarray(np.asarray(row_ptr), dtype=np.int64)
            cl = np.ascontiguousarray(np.asarray(col), dtype=np.int32)
            vl = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
            self._keep = (rp, cl, vl)
            args = (rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                    vl.ctypes.data_as(ctypes.c_void_p), 0)
        check(L.mwcg_create_csr(int(n), args[0], args[1], args[2], args[3], _stream(), ctypes.byref(self._h)))
        self._keep = None
        self.n = int(n)
        self.nnz = int(L.mwcg_nnz(self._h))

    @classmethod
    def from_csr(cls, A) -> "CSRMatrix":
        """From any object with n, row_ptr, col, val (e.g. problems.CSR)."""
        return cls(A.n, A.row_ptr, A.col, A.val)

    @property
    def handle(self):
        return self._h

    @property
    def plan(self) -> tuple[int, int, int]:
        p = Plan()
        check(_capi.load().mwcg_get_plan(self._h, ctypes.byref(p)))
        return (p.V, p.T, p.G)

    @plan.setter
    def plan(self, vtg):
        """Pin (V, T, G) for every arithmetic; None returns to the automatic plans."""
        if vtg is None:
            check(_capi.load().mwcg_set_plan(self._h, None))
            return
        p = Plan(*[int(v) for v in vtg])
        check(_capi.load().mwcg_set_plan(self._h, ctypes.byref(p)))

    def plan_for(self, arith) -> tuple[int, int, int]:
        """The plan a solve in `arith` uses (timed at the first call in it)."""
        return self.tuning(arith)[0]

    def tuning(self, arith):
        """(plan, {V: measured SpMV ms}) of an arithmetic's automatic plan."""
        p = Plan()
        ms = (ctypes.c_double * 6)()
        check(_capi.load().mwcg_get_plan_for(self._h, arith_id(arith), _stream(), ctypes.byref(p), ms))
        return (p.V, p.T, p.G), {1 << j: ms[j] for j in range(6) if ms[j] > 0}

    @property
    def normalization(self) -> tuple[int, int]:
        """(every, mask) of the quasi arithmetics' normalisation policy (mwcg.h)."""
        e, m = ctypes.c_int32(0), ctypes.c_uint32(0)
        check(_capi.load().mwcg_get_normalization(self._h, ctypes.byref(e), ctypes.byref(m)))
        return (e.value, m.value)

    @normalization.setter
    def normalization(self, policy):
        """policy = (every, mask), mask an int or an iterable of "r", "x", "p", "q", "sum"."""
        every, mask = policy
        if not isinstance(mask, int):
            mask = sum(_capi.NORM[k] for k in set(mask))
        check(_capi.load().mwcg_set_normalization(self._h, int(every), int(mask)))

    @property
    def preconditioner(self) -> str:
        """"none" (Algorithm 1) or "jacobi" (M^-1 = diag(fl(1/a_ii)), mwcg.h)."""
        k = ctypes.c_int(0)
        check(_capi.load().mwcg_get_preconditioner(self._h, ctypes.byref(k)))
        return {v: n for n, v in _capi.PRECOND.items()}[k.value]

    @preconditioner.setter
    def preconditioner(self, kind: str):
        if kind not in _capi.PRECOND:
            raise ValueError(f"unknown preconditioner {kind!r}")
        check(_capi.load().mwcg_set_preconditioner(self._h, _capi.PRECOND[kind]))

    def update_values(self, val) -> None:
        L = _capi.load()
        if isinstance(val, torch.Tensor) and val.is_cuda:
            v = val.to(torch.float64).contiguous()
            check(L.mwcg_update_values(self._h, ctypes.c_void_p(v.data_ptr()), 1, _stream()))
        else:
            v = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
            check(L.mwcg_update_values(self._h, v.ctypes.data_as(ctypes.c_void_p), 0, _stream()))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _capi.load().mwcg_destroy_csr(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class SolveResult:
    x: torch.Tensor          # (w, n) multi-word solution
    iters: int
    relres: float
    status: int              # 0 converged, 1 maxit, 2 breakdown, 3 bad preconditioner, 4 x out of range (QQF)
    history: torch.Tensor | None = None

    @property
    def converged(self) -> bool:
        return self.status == 0


def solve(A: CSRMatrix, b: torch.Tensor, arith="qtw", tol: float = 1e-14, maxit: int = 20000,
          x0: torch.Tensor | None = None, history: bool = False) -> SolveResult:
    """CG on A x = b in the given arithmetic (device tensors)."""
    a = arith_id(arith)
    x = torch.zeros((SLOTS[a], A.n), dtype=torch.float64, device=b.device) if x0 is None else \
        _to_abi(a, x0, A.n).clone()
    it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
    L = _capi.load()
    hist = None
    if history:
        hist = torch.full((max(int(maxit), 1),), float("nan"), dtype=torch.float64, device=b.device)
        st = check(L.mwcg_solve_history(A.handle, _ptr(b), _ptr(x), a, float(tol), int(maxit), _ptr(hist), _stream(),
                                        ctypes.byref(it), ctypes.byref(rr)))
        hist = hist[: it.value]
    else:
        st = check(L.mwcg_solve(A.handle, _ptr(b), _ptr(x), a, float(tol), int(maxit), _stream(),
                                ctypes.byref(it), ctypes.byref(rr)))
    return SolveResult(_from_abi(a, x, A.n), it.value, rr.value, st, hist)


def solve_bicgstab(A: CSRMatrix, b: torch.Tensor, arith="qtw", tol: float = 1e-14, maxit: int = 20000,
                   x0: torch.Tensor | None = None, history: bool = False) -> SolveResult:
    """BiCGStab on A x = b (A may be nonsymmetric) in the given arithmetic (device tensors)."""
    a = arith_id(arith)
    x = torch.zeros((SLOTS[a], A.n), dtype=torch.float64, device=b.device) if x0 is None else \
        _to_abi(a, x0, A.n).clone()
    it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
    hist = None
    if history:
        hist = torch.full((max(int(maxit), 1),), float("nan"), dtype=torch.float64, device=b.device)
    st = check(_capi.load().mwcg_solve_bicgstab(A.handle, _ptr(b), _ptr(x), a, float(tol), int(maxit),
                                                _ptr(hist) if history else None, _stream(), ctypes.byref(it),
                                                ctypes.byref(rr)))
    if history:
        hist = hist[: it.value]
    return SolveResult(_from_abi(a, x, A.n), it.value, rr.value, st, hist)


def solve_host(A: CSRMatrix, b: np.ndarray, arith="qtw", tol: float = 1e-14, maxit: int = 20000,
               x0: np.ndarray | None = None):
    """CG with host (numpy) buffers; the copies are part of the call.  Returns (x, iters, relres, status)."""
    a = arith_id(arith)
    w = WORDS[a]
    bb = np.ascontiguousarray(b, dtype=np.float64)
    if a in FP32_WORDS:
        x = np.zeros((SLOTS[a], A.n)) if x0 is None else _pack_np(x0, A.n)
    else:
        x = np.zeros((w, A.n)) if x0 is None else \
            np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(w, A.n)).copy()
    it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
    st = check(_capi.load().mwcg_solve_host(A.handle, bb.ctypes.data_as(ctypes.c_void_p),
                                            x.ctypes.data_as(ctypes.c_void_p), a, float(tol), int(maxit), _stream(),
                                            ctypes.byref(it), ctypes.byref(rr)))
    return (_unpack_np(x, A.n) if a in FP32_WORDS else x), it.value, rr.value, st


def solve_batched(As, bs, arith, tol, maxit, x0s=None):
    """Many independent systems in one persistent launch.  Returns a list of SolveResult."""
    ns = len(As)
    ar = [arith_id(a) for a in (arith if isinstance(arith, (list, tuple)) else [arith] * ns)]
    tl = list(tol) if isinstance(tol, (list, tuple)) else [float(tol)] * ns
    mi = list(maxit) if isinstance(maxit, (list, tuple)) else [int(maxit)] * ns
    xs = []
    for s in range(ns):
        n = As[s].n
        if x0s is None or x0s[s] is None:
            xs.append(torch.zeros((SLOTS[ar[s]], n), dtype=torch.float64, device=bs[s].device))
        else:                                   # the ABI layout (QQF / QF: packed FP32 words), a copy
            xs.append(_to_abi(ar[s], x0s[s], n).clone())
    P = ctypes.c_void_p
    hA = (P * ns)(*[A.handle.value for A in As])
    hb = (P * ns)(*[b.data_ptr() for b in bs])
    hx = (P * ns)(*[x.data_ptr() for x in xs])
    har = (ctypes.c_int32 * ns)(*ar)
    htl = (ctypes.c_double * ns)(*tl)
    hmi = (ctypes.c_int32 * ns)(*mi)
    it = (ctypes.c_int32 * ns)()
    rr = (ctypes.c_double * ns)()
    stt = (ctypes.c_int32 * ns)()
    for b in bs:
        _ptr(b)
    check(_capi.load().mwcg_solve_batched(ns, hA, hb, hx, har, htl, hmi, _stream(), it, rr, stt))
    return [SolveResult(_from_abi(ar[s], xs[s], As[s].n), it[s], rr[s], stt[s]) for s in range(ns)]


def batched_cluster_size() -> int:
    """CTAs per worker cluster of solve_batched (its systems use plan {V, 256, this})."""
    return int(_capi.load().mwcg_batched_cluster_size())


def adjoint(A: CSRMatrix, x: torch.Tensor, gx: torch.Tensor, arith="qtw", tol: float = 1e-20, maxit: int = 20000):
    """Gradients of L with dL/dx = gx: returns (g_b[n], g_val[nnz], iters, relres, status)."""
    a = arith_id(arith)
    g_b = torch.empty(A.n, dtype=torch.float64, device=gx.device)
    g_val = torch.empty(A.nnz, dtype=torch.float64, device=gx.device)
    it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
    xc, gc = _to_abi(a, x, A.n), gx.to(torch.float64).contiguous()   # held until the call returns
    st = check(_capi.load().mwcg_adjoint(A.handle, _ptr(xc), _ptr(gc), a, float(tol), int(maxit), _stream(),
                                         _ptr(g_b), _ptr(g_val), ctypes.byref(it), ctypes.byref(rr)))
    return g_b, g_val, it.value, rr.value, st


def spmv(A: CSRMatrix, arith, p: torch.Tensor) -> torch.Tensor:
    a = arith_id(arith)
    pp = _to_abi(a, p, A.n)
    q = torch.empty_like(pp)
    check(_capi.load().mwcg_spmv(A.handle, a, _ptr(pp), _ptr(q), _stream()))
    return _from_abi(a, q, A.n)


def dot(arith, u: torch.Tensor, v: torch.Tensor, G: int) -> np.ndarray:
    a = arith_id(arith)
    out = np.zeros(WORDS[a])
    n = u.shape[-1]
    uu, vv = _to_abi(a, u, n), _to_abi(a, v, n)      # held until the call returns
    check(_capi.load().mwcg_dot(a, n, _ptr(uu), _ptr(vv), int(G), _stream(), out.ctypes.data_as(ctypes.c_void_p)))
    return out


_OPS = {"add": 0, "mul": 1, "dxmul": 2, "div": 3, "normalize": 4, "collapse": 5}


def word_op(op: str, arith, a: torch.Tensor, b: torch.Tensor | None = None) -> torch.Tensor:
    """Element-wise word operation on the device (see mwcg_word_op)."""
    k = arith_id(arith)
    o = _OPS[op]
    n = a.shape[-1]
    if k in FP32_WORDS:                 # FP32 words: pack the multi-word operands
        a = a if o == 2 else _to_abi(k, a, n)
        b = None if b is None else _to_abi(k, b, n)
    c = torch.empty(n if o == 5 else (SLOTS[k], n), dtype=torch.float64, device=a.device)
    check(_capi.load().mwcg_word_op(o, k, n, _ptr(a), _ptr(b), _ptr(c), _stream()))
    return c if o == 5 else _from_abi(k, c, n)


def collapse(x: torch.Tensor) -> torch.Tensor:
    """FP64 value of a (w, n) multi-word vector, lowest word first (QQF: float32 (4, n))."""
    if x.dtype == torch.float32:
        return word_op("collapse", "qqf", x)
    w, n = (1, x.shape[0]) if x.dim() == 1 else x.shape
    y = torch.empty(n, dtype=torch.float64, device=x.device)
    xc = x.contiguous()                                 # held until the call returns
    check(_capi.load().mwcg_collapse(_ptr(xc), int(w), int(n), _ptr(y), _stream()))
    return y


class MWCGSolve(torch.autograd.Function):
    """x = A(values)^{-1} b with a hand-written backward (adjoint CG in the same
    arithmetic, then the sparsity-masked -lambda_i x_j gradient).  Only the
    multi-word solution x is saved for backward."""

    @staticmethod
    def forward(ctx, values, b, A: CSRMatrix, arith, tol, maxit, adj_tol=None):
        A.update_values(values.detach())
        res = solve(A, b.detach().contiguous(), arith, tol, maxit)
        if res.status != 0:
            raise RuntimeError(f"forward CG did not converge (status {res.status}, relres {res.relres:.3e})")
        ctx.A, ctx.arith, ctx.maxit = A, arith, maxit
        ctx.adj_tol = tol if adj_tol is None else adj_tol
        ctx.save_for_backward(res.x)
        return collapse(res.x)

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        g_b, g_val, it, rr, st = adjoint(ctx.A, x, gx.contiguous().to(torch.float64), ctx.arith, ctx.adj_tol,
                                         ctx.maxit)
        if st != 0:
            raise RuntimeError(f"adjoint CG did not converge (status {st}, relres {rr:.3e})")
        return g_val, g_b, None, None, None, None, None


def solve_differentiable(A: CSRMatrix, values: torch.Tensor, b: torch.Tensor, arith="qtw", tol=1e-20,
                         maxit=20000, adj_tol=None) -> torch.Tensor:
    return MWCGSolve.apply(values, b, A, arith, tol, maxit, adj_tol)
