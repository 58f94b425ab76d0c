"""Jacobi-preconditioned CG on the CUDA path vs the oracle, bit for bit.

M^-1 = diag(fl(1/a_ii)) (mwcg_set_preconditioner).  Every path that runs the
solver -- the CUDA graph, the host-launched (eager) kernels, the one-cluster
launch for small systems, the batched persistent kernel and the adjoint --
must give the oracle's bits, including the undefined-preconditioner status.
"""
import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu

ARITHS = ["fp64", "dw", "qdw", "tw", "qtw", "qdw_nn", "qtw_nn", "qw", "qqw", "qqw_nn"]
W = {"fp64": 1, "dw": 2, "qdw": 2, "tw": 3, "qtw": 3, "qdw_nn": 2, "qtw_nn": 3, "qw": 4, "qqw": 4, "qqw_nn": 4}
R, X, PP, Q, SUM = 1, 2, 4, 8, 16


@pytest.fixture(scope="module")
def mw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_13536_gb300 import build, solver
    build.build()
    return solver


def same_bits(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    if not np.array_equal(na, nb):
        return False
    return np.array_equal(a.view(np.uint64)[~na], b.view(np.uint64)[~nb])


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _check(mw, orc, M, A, b, arith, tol, maxit, tag, norm=None, x0=None):
    if norm is not None:
        M.normalization = norm
    r = mw.solve(M, dev(b), arith, tol, maxit, history=True, x0=None if x0 is None else dev(x0))
    xo, ito, rro, sto, ho = orc.cg(arith, A, b, x0=x0, tol=tol, maxit=maxit, plan=M.plan, history=True,
                                   norm=norm, precond="jacobi")
    assert (r.iters, r.status) == (ito, sto), (tag, arith, norm, r.iters, ito, r.status, sto)
    assert same_bits(np.array([r.relres]), np.array([rro])), (tag, arith, r.relres, rro)
    assert same_bits(r.x.cpu().numpy(), xo), (tag, arith, norm)
    if r.iters:
        assert same_bits(r.history.cpu().numpy(), ho), (tag, arith)
    return r


@pytest.mark.parametrize("arith", ARITHS)
def test_graph_path_all_arithmetics(mw, orc, arith):
    """Variable-coefficient diffusion (Jacobi changes the iterates) and a
    power-law graph Laplacian in its automatic plan."""
    for A, seed, tol, maxit in ((P.diffusion_2d(90, 3), 31, 1e-26, 400),
                                (P.power_law_laplacian(5000, seed=7, mean_deg=12, max_deg=300), 32, 1e-26, 300)):
        b = P.rhs_uniform(A.n, seed)
        M = mw.CSRMatrix.from_csr(A)
        M.preconditioner = "jacobi"
        _check(mw, orc, M, A, b, arith, tol, maxit, A.name)


@pytest.mark.parametrize("arith", ["qdw", "qtw", "qqw"])
def test_with_normalisation_policies(mw, orc, arith):
    A = P.laplacian_3d(24, 1e-3)
    b = P.rhs_uniform(A.n, 33)
    M = mw.CSRMatrix.from_csr(A)
    M.plan = (2, 256, 37)
    M.preconditioner = "jacobi"
    for norm in ((1, R), (1, R | X | PP | Q | SUM), (2, R | PP), (0, R), (2, R)):
        _check(mw, orc, M, A, b, arith, 1e-30, 150, "policy", norm=norm)


@pytest.mark.parametrize("arith", ["fp64", "dw", "qtw", "tw", "qqw", "qw"])
def test_single_cluster_path(mw, orc, arith):
    A = P.diffusion_2d(40, 5)
    b = P.rhs_uniform(A.n, 34)
    M = mw.CSRMatrix.from_csr(A)
    M.preconditioner = "jacobi"
    _check(mw, orc, M, A, b, arith, 1e-30, 400, "cluster")
    M.plan = (4, 256, M.plan[2])
    x0 = np.random.default_rng(3).standard_normal((W[arith], A.n)) * np.array([1.0, 1e-17, 1e-34, 1e-51][:W[arith]])[:, None]
    _check(mw, orc, M, A, b, arith, 1e-30, 400, "cluster V=4 x0", x0=x0)


def test_eager_launches(mw, orc, monkeypatch):
    monkeypatch.setenv("MWCG_EAGER", "1")
    A = P.diffusion_2d(70, 6)
    b = P.rhs_uniform(A.n, 35)
    M = mw.CSRMatrix.from_csr(A)
    M.preconditioner = "jacobi"
    for ar in ("qtw", "fp64"):
        _check(mw, orc, M, A, b, ar, 1e-30, 120, "eager")


def test_switching_preconditioner_and_values(mw, orc):
    """Toggle the preconditioner between solves; change the values (the
    weights must follow the new diagonal)."""
    A = P.diffusion_2d(60, 8)
    b = P.rhs_uniform(A.n, 36)
    M = mw.CSRMatrix.from_csr(A)
    for kind in ("jacobi", "none", "jacobi"):
        M.preconditioner = kind
        r = mw.solve(M, dev(b), "qdw", 1e-26, 500)
        xo, ito, rro, sto = orc.cg("qdw", A, b, tol=1e-26, maxit=500, plan=M.plan,
                                   precond=None if kind == "none" else "jacobi")
        assert (r.iters, r.status) == (ito, sto) and same_bits(r.x.cpu().numpy(), xo), kind
    # D A D with d_i in {1, 2}: still SPD, every value exact, a new diagonal.
    d = np.where(np.arange(A.n) % 3 == 0, 2.0, 1.0)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    A2 = A.with_values(A.val * d[rows] * d[A.col])
    M.update_values(A2.val)
    _check(mw, orc, M, A2, b, "qdw", 1e-26, 500, "new values")


def test_undefined_preconditioner(mw, orc):
    A = P.laplacian_2d(30)
    b = P.rhs_uniform(A.n, 37)
    for bad in ("zero", "negative", "missing"):
        B = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
        k0 = [k for k in range(B.row_ptr[7], B.row_ptr[8]) if B.col[k] == 7][0]
        if bad == "zero":
            B.val[k0] = 0.0
        elif bad == "negative":
            B.val[k0] = -4.0
        else:
            B.col[k0] = 6 if B.col[k0 - 1] != 6 else 8
        M = mw.CSRMatrix.from_csr(B)
        M.preconditioner = "jacobi"
        x0 = np.full((3, A.n), 0.25)      # three words: QTW
        r = mw.solve(M, dev(b), "qtw", 1e-20, 100, x0=dev(x0))
        xo, ito, rro, sto = orc.cg("qtw", B, b, x0=x0, tol=1e-20, maxit=100, plan=M.plan, precond="jacobi")
        assert (r.status, r.iters, sto, ito) == (3, 0, 3, 0), bad
        assert np.array_equal(r.x.cpu().numpy(), x0)
        M.preconditioner = "none"                 # the plain solver does not need the diagonal
        r = mw.solve(M, dev(b), "fp64", 1e-10, 3)
        assert r.status in (0, 1, 2)


def test_batched_mixed_preconditioning(mw, orc):
    import torch
    systems = [(P.diffusion_2d(35, 1), "qtw", "jacobi"), (P.laplacian_3d(14, 1e-3), "qdw", "none"),
               (P.diffusion_2d(30, 7), "qqw", "jacobi"), (P.laplacian_2d(22), "qw", "none"),
               (P.power_law_laplacian(2000, seed=9, mean_deg=10, max_deg=120), "dw", "jacobi"),
               (P.diffusion_2d(20, 2), "fp64", "jacobi"), (P.laplacian_2d(25), "tw", "none"),
               (P.diffusion_2d(28, 4), "qtw_nn", "jacobi")]
    bad = P.laplacian_2d(12)
    bad = P.CSR(bad.n, bad.row_ptr.copy(), bad.col.copy(), bad.val.copy())
    kd = [k for k in range(bad.row_ptr[3], bad.row_ptr[4]) if bad.col[k] == 3][0]
    bad.val[kd] = 0.0                               # undefined Jacobi weight
    systems.append((bad, "qdw", "jacobi"))
    Ms, bs = [], []
    for k, (A, ar, pc) in enumerate(systems):
        M = mw.CSRMatrix.from_csr(A)
        M.preconditioner = pc
        Ms.append(M)
        bs.append(torch.as_tensor(P.rhs_uniform(A.n, 60 + k), device="cuda"))
    res = mw.solve_batched(Ms, bs, [s[1] for s in systems], 1e-26, 600)
    C = mw.batched_cluster_size()
    for (A, ar, pc), M, b, r in zip(systems, Ms, bs, res):
        xo, ito, rro, sto = orc.cg(ar, A, b.cpu().numpy(), tol=1e-26, maxit=600, plan=(M.plan[0], 256, C),
                                   precond=None if pc == "none" else "jacobi")
        assert (r.iters, r.status) == (ito, sto), (A.name, ar, pc)
        assert same_bits(r.x.cpu().numpy(), xo), (A.name, ar, pc)
    assert res[-1].status == 3


@pytest.mark.parametrize("arith", ["qtw", "dw", "qqw"])
def test_adjoint_gradients(mw, orc, arith):
    import torch
    A = P.diffusion_2d(50, 10)
    b = P.rhs_uniform(A.n, 38)
    wv = P.rhs_uniform(A.n, 39)
    M = mw.CSRMatrix.from_csr(A)
    M.preconditioner = "jacobi"
    r = mw.solve(M, dev(b), arith, 1e-28, 2000)
    xo, *_ = orc.cg(arith, A, b, tol=1e-28, maxit=2000, plan=M.plan, precond="jacobi")
    assert same_bits(r.x.cpu().numpy(), xo)
    g_b, g_val, it, rr, st = mw.adjoint(M, r.x, dev(wv), arith, 1e-28, 2000)
    gbo, gvo, lam, ito, rro, sto = orc.adjoint(arith, A, xo, wv, 1e-28, 2000, plan=M.plan, precond="jacobi")
    assert (it, st) == (ito, sto)
    assert same_bits(g_b.cpu().numpy(), gbo) and same_bits(g_val.cpu().numpy(), gvo)


def test_preconditioner_arguments(mw):
    M = mw.CSRMatrix.from_csr(P.laplacian_2d(8))
    assert M.preconditioner == "none"
    M.preconditioner = "jacobi"
    assert M.preconditioner == "jacobi"
    with pytest.raises(ValueError):
        M.preconditioner = "ilu"
    from paper_2510_13536_gb300 import _capi
    import ctypes
    with pytest.raises(_capi.MWCGError):
        _capi.check(_capi.load().mwcg_set_preconditioner(M.handle, ctypes.c_int(7)))
    assert M.preconditioner == "jacobi"
