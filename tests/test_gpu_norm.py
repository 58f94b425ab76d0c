"""Normalisation policy of the quasi arithmetics on the CUDA path vs the oracle.

The policy {every, mask} (mwcg_set_normalization) generalises Sec. IV-D's
normalisation of r after its AXPY.  Every path that runs CG -- the CUDA graph,
the host-launched (eager) kernels, the single-cluster launch for small
systems and the batched persistent kernel -- must give the oracle's bits for
every policy, including the ones that break down.
"""
import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu

R, X, PP, Q, SUM = 1, 2, 4, 8, 16
ALL = R | X | PP | Q | SUM
POLICIES = [(0, R), (1, R | X), (1, R | PP), (1, R | Q), (1, R | SUM), (1, ALL), (2, ALL), (3, R | Q | SUM),
            (2, R)]


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


def _check(mw, orc, M, A, b, arith, norm, tol, maxit, tag):
    M.normalization = norm
    r = mw.solve(M, dev(b), arith, tol, maxit, history=True)
    xo, ito, rro, sto, ho = orc.cg(arith, A, b, tol=tol, maxit=maxit, plan=M.plan, history=True, norm=norm)
    assert (r.iters, r.status) == (ito, sto), (tag, arith, norm, r.iters, ito, r.status, sto)
    assert same_bits(np.array([r.relres]), np.array([rro])), (tag, arith, norm)
    assert same_bits(r.x.cpu().numpy(), xo), (tag, arith, norm)
    assert same_bits(r.history.cpu().numpy(), ho), (tag, arith, norm)


@pytest.mark.parametrize("arith", ["qdw", "qtw", "qqw"])
def test_graph_path_every_policy(mw, orc, arith):
    """3-D Laplacian 24^3 (54 tiles: the CUDA-graph path) in plan V=2 so that the
    lane-tree combines of NORM_SUM are exercised."""
    A = P.laplacian_3d(24, 1e-3)
    b = P.rhs_uniform(A.n, 21)
    M = mw.CSRMatrix.from_csr(A)
    M.plan = (2, 256, 37)
    for norm in POLICIES:
        _check(mw, orc, M, A, b, arith, norm, 1e-30, 120, "graph")


@pytest.mark.parametrize("arith", ["qdw", "qtw"])
def test_power_law_auto_plan(mw, orc, arith):
    """Irregular rows in the automatic plan (several lanes per row)."""
    A = P.power_law_laplacian(6000, seed=31, mean_deg=20, max_deg=400)
    b = P.rhs_uniform(A.n, 32)
    M = mw.CSRMatrix.from_csr(A)
    for norm in ((1, ALL), (1, R | SUM), (2, R | Q)):
        _check(mw, orc, M, A, b, arith, norm, 1e-30, 150, "power-law")


@pytest.mark.parametrize("arith", ["qdw", "qtw", "qqw"])
def test_single_cluster_path(mw, orc, arith):
    """A 2-D Laplacian small enough for the one-cluster launch."""
    A = P.laplacian_2d(40)
    b = P.rhs_uniform(A.n, 22)
    M = mw.CSRMatrix.from_csr(A)
    for norm in POLICIES:
        _check(mw, orc, M, A, b, arith, norm, 1e-30, 200, "cluster")
    M.plan = (4, 256, M.plan[2])
    for norm in ((1, R | SUM), (1, ALL)):
        _check(mw, orc, M, A, b, arith, norm, 1e-30, 200, "cluster V=4")


def test_eager_launches(mw, orc, monkeypatch):
    """The host-launched kernels pick the same SpMV variant as the graph."""
    monkeypatch.setenv("MWCG_EAGER", "1")
    A = P.laplacian_3d(20)
    b = P.rhs_uniform(A.n, 23)
    M = mw.CSRMatrix.from_csr(A)
    for norm in ((1, R | SUM), (0, R), (1, ALL)):
        _check(mw, orc, M, A, b, "qtw", norm, 1e-30, 60, "eager")


def test_policy_switch_rebuilds_the_graph(mw, orc):
    """Switching NORM_SUM on and off between solves on one handle."""
    A = P.laplacian_3d(20)
    b = P.rhs_uniform(A.n, 24)
    M = mw.CSRMatrix.from_csr(A)
    for norm in ((1, R), (1, R | SUM), (1, R), (0, SUM), (1, R | SUM)):
        _check(mw, orc, M, A, b, "qdw", norm, 1e-30, 80, "switch")


def test_batched_policies(mw, orc):
    import torch
    systems = [(P.laplacian_2d(30), "qtw", (1, ALL)), (P.laplacian_3d(12), "qdw", (2, R | Q)),
               (P.diffusion_2d(25, seed=3), "qtw", (0, R)), (P.laplacian_2d(20), "qdw", (1, R | SUM)),
               (P.power_law_laplacian(1500, seed=5, mean_deg=10, max_deg=100), "qtw", (3, R | X | SUM))]
    Ms, bs = [], []
    for k, (A, ar, norm) in enumerate(systems):
        M = mw.CSRMatrix.from_csr(A)
        M.normalization = norm
        Ms.append(M)
        bs.append(torch.as_tensor(P.rhs_uniform(A.n, 40 + k), device="cuda"))
    res = mw.solve_batched(Ms, bs, [s[1] for s in systems], 1e-30, 300)
    C = mw.batched_cluster_size()
    for (A, ar, norm), M, b, r in zip(systems, Ms, bs, res):
        xo, ito, rro, sto = orc.cg(ar, A, b.cpu().numpy(), tol=1e-30, maxit=300, plan=(M.plan[0], 256, C), norm=norm)
        assert (r.iters, r.status) == (ito, sto), (A.name, ar, norm)
        assert same_bits(r.x.cpu().numpy(), xo), (A.name, ar, norm)


def test_policy_arguments(mw):
    from paper_2510_13536_gb300._capi import MWCGError
    M = mw.CSRMatrix.from_csr(P.laplacian_2d(8))
    assert M.normalization == (1, R)
    M.normalization = (4, ["q", "sum", "r"])
    assert M.normalization == (4, R | Q | SUM)
    with pytest.raises(MWCGError):
        M.normalization = (-1, R)
    with pytest.raises(MWCGError):
        M.normalization = (1, 32)
    assert M.normalization == (4, R | Q | SUM)
