"""BiCGStab on the CUDA path vs the oracle, bit for bit (mwcg_solve_bicgstab).

Nonsymmetric upwind convection-diffusion systems and a power-law graph
Laplacian, every arithmetic, explicit and automatic plans, the host-launched
kernels, the early exit on ||s||, breakdown and the special cases.
"""
import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu

ARITHS = ["fp64", "dw", "qdw", "tw", "qtw", "qdw_nn", "qtw_nn", "qw", "qqw", "qqw_nn"]
W = {"fp64": 1, "dw": 2, "qdw": 2, "tw": 3, "qtw": 3, "qdw_nn": 2, "qtw_nn": 3, "qw": 4, "qqw": 4, "qqw_nn": 4}
TOL = {"fp64": 1e-14, "dw": 1e-28, "qdw": 1e-28, "tw": 1e-40, "qtw": 1e-40, "qdw_nn": 1e-28, "qtw_nn": 1e-40,
       "qw": 1e-55, "qqw": 1e-55, "qqw_nn": 1e-55}


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


def _check(mw, orc, M, A, b, arith, tol, maxit, tag, x0=None):
    r = mw.solve_bicgstab(M, dev(b), arith, tol, maxit, history=True, x0=None if x0 is None else dev(x0))
    xo, ito, rro, sto, ho = orc.bicgstab(arith, A, b, x0=x0, tol=tol, maxit=maxit, plan=M.plan, history=True)
    assert (r.iters, r.status) == (ito, sto), (tag, arith, r.iters, ito, r.status, sto)
    assert same_bits(np.array([r.relres]), np.array([rro])), (tag, arith, r.relres, rro)
    assert same_bits(r.x.cpu().numpy(), xo), (tag, arith)
    if r.iters:
        assert same_bits(r.history.cpu().numpy(), ho), (tag, arith)
    return r


@pytest.mark.parametrize("arith", ARITHS)
def test_convection_diffusion_every_arithmetic(mw, orc, arith):
    A = P.convection_diffusion_2d(72, 2.0)
    b = P.rhs_uniform(A.n, 51)
    M = mw.CSRMatrix.from_csr(A)
    r = _check(mw, orc, M, A, b, arith, TOL[arith], 800, "cd72")
    assert r.status == 0 or arith.endswith("_nn")          # the NN variants may break down
    M.plan = (2, 256, 37)
    _check(mw, orc, M, A, b, arith, TOL[arith], 800, "cd72 V=2")


@pytest.mark.parametrize("arith", ["fp64", "dw", "qtw", "qqw"])
def test_irregular_rows_and_small_systems(mw, orc, arith):
    A = P.power_law_laplacian(5000, seed=17, mean_deg=12, max_deg=300)
    b = P.rhs_uniform(A.n, 52)
    M = mw.CSRMatrix.from_csr(A)
    _check(mw, orc, M, A, b, arith, 1e-25, 400, "powerlaw")
    A = P.convection_diffusion_2d(16, 8.0)                  # 256 rows: one tile
    b = P.rhs_uniform(A.n, 53)
    M = mw.CSRMatrix.from_csr(A)
    x0 = np.random.default_rng(5).standard_normal((W[arith], A.n)) * np.array([1.0, 1e-17, 1e-34, 1e-51][:W[arith]])[:, None]
    _check(mw, orc, M, A, b, arith, TOL[arith], 400, "cd16 x0", x0=x0)


def test_eager_launches(mw, orc, monkeypatch):
    monkeypatch.setenv("MWCG_EAGER", "1")
    A = P.convection_diffusion_2d(40, 4.0)
    b = P.rhs_uniform(A.n, 54)
    M = mw.CSRMatrix.from_csr(A)
    for ar in ("qtw", "fp64", "qqw"):
        _check(mw, orc, M, A, b, ar, TOL[ar], 300, "eager")


def test_closed_forms_and_breakdown(mw, orc):
    n = 300
    b = P.rhs_uniform(n, 55)
    for d in (2.0, -2.0):
        A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, d))
        M = mw.CSRMatrix.from_csr(A)
        for ar in ARITHS:
            r = _check(mw, orc, M, A, b, ar, 1e-30, 5, f"diag {d}")
            assert (r.status, r.iters, r.relres) == (0, 1, 0.0)
    R = P.CSR(2, np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32), np.array([1.0, -1.0]))
    M = mw.CSRMatrix.from_csr(R)
    for ar in ARITHS:
        r = _check(mw, orc, M, R, np.array([1.0, 0.0]), ar, 1e-30, 5, "rotation")
        assert (r.status, r.iters) == (2, 1)


def test_special_cases(mw, orc):
    A = P.convection_diffusion_2d(20, 1.0)
    b = P.matvec_exact(A, np.ones(A.n))
    M = mw.CSRMatrix.from_csr(A)
    for ar in ARITHS:
        w = W[ar]
        r = mw.solve_bicgstab(M, dev(np.zeros(A.n)), ar, 1e-10, 50, x0=dev(np.ones((w, A.n))))
        assert (r.iters, r.status, r.relres) == (0, 0, 0.0) and np.all(r.x.cpu().numpy() == 0)
        x0 = np.zeros((w, A.n))
        x0[0] = 1.0
        r = mw.solve_bicgstab(M, dev(b), ar, 1e-10, 50, x0=dev(x0))
        assert (r.iters, r.status) == (0, 0) and np.all(r.x.cpu().numpy() == x0)
        r = mw.solve_bicgstab(M, dev(b), ar, 1e-10, 0)
        xo, ito, rro, sto = orc.bicgstab(ar, A, b, tol=1e-10, maxit=0, plan=M.plan)
        assert (r.iters, r.status) == (ito, sto) == (0, 1) and r.relres == rro
        _check(mw, orc, M, A, b, ar, 1e-300, 3, "maxit")


def test_empty_system(mw):
    import torch
    E = P.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    M = mw.CSRMatrix.from_csr(E)
    for ar in ("fp64", "qtw", "qqw"):
        b = torch.zeros(0, dtype=torch.float64, device="cuda")
        r = mw.solve_bicgstab(M, b, ar, 1e-10, 10)
        assert (r.iters, r.status, r.relres) == (0, 0, 0.0) and r.x.numel() == 0
        M.preconditioner = "jacobi"
        r = mw.solve(M, b, ar, 1e-10, 10)
        assert (r.iters, r.status, r.relres) == (0, 0, 0.0)
        M.preconditioner = "none"
