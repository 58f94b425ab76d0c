"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

The kernels and the oracle follow the same operation sequences and, given the
same plan {V, T, G}, the same summation order, so the comparison is bit for
bit: word operations, SpMV, dots, every CG iterate, iteration counts, final
residuals and statuses.
"""
import random
import re

import numpy as np
import pytest

from mwref import rand_mw
from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu

ARITHS = ["fp64", "dw", "qdw", "tw", "qtw", "qdw_nn", "qtw_nn", "qw", "qqw", "qqw_nn"]
W = {"fp64": 1, "dw": 2, "qdw": 2, "tw": 3, "qtw": 3, "qdw_nn": 2, "qtw_nn": 3, "qw": 4, "qqw": 4, "qqw_nn": 4}
SCALE = np.array([1.0, 1e-17, 1e-34, 1e-51])


@pytest.fixture(scope="module")
def mw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_13536_gb300 import build, solver
    build.build()
    return solver


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def same_bits(a, b):
    """Bit-identical, except that any two NaNs match: the GPU and the host CPU
    produce different NaN payloads/signs for the same invalid operation."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    if not np.array_equal(na, nb):
        return False
    return np.array_equal(bits(a)[~na], bits(b)[~nb])


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _inputs(rng, n, w):
    a = rand_mw(rng, n, w, emin=-40, emax=40)
    b = rand_mw(rng, n, w, emin=-40, emax=40)
    # Adversarial rows: cancellation, exact zeros, signed zeros, tiny lower words.
    k = n // 4
    b[:, :k] = -a[:, :k] * (1 + np.array([rng.choice((0.0, 2.0 ** -rng.randint(1, 60))) for _ in range(k)]))
    b[:, k:k + 8] = 0.0
    b[0, k + 8:k + 16] = -0.0
    return a, b


@pytest.mark.parametrize("arith", ARITHS)
def test_word_ops_bit_exact(mw, orc, arith):
    rng = random.Random(100 + W[arith])
    w = W[arith]
    n = 4000
    a, b = _inputs(rng, n, w)
    s = a[0].copy()
    da, db, ds = dev(a), dev(b), dev(s)
    assert same_bits(host(mw.word_op("add", arith, da, db)), orc.add(arith, a, b))
    assert same_bits(host(mw.word_op("mul", arith, da, db)), orc.mul(arith, a, b))
    assert same_bits(host(mw.word_op("dxmul", arith, ds, db)), orc.dxmul(arith, s, b))
    nz = np.abs(b[0]) > 0
    assert same_bits(host(mw.word_op("div", arith, dev(a[:, nz]), dev(b[:, nz]))), orc.div(arith, a[:, nz], b[:, nz]))
    assert same_bits(host(mw.word_op("normalize", arith, da)), orc.normalize(arith, a))
    assert same_bits(host(mw.word_op("collapse", arith, da)), orc.collapse(arith, a))


def _matrices():
    out = [P.laplacian_2d(37), P.laplacian_3d(11, 1e-3),
           P.power_law_laplacian(3000, seed=5, mean_deg=12, max_deg=300),
           P.diffusion_2d(40, seed=3)]
    # A matrix with empty rows and a ragged tail (n not a multiple of any tile).
    A = P.power_law_laplacian(1111, seed=9, mean_deg=6, max_deg=80)
    rp = A.row_ptr.copy()
    keep = np.ones(A.nnz, dtype=bool)
    for i in (0, 5, 500, 1110):
        keep[rp[i]:rp[i + 1]] = False
    cnt = np.array([keep[rp[i]:rp[i + 1]].sum() for i in range(A.n)])
    rp2 = np.zeros(A.n + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp2[1:])
    out.append(P.CSR(A.n, rp2, A.col[keep], A.val[keep], "with_empty_rows"))
    out.append(_drop_rows(P.laplacian_2d(45), (0, 33, 700, 2024), "stencil_with_empty_rows"))
    return out


def _drop_rows(A, rows, name):
    """A with the entries of `rows` removed (empty rows, same n)."""
    rp = A.row_ptr
    keep = np.ones(A.nnz, dtype=bool)
    for i in rows:
        keep[rp[i]:rp[i + 1]] = False
    cnt = np.array([keep[rp[i]:rp[i + 1]].sum() for i in range(A.n)])
    rp2 = np.zeros(A.n + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp2[1:])
    return P.CSR(A.n, rp2, A.col[keep], A.val[keep], name)


@pytest.mark.parametrize("arith", ARITHS)
def test_spmv_bit_exact_all_lane_splits(mw, orc, arith):
    rng = np.random.default_rng(7)
    w = W[arith]
    for A in _matrices():
        M = mw.CSRMatrix.from_csr(A)
        p = rng.standard_normal((w, A.n)) * SCALE[:w, None]
        for V in (1, 2, 4, 8, 16, 32):
            M.plan = (V, 256, 5)
            q = host(mw.spmv(M, arith, dev(p)))
            assert same_bits(q, orc.spmv(arith, A, p, V)), (A.name, V)


@pytest.mark.parametrize("arith", ["fp64", "dw", "qtw", "tw", "qqw", "qw"])
def test_dot_bit_exact(mw, orc, arith):
    rng = np.random.default_rng(8)
    w = W[arith]
    for n in (1, 7, 255, 256, 257, 5000, 65536 + 3):
        u = rng.standard_normal((w, n)) * SCALE[:w, None]
        v = rng.standard_normal((w, n)) * SCALE[:w, None]
        for G in (1, 3, 152, 1024):
            d = mw.dot(arith, dev(u), dev(v), G)
            assert same_bits(d, orc.dot(arith, u, v, 256, G)), (n, G)


CG_CASES = [
    ("lap2d_64_twin", lambda: (P.laplacian_2d(64), None), 1e-12, 2000),
    ("lap3d_20", lambda: (P.laplacian_3d(20), 1), 1e-14, 3000),
    ("powerlaw_6000", lambda: (P.power_law_laplacian(6000, seed=11, mean_deg=20, max_deg=400), 2), 1e-10, 3000),
    ("diffusion_48", lambda: (P.diffusion_2d(48, seed=4), 3), 1e-14, 3000),
]


@pytest.mark.parametrize("case", CG_CASES, ids=[c[0] for c in CG_CASES])
@pytest.mark.parametrize("arith", ARITHS)
def test_cg_bit_exact_against_mirrored_oracle(mw, orc, arith, case):
    name, make, tol, maxit = case
    A, seed = make()
    b = P.rhs_ones_exact(A) if seed is None else P.rhs_uniform(A.n, seed)
    M = mw.CSRMatrix.from_csr(A)
    V, T, G = M.plan_for(arith)                 # the automatic (timed) plan of this arithmetic
    r = mw.solve(M, dev(b), arith, tol, maxit)
    xo, ito, rro, sto = orc.cg(arith, A, b, tol=tol, maxit=maxit, plan=(V, T, G))
    assert (r.iters, r.status) == (ito, sto), (name, arith)
    assert same_bits(np.array([r.relres]), np.array([rro]))
    assert same_bits(host(r.x), xo)


@pytest.mark.parametrize("arith", ["fp64", "dw", "qtw", "qqw", "qqf"])
def test_value_updates_then_solve(mw, orc, arith):
    """New values from the host, then from the device, on a stencil with empty
    rows and a ragged tail: the solve and the SpMV equal the oracle's on the
    new matrix, bit for bit."""
    import torch
    A = _drop_rows(P.laplacian_3d(13, 1e-2), (7, 2196), "lap3d_13_holes")   # 2197 rows
    ln = np.diff(A.row_ptr)
    dt = np.float32 if arith == "qqf" else np.float64      # FP32 words travel as float32
    b = P.rhs_uniform(A.n, 21)
    b[ln == 0] = 0.0                               # an empty row's equation is 0 = 0
    M = mw.CSRMatrix.from_csr(A)
    M.plan = (1, 256, 11)
    rng = np.random.default_rng(22)
    rows = np.repeat(np.arange(A.n), ln)
    diag = A.col == rows
    for step, on_device in ((0, False), (1, False), (2, True)):
        val = A.val.copy()
        if step:
            val[diag] += rng.uniform(0.5, 1.0, diag.sum())       # still diagonally dominant
        A2 = A.with_values(val)
        if step:
            M.update_values(torch.as_tensor(val, device="cuda") if on_device else val)
        r = mw.solve(M, dev(b), arith, 1e-13, 3000)
        xo, ito, rro, sto = orc.cg(arith, A2, b, tol=1e-13, maxit=3000, plan=(1, 256, 11))
        assert (r.iters, r.status) == (ito, sto), (arith, step)
        assert same_bits(host(r.x), xo), (arith, step)
        q = host(mw.spmv(M, arith, torch.as_tensor(xo.astype(dt), device="cuda")))
        assert same_bits(q, orc.spmv(arith, A2, xo, 1)), (arith, step)


def test_device_arrays_checked_on_the_device(mw, orc):
    """A handle from device arrays: its entries are checked on the device and
    the first bad entry is reported as the host check reports it; valid
    arrays give the same solve as host arrays."""
    import torch
    from paper_2510_13536_gb300._capi import MWCGError
    A = P.laplacian_3d(12)
    rp = torch.as_tensor(A.row_ptr, device="cuda")
    col = torch.as_tensor(A.col, device="cuda")
    val = torch.as_tensor(A.val, device="cuda")
    bad_col, bad_val = col.clone(), val.clone()
    bad_col[5000] = A.n
    bad_val[4000] = float("nan")
    bad_val[6000] = float("inf")
    for c, v, msg in ((bad_col, val, f"col[5000] = {A.n} out of range"), (col, bad_val, "val[4000] is not finite"),
                      (bad_col, bad_val, "val[4000] is not finite")):
        with pytest.raises(MWCGError, match=re.escape(msg)):
            mw.CSRMatrix(A.n, rp, c, v)
        with pytest.raises(MWCGError, match=re.escape(msg)):
            mw.CSRMatrix(A.n, A.row_ptr, c.cpu().numpy(), v.cpu().numpy())
    b = P.rhs_uniform(A.n, 31)
    Md, Mh = mw.CSRMatrix(A.n, rp, col, val), mw.CSRMatrix.from_csr(A)
    for M in (Md, Mh):
        M.plan = (1, 256, 7)
    rd, rh = mw.solve(Md, dev(b), "qtw", 1e-14, 500), mw.solve(Mh, dev(b), "qtw", 1e-14, 500)
    assert (rd.iters, rd.status) == (rh.iters, rh.status) and same_bits(host(rd.x), host(rh.x))


@pytest.mark.parametrize("arith", ["dw", "qtw", "fp64"])
def test_cg_explicit_plans_and_x0(mw, orc, arith):
    A = P.power_law_laplacian(2500, seed=13, mean_deg=15, max_deg=200)
    b = P.rhs_uniform(A.n, 14)
    w = W[arith]
    x0 = np.random.default_rng(15).standard_normal((w, A.n)) * np.array([1.0, 1e-17, 1e-34][:w])[:, None]
    M = mw.CSRMatrix.from_csr(A)
    for plan in ((1, 256, 1), (4, 256, 7), (32, 256, 300)):
        M.plan = plan
        r = mw.solve(M, dev(b), arith, 1e-11, 5000, x0=dev(x0))
        xo, ito, rro, sto = orc.cg(arith, A, b, x0=x0, tol=1e-11, maxit=5000, plan=plan)
        assert (r.iters, r.status) == (ito, sto) and same_bits(host(r.x), xo), plan


def test_cg_special_cases(mw, orc):
    A = P.laplacian_2d(16)
    b = P.rhs_ones_exact(A)
    M = mw.CSRMatrix.from_csr(A)
    for arith in ARITHS:
        plan = M.plan_for(arith)
        w = W[arith]
        # b = 0 -> x = 0, zero iterations
        r = mw.solve(M, dev(np.zeros(A.n)), arith, 1e-10, 100, x0=dev(np.ones((w, A.n))))
        assert (r.iters, r.status, r.relres) == (0, 0, 0.0) and np.all(host(r.x) == 0)
        # exact x0 -> zero iterations
        x0 = np.zeros((w, A.n))
        x0[0] = 1.0
        r = mw.solve(M, dev(b), arith, 1e-10, 100, x0=dev(x0))
        assert (r.iters, r.status) == (0, 0) and same_bits(host(r.x), x0)
        # maxit = 0
        r = mw.solve(M, dev(b), arith, 1e-10, 0)
        xo, ito, rro, sto = orc.cg(arith, A, b, tol=1e-10, maxit=0, plan=plan)
        assert (r.iters, r.status) == (ito, sto) == (0, 1) and r.relres == rro
        # maxit reached
        r = mw.solve(M, dev(b), arith, 1e-30, 3)
        xo, ito, rro, sto = orc.cg(arith, A, b, tol=1e-30, maxit=3, plan=plan)
        assert (r.iters, r.status) == (3, 1) == (ito, sto) and same_bits(host(r.x), xo)
        # NaN in b -> breakdown on the first pass
        bb = b.copy()
        bb[7] = np.nan
        r = mw.solve(M, dev(bb), arith, 1e-10, 100)
        assert (r.iters, r.status) == (1, 2)
    # negative definite -> breakdown on the first pass
    Mneg = mw.CSRMatrix.from_csr(A.with_values(-A.val))
    for arith in ARITHS:
        r = mw.solve(Mneg, dev(b), arith, 1e-10, 100)
        assert (r.iters, r.status) == (1, 2)


def test_history_and_host_buffers(mw, orc):
    A = P.laplacian_3d(16)
    b = P.rhs_uniform(A.n, 5)
    M = mw.CSRMatrix.from_csr(A)
    r = mw.solve(M, dev(b), "qtw", 1e-13, 2000, history=True)
    xo, ito, rro, sto, ho = orc.cg("qtw", A, b, tol=1e-13, maxit=2000, plan=M.plan, history=True)
    assert same_bits(host(r.history), ho)
    xh, ith, rrh, sth = mw.solve_host(M, b, "qtw", 1e-13, 2000)
    assert (ith, sth) == (r.iters, r.status) and same_bits(xh, host(r.x))


def test_repeated_solves_reuse_graph(mw):
    A = P.laplacian_2d(50)
    M = mw.CSRMatrix.from_csr(A)
    b = dev(P.rhs_uniform(A.n, 1))
    r1 = mw.solve(M, b, "qdw", 1e-12, 1000)
    r2 = mw.solve(M, b, "qdw", 1e-12, 1000)
    r3 = mw.solve(M, b, "dw", 1e-12, 1000)
    r4 = mw.solve(M, b, "qdw", 1e-12, 1000)
    assert same_bits(host(r1.x), host(r2.x)) and same_bits(host(r1.x), host(r4.x))
    assert r3.status == 0


def test_adjoint_bit_exact_and_against_exact(mw, orc):
    A = P.diffusion_2d(24, seed=8)
    b = P.rhs_normal(A.n, 9)
    wv = P.rhs_normal(A.n, 10)
    M = mw.CSRMatrix.from_csr(A)
    for arith, tol in (("qtw", 1e-28), ("dw", 1e-24), ("fp64", 1e-13)):
        r = mw.solve(M, dev(b), arith, tol, 5000)
        g_b, g_val, it, rr, st = mw.adjoint(M, r.x, dev(wv), arith, tol, 5000)
        gbo, gvo, lam, ito, rro, sto = orc.adjoint(arith, A, host(r.x), wv, tol, 5000, plan=M.plan)
        assert (it, st) == (ito, sto)
        assert same_bits(host(g_b), gbo) and same_bits(host(g_val), gvo)
