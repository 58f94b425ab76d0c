"""Full-size checks on the 128^3 Poisson workload, in the recorded plan (the one bench.py times for QTW).

The expected values come from the CPU oracle's complete solve
(tests/golden/fullsize_c2.json, written by tests/golden/make_fullsize.py):
iteration count, status, the bits of the final residual and the SHA-256 of
every bit of the multi-word solution.  The exact-solution twin (b = A*1)
checks the forward error against x* = 1, a property that holds at any size.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "fullsize_c2.json")


@pytest.fixture(scope="module")
def mw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_13536_gb300 import build, solver
    build.build()
    return solver


@pytest.fixture(scope="module")
def c2(mw):
    import torch
    A, b, tol, maxit = P.workload("c2")
    M = mw.CSRMatrix.from_csr(A)
    return A, M, torch.as_tensor(b, device="cuda"), tol, maxit


@pytest.mark.parametrize("arith", ["fp64", "dw", "qtw", "qqf", "qf"])
def test_c2_solution_bits_match_oracle_full_solve(mw, c2, arith):
    g = json.load(open(GOLD))
    if arith not in g:
        pytest.skip(f"no oracle record for {arith}")
    A, M, b, tol, maxit = c2
    if arith == "qtw":                 # the headline arithmetic: its automatic plan is the recorded one
        assert tuple(g["plan"]) == M.plan_for(arith), "the solver's automatic plan differs from the recorded one"
    M.plan = tuple(g["plan"])          # every arithmetic solved in the recorded plan
    r = mw.solve(M, b, arith, tol, maxit)
    M.plan = None
    e = g[arith]
    assert (r.iters, r.status) == (e["iters"], e["status"])
    assert float(r.relres).hex() == e["relres_hex"]
    x = r.x.cpu().numpy().astype(np.float64)      # QQF's / QF's FP32 words as the oracle stores them
    for i, words in e["samples"].items():
        assert [float(x[k, int(i)]).hex() for k in range(x.shape[0])] == words
    assert hashlib.sha256(np.ascontiguousarray(x).view(np.uint64).tobytes()).hexdigest() == e["x_sha256"]


@pytest.mark.parametrize("arith,bound", [("fp64", 1e-9), ("dw", 1e-10), ("qdw", 1e-10), ("qtw", 1e-10),
                                         ("qqf", 1e-10), ("qf", 1e-10)])
def test_c2_twin_forward_error(mw, arith, bound):
    import torch
    A, b, tol, maxit = P.workload("c2_twin")
    M = mw.CSRMatrix.from_csr(A)
    r = mw.solve(M, torch.as_tensor(b, device="cuda"), arith, tol, maxit)
    assert r.status == 0 and r.relres < tol
    x = mw.collapse(r.x).cpu().numpy()
    err = np.linalg.norm(x - 1.0) / np.sqrt(A.n)
    assert err < bound, err
