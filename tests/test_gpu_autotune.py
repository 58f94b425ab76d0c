"""The plan autotuner on the device.

Each arithmetic gets its own automatic plan: the cost model's lane count V,
checked at the first call by timing the SpMV under the model's best
candidates.  Checked here:
* on an irregular power-law graph Laplacian (rows of 5 to 1000 entries), the
  plan chosen for DW, FP64 and QTW is within 10% of the fastest of an
  independent sweep over every lane count (CUDA events around each SpMV
  launch, mwcg_profile_kernels, plan pinned per V), and a solve in the
  chosen plan equals the oracle's in that plan bit for bit;
* a pinned plan applies to every arithmetic and reports no timings, and
  unpinning returns to the automatic plans.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_13536_gb300 import build, solver
    build.build()
    return solver


@pytest.fixture(scope="module")
def graph():
    return P.power_law_laplacian(200_000, seed=41, mean_deg=30, max_deg=1000)


def _spmv_ms(mw, M, arith, b, V, G):
    """Mean SpMV launch time (ms) over 5 CG iterations in plan (V, 256, G)."""
    import torch
    from paper_2510_13536_gb300 import _capi
    M.plan = (V, 256, G)
    x = torch.zeros((mw.words(arith), M.n), dtype=torch.float64, device="cuda")
    kms = (ctypes.c_double * 3)()
    _capi.check(_capi.load().mwcg_profile_kernels(
        M.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), mw.arith_id(arith), 5,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), kms))
    return kms[0]


@pytest.mark.parametrize("arith", ["dw", "fp64", "qtw"])
def test_tuned_lane_count_is_near_the_measured_best(mw, orc, graph, arith):
    import torch
    A = graph
    b = P.rhs_normal(A.n, 42)
    db = torch.as_tensor(b, device="cuda")
    M = mw.CSRMatrix.from_csr(A)
    plan, timed = M.tuning(arith)
    V, T, G = plan
    sweep = {v: min(_spmv_ms(mw, M, arith, db, v, G) for _ in range(2)) for v in (1, 2, 4, 8, 16, 32)}
    best = min(sweep.values())
    assert sweep[V] <= 1.10 * best, (arith, plan, timed, sweep)
    # A solve in the tuned plan equals the oracle's in that plan.
    M.plan = None
    assert M.plan_for(arith) == plan
    r = mw.solve(M, db, arith, 0.0, 15)
    xo, ito, rro, sto = orc.cg(arith, A, b, tol=0.0, maxit=15, plan=plan)
    assert (r.iters, r.status) == (ito, sto) == (15, 1)
    assert np.array_equal(r.x.cpu().numpy().view(np.uint64), xo.view(np.uint64))


def test_pinned_plan_applies_to_every_arithmetic(mw):
    A = P.laplacian_3d(40)
    M = mw.CSRMatrix.from_csr(A)
    auto = {ar: M.plan_for(ar) for ar in ("fp64", "dw", "qtw", "qqf")}
    assert all(p[1] == 256 for p in auto.values())
    M.plan = (2, 256, 37)
    for ar in ("fp64", "dw", "qtw", "qqf"):
        plan, timed = M.tuning(ar)
        assert plan == (2, 256, 37) and timed == {}
    M.plan = None
    assert {ar: M.plan_for(ar) for ar in auto} == auto
