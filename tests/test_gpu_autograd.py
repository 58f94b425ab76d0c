"""torch.autograd wrapper (MWCGSolve) on the GPU: forward = mwcg_solve, backward =
adjoint CG + sparsity-masked -lambda_i x_j, bit-exact against the oracle."""
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


@pytest.mark.parametrize("arith,tol", [("qtw", 1e-26), ("dw", 1e-22), ("fp64", 1e-12)])
def test_autograd_gradients_equal_oracle_adjoint(mw, orc, arith, tol):
    import torch
    A = P.diffusion_2d(30, seed=31)
    b = P.rhs_normal(A.n, 32)
    wv = P.rhs_normal(A.n, 33)
    M = mw.CSRMatrix.from_csr(A)
    vals = torch.as_tensor(A.val, device="cuda").clone().requires_grad_(True)
    bb = torch.as_tensor(b, device="cuda").clone().requires_grad_(True)
    x = mw.solve_differentiable(M, vals, bb, arith, tol, 5000)
    loss = torch.dot(torch.as_tensor(wv, device="cuda"), x)
    loss.backward()
    xo, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=5000, plan=M.plan)
    assert st == 0
    g_b, g_val, lam, it2, rr2, st2 = orc.adjoint(arith, A, xo, wv, tol, 5000, plan=M.plan)
    xc = orc.collapse(arith, xo) if xo.shape[0] > 1 else xo[0]
    assert np.array_equal(x.detach().cpu().numpy().view(np.uint64), xc.view(np.uint64))
    assert np.array_equal(vals.grad.cpu().numpy().view(np.uint64), g_val.view(np.uint64))
    assert np.array_equal(bb.grad.cpu().numpy().view(np.uint64), g_b.view(np.uint64))


def test_values_update_changes_the_solve(mw):
    import torch
    A = P.laplacian_2d(20)
    M = mw.CSRMatrix.from_csr(A)
    b = torch.as_tensor(P.rhs_uniform(A.n, 1), device="cuda")
    r1 = mw.solve(M, b, "dw", 1e-20, 1000)
    M.update_values(2.0 * A.val)                      # A -> 2A: x -> x/2 exactly in spirit
    r2 = mw.solve(M, b, "dw", 1e-20, 1000)
    x1, x2 = mw.collapse(r1.x), mw.collapse(r2.x)
    assert float(torch.max(torch.abs(x1 - 2 * x2))) < 1e-14
    with pytest.raises(RuntimeError):
        M.update_values(np.full(A.nnz, np.nan))
    # Device values are checked on the device; a rejected update leaves A as it was.
    v = torch.as_tensor(A.val, device="cuda") * 2.0
    v[123] = float("inf")
    v[400] = float("nan")
    with pytest.raises(RuntimeError, match=r"val\[123\]"):
        M.update_values(v)
    r3 = mw.solve(M, b, "dw", 1e-20, 1000)
    assert torch.equal(r3.x, r2.x)
    M.update_values(torch.as_tensor(A.val, device="cuda"))
    r4 = mw.solve(M, b, "dw", 1e-20, 1000)
    assert torch.equal(r4.x, r1.x)


def test_pipe_probe_reports_rates(mw):
    import torch
    from paper_2510_13536_gb300 import _capi
    L = _capi.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    scratch = torch.empty(sms * 8 * 256, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rates = []
    for kind in range(5):
        v = ctypes.c_double(0.0)
        assert L.mwcg_probe_peak(kind, ctypes.c_void_p(scratch.data_ptr()), scratch.numel() * 8, s,
                                 ctypes.byref(v)) == 0
        rates.append(v.value)
    assert all(r > 1e10 for r in rates)
    assert rates[2] > 10 * rates[0]                  # the integer pipe is far wider than the FP64 pipe
    assert L.mwcg_probe_peak(0, ctypes.c_void_p(scratch.data_ptr()), 16, s, ctypes.byref(ctypes.c_double())) == -1
