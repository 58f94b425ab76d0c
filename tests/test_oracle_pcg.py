"""Pins of the oracle's Jacobi-preconditioned CG (an extension; Sec. VI names
preconditioning as future work).

M^-1 = diag(w), w_i = fl(1 / a_ii), applied as the arithmetic's FP64 x
multi-word product; the stopping residual stays FP64 (Sec. IV-C).  Independent
references:
 * textbook PCG in exact rationals (with the same FP64 w taken exactly);
 * plain CG, already pinned: with a constant power-of-two diagonal, w scales
   exactly, so every PCG quantity is a power-of-two multiple of the CG one
   and x must come out bit for bit the same;
 * exact-solution systems (b = A x*), closed forms and special cases.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from mwref import col, dense_fraction, pcg_exact, val
from paper_2510_13536_gb300 import problems as P

LEVEL = {"fp64": 1e-11, "dw": 1e-26, "qdw": 1e-25, "tw": 1e-40, "qtw": 1e-39}
W = {"fp64": 1, "dw": 2, "qdw": 2, "tw": 3, "qtw": 3}


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


@pytest.mark.parametrize("arith", ["fp64", "dw", "qdw", "qtw"])
@pytest.mark.parametrize("plan", [None, (1, 256, 3), (4, 256, 2)])
def test_power_of_two_diagonal_reproduces_cg(orc, arith, plan):
    """2-D 5-point Laplacian (diagonal 4): z = r/4 exactly, so PCG's p, q, rho,
    p^T q are CG's times 1/4, 1/4, 1/4, 1/16, alpha is CG's times 4, and x is
    CG's bit for bit.  (TW is left out: its restatement is not exactly
    scale-equivariant in every branch.)"""
    A = P.laplacian_2d(20)
    b = P.rhs_uniform(A.n, 3)
    for norm in (None, (2, 1 | 4)):
        if norm is not None and arith not in ("qdw", "qtw"):
            continue
        x1, i1, _, s1 = orc.cg(arith, A, b, tol=0.0, maxit=40, plan=plan, norm=norm)
        x2, i2, _, s2 = orc.cg(arith, A, b, tol=0.0, maxit=40, plan=plan, norm=norm, precond="jacobi")
        assert (i1, s1) == (i2, s2) == (40, 1)
        assert np.array_equal(_bits(x1), _bits(x2)), (arith, plan, norm)


@pytest.mark.parametrize("arith", ["fp64", "dw", "qdw", "tw", "qtw"])
def test_iterates_follow_exact_pcg(orc, arith):
    A = P.random_spd_small(9, seed=3)
    b = P.rhs_uniform(A.n, 4)
    d = np.array([A.val[k] for i in range(A.n) for k in range(A.row_ptr[i], A.row_ptr[i + 1]) if A.col[k] == i])
    w = 1.0 / d
    xs, rrs = pcg_exact(dense_fraction(A), b, w, 6)
    bn = math.sqrt(float(sum(Fraction(float(v)) ** 2 for v in b)))
    for k in (1, 2, 4, 6):
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-300, maxit=k, precond="jacobi")
        assert it == k and st == 1
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            got = sum(Fraction(float(v)) for v in x[:, i])
            assert abs(float(got - xs[k - 1][i])) <= LEVEL[arith] * float(scale), (arith, k, i)
        assert rr == pytest.approx(math.sqrt(float(rrs[k - 1])) / bn, rel=1e-9, abs=1e-300)


@pytest.mark.parametrize("arith,tol,bound", [("dw", 1e-26, 1e-23), ("qdw", 1e-26, 1e-23),
                                             ("qtw", 1e-38, 1e-35), ("fp64", 1e-14, 1e-11)])
def test_exact_solution_of_dyadic_diffusion(orc, arith, tol, bound):
    A = P.diffusion_2d(24, 11, dyadic=True)
    xs = P.random_signs(A.n, 12)
    b = P.matvec_grid_exact(A, xs)
    x, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=5000, plan=(1, 256, 3), precond="jacobi")
    assert st == 0
    err = math.sqrt(sum(float(sum(Fraction(float(v)) for v in x[:, i]) - Fraction(float(xs[i]))) ** 2
                        for i in range(A.n)) / A.n)
    assert err <= bound, err
    _, it_cg, _, st_cg = orc.cg(arith, A, b, tol=tol, maxit=5000, plan=(1, 256, 3))
    assert st_cg == 0 and it < it_cg            # the diagonal scaling pays on variable coefficients


def test_diagonal_system_closed_form(orc):
    """A = 2I: w = 1/2, z0 = r0/2, alpha = 1, x1 = b/2 exactly and r1 = 0."""
    n = 50
    A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    b = P.rhs_uniform(n, 1)
    for arith in W:
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-30, maxit=5, precond="jacobi")
        assert (st, it, rr) == (0, 1, 0.0)
        assert np.all(x[0] == b / 2) and np.all(x[1:] == 0)


def test_special_cases(orc):
    A = P.laplacian_2d(8)
    b = P.rhs_ones_exact(A)
    for arith in W:
        w = W[arith]
        x, it, rr, st = orc.cg(arith, A, np.zeros(A.n), x0=np.ones((w, A.n)), tol=1e-10, maxit=50,
                               precond="jacobi")
        assert (st, it, rr) == (0, 0, 0.0) and np.all(x == 0)
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-10, maxit=0, precond="jacobi")
        assert (st, it) == (1, 0) and rr == 1.0 and np.all(x == 0)
        # a diagonal entry that is zero, negative or missing: status 3, x0 untouched
        for bad in ("zero", "negative", "missing"):
            B = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
            k0 = [k for k in range(B.row_ptr[5], B.row_ptr[6]) if B.col[k] == 5][0]
            if bad == "zero":
                B.val[k0] = 0.0
            elif bad == "negative":
                B.val[k0] = -4.0
            else:
                B.col[k0] = 4 if B.col[k0 - 1] != 4 else 6      # off the diagonal
            x0 = np.full((w, A.n), 0.5)
            x, it, rr, st = orc.cg(arith, B, b, x0=x0, tol=1e-10, maxit=50, precond="jacobi")
            assert (st, it) == (3, 0) and np.all(x == x0), (arith, bad)


# ---------------------------------------------------------------------------
# QQF and QF (four FP32 words): the same recurrence with the scaled iteration
# of their CG (r~ = 2^-E r, z~ = w (x) r~, shift from the FP64 residual sum).
# ---------------------------------------------------------------------------
FP32W = ["qqf", "qf"]
LEVEL32 = {"qqf": 1e-20, "qf": 1e-27}        # QQF is quasi: its lower words drift (1.1e-21 here)


def _sum_words(x, i):
    return sum(Fraction(float(v)) for v in x[:, i])


@pytest.mark.parametrize("arith", FP32W)
@pytest.mark.parametrize("plan", [None, (1, 256, 3)])
def test_fp32_words_power_of_two_diagonal_reproduces_cg(orc, arith, plan):
    """Diagonal 4: z~ = r~/4 exactly and every scaled quantity is a power-of-two
    multiple of CG's, so x is CG's bit for bit (the shifts may differ: the
    scaling is exact)."""
    A = P.laplacian_2d(20)
    b = P.rhs_uniform(A.n, 3)
    x1, i1, _, s1 = orc.cg(arith, A, b, tol=0.0, maxit=40, plan=plan)
    x2, i2, _, s2 = orc.cg(arith, A, b, tol=0.0, maxit=40, plan=plan, precond="jacobi")
    assert (i1, s1) == (i2, s2) == (40, 1)
    assert np.array_equal(_bits(x1), _bits(x2)), (arith, plan)


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_follow_exact_pcg(orc, arith):
    A = P.random_spd_small(9, seed=3)
    b = P.rhs_uniform(A.n, 4)
    d = np.array([A.val[k] for i in range(A.n) for k in range(A.row_ptr[i], A.row_ptr[i + 1]) if A.col[k] == i])
    xs, rrs = pcg_exact(dense_fraction(A), b, 1.0 / d, 6)
    bn = math.sqrt(float(sum(Fraction(float(v)) ** 2 for v in b)))
    for k in (1, 2, 4, 6):
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-300, maxit=k, precond="jacobi")
        assert it == k and st == 1
        assert np.all(x.astype(np.float32).astype(np.float64) == x)       # FP32 words
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            assert abs(float(_sum_words(x, i) - xs[k - 1][i])) <= LEVEL32[arith] * float(scale), (arith, k, i)
        assert rr == pytest.approx(math.sqrt(float(rrs[k - 1])) / bn, rel=1e-9, abs=1e-300)


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_exact_solution_of_dyadic_diffusion(orc, arith):
    A = P.diffusion_2d(24, 11, dyadic=True)
    xs = P.random_signs(A.n, 12)
    b = P.matvec_grid_exact(A, xs)
    x, it, rr, st = orc.cg(arith, A, b, tol=1e-24, maxit=5000, plan=(1, 256, 3), precond="jacobi")
    assert st == 0
    err = math.sqrt(sum(float(_sum_words(x, i) - Fraction(float(xs[i]))) ** 2 for i in range(A.n)) / A.n)
    assert err <= 1e-21, err
    _, it_cg, _, st_cg = orc.cg(arith, A, b, tol=1e-24, maxit=5000, plan=(1, 256, 3))
    assert st_cg == 0 and it < it_cg


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_scaling_is_invisible(orc, arith):
    """b 2^k: the same iterations and residual history (E absorbs k), and x
    2^k at k = +40.  At k = -40 x's lowest words (about 1e-37 after the
    scaling) have error terms in FP32's subnormal range, so x is unscaled
    FP32 words that no longer scale exactly."""
    A = P.laplacian_2d(24, 1e-3)
    b = P.rhs_uniform(A.n, 9)
    x0, i0, r0, s0, h0 = orc.cg(arith, A, b, tol=1e-22, maxit=2000, precond="jacobi", history=True)
    assert s0 == 0
    for k in (-40, 40):
        x, it, rr, st, h = orc.cg(arith, A, b * 2.0 ** k, tol=1e-22, maxit=2000, precond="jacobi", history=True)
        assert (it, st, rr) == (i0, s0, r0) and np.array_equal(h, h0)
        if k > 0:
            assert np.array_equal(x, x0 * 2.0 ** k)


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_closed_form_and_special_cases(orc, arith):
    n = 50
    A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    b = P.rhs_uniform(n, 1)
    x, it, rr, st = orc.cg(arith, A, b, tol=1e-30, maxit=5, precond="jacobi")
    assert (st, it, rr) == (0, 1, 0.0)                      # A = 2I: x1 = b/2, r1 = 0
    assert all(_sum_words(x, i) == Fraction(float(b[i])) / 2 for i in range(n))
    A = P.laplacian_2d(8)
    b = P.rhs_ones_exact(A)
    x, it, rr, st = orc.cg(arith, A, np.zeros(A.n), x0=np.ones((4, A.n)), tol=1e-10, maxit=50, precond="jacobi")
    assert (st, it, rr) == (0, 0, 0.0) and np.all(x == 0)
    x, it, rr, st = orc.cg(arith, A, b, tol=1e-10, maxit=0, precond="jacobi")
    assert (st, it) == (1, 0) and rr == 1.0 and np.all(x == 0)
    B = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    B.val[[k for k in range(B.row_ptr[5], B.row_ptr[6]) if B.col[k] == 5][0]] = -4.0
    x0 = np.full((4, A.n), 0.5)
    x, it, rr, st = orc.cg(arith, B, b, x0=x0, tol=1e-10, maxit=50, precond="jacobi")
    assert (st, it) == (3, 0) and np.all(x == x0)
    with pytest.raises(ValueError):                          # the policy is fixed for FP32 words
        orc.cg(arith, A, b, tol=1e-10, maxit=50, precond="jacobi", norm=(2, 1))
