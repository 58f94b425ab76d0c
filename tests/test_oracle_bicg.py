"""Pins of the oracle's BiCGStab (an extension for nonsymmetric systems; Sec.
VI names other iterative methods as future work).

Independent references: textbook BiCGStab in exact rationals, exact-solution
systems (b = A x* with dyadic nonsymmetric A), and closed forms -- A = +-2I
(one step, the early exit on ||s||), a rotation (rh^T v = 0: breakdown).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from mwref import bicgstab_exact, col, dense_fraction, val
from paper_2510_13536_gb300 import problems as P

ALL = ["fp64", "dw", "qdw", "tw", "qtw", "qw", "qqw"]
W = {"fp64": 1, "dw": 2, "qdw": 2, "tw": 3, "qtw": 3, "qw": 4, "qqw": 4}
LEVEL = {"fp64": 1e-10, "dw": 1e-25, "qdw": 1e-24, "tw": 1e-38, "qtw": 1e-37, "qw": 1e-52, "qqw": 1e-51}


def _nonsym_small(n, seed):
    """Diagonally dominant nonsymmetric matrix with dyadic entries."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        off = 0.0
        for j in range(n):
            if j != i and (abs(i - j) == 1 or rng.random() < 0.3):
                w = float(rng.integers(-8, 9)) / 4.0
                if w != 0.0:
                    rows.append(i), cols.append(j), vals.append(w)
                    off += abs(w)
        rows.append(i), cols.append(i), vals.append(off + float(rng.integers(1, 5)) / 2.0)
    return P._from_coo(n, np.array(rows), np.array(cols), np.array(vals), f"nonsym_{n}")


@pytest.mark.parametrize("arith", ALL)
def test_iterates_follow_exact_bicgstab(orc, arith):
    A = _nonsym_small(9, 3)
    b = P.rhs_uniform(A.n, 4)
    xs = bicgstab_exact(dense_fraction(A), b, 4)
    for k in range(1, len(xs) + 1):
        x, it, rr, st = orc.bicgstab(arith, A, b, tol=1e-300, maxit=k)
        assert it == k and st == 1, (arith, k, it, st)
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            assert abs(float(val(col(x, i)) - xs[k - 1][i])) <= LEVEL[arith] * float(scale), (arith, k, i)


@pytest.mark.parametrize("arith,tol,bound", [("fp64", 1e-14, 1e-11), ("dw", 1e-28, 1e-25), ("qtw", 1e-40, 1e-37),
                                             ("qqw", 1e-55, 1e-52)])
def test_exact_solution_of_convection_diffusion(orc, arith, tol, bound):
    A = P.convection_diffusion_2d(24, 2.0)
    xs = P.random_signs(A.n, 5)
    b = P.matvec_exact(A, xs)
    x, it, rr, st = orc.bicgstab(arith, A, b, tol=tol, maxit=3000, plan=(1, 256, 3))
    assert st == 0, (it, rr)
    err = math.sqrt(sum(float(val(col(x, i)) - Fraction(float(xs[i]))) ** 2 for i in range(A.n)) / A.n)
    assert err <= bound, err


def test_closed_forms(orc):
    n = 40
    b = P.rhs_uniform(n, 1)
    for d in (2.0, -2.0):
        A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, d))
        for arith in ALL:
            # r0 = b, v = d b, alpha = 1/d, s = 0: the early exit, x = b/d exactly.
            x, it, rr, st = orc.bicgstab(arith, A, b, tol=1e-30, maxit=5)
            assert (st, it, rr) == (0, 1, 0.0), (arith, d)
            assert np.all(x[0] == b / d) and np.all(x[1:] == 0)
    # Rotation [[0, 1], [-1, 0]], b = (1, 0): v = A r0 = (0, -1), rh^T v = 0.
    R = P.CSR(2, np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32), np.array([1.0, -1.0]))
    for arith in ALL:
        x, it, rr, st = orc.bicgstab(arith, R, np.array([1.0, 0.0]), tol=1e-30, maxit=5)
        assert (st, it) == (2, 1), arith


def test_special_cases(orc):
    A = P.convection_diffusion_2d(8, 1.0)
    xs = np.ones(A.n)
    b = P.matvec_exact(A, xs)
    for arith in ALL:
        w = W[arith]
        x, it, rr, st = orc.bicgstab(arith, A, np.zeros(A.n), x0=np.ones((w, A.n)), tol=1e-10, maxit=50)
        assert (st, it, rr) == (0, 0, 0.0) and np.all(x == 0)
        x0 = np.zeros((w, A.n))
        x0[0] = 1.0
        x, it, rr, st = orc.bicgstab(arith, A, b, x0=x0, tol=1e-10, maxit=50)
        assert (st, it) == (0, 0) and np.all(x == x0)
        x, it, rr, st = orc.bicgstab(arith, A, b, tol=1e-10, maxit=0)
        assert (st, it) == (1, 0) and rr == 1.0 and np.all(x == 0)


def test_nonsymmetric_system_needs_bicgstab(orc):
    """CG is not defined for nonsymmetric A; on the convection-dominated system
    it fails to converge where BiCGStab converges."""
    A = P.convection_diffusion_2d(32, 8.0)
    b = P.rhs_uniform(A.n, 6)
    _, it_b, rr_b, st_b = orc.bicgstab("qtw", A, b, tol=1e-30, maxit=2000)
    _, it_c, rr_c, st_c = orc.cg("qtw", A, b, tol=1e-30, maxit=2000)
    assert st_b == 0 and st_c != 0, (it_b, rr_b, it_c, rr_c, st_c)


# ---------------------------------------------------------------------------
# QQF and QF (four FP32 words): the same recurrence with the scaled iteration
# of their CG (r, p, v, s, t at 2^E, the shadow residual at 2^E0).
# ---------------------------------------------------------------------------
FP32W = ["qqf", "qf"]
LEVEL32 = {"qqf": 1e-25, "qf": 1e-28}        # QQF is quasi: its lower words drift


def _sum_words(x, i):
    return sum(Fraction(float(v)) for v in x[:, i])


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_follow_exact_bicgstab(orc, arith):
    A = _nonsym_small(9, 3)
    b = P.rhs_uniform(A.n, 4)
    xs = bicgstab_exact(dense_fraction(A), b, 4)
    for k in range(1, len(xs) + 1):
        x, it, rr, st = orc.bicgstab(arith, A, b, tol=1e-300, maxit=k)
        assert it == k and st == 1, (arith, k, it, st)
        assert np.all(x.astype(np.float32).astype(np.float64) == x)       # FP32 words
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            assert abs(float(_sum_words(x, i) - xs[k - 1][i])) <= LEVEL32[arith] * float(scale), (arith, k, i)


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_exact_solution_of_convection_diffusion(orc, arith):
    A = P.convection_diffusion_2d(24, 2.0)
    xs = P.random_signs(A.n, 5)
    b = P.matvec_exact(A, xs)
    x, it, rr, st = orc.bicgstab(arith, A, b, tol=1e-24, maxit=3000, plan=(1, 256, 3))
    assert st == 0, (it, rr)
    err = math.sqrt(sum(float(_sum_words(x, i) - Fraction(float(xs[i]))) ** 2 for i in range(A.n)) / A.n)
    assert err <= 1e-22, err


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_scaling_is_invisible(orc, arith):
    """b 2^k: the same iterations and residual history (E absorbs k), x 2^k at
    k = +40 (at k = -40 x's lowest words reach FP32's subnormal range), and at
    k = +300 the first x update overflows FP32: status 4."""
    A = P.convection_diffusion_2d(16, 1.0)
    b = P.rhs_uniform(A.n, 6)
    x0, i0, r0, s0, h0 = orc.bicgstab(arith, A, b, tol=1e-22, maxit=2000, history=True)
    assert s0 == 0
    for k in (-40, 40):
        x, it, rr, st, h = orc.bicgstab(arith, A, b * 2.0 ** k, tol=1e-22, maxit=2000, history=True)
        assert (it, st, rr) == (i0, s0, r0) and np.array_equal(h, h0), k
        if k > 0:
            assert np.array_equal(x, x0 * 2.0 ** k)
    x, it, rr, st = orc.bicgstab(arith, A, b * 2.0 ** 300, tol=1e-22, maxit=2000)
    assert (st, it) == (4, 1)


@pytest.mark.parametrize("arith", FP32W)
def test_fp32_words_closed_forms_and_special_cases(orc, arith):
    n = 40
    b = P.rhs_uniform(n, 1)
    for d in (2.0, -2.0):
        A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, d))
        x, it, rr, st = orc.bicgstab(arith, A, b, tol=1e-30, maxit=5)
        assert (st, it, rr) == (0, 1, 0.0), d                     # the early exit, x = b / d exactly
        assert all(_sum_words(x, i) == Fraction(float(b[i])) / Fraction(d) for i in range(n))
    R = P.CSR(2, np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32), np.array([1.0, -1.0]))
    x, it, rr, st = orc.bicgstab(arith, R, np.array([1.0, 0.0]), tol=1e-30, maxit=5)
    assert (st, it) == (2, 1)                                      # rotation: rh^T v = 0
    A = P.convection_diffusion_2d(8, 1.0)
    x, it, rr, st = orc.bicgstab(arith, A, np.zeros(A.n), x0=np.ones((4, A.n)), tol=1e-10, maxit=50)
    assert (st, it, rr) == (0, 0, 0.0) and np.all(x == 0)
    x, it, rr, st = orc.bicgstab(arith, A, P.matvec_exact(A, np.ones(A.n)), tol=1e-10, maxit=0)
    assert (st, it) == (1, 0) and rr == 1.0 and np.all(x == 0)
    # Same iterations as DW on the convection-dominated system.
    A = P.convection_diffusion_2d(32, 8.0)
    b = P.rhs_uniform(A.n, 6)
    _, it_f, _, st_f = orc.bicgstab(arith, A, b, tol=1e-14, maxit=3000, plan=(1, 256, 7))
    _, it_d, _, st_d = orc.bicgstab("dw", A, b, tol=1e-14, maxit=3000, plan=(1, 256, 7))
    assert st_f == st_d == 0 and it_f == it_d
