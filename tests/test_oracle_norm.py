"""Pins of the oracle's normalisation policy (an extension of Sec. IV-D).

Sec. IV-D normalises the quasi arithmetics' residual r once per iteration,
after its AXPY, and leaves frequency and placement open (Sec. VI).  The policy
{every, mask} normalises r, x, p, q = A p or the SpMV running sum on the
iterations it with it % every == 0.  Facts fixed independently of the policy
code:
 * every = 0 never normalises: bit-identical to the NN variants of
   Sec. V-B3, whose normalisation is the identity (word-level pins).
 * {1, R} is Sec. IV-D's placement: bit-identical to the default solver.
 * every > maxit: no iteration normalises, so the run equals the NN run.
 * Normalisation is error free (word-level pins), so policies that keep r
   normalised still reach the exact solution of an exact-right-hand-side
   system to the arithmetic's level (checked in exact rationals).
 * Normalised x is in normalised form: QuickTwoSum gives fl(x1 + x2) = x1,
   VecSum3 gives |x2| <= ulp(x1).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

R, X, PP, Q, SUM = 1, 2, 4, 8, 16
PLANS = [None, (1, 256, 2), (4, 256, 3)]


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


def _same(a, b):
    xa, ia, ra, sa, ha = a
    xb, ib, rb, sb, hb = b
    return (np.array_equal(_bits(xa), _bits(xb)) and ia == ib and sa == sb
            and (ra == rb or (math.isnan(ra) and math.isnan(rb)))
            and np.array_equal(_bits(ha), _bits(hb)))


def _system():
    A = P.laplacian_2d(12)
    return A, P.rhs_uniform(A.n, 11)


@pytest.mark.parametrize("arith", ["qdw", "qtw"])
@pytest.mark.parametrize("plan", PLANS)
def test_every_zero_is_the_nn_variant(orc, arith, plan):
    A, b = _system()
    nn = orc.cg(arith + "_nn", A, b, tol=1e-35, maxit=60, plan=plan, history=True)
    for mask in (R, R | X | PP | Q | SUM, Q, SUM):
        got = orc.cg(arith, A, b, tol=1e-35, maxit=60, plan=plan, history=True, norm=(0, mask))
        assert _same(got, nn), (arith, mask)


@pytest.mark.parametrize("arith", ["qdw", "qtw", "dw", "tw", "fp64"])
@pytest.mark.parametrize("plan", PLANS)
def test_every_iteration_on_r_is_the_default(orc, arith, plan):
    A, b = _system()
    ref = orc.cg(arith, A, b, tol=1e-35, maxit=60, plan=plan, history=True)
    got = orc.cg(arith, A, b, tol=1e-35, maxit=60, plan=plan, history=True, norm=(1, R))
    assert _same(got, ref)


@pytest.mark.parametrize("arith", ["dw", "tw", "fp64"])
def test_non_quasi_arithmetics_ignore_the_policy(orc, arith):
    """DW/TW results are normalised by every operation (Sec. III); FP64 has one word."""
    A, b = _system()
    ref = orc.cg(arith, A, b, tol=1e-35, maxit=40, plan=(1, 256, 2), history=True)
    for norm in ((0, R), (3, R | X | PP | Q | SUM)):
        got = orc.cg(arith, A, b, tol=1e-35, maxit=40, plan=(1, 256, 2), history=True, norm=norm)
        assert _same(got, ref)


@pytest.mark.parametrize("arith", ["qdw", "qtw"])
def test_every_beyond_maxit_never_normalises(orc, arith):
    A, b = _system()
    nn = orc.cg(arith + "_nn", A, b, tol=1e-35, maxit=15, plan=(1, 256, 2), history=True)
    got = orc.cg(arith, A, b, tol=1e-35, maxit=15, plan=(1, 256, 2), history=True,
                 norm=(16, R | X | PP | Q | SUM))
    assert _same(got, nn)


@pytest.mark.parametrize("arith", ["qdw", "qtw"])
def test_each_placement_changes_the_iterates(orc, arith):
    """A placement that is silently skipped would leave the NN bits unchanged."""
    A, b = _system()
    nn = orc.cg(arith + "_nn", A, b, tol=1e-35, maxit=30, plan=(2, 256, 2), history=True)
    for mask in (R, X, PP, Q, SUM):
        got = orc.cg(arith, A, b, tol=1e-35, maxit=30, plan=(2, 256, 2), history=True, norm=(1, mask))
        assert not np.array_equal(_bits(got[0]), _bits(nn[0])) or not np.array_equal(
            _bits(got[4]), _bits(nn[4])), (arith, mask)


@pytest.mark.parametrize("arith,tol,bound", [("qdw", 1e-28, 1e-26), ("qtw", 1e-40, 1e-38)])
@pytest.mark.parametrize("norm", [(1, R), (1, R | X | PP | Q | SUM), (1, R | Q), (1, R | SUM), (1, R | X),
                                  (2, R | X | PP | Q | SUM)])
def test_policies_that_normalise_r_reach_the_exact_solution(orc, arith, tol, bound, norm):
    """16x16 5-point Laplacian, x* = +-1, b = A x* (integers, exact): the exact
    solution is x*, and the error is measured in exact rationals.  (Leaving r
    unnormalised on some iterations, e.g. {2, R}, breaks down before these
    tolerances: a cancelling r update leaves its value in the lower words,
    which the next quasi product partly drops.)"""
    A = P.laplacian_2d(16)
    xs = P.random_signs(A.n, 5)
    b = P.matvec_exact(A, xs)
    x, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=2000, plan=(2, 256, 3), norm=norm)
    assert st == 0, (it, rr)
    err2 = sum((sum(Fraction(float(w)) for w in x[:, i]) - Fraction(float(xs[i]))) ** 2 for i in range(A.n))
    assert math.sqrt(float(err2) / A.n) <= bound


def test_normalised_x_is_in_normalised_form(orc):
    A, b = _system()
    x, it, rr, st = orc.cg("qdw", A, b, tol=1e-28, maxit=500, plan=(1, 256, 2), norm=(1, R | X))
    assert st == 0
    assert np.all(x[0] + x[1] == x[0])                      # QuickTwoSum postcondition
    x, it, rr, st = orc.cg("qtw", A, b, tol=1e-40, maxit=500, plan=(1, 256, 2), norm=(1, R | X))
    assert st == 0
    ulp = np.vectorize(math.ulp)
    assert np.all(np.abs(x[1]) <= ulp(x[0]))                # VecSum3 leading pair
