"""Pins of the oracle's CG (Algorithm 1, Sec. IV-C, IV-D) against exact arithmetic.

Independent references: textbook CG run in exact rationals, an exact rational
direct solve, the finite-termination property of CG, exact-solution systems
(b = A·1, Sec. V-A) and special cases whose answer is fixed by the algorithm.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from mwref import cg_exact, col, dense_fraction, fnorm, solve_exact, val
from paper_2510_13536_gb300 import problems as P

ALL = ["fp64", "dw", "qdw", "tw", "qtw"]
W = {"fp64": 1, "dw": 2, "qdw": 2, "tw": 3, "qtw": 3, "qdw_nn": 2, "qtw_nn": 3}
# Agreement level with exact CG iterates after a few steps, per arithmetic.
LEVEL = {"fp64": 1e-11, "dw": 1e-26, "qdw": 1e-25, "tw": 1e-40, "qtw": 1e-39}


def _xval(x, i):
    return val(col(x, i))


@pytest.mark.parametrize("arith", ALL)
def test_iterates_follow_exact_cg(orc, arith):
    """After k passes the oracle's x_k equals textbook CG's x_k (exact rationals)
    up to the arithmetic's rounding level; its relres is ||r_k|| / ||b||."""
    A = P.random_spd_small(9, seed=3)
    b = P.rhs_uniform(A.n, 4)
    M = dense_fraction(A)
    xs, rhos = cg_exact(M, b, 6)
    bn = fnorm([Fraction(float(v)) for v in b])
    for k in (1, 2, 4, 6):
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-300, maxit=k)
        assert it == k and st == 1
        xe = xs[k - 1]
        scale = max(abs(v) for v in xe)
        err = max(abs(_xval(x, i) - xe[i]) for i in range(A.n)) / scale
        assert float(err) <= LEVEL[arith], (k, float(err))
        rel_exact = math.sqrt(float(rhos[k - 1])) / bn
        assert abs(rr - rel_exact) <= 1e-9 * rel_exact


@pytest.mark.parametrize("arith", ["tw", "qtw", "dw", "qdw"])
def test_finite_termination(orc, arith):
    """In exact arithmetic CG ends in at most n steps; in 106/159-bit arithmetic a
    well-conditioned n = 16 system reaches the arithmetic's floor in n + 2 steps."""
    A = P.random_spd_small(16, seed=5, shift_exp=0)
    b = P.rhs_uniform(A.n, 6)
    tol = 1e-38 if W[arith] == 3 else 1e-24
    x, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=200)
    assert st == 0 and it <= A.n + 2, (it, rr)


@pytest.mark.parametrize("arith", ALL)
def test_forward_error_against_exact_solve(orc, arith):
    A = P.random_spd_small(24, seed=7, shift_exp=-4)
    b = P.rhs_uniform(A.n, 8)
    xe = solve_exact(dense_fraction(A), b)
    tol = {"fp64": 1e-14, "dw": 1e-28, "qdw": 1e-28, "tw": 1e-42, "qtw": 1e-42}[arith]
    x, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=2000)
    assert st == 0
    num = math.sqrt(sum(float(_xval(x, i) - xe[i]) ** 2 for i in range(A.n)))
    err = num / fnorm(xe)
    bound = {"fp64": 1e-10, "dw": 1e-24, "qdw": 1e-24, "tw": 1e-38, "qtw": 1e-38}[arith]
    assert err <= bound, err


@pytest.mark.parametrize("arith", ["fp64", "dw"])
def test_exact_solution_twin_2d_poisson(orc, arith):
    """64x64 5-point Laplacian with b = A·1 (exact): x* = 1 (Sec. V-A method)."""
    A = P.laplacian_2d(64)
    b = P.rhs_ones_exact(A)
    x, it, rr, st = orc.cg(arith, A, b, tol=1e-12, maxit=2000)
    assert st == 0 and rr < 1e-12
    xc = orc.collapse(arith, x) if W[arith] > 1 else x[0]
    assert np.max(np.abs(xc - 1.0)) < 1e-9


def test_special_cases(orc):
    A = P.laplacian_2d(8)
    b = P.rhs_ones_exact(A)
    for arith in ALL:
        w = W[arith]
        # b = 0: x = 0, no iterations.
        x, it, rr, st = orc.cg(arith, A, np.zeros(A.n), x0=np.ones((w, A.n)), tol=1e-10, maxit=50)
        assert st == 0 and it == 0 and rr == 0.0 and np.all(x == 0)
        # x0 already exact: r0 = 0, no iterations, x0 returned.
        x0 = np.zeros((w, A.n))
        x0[0] = 1.0
        x, it, rr, st = orc.cg(arith, A, b, x0=x0, tol=1e-10, maxit=50)
        assert st == 0 and it == 0 and np.all(x == x0)
        # maxit = 0: status 1, x0 untouched.
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-10, maxit=0)
        assert st == 1 and it == 0 and np.all(x == 0) and rr == 1.0
        # Negative definite: p^T q < 0 on the first pass -> breakdown.
        x, it, rr, st = orc.cg(arith, A.with_values(-A.val), b, tol=1e-10, maxit=50)
        assert st == 2 and it == 1
        # NaN in b -> breakdown on the first pass.
        bb = b.copy()
        bb[3] = np.nan
        x, it, rr, st = orc.cg(arith, A, bb, tol=1e-10, maxit=50)
        assert st == 2 and it == 1


def test_relres_is_fp64_collapse_over_bnorm(orc):
    """Sec. IV-C: the stopping residual is FP64: sqrt(collapse(rho))/||b||.  With
    maxit = 1 from x0 = 0 on a diagonal system the first residual is known in
    closed form: A = 2I gives alpha = 1/2, x1 = b/2, r1 = 0."""
    n = 50
    A = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    b = P.rhs_uniform(n, 1)
    for arith in ALL:
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-30, maxit=5)
        assert st == 0 and it == 1 and rr == 0.0
        assert np.all(x[0] == b / 2)


def test_unnormalised_quasi_does_not_converge(orc):
    """Sec. V-B3: without the per-iteration normalisation of r, quasi CG fails to
    converge, while the normalised variants converge."""
    A = P.laplacian_2d(32, 1e-6)
    b = P.rhs_uniform(A.n, 3)
    for arith, nn, tol in (("qdw", "qdw_nn", 1e-28), ("qtw", "qtw_nn", 1e-40)):
        _, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=3000)
        assert st == 0, arith
        _, it2, rr2, st2 = orc.cg(nn, A, b, tol=tol, maxit=3000)
        assert st2 != 0, (nn, it2, rr2)


def test_mirrored_order_visits_every_leaf_once(orc):
    """The mirrored (tile / block / tree) reduction must add each row exactly once:
    with integer data every order gives the exact sum n(n+1)/2."""
    for n in (1, 5, 255, 256, 257, 1000, 4099):
        u = np.ones(n)
        v = np.arange(1, n + 1, dtype=np.float64)
        for (R, G) in ((0, 1), (32, 1), (64, 3), (256, 7), (128, 1000)):
            assert orc.dot("fp64", u, v, R, G)[0] == n * (n + 1) / 2
            d = orc.dot("qtw", np.vstack([u, 0 * u, 0 * u]), np.vstack([v, 0 * v, 0 * v]), R, G)
            assert val(d) == Fraction(n * (n + 1), 2)


def test_lane_split_spmv_exact_on_integer_data(orc):
    """Any lane split V of a row sums every entry once: on integer data every V
    matches the plain row sum."""
    A = P.power_law_laplacian(2000, seed=3, mean_deg=12, max_deg=200, dyadic=True)
    A = A.with_values(np.round(A.val * 4.0))           # small integers, exact sums
    p = np.vstack([np.arange(A.n, dtype=np.float64) % 7 - 3, np.zeros(A.n), np.zeros(A.n)])
    ref = orc.spmv("qtw", A, p, 0)
    for V in (1, 2, 4, 8, 16, 32):
        q = orc.spmv("qtw", A, p, V)
        assert np.all(orc.collapse("qtw", q) == orc.collapse("qtw", ref)), V


def test_mirrored_and_plain_agree_to_rounding(orc):
    A = P.laplacian_3d(12)
    b = P.rhs_uniform(A.n, 2)
    for arith, tol in (("dw", 1e-26), ("qtw", 1e-36)):
        x1, it1, r1, s1 = orc.cg(arith, A, b, tol=tol, maxit=1000)
        x2, it2, r2, s2 = orc.cg(arith, A, b, tol=tol, maxit=1000, plan=(2, 256, 5))
        assert s1 == s2 == 0 and abs(it1 - it2) <= 2
        d = np.max(np.abs(orc.collapse(arith, x1) - orc.collapse(arith, x2)))
        assert d < 1e-20


def test_adjoint_gradient_against_exact(orc):
    """dL/dval_k = -lambda_i x_j and dL/db = lambda with lambda = A^-1 w (exact
    rational reference, every stored entry treated as independent)."""
    A = P.random_spd_small(14, seed=11, shift_exp=-2)
    b = P.rhs_uniform(A.n, 12)
    wv = P.rhs_normal(A.n, 13)
    M = dense_fraction(A)
    xe = solve_exact(M, b)
    le = solve_exact(M, wv)                     # A symmetric: A^T lambda = w
    for arith, tol, lvl in (("fp64", 1e-15, 1e-9), ("dw", 1e-30, 1e-24), ("qtw", 1e-42, 1e-36)):
        x, it, rr, st = orc.cg(arith, A, b, tol=tol, maxit=500)
        g_b, g_val, lam, it2, rr2, st2 = orc.adjoint(arith, A, x, wv, tol, 500)
        assert st == 0 and st2 == 0
        for i in range(A.n):
            assert abs(g_b[i] - float(le[i])) <= lvl * max(1.0, abs(float(le[i])))
        for i in range(A.n):
            for k in range(int(A.row_ptr[i]), int(A.row_ptr[i + 1])):
                ge = -float(le[i] * xe[int(A.col[k])])
                assert abs(g_val[k] - ge) <= lvl * max(1.0, abs(ge))


def test_adjoint_matches_tw_finite_differences(orc):
    """Central differences of L = w^T x taken with TW solves, perturbing a
    symmetric pair (a_ij, a_ji) together so A stays SPD: dL = g_ij + g_ji."""
    A = P.diffusion_2d(6, seed=21)
    b = P.rhs_normal(A.n, 22)
    wv = P.rhs_normal(A.n, 23)
    x, *_ = orc.cg("qtw", A, b, tol=1e-40, maxit=500)
    _, g_val, *_ = orc.adjoint("qtw", A, x, wv, 1e-40, 500)
    rng = random.Random(5)
    rp, cl = A.row_ptr, A.col
    for _ in range(6):
        i = rng.randrange(A.n)
        k = rng.randrange(int(rp[i]), int(rp[i + 1]))
        j = int(cl[k])
        kt = [kk for kk in range(int(rp[j]), int(rp[j + 1])) if int(cl[kk]) == i][0]
        h = 1e-12 * abs(A.val[k])
        Ls = []
        for sgn in (1, -1):
            v = A.val.copy()
            v[k] += sgn * h
            if kt != k:
                v[kt] += sgn * h
            xs, *_ = orc.cg("tw", A.with_values(v), b, tol=1e-44, maxit=800)
            xsv = [val(col(xs, t)) for t in range(A.n)]
            Ls.append(sum(Fraction(float(wv[t])) * xsv[t] for t in range(A.n)))
        hh = Fraction(float(A.val[k] + h)) - Fraction(float(A.val[k]))   # the step actually taken
        fd = float((Ls[0] - Ls[1]) / (2 * hh))
        an = g_val[k] + (g_val[kt] if kt != k else 0.0)
        assert abs(fd - an) <= 1e-8 * abs(an), (i, j, fd, an)
