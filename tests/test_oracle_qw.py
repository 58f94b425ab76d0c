"""Pins of the oracle's four-word arithmetics QW and QQW (an extension; Sec. I lists both).

The paper lists QW (Hida et al.) and QQW (Ozaki and Imamura) among the
multi-word arithmetics (Sec. I) but evaluates neither and prints no
algorithm.  The oracle's readings: QQW continues QTW's Algorithms 7-10 one
level down (VecSum4 as its normalisation); QW is QQW followed by the
error-free VecSum and a renormalisation to four non-overlapping words.  What
fixes them independently of that code:
 * exact rational arithmetic: the error envelopes of add / mul / FP64 x MW /
   division at the quad-word level (~2^-212, Sec. I);
 * with zero lower words, add / mul / dxmul return the exact TwoSum / TwoProd;
 * normalisation (VecSum4) and QW's renormalisation are error free;
 * QW words do not overlap (|c_{k+1}| <= ulp(c_k));
 * CG in QQW / QW follows exact CG, reaches an exact solution at the quad-word
   level, and QQW without normalisation fails where QQW converges (Sec. V-B3).
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from mwref import cg_exact, col, dense_fraction, fnorm, rand_mw, solve_exact, val
from paper_2510_13536_gb300 import problems as P

N = 1500
U = Fraction(1, 2 ** 53)
ENV4 = Fraction(1, 2 ** 205)          # relative, for normalised operands


def rel_err(got, exact):
    return abs(got - exact) / abs(exact) if exact != 0 else abs(got)


@pytest.mark.parametrize("arith", ["qqw", "qw"])
def test_mul_and_dxmul_error_envelope(orc, arith):
    rng = random.Random(41)
    a, b = rand_mw(rng, N, 4), rand_mw(rng, N, 4)
    c = orc.mul(arith, a, b)
    s = np.array([float(rand_mw(rng, 1, 1)[0, 0]) for _ in range(N)])
    d = orc.dxmul(arith, s, b)
    for i in range(N):
        assert rel_err(val(col(c, i)), val(col(a, i)) * val(col(b, i))) <= ENV4, (arith, i)
        assert rel_err(val(col(d, i)), Fraction(s[i]) * val(col(b, i))) <= ENV4, (arith, i)


@pytest.mark.parametrize("arith", ["qqw", "qw"])
def test_add_error_envelope(orc, arith):
    """Absolute bound relative to |a| + |b| for any signs (cancellation)."""
    rng = random.Random(42)
    a, b = rand_mw(rng, N, 4), rand_mw(rng, N, 4)
    c = orc.add(arith, a, b)
    for i in range(N):
        va, vb = val(col(a, i)), val(col(b, i))
        assert abs(val(col(c, i)) - (va + vb)) <= ENV4 * (abs(va) + abs(vb))


@pytest.mark.parametrize("arith", ["qqw", "qw"])
def test_division_accuracy(orc, arith):
    rng = random.Random(43)
    a, b = rand_mw(rng, N, 4), rand_mw(rng, N, 4)
    c = orc.div(arith, a, b)
    for i in range(N):
        assert rel_err(val(col(c, i)), val(col(a, i)) / val(col(b, i))) <= Fraction(1, 2 ** 200)


def test_precision_is_quad_word(orc):
    """Sec. I: four words of 53 bits give about 212 bits: the worst product
    error over random operands lies between 2^-216 and 2^-205."""
    rng = random.Random(44)
    a, b = rand_mw(rng, 800, 4), rand_mw(rng, 800, 4)
    for arith in ("qqw", "qw"):
        c = orc.mul(arith, a, b)
        worst = max(rel_err(val(col(c, i)), val(col(a, i)) * val(col(b, i))) for i in range(800))
        assert Fraction(1, 2 ** 216) <= worst <= Fraction(1, 2 ** 205), (arith, float(worst))


def test_zero_lower_words_reduce_to_error_free_transforms(orc):
    rng = random.Random(45)
    a1 = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-40, 40) for _ in range(N)])
    b1 = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-40, 40) for _ in range(N)])
    z = np.zeros(N)
    A = np.vstack([a1, z, z, z])
    B = np.vstack([b1, z, z, z])
    for arith in ("qqw", "qw", "qqw_nn"):
        s, p, d = orc.add(arith, A, B), orc.mul(arith, A, B), orc.dxmul(arith, a1, B)
        for i in range(0, N, 7):
            assert val(col(s, i)) == Fraction(a1[i]) + Fraction(b1[i])
            assert val(col(p, i)) == Fraction(a1[i]) * Fraction(b1[i])
            assert val(col(d, i)) == Fraction(a1[i]) * Fraction(b1[i])
            assert s[0, i] == a1[i] + b1[i] and p[0, i] == a1[i] * b1[i]


def test_normalisation_is_error_free_and_qw_does_not_overlap(orc):
    rng = random.Random(46)
    a = rand_mw(rng, 600, 4)
    a[1] *= np.array([rng.uniform(0.5, 3e15) for _ in range(600)])     # overlapping words
    c = orc.normalize("qqw", a)
    for i in range(600):
        assert val(col(c, i)) == val(col(a, i))
        assert c[0, i] == a[0, i] + a[1, i]            # VecSum4's leading word
    assert np.all(orc.normalize("qqw_nn", a) == a)
    ulp = np.vectorize(math.ulp)
    x, y = rand_mw(rng, N, 4), rand_mw(rng, N, 4)
    for c in (orc.add("qw", x, y), orc.mul("qw", x, y), orc.dxmul("qw", x[0], y), orc.div("qw", x, y)):
        for k in range(3):
            assert np.all(np.abs(c[k + 1]) <= ulp(c[k])), k


def test_exact_cancellation_and_collapse(orc):
    rng = random.Random(47)
    a = rand_mw(rng, 300, 4)
    for arith in ("qqw", "qw"):
        assert np.all(orc.add(arith, a, -a) == 0.0)
    # collapse lowest first: fl(c1 + fl(c2 + fl(c3 + c4))).  Worked by hand with
    # c = (1, 2^-53, 2^-106, 2^-106): c3 + c4 = 2^-105 exactly, c2 + 2^-105 is
    # representable, and 1 + (2^-53 + 2^-105) lies above the tie: 1 + 2^-52.
    # Any other association meets a tie first and rounds to even, giving 1.
    t = np.array([[1.0], [2.0 ** -53], [2.0 ** -106], [2.0 ** -106]])
    for arith in ("qqw", "qw"):
        assert orc.collapse(arith, t)[0] == 1.0 + 2.0 ** -52


@pytest.mark.parametrize("arith", ["qqw", "qw"])
def test_cg_iterates_follow_exact_cg(orc, arith):
    A = P.random_spd_small(9, seed=3)
    b = P.rhs_uniform(A.n, 4)
    xs, _ = cg_exact(dense_fraction(A), b, 6)
    for k in (1, 3, 6):
        x, it, rr, st = orc.cg(arith, A, b, tol=1e-300, maxit=k)
        assert it == k and st == 1
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            assert abs(float(val(col(x, i)) - xs[k - 1][i])) <= 1e-54 * float(scale), (arith, k, i)


@pytest.mark.parametrize("arith", ["qqw", "qw"])
def test_forward_error_against_exact_solve(orc, arith):
    A = P.random_spd_small(24, seed=7, shift_exp=-4)
    b = P.rhs_uniform(A.n, 8)
    xe = solve_exact(dense_fraction(A), b)
    x, it, rr, st = orc.cg(arith, A, b, tol=1e-58, maxit=3000)
    assert st == 0
    err = math.sqrt(sum(float(val(col(x, i)) - xe[i]) ** 2 for i in range(A.n))) / fnorm(xe)
    assert err <= 1e-55, err


def test_unnormalised_qqw_does_not_converge(orc):
    A = P.laplacian_2d(32, 1e-6)
    b = P.rhs_uniform(A.n, 3)
    _, it, rr, st = orc.cg("qqw", A, b, tol=1e-55, maxit=3000)
    assert st == 0
    _, it2, rr2, st2 = orc.cg("qqw_nn", A, b, tol=1e-55, maxit=3000)
    assert st2 != 0, (it2, rr2)
