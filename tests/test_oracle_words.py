"""Pins of the oracle's word algorithms (Sec. III) against exact arithmetic.

Every check here compares the oracle with something independent of it: exact
rationals (``fractions.Fraction``), the IEEE operations of the Python host, the
operation counts printed in the paper (tests/golden/op_counts.json), published
error-bound envelopes, or algebraic identities.
"""
import json
import math
import os
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

from mwref import U, col, rand_mw, rel_err, split, val

GOLD = os.path.join(os.path.dirname(__file__), "golden")
N = 1500


def _adversarial_pairs(rng, n):
    """Doubles with huge exponent gaps, cancellation, signed zeros and subnormals."""
    a, b = [], []
    specials = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1.0, -1.0,
                2.0 ** 1000, -(2.0 ** 1000), 1.0 + 2.0 ** -52, 2.0 ** -1074 * 3]
    for _ in range(n):
        kind = rng.randrange(6)
        x = rng.uniform(1, 2) * 2.0 ** rng.randint(-60, 60) * rng.choice((1, -1))
        if kind == 0:
            y = rng.uniform(1, 2) * 2.0 ** rng.randint(-60, 60) * rng.choice((1, -1))
        elif kind == 1:       # near cancellation
            y = -x * (1 + rng.choice((1, -1)) * rng.random() * 2.0 ** -rng.randint(1, 52))
        elif kind == 2:       # gap around the rounding point
            y = x * 2.0 ** -rng.randint(50, 56) * rng.uniform(-1, 1)
        elif kind == 3:
            y = rng.choice(specials)
        elif kind == 4:       # subnormal range
            x = rng.uniform(-1, 1) * 2.0 ** -1060
            y = rng.uniform(-1, 1) * 2.0 ** -1070
        else:
            x = rng.choice(specials)
            y = rng.choice(specials)
        a.append(x)
        b.append(y)
    return np.array(a), np.array(b)


def test_two_sum_is_error_free(orc):
    rng = random.Random(1)
    a, b = _adversarial_pairs(rng, 4000)
    x, y = orc.two_sum(a, b)
    for i in range(a.size):
        assert x[i] == a[i] + b[i]                      # x = fl(a+b), host IEEE RNE
        assert Fraction(x[i]) + Fraction(y[i]) == Fraction(a[i]) + Fraction(b[i])


def test_quick_two_sum_error_free_when_ordered(orc):
    rng = random.Random(2)
    a, b = _adversarial_pairs(rng, 4000)
    swap = np.abs(a) < np.abs(b)
    a2, b2 = np.where(swap, b, a), np.where(swap, a, b)
    x, y = orc.quick_two_sum(a2, b2)
    for i in range(a.size):
        assert x[i] == a2[i] + b2[i]
        assert Fraction(x[i]) + Fraction(y[i]) == Fraction(a2[i]) + Fraction(b2[i])


def test_two_prod_is_error_free(orc):
    rng = random.Random(3)
    a = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-400, 400) for _ in range(4000)])
    b = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-400, 400) for _ in range(4000)])
    x, y = orc.two_prod(a, b)
    for i in range(a.size):
        assert x[i] == a[i] * b[i]
        assert Fraction(x[i]) + Fraction(y[i]) == Fraction(a[i]) * Fraction(b[i])


def _count(orc, fn, n=64):
    orc.ops_reset()
    fn(n)
    c = orc.ops_get()
    assert c % n == 0
    return c // n


def test_tw_operation_counts_reported(orc):
    """TW is this project's restatement of a scheme the paper cites without
    printing it (Sec. III, TW paragraph: 42 + alpha operations for the
    addition, 38 + alpha for the multiplication).  The restatement's counts
    are pinned here and compared with the paper's, not made equal to them:
    the addition is a VecSum over the six merged words (5 TwoSums, 30
    operations) plus a renormalisation of 3 to 5 QuickTwoSums (9 to 15: the
    branch-dependent part); the multiplication is 36 operations plus a
    two-QuickTwoSum renormalisation, 42 on every input.  Relative to the
    paper's fixed parts that is 12 fewer for the addition and 2 fewer for
    the multiplication, with a larger renormalisation (42 - 38 = 4 more in
    total for the multiplication)."""
    g = json.load(open(os.path.join(GOLD, "op_counts.json")))["tw_paper"]
    rng = random.Random(9)
    adds, muls = [], []
    for _ in range(1500):
        a, b = rand_mw(rng, 1, 3), rand_mw(rng, 1, 3)
        for op, out in ((orc.add, adds), (orc.mul, muls)):
            orc.ops_reset()
            op("tw", a, b)
            out.append(orc.ops_get())
    assert set(muls) == {42}
    assert min(adds) >= 30 + 9 and max(adds) <= 30 + 15 and all((c - 30) % 3 == 0 for c in adds)
    mean_add = sum(adds) / len(adds)
    # Reported: restatement (fixed + branch part) against the paper's fixed part.
    print(f"TW add: {mean_add:.1f} ops mean (30 + 9..15) vs paper {g['add_fixed']} + alpha; "
          f"TW mul: 42 ops (36 + 6) vs paper {g['mul_fixed']} + alpha")
    assert 30 < g["add_fixed"] and 36 < g["mul_fixed"]


def test_operation_counts_match_paper(orc):
    g = json.load(open(os.path.join(GOLD, "op_counts.json")))
    rng = random.Random(4)
    a2, b2 = rand_mw(rng, 64, 2), rand_mw(rng, 64, 2)
    a3, b3 = rand_mw(rng, 64, 3), rand_mw(rng, 64, 3)
    s = a2[0]
    assert _count(orc, lambda n: orc.two_sum(a2[0], b2[0])) == g["two_sum"]
    assert _count(orc, lambda n: orc.quick_two_sum(a2[0], b2[0])) == g["quick_two_sum"]
    assert _count(orc, lambda n: orc.two_prod(a2[0], b2[0])) == g["two_prod"]
    assert _count(orc, lambda n: orc.add("dw", a2, b2)) == g["dw_add"]
    assert _count(orc, lambda n: orc.mul("dw", a2, b2)) == g["dw_mul"]
    assert _count(orc, lambda n: orc.add("qdw", a2, b2)) == g["qdw_add"]
    assert _count(orc, lambda n: orc.mul("qdw", a2, b2)) == g["qdw_mul"]
    assert _count(orc, lambda n: orc.add("qtw", a3, b3)) == g["qtw_add"]
    assert _count(orc, lambda n: orc.mul("qtw", a3, b3)) == g["qtw_mul"]
    assert _count(orc, lambda n: orc.vecsum3(a3)) == g["vecsum3"]
    assert _count(orc, lambda n: orc.dxmul("qtw", s, b3)) == g["dx_qtw_mul"]
    # Derived FP64 x MW products (Sec. III, last paragraph): operations on the
    # zero lower words are dropped -> DW 7-1, QDW 4-1.
    assert _count(orc, lambda n: orc.dxmul("dw", s, b2)) == g["dw_mul"] - 1
    assert _count(orc, lambda n: orc.dxmul("qdw", s, b2)) == g["qdw_mul"] - 1


# Error envelopes (relative, exact rational check).  Bounds proposed for
# this project from the published analyses the paper cites; the paper prints
# none.  u = 2^-53.
ENV = {
    ("dw", "mul"): 8 * U ** 2,
    ("qdw", "mul"): 8 * U ** 2,
    ("qtw", "mul"): 64 * U ** 3,
    ("tw", "mul"): Fraction(1, 2 ** 150),
    ("tw", "add"): Fraction(1, 2 ** 150),
}


@pytest.mark.parametrize("arith,w", [("dw", 2), ("qdw", 2), ("qtw", 3), ("tw", 3)])
def test_mul_error_envelope(orc, arith, w):
    rng = random.Random(5 + w)
    a, b = rand_mw(rng, N, w), rand_mw(rng, N, w)
    c = orc.mul(arith, a, b)
    env = ENV[(arith, "mul")]
    for i in range(N):
        exact = val(col(a, i)) * val(col(b, i))
        assert rel_err(val(col(c, i)), exact) <= env, (arith, i)


@pytest.mark.parametrize("arith,w", [("dw", 2), ("qdw", 2), ("qtw", 3), ("tw", 3)])
def test_dxmul_error_envelope(orc, arith, w):
    rng = random.Random(11 + w)
    b = rand_mw(rng, N, w)
    a = np.array([float(rand_mw(rng, 1, 1)[0, 0]) for _ in range(N)])
    c = orc.dxmul(arith, a, b)
    env = ENV[(arith, "mul")]
    for i in range(N):
        exact = Fraction(a[i]) * val(col(b, i))
        assert rel_err(val(col(c, i)), exact) <= env


def test_add_error_envelopes(orc):
    rng = random.Random(7)
    # DW (the one-TwoSum variant): relative bound for same-sign operands only.
    a, b = rand_mw(rng, N, 2, signed=False), rand_mw(rng, N, 2, signed=False)
    c = orc.add("dw", a, b)
    for i in range(N):
        ex = val(col(a, i)) + val(col(b, i))
        assert rel_err(val(col(c, i)), ex) <= 8 * U ** 2
    # QDW / QTW: absolute bound relative to |a| + |b| for any signs.
    for arith, w, env in (("qdw", 2, 8 * U ** 2), ("qtw", 3, 64 * U ** 3)):
        a, b = rand_mw(rng, N, w), rand_mw(rng, N, w)
        c = orc.add(arith, a, b)
        for i in range(N):
            va, vb = val(col(a, i)), val(col(b, i))
            assert abs(val(col(c, i)) - (va + vb)) <= env * (abs(va) + abs(vb))
    # TW: relative bound for any signs (VecSum is error-free; only the
    # renormalisation to three words rounds).
    a, b = rand_mw(rng, N, 3), rand_mw(rng, N, 3)
    c = orc.add("tw", a, b)
    for i in range(N):
        ex = val(col(a, i)) + val(col(b, i))
        assert rel_err(val(col(c, i)), ex) <= ENV[("tw", "add")]


def test_add_cancellation_cases(orc):
    """Exact cancellation: a + (-a) must be exactly zero in every arithmetic."""
    rng = random.Random(8)
    for arith, w in (("dw", 2), ("qdw", 2), ("qtw", 3), ("tw", 3)):
        a = rand_mw(rng, 200, w)
        c = orc.add(arith, a, -a)
        assert np.all(c == 0.0), arith


def test_normalized_results_do_not_overlap(orc):
    rng = random.Random(9)
    a, b = rand_mw(rng, N, 2), rand_mw(rng, N, 2)
    for c in (orc.add("dw", a, b), orc.mul("dw", a, b), orc.dxmul("dw", a[0], b)):
        assert np.all(c[0] + c[1] == c[0])                       # fl(c1+c2) = c1 (Sec. III)
    # TW: the renormalisation with branches yields ulp-nonoverlapping words,
    # |c2| <= ulp(c1) and |c3| <= ulp(c2) (the property that renormalisation
    # guarantees; the product even meets fl(c1+c2) = c1).
    a, b = rand_mw(rng, N, 3), rand_mw(rng, N, 3)
    ulp = np.vectorize(math.ulp)
    for c in (orc.add("tw", a, b), orc.mul("tw", a, b), orc.dxmul("tw", a[0], b)):
        assert np.all(np.abs(c[1]) <= ulp(c[0]))
        assert np.all(np.abs(c[2]) <= ulp(c[1]))
    c = orc.mul("tw", a, b)
    assert np.all(c[0] + c[1] == c[0]) and np.all(c[1] + c[2] == c[1])


def test_zero_lower_words_reduce_to_error_free_transforms(orc):
    """With zero lower words every add/mul must return the exact TwoSum/TwoProd pair."""
    rng = random.Random(10)
    a1 = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-40, 40) for _ in range(N)])
    b1 = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-40, 40) for _ in range(N)])
    z = np.zeros(N)
    for arith, w in (("dw", 2), ("qdw", 2), ("qtw", 3), ("tw", 3)):
        A = np.vstack([a1] + [z] * (w - 1))
        B = np.vstack([b1] + [z] * (w - 1))
        s = orc.add(arith, A, B)
        p = orc.mul(arith, A, B)
        d = orc.dxmul(arith, a1, B)
        for i in range(0, N, 7):
            assert val(col(s, i)) == Fraction(a1[i]) + Fraction(b1[i])
            assert val(col(p, i)) == Fraction(a1[i]) * Fraction(b1[i])
            assert val(col(d, i)) == Fraction(a1[i]) * Fraction(b1[i])
            assert s[0, i] == a1[i] + b1[i] and p[0, i] == a1[i] * b1[i]


def _same_up_to_zero_sign(x, y):
    return np.all((x == y) | ((x == 0) & (y == 0)))


def test_fp64_times_mw_is_zero_padded_product(orc):
    """Sec. III: FP64 x MW omits work on lower words assumed zero.  For DW, QDW
    and TW those omissions are identities, so the result equals the full
    product with the FP64 operand zero-padded (up to the sign of zero)."""
    rng = random.Random(12)
    for arith, w in (("dw", 2), ("qdw", 2), ("tw", 3)):
        b = rand_mw(rng, N, w)
        a = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30) for _ in range(N)])
        A = np.vstack([a] + [np.zeros(N)] * (w - 1))
        assert _same_up_to_zero_sign(orc.dxmul(arith, a, b), orc.mul(arith, A, b)), arith


def test_vecsum3_is_error_free(orc):
    rng = random.Random(13)
    a = rand_mw(rng, N, 3)
    a[1] *= np.array([rng.uniform(0.5, 3e15) for _ in range(N)])   # make the words overlap
    c = orc.vecsum3(a)
    for i in range(N):
        assert val(col(c, i)) == val(col(a, i))
        assert c[0, i] == a[0, i] + a[1, i]


def test_quasi_normalization_is_error_free(orc):
    rng = random.Random(14)
    for arith, w in (("qdw", 2), ("qtw", 3)):
        a = rand_mw(rng, 500, w)
        c = orc.normalize(arith, a)
        for i in range(500):
            assert val(col(c, i)) == val(col(a, i))
        assert np.all(orc.normalize(arith + "_nn", a) == a)      # the NN variants never normalise


@pytest.mark.parametrize("arith,w,env", [("dw", 2, 8 * U ** 2), ("qdw", 2, 8 * U ** 2),
                                         ("qtw", 3, Fraction(1, 2 ** 150)), ("tw", 3, Fraction(1, 2 ** 150)),
                                         ("fp64", 1, U)])
def test_division_accuracy(orc, arith, w, env):
    rng = random.Random(15 + w)
    a, b = rand_mw(rng, N, w), rand_mw(rng, N, w)
    c = orc.div(arith, a, b)
    for i in range(N):
        exact = val(col(a, i)) / val(col(b, i))
        assert rel_err(val(col(c, i)), exact) <= env


def test_collapse_rounds_lowest_first(orc):
    # fl(c1 + fl(c2 + c3)); c2 + c3 = 2^-53 exactly here so the tie goes to even.
    a = np.array([[1.0], [2.0 ** -54], [2.0 ** -54]])
    assert orc.collapse("qtw", a)[0] == 1.0 + 2.0 ** -53 == 1.0   # 1 + 2^-53 rounds to even = 1
    a = np.array([[1.0], [2.0 ** -53], [2.0 ** -80]])
    assert orc.collapse("tw", a)[0] == 1.0 + 2.0 ** -52            # above the tie, rounds up


def test_precision_classes(orc):
    """Sec. I: DW ~ 106 bits, TW ~ 159 bits of precision.  The worst relative
    error of a product over random operands sits between 2^-(bits+2) ... 2^-(bits-6)."""
    g = json.load(open(os.path.join(GOLD, "precision_bits.json")))
    rng = random.Random(16)
    for arith, w, bits in (("dw", 2, g["dw_bits"]), ("tw", 3, g["tw_bits"])):
        a, b = rand_mw(rng, 800, w), rand_mw(rng, 800, w)
        c = orc.mul(arith, a, b)
        worst = max(rel_err(val(col(c, i)), val(col(a, i)) * val(col(b, i))) for i in range(800))
        assert Fraction(1, 2 ** (bits + 4)) <= worst <= Fraction(1, 2 ** (bits - 8)), (arith, float(worst))


def test_printed_left_to_right_order_dwadd(orc):
    """Algorithm 5 writes e = fl(e + a2 + b2), evaluated left to right.  Worked by hand:
    a = (1, 2^-123), b = (2^-70, -2^-123).  TwoSum(1, 2^-70) = (1, 2^-70) exactly.
    fl(2^-70 + 2^-123) is a tie (half an ulp of 2^-70) and rounds to even, 2^-70;
    then fl(2^-70 - 2^-123) = 2^-70 - 2^-123 is representable.  QuickTwoSum(1, e)
    keeps both words.  (The other association would give e = 2^-70.)"""
    a = np.array([[1.0], [2.0 ** -123]])
    b = np.array([[2.0 ** -70], [-(2.0 ** -123)]])
    for arith in ("dw", "qdw"):
        c = orc.add(arith, a, b)
        assert c[0, 0] == 1.0 and c[1, 0] == 2.0 ** -70 - 2.0 ** -123


def test_printed_left_to_right_order_qtwadd(orc):
    """Algorithm 7 writes c3 = fl(a3 + b3 + e2 + e3).  Worked by hand:
    a = (1, 2^-54, 2^-108), b = (1, 2^-200, -2^-108): TwoSum(1,1) = (2, 0);
    TwoSum(2^-54, 2^-200) = (2^-54, 2^-200); TwoSum(2^-54, 0) = (2^-54, 0);
    c3 = ((2^-108 - 2^-108) + 2^-200) + 0 = 2^-200.  Any association that adds
    e2 to a3 or b3 first loses 2^-200 (below half an ulp of 2^-108) and gives 0."""
    a = np.array([[1.0], [2.0 ** -54], [2.0 ** -108]])
    b = np.array([[1.0], [2.0 ** -200], [-(2.0 ** -108)]])
    c = orc.add("qtw", a, b)
    assert c[:, 0].tolist() == [2.0, 2.0 ** -54, 2.0 ** -200]
