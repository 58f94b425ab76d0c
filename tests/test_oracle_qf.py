"""Pins of the oracle's QF: QQF (four FP32 words) with every addition and
product followed by VecSum4, the non-quasi counterpart as DW is to QDW
(Sec. III).  The paper prints no FP32-word algorithm (Sec. II, Sec. VI).

What fixes it independently of that code:
 * exact rationals: the quad-float error envelopes of add / mul / division;
 * every QF result is already normalised (VecSum4 leaves it unchanged),
   which QQF's results are not;
 * with zero lower words, add / mul are the exact FP32 TwoSum / TwoProd;
 * CG in QF follows exact CG, and the scaled iteration is invisible (b 2^k);
 * on an ill-conditioned power-law graph Laplacian, where QQF's operand-
   relative errors break the iteration down, QF converges in fewer
   iterations than FP64 and about as many as QDW.
"""
import random
from fractions import Fraction

import numpy as np

from mwref import cg_exact, col, dense_fraction, val
from paper_2510_13536_gb300 import problems as P
from test_oracle_qqf import rand_mwf, rel_err

N = 1200


def test_envelopes_and_normalised_results(orc):
    rng = random.Random(71)
    a, b = rand_mwf(rng, N), rand_mwf(rng, N)
    for op, env in (("add", 2 ** -93), ("mul", 2 ** -91), ("div", 2 ** -89)):
        c = getattr(orc, op)("qf", a, b)
        for i in range(0, N, 3):
            va, vb = val(col(a, i)), val(col(b, i))
            if op == "add":
                assert abs(val(col(c, i)) - (va + vb)) <= Fraction(env) * (abs(va) + abs(vb))
            else:
                assert rel_err(val(col(c, i)), va * vb if op == "mul" else va / vb) <= Fraction(env)
        assert np.array_equal(orc.normalize("qf", c), c), op
    s64 = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30) for _ in range(N)])
    d = orc.dxmul("qf", s64, b)                          # FP64 x QF, as in the SpMV
    for i in range(0, N, 3):
        assert rel_err(val(col(d, i)), Fraction(s64[i]) * val(col(b, i))) <= Fraction(2 ** -89)
    assert np.array_equal(orc.normalize("qf", d), d)
    # QQF's sums and products are not in normalised form: the pin discriminates.
    assert not np.array_equal(orc.normalize("qqf", orc.dxmul("qqf", s64, b)), orc.dxmul("qqf", s64, b))
    assert not np.array_equal(orc.normalize("qqf", orc.add("qqf", a, b)), orc.add("qqf", a, b))
    assert not np.array_equal(orc.normalize("qqf", orc.mul("qqf", a, b)), orc.mul("qqf", a, b))


def test_zero_lower_words_give_exact_twosum_twoprod(orc):
    rng = random.Random(72)
    a1 = np.array([float(np.float32(rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30))) for _ in range(N)])
    b1 = np.array([float(np.float32(rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30))) for _ in range(N)])
    z = np.zeros(N)
    A, B = np.vstack([a1, z, z, z]), np.vstack([b1, z, z, z])
    s, p = orc.add("qf", A, B), orc.mul("qf", A, B)
    for i in range(0, N, 5):
        assert val(col(s, i)) == Fraction(a1[i]) + Fraction(b1[i])
        assert val(col(p, i)) == Fraction(a1[i]) * Fraction(b1[i])


def test_cg_iterates_follow_exact_cg(orc):
    A = P.random_spd_small(9, seed=3)
    b = P.rhs_uniform(A.n, 4)
    xs, _ = cg_exact(dense_fraction(A), b, 6)
    for k in (1, 3, 6):
        x, it, rr, st = orc.cg("qf", A, b, tol=1e-300, maxit=k)
        assert it == k and st == 1
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            assert abs(float(val(col(x, i)) - xs[k - 1][i])) <= 1e-24 * float(scale), (k, i)


def test_scaling_is_invisible(orc):
    A = P.laplacian_2d(20, 1e-3)
    b = P.rhs_uniform(A.n, 9)
    x, it, rr, st, h = orc.cg("qf", A, b, tol=1e-22, maxit=2000, history=True)
    assert st == 0
    for k in (20, -20, -300):
        x2, it2, rr2, st2, h2 = orc.cg("qf", A, b * 2.0 ** k, tol=1e-22, maxit=2000, history=True)
        assert (it2, rr2) == (it, rr) and np.array_equal(h2, h), k
        if abs(k) <= 20:            # x's lowest words (~1e-25 |x|) stay above FP32's subnormals
            assert st2 == 0 and np.array_equal(x2, x * 2.0 ** k), k
        else:                       # the whole solution under FP32's normal range
            assert st2 == 4, k
    x2, it2, rr2, st2, h2 = orc.cg("qf", A, b * 2.0 ** 300, tol=1e-22, maxit=2000, history=True)
    assert (st2, it2) == (4, 1) and np.array_equal(h2, h[:1])        # x overflows at the first update


def test_converges_where_qqf_breaks_down(orc):
    """Power-law graph Laplacian, n = 2000 (lognormal weights, isolated nodes
    at 1e-8): strongly cancelling rows.  QQF breaks down; QF converges faster
    than FP64, with about QDW's iteration count."""
    A = P.power_law_laplacian(2000, seed=7, mean_deg=12, max_deg=300)
    b = P.rhs_uniform(A.n, 32)
    runs = {ar: orc.cg(ar, A, b, tol=1e-14, maxit=20000) for ar in ("fp64", "qdw", "qqf", "qf")}
    it = {ar: r[1] for ar, r in runs.items()}
    st = {ar: r[3] for ar, r in runs.items()}
    assert st["qqf"] == 2 and st["qf"] == st["qdw"] == st["fp64"] == 0, st
    assert it["qf"] < it["fp64"] and it["qf"] <= 1.1 * it["qdw"], it
