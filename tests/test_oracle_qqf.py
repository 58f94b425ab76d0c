"""Pins of the oracle's FP32-word arithmetic QQF and its scaled CG.

Sec. II notes multi-word arithmetic built from FP32 words where FP64 is
missing, and Sec. VI names processors with little FP64 throughput; the paper
prints no FP32-word algorithm.  The oracle's readings: QQF is QQW's sequence
with FP32 words and operations (about 96 bits); FP64 inputs enter through an
exact three-word split by significand bits; CG keeps r and p scaled by a
power of two so that FP32's exponent range covers a shrinking residual.
What fixes them independently of that code:
 * exact rational arithmetic: the error envelopes of add / mul / FP64 x QQF /
   division at the quad-float level (about 2^-90);
 * the split is the truncation to 24 significant bits plus the exact rest,
   computed here from math.frexp; outside its range it is numpy's FP32
   rounding;
 * with zero lower words, add / mul are the exact FP32 TwoSum / TwoProd;
 * the normalisation (VecSum4) is error free;
 * CG in QQF follows exact CG; its forward error reaches the quad-float level;
 * the scaling is invisible: b 2^k gives the same iterations, the same
   residual history bit for bit, and (inside FP32's range) x 2^k exactly.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from mwref import cg_exact, col, dense_fraction, fnorm, solve_exact, val
from paper_2510_13536_gb300 import problems as P

N = 1500


def f32(x: float) -> float:
    return float(np.float32(x))


def rand_mwf(rng: random.Random, n: int, emin: int = -20, emax: int = 20) -> np.ndarray:
    """(4, n) nearest-rounding FP32 expansions of random ~110-bit values."""
    out = np.empty((4, n))
    for i in range(n):
        m = rng.getrandbits(110) | (1 << 109)
        v = Fraction(m, 1 << 110) * Fraction(2) ** rng.randint(emin, emax)
        if rng.random() < 0.5:
            v = -v
        rem = v
        for k in range(4):
            out[k, i] = f32(float(rem))
            rem -= Fraction(out[k, i])
    return out


def rel_err(got, exact):
    return abs(got - exact) / abs(exact) if exact != 0 else abs(got)


def is_f32(a) -> bool:
    a = np.asarray(a, dtype=np.float64)
    return bool(np.all(a.astype(np.float32).astype(np.float64) == a))


def trunc24(s: float) -> float:
    """s truncated to 24 significant bits (toward zero)."""
    m, e = math.frexp(s)                         # s = m 2^e, 1/2 <= |m| < 1
    t = math.floor(abs(m) * 2 ** 24)
    return math.copysign(math.ldexp(t, e - 24), s)


def test_split_is_exact_and_by_significand_bits(orc):
    rng = random.Random(51)
    s = np.array([rng.uniform(1, 2) * rng.choice([-1, 1]) * 2.0 ** rng.randint(-97, 126) for _ in range(N)])
    one = np.zeros((4, N))
    one[0] = 1.0
    d = orc.dxmul("qqf", s, one)                 # the split times one: the split itself
    assert is_f32(d)
    for i in range(N):
        assert val(col(d, i)) == Fraction(s[i])
        assert d[0, i] == trunc24(s[i]) and d[3, i] == 0.0
        assert abs(d[1, i]) < math.ldexp(1.0, math.frexp(d[0, i])[1] - 24)
    # Outside 2^-97 <= |s| < 2^128: FP32 rounding of the value and of the rests.
    odd = np.array([0.0, -0.0, 5e-310, -3.3e-320, 1.3 * 2.0 ** -100, -7.1e-35, 2.0 ** -98])
    one = np.zeros((4, odd.size))
    one[0] = 1.0
    d = orc.dxmul("qqf", odd, one)
    for i, v in enumerate(odd):
        a0 = f32(v)
        a1 = f32(v - a0)
        a2 = f32((v - a0) - a1)
        assert (d[0, i], d[1, i], d[2, i]) == (a0, a1, a2), v
        assert math.copysign(1.0, d[0, i]) == math.copysign(1.0, a0)


@pytest.mark.parametrize("op,env", [("add", 2 ** -93), ("mul", 2 ** -91), ("div", 2 ** -89)])
def test_error_envelopes(orc, op, env):
    """Exact rationals; add relative to |a| + |b| (any signs), the others relative."""
    rng = random.Random(52)
    a, b = rand_mwf(rng, N), rand_mwf(rng, N)
    c = getattr(orc, op)("qqf", a, b)
    assert is_f32(c)
    env = Fraction(env)
    worst = Fraction(0)
    for i in range(N):
        va, vb = val(col(a, i)), val(col(b, i))
        if op == "add":
            e = abs(val(col(c, i)) - (va + vb)) / (abs(va) + abs(vb))
        else:
            e = rel_err(val(col(c, i)), va * vb if op == "mul" else va / vb)
        worst = max(worst, e)
    assert worst <= env, (op, math.log2(worst))
    # quad-float, not more: 24 x 4 bits less the quasi truncation.
    assert worst >= Fraction(1, 2 ** 102), (op, math.log2(worst))


def test_fp64_times_qqf_envelope(orc):
    rng = random.Random(53)
    b = rand_mwf(rng, N)
    s = np.array([rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30) for _ in range(N)])
    d = orc.dxmul("qqf", s, b)
    for i in range(N):
        assert rel_err(val(col(d, i)), Fraction(s[i]) * val(col(b, i))) <= Fraction(1, 2 ** 89)


def test_zero_lower_words_give_exact_twosum_twoprod(orc):
    rng = random.Random(54)
    a1 = np.array([f32(rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30)) for _ in range(N)])
    b1 = np.array([f32(rng.uniform(-2, 2) * 2.0 ** rng.randint(-30, 30)) for _ in range(N)])
    z = np.zeros(N)
    A, B = np.vstack([a1, z, z, z]), np.vstack([b1, z, z, z])
    s, p = orc.add("qqf", A, B), orc.mul("qqf", A, B)
    for i in range(0, N, 5):
        assert val(col(s, i)) == Fraction(a1[i]) + Fraction(b1[i])
        assert val(col(p, i)) == Fraction(a1[i]) * Fraction(b1[i])
        assert s[0, i] == float(np.float32(a1[i]) + np.float32(b1[i]))
        assert p[0, i] == float(np.float32(a1[i]) * np.float32(b1[i]))


def test_normalisation_is_error_free(orc):
    rng = random.Random(55)
    a = rand_mwf(rng, 600)
    a[1] = np.array([f32(a[1, i] * rng.uniform(0.5, 3e6)) for i in range(600)])     # overlapping words
    c = orc.normalize("qqf", a)
    assert is_f32(c)
    for i in range(600):
        assert val(col(c, i)) == val(col(a, i))
        assert c[0, i] == float(np.float32(a[0, i]) + np.float32(a[1, i]))


def test_collapse_lowest_first_in_fp64(orc):
    # (1, 2^-53, 2^-106, 2^-106) are FP32 numbers; lowest first: 2^-106 + 2^-106
    # = 2^-105, 2^-53 + 2^-105 exact, and 1 + that lies above the tie: 1 + 2^-52.
    t = np.array([[1.0], [2.0 ** -53], [2.0 ** -106], [2.0 ** -106]])
    assert orc.collapse("qqf", t)[0] == 1.0 + 2.0 ** -52
    rng = random.Random(56)
    a = rand_mwf(rng, 300)
    assert np.all(orc.add("qqf", a, -a) == 0.0)


def test_cg_iterates_follow_exact_cg(orc):
    A = P.random_spd_small(9, seed=3)
    b = P.rhs_uniform(A.n, 4)
    xs, _ = cg_exact(dense_fraction(A), b, 6)
    for k in (1, 3, 6):
        x, it, rr, st = orc.cg("qqf", A, b, tol=1e-300, maxit=k)
        assert it == k and st == 1 and is_f32(x)
        scale = max(abs(v) for v in xs[k - 1])
        for i in range(A.n):
            assert abs(float(val(col(x, i)) - xs[k - 1][i])) <= 1e-24 * float(scale), (k, i)


def test_forward_error_against_exact_solve(orc):
    A = P.random_spd_small(24, seed=7, shift_exp=-4)
    b = P.rhs_uniform(A.n, 8)
    xe = solve_exact(dense_fraction(A), b)
    x, it, rr, st = orc.cg("qqf", A, b, tol=1e-24, maxit=3000)
    assert st == 0
    err = math.sqrt(sum(float(val(col(x, i)) - xe[i]) ** 2 for i in range(A.n))) / fnorm(xe)
    assert err <= 1e-22, err


def test_scaling_is_invisible(orc):
    """b 2^k: E absorbs k, so the scaled iteration is the same bit for bit.
    x is held unscaled: at k = -300 every word of the solution is far below
    FP32's normal range and at k = +300 the first update overflows; both
    solves report the out-of-range status (4) instead of convergence."""
    A = P.laplacian_2d(24, 1e-3)
    b = P.rhs_uniform(A.n, 9)
    x, it, rr, st, h = orc.cg("qqf", A, b, tol=1e-22, maxit=2000, history=True)
    assert st == 0
    for k in (40, -40, -300):
        x2, it2, rr2, st2, h2 = orc.cg("qqf", A, b * 2.0 ** k, tol=1e-22, maxit=2000, history=True)
        assert (it2, rr2) == (it, rr), k
        assert np.array_equal(h2, h), k
        if abs(k) <= 40:                          # x itself must stay within FP32's range
            assert st2 == 0 and np.array_equal(x2, x * 2.0 ** k), k
        else:
            assert st2 == 4 and np.max(np.abs(x2[0])) < 2.0 ** -126, k
    x2, it2, rr2, st2, h2 = orc.cg("qqf", A, b * 2.0 ** 300, tol=1e-22, maxit=2000, history=True)
    assert (st2, it2) == (4, 1) and np.array_equal(h2, h[:1]) and not np.all(np.isfinite(x2[0]))


def test_tracks_double_word_cg(orc):
    """QQF (about 96 bits) and DW (106) take the same CG path on a 2-D Laplacian."""
    A = P.laplacian_2d(32)
    b = P.rhs_uniform(A.n, 3)
    xq, itq, rrq, stq = orc.cg("qqf", A, b, tol=1e-22, maxit=3000)
    xd, itd, rrd, std_ = orc.cg("dw", A, b, tol=1e-22, maxit=3000)
    _, itf, _, _ = orc.cg("fp64", A, b, tol=1e-22, maxit=3000)
    assert stq == std_ == 0 and itq == itd < itf
    assert abs(rrq - rrd) <= 1e-8 * rrd
    xq64, xd64 = orc.collapse("qqf", xq), orc.collapse("dw", xd)
    assert np.max(np.abs(xq64 - xd64)) <= 1e-20 * np.max(np.abs(xd64))


@pytest.mark.parametrize("ar", ["qqf", "qf"])
def test_adjoint_gradient_equals_triple_word(orc, ar):
    """The adjoint in FP32 words (lambda by the scaled CG, g_val = -lambda_i x_j
    in the arithmetic, collapsed) against TW's, whose adjoint is pinned to exact
    rational gradients and central differences: solved to 1e-24 both are
    exact to FP64, so the collapsed gradients agree to a few ulps."""
    for A in (P.laplacian_3d(8, 1e-2), P.diffusion_2d(20, seed=5)):
        b = P.rhs_uniform(A.n, 5)
        w = np.random.default_rng(3).standard_normal(A.n)
        x, it, _, st = orc.cg(ar, A, b, tol=1e-24, maxit=5000)
        xt, itt, _, stt = orc.cg("tw", A, b, tol=1e-24, maxit=5000)
        assert st == stt == 0
        g_b, g_val, lam, it2, _, st2 = orc.adjoint(ar, A, x, w, 1e-24, 5000)
        t_b, t_val, _, _, _, _ = orc.adjoint("tw", A, xt, w, 1e-24, 5000)
        assert st2 == 0 and is_f32(lam) and g_val.shape == (A.nnz,)
        assert np.max(np.abs(g_b - t_b)) <= 4e-16 * np.max(np.abs(t_b))
        assert np.max(np.abs(g_val - t_val)) <= 4e-16 * np.max(np.abs(t_val))
        # A mutation of the formula (the sign, or lambda and x swapped on a
        # nonsymmetric pattern of values) would fail: g_val is -lambda_row x_col.
        rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
        lam64, x64 = orc.collapse(ar, lam), orc.collapse(ar, x)
        assert np.allclose(g_val, -lam64[rows] * x64[A.col], rtol=1e-12, atol=0)


def test_special_cases(orc):
    A = P.laplacian_2d(10)
    x, it, rr, st = orc.cg("qqf", A, np.zeros(A.n), x0=np.ones((4, A.n)), tol=1e-10, maxit=20)
    assert (it, st, rr) == (0, 0, 0.0) and np.all(x == 0.0)
    b = P.matvec_exact(A, np.ones(A.n))
    x0 = np.zeros((4, A.n))
    x0[0] = 1.0
    x, it, rr, st = orc.cg("qqf", A, b, x0=x0, tol=1e-10, maxit=20)     # r0 = 0 exactly
    assert (it, st, rr) == (0, 0, 0.0) and np.array_equal(x, x0)
    x, it, rr, st = orc.cg("qqf", A, b, tol=1e-10, maxit=0)
    assert (it, st) == (0, 1) and rr == 1.0
    with pytest.raises(ValueError):
        orc.cg("qqf", A, b, norm=(2, 1))
    with pytest.raises(ValueError):                 # Jacobi PCG keeps the fixed policy too
        orc.cg("qqf", A, b, precond="jacobi", norm=(2, 1))
    x, it, rr, st = orc.bicgstab("qqf", A, b, tol=1e-20, maxit=200)   # BiCGStab runs scaled too
    assert st == 0 and it > 0
