"""The integer-pipe rounding-error routine (csrc/mw_int.cuh) checked on the CPU.

mw_int.cuh compiles as plain C++; a small shim exposes it to numpy.  Its
result must equal, bit for bit, the error term of the printed TwoSum
(Algorithm 2) and, where QuickTwoSum's precondition holds, of QuickTwoSum
(Algorithm 3), evaluated here with numpy's IEEE float64 operations; on a
subset it is also checked against exact rational arithmetic.
"""
import ctypes
import os
import random
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_13536_gb300", "csrc")

SHIM = r"""
#include "mw_int.cuh"
extern "C" void add_error_batch(long n, const double* a, const double* b, const double* x, double* y, int* ok) {
  for (long i = 0; i < n; ++i) { double t = 0.0; ok[i] = mwi::add_error(a[i], b[i], x[i], t) ? 1 : 0; y[i] = t; }
}
#include <cmath>
extern "C" void mul_error_batch(long n, const double* a, const double* b, double* e, double* ref, int* ok) {
  for (long i = 0; i < n; ++i) {
    const double p = a[i] * b[i];
    double t = 0.0;
    ok[i] = mwi::mul_error(a[i], b[i], p, t) ? 1 : 0;
    e[i] = t;
    ref[i] = std::fma(a[i], b[i], -p);
  }
}
extern "C" void add_rn_batch(long n, const double* a, const double* b, double* x, double* ref, int* ok) {
  for (long i = 0; i < n; ++i) {
    double t = 0.0;
    ok[i] = mwi::add_rn(a[i], b[i], t) ? 1 : 0;
    x[i] = t;
    ref[i] = a[i] + b[i];
  }
}
extern "C" void pow2_dx_batch(long n, int w, const double* a, const double* b, double* c, int* ok) {
  for (long i = 0; i < n; ++i) {
    bool g = mwi::is_pow2(a[i]);
    for (int k = 0; k < w && g; ++k) {
      double t = 0.0;
      g = mwi::pow2_scale(a[i], b[k * n + i], k > 0, t);
      c[k * n + i] = t;
    }
    ok[i] = g ? 1 : 0;
  }
}
template <int W>
static void pow2_product_batch_w(long n, const double* a, const double* b, double* c, int* ok) {
  for (long i = 0; i < n; ++i) {
    double bw[W], cw[W];
    for (int k = 0; k < W; ++k) bw[k] = b[k * n + i];
    ok[i] = mwi::pow2_product<W>(a[i], bw, cw) ? 1 : 0;
    for (int k = 0; k < W; ++k) c[k * n + i] = cw[k];
  }
}
extern "C" void pow2_product_batch(long n, int w, const double* a, const double* b, double* c, int* ok) {
  if (w == 2) pow2_product_batch_w<2>(n, a, b, c, ok);
  else if (w == 3) pow2_product_batch_w<3>(n, a, b, c, ok);
  else pow2_product_batch_w<4>(n, a, b, c, ok);
}
extern "C" void quick_exact_batch(long n, const double* a, const double* b, int* ok) {
  for (long i = 0; i < n; ++i) ok[i] = mwi::quick_exact(a[i], b[i]) ? 1 : 0;
}
"""


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    d = tmp_path_factory.mktemp("mwi")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    lib = d / "libmwi.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC,
                    "-o", str(lib), str(src)], check=True)
    L = ctypes.CDLL(str(lib))
    P = ctypes.c_void_p
    L.add_error_batch.argtypes = [ctypes.c_long, P, P, P, P, P]
    L.quick_exact_batch.argtypes = [ctypes.c_long, P, P, P]
    L.mul_error_batch.argtypes = [ctypes.c_long, P, P, P, P, P]
    L.add_rn_batch.argtypes = [ctypes.c_long, P, P, P, P, P]
    L.pow2_dx_batch.argtypes = [ctypes.c_long, ctypes.c_int, P, P, P, P]
    L.pow2_product_batch.argtypes = [ctypes.c_long, ctypes.c_int, P, P, P, P]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def add_error(L, a, b, x):
    y = np.zeros_like(a)
    ok = np.zeros(a.size, dtype=np.int32)
    L.add_error_batch(a.size, _p(a), _p(b), _p(x), _p(y), _p(ok))
    return y, ok.astype(bool)


def printed_two_sum(a, b):
    with np.errstate(all="ignore"):
        s = a + b
        z = s - a
        y = (a - (s - z)) + (b - z)
    return s, y


def printed_quick_two_sum(a, b):
    with np.errstate(all="ignore"):
        s = a + b
        y = (a - s) + b
    return s, y


def inputs(seed, n):
    rng = np.random.default_rng(seed)
    e = rng.integers(-1000, 1000, size=n)
    a = rng.uniform(1, 2, size=n) * np.exp2(e) * rng.choice([-1.0, 1.0], size=n)
    kind = rng.integers(0, 8, size=n)
    gap = rng.integers(-60, 61, size=n)
    b = rng.uniform(1, 2, size=n) * np.exp2(np.clip(e + gap, -1074, 1023)) * rng.choice([-1.0, 1.0], size=n)
    # near cancellation
    m = kind == 1
    b[m] = -a[m] * (1 + rng.choice([-1.0, 1.0], size=m.sum()) * rng.uniform(0, 1, m.sum()) *
                    np.exp2(-rng.integers(1, 54, m.sum())))
    # exact half-ulp ties and neighbours around the rounding point
    m = kind == 2
    k = rng.integers(50, 58, m.sum())
    b[m] = np.ldexp(np.sign(rng.uniform(-1, 1, m.sum())) * rng.integers(1, 4, m.sum()), np.frexp(a[m])[1] - k)
    # integers / small dyadics (many exact sums)
    m = kind == 3
    a[m] = rng.integers(-2 ** 53, 2 ** 53, m.sum()).astype(np.float64)
    b[m] = rng.integers(-2 ** 20, 2 ** 20, m.sum()).astype(np.float64)
    # powers of two against small opposite values
    m = kind == 4
    a[m] = np.exp2(rng.integers(-500, 500, m.sum())) * rng.choice([-1.0, 1.0], m.sum())
    b[m] = -a[m] * rng.uniform(0, 1, m.sum()) * np.exp2(-rng.integers(40, 60, m.sum()))
    # zeros, signed zeros, tiny and huge values, infinities, NaN
    m = np.nonzero(kind == 5)[0]
    sp = np.array([0.0, -0.0, 5e-324, -2.2250738585072014e-308, 1e-300, 1.7e308, -1.7e308, np.inf, -np.inf, np.nan])
    b[m] = sp[rng.integers(0, sp.size, m.size)]
    m2 = m[::3]
    a[m2] = sp[rng.integers(0, sp.size, m2.size)]
    return a, b


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_printed_two_sum(shim, seed):
    a, b = inputs(seed, 400_000)
    for (u, v) in ((a, b), (b, a)):
        x, y_ref = printed_two_sum(u, v)
        y, ok = add_error(shim, u, v, x)
        fin = np.isfinite(u) & np.isfinite(v) & np.isfinite(x)
        # Where the integer path applies, the bits agree with the printed sequence.
        assert np.array_equal(y[ok].view(np.uint64), y_ref[ok].view(np.uint64))
        # It declines only for non-finite/overflow-prone or tiny operands.
        big = np.maximum(np.abs(u), np.abs(v))
        small = np.minimum(np.abs(u), np.abs(v))
        expected_decline = ~fin | (big >= 2.0 ** 1023) | ((small < 2.0 ** (110 - 1023)) & (small != 0))
        assert np.array_equal(~ok, expected_decline)
        assert ok.mean() > 0.8


def test_matches_printed_quick_two_sum_when_precondition_holds(shim):
    a, b = inputs(7, 400_000)
    q = np.zeros(a.size, dtype=np.int32)
    shim.quick_exact_batch(a.size, _p(a), _p(b), _p(q))
    q = q.astype(bool)
    x, y_ref = printed_quick_two_sum(a, b)
    y, ok = add_error(shim, a, b, x)
    m = q & ok
    assert m.sum() > 100_000
    assert np.array_equal(y[m].view(np.uint64), y_ref[m].view(np.uint64))


def test_exact_rational_error(shim):
    a, b = inputs(11, 20_000)
    with np.errstate(all="ignore"):
        x = a + b
    y, ok = add_error(shim, a, b, x)
    idx = np.nonzero(ok)[0]
    for i in idx[::7]:
        assert Fraction(float(y[i])) == Fraction(float(a[i])) + Fraction(float(b[i])) - Fraction(float(x[i]))
        assert not (y[i] == 0 and np.signbit(y[i]))        # zero error is +0, as the printed sequence gives


def test_mul_error_matches_two_prod_fma(shim):
    """The integer product error equals fma(a, b, -fl(a*b)) (TwoProdFMA) bit for bit."""
    rng = np.random.default_rng(17)
    n = 400_000
    a = rng.uniform(1, 2, n) * np.exp2(rng.integers(-540, 540, n)) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1, 2, n) * np.exp2(rng.integers(-540, 540, n)) * rng.choice([-1.0, 1.0], n)
    m = rng.integers(0, 6, n)
    b[m == 1] = 1.0 + np.ldexp(rng.integers(0, 2 ** 20, (m == 1).sum()).astype(float), -52)   # short significands
    a[m == 2] = np.round(a[m == 2] * 2 ** 10) / 2 ** 10                                     # exact products
    sp = np.array([0.0, -0.0, 5e-324, 1e-310, 1e308, -1e308, np.inf, np.nan, 1.0, -1.0])
    k = np.nonzero(m == 3)[0]
    b[k] = sp[rng.integers(0, sp.size, k.size)]
    k = np.nonzero(m == 4)[0]                                                               # tiny products
    a[k] = np.exp2(rng.integers(-1022, -500, k.size)) * rng.uniform(1, 2, k.size)
    b[k] = np.exp2(rng.integers(-500, -1, k.size)) * rng.uniform(1, 2, k.size)
    e = np.zeros(n)
    ref = np.zeros(n)
    ok = np.zeros(n, dtype=np.int32)
    with np.errstate(all="ignore"):
        shim.mul_error_batch(n, _p(a), _p(b), _p(e), _p(ref), _p(ok))
    ok = ok.astype(bool)
    assert ok.mean() > 0.7
    assert np.array_equal(e[ok].view(np.uint64), ref[ok].view(np.uint64))


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_integer_add_matches_ieee_addition(shim, seed):
    """add_rn equals the IEEE round-to-nearest-even sum bit for bit (ties, cancellation,
    carries, zeros), declining only for non-finite/overflow-prone/subnormal cases."""
    a, b = inputs(seed, 500_000)
    rng = np.random.default_rng(seed)
    m = rng.integers(0, 4, a.size)
    # exact ties: b = +-(k + 1/2) ulp(a) and carries into a new binade
    k = m == 1
    ulp = np.spacing(np.abs(a[k]))
    b[k] = np.sign(rng.uniform(-1, 1, k.sum())) * ulp * (rng.integers(0, 4, k.sum()) + 0.5)
    k = m == 2
    a[k] = np.nextafter(np.exp2(rng.integers(-100, 100, k.sum())), 0) * rng.choice([-1.0, 1.0], k.sum())
    b[k] = np.spacing(np.abs(a[k])) * rng.uniform(0.1, 3, k.sum()) * np.sign(a[k]) * rng.choice([-1.0, 1.0], k.sum())
    for (u, v) in ((a, b), (b, a)):
        x = np.zeros_like(u)
        ref = np.zeros_like(u)
        ok = np.zeros(u.size, dtype=np.int32)
        with np.errstate(all="ignore"):
            shim.add_rn_batch(u.size, _p(u), _p(v), _p(x), _p(ref), _p(ok))
        ok = ok.astype(bool)
        assert ok.mean() > 0.7
        assert np.array_equal(x[ok].view(np.uint64), ref[ok].view(np.uint64))


@pytest.mark.parametrize("arith,w", [("qtw", 3), ("qdw", 2)])
def test_power_of_two_product_matches_printed_dxmul(shim, orc, arith, w):
    """For a = +-2^k the exact-scaling path equals the printed FP64 x MW product
    (Algorithm 10 / its QDW analogue) of the oracle bit for bit, zero words included."""
    rng = np.random.default_rng(31 + w)
    n = 200_000
    a = np.exp2(rng.integers(-60, 61, n).astype(float)) * rng.choice([-1.0, 1.0], n)
    a[::7] = rng.uniform(1, 2, a[::7].size)                      # non powers of two: declined
    a[::11] = rng.choice([1.0, -1.0, 0.5, -2.0], a[::11].size)
    b = np.empty((w, n))
    b[0] = rng.uniform(-2, 2, n) * np.exp2(rng.integers(-300, 300, n))
    for k in range(1, w):
        b[k] = b[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -53
    z = rng.integers(0, 6, n)
    b[1, z == 1] = 0.0
    b[1, z == 2] = -0.0
    b[w - 1, z == 3] = -0.0
    b[0, z == 4] = -0.0
    b[:, z == 5] *= 2.0 ** 900                                    # near overflow after scaling
    c = np.zeros((w, n))
    ok = np.zeros(n, dtype=np.int32)
    shim.pow2_dx_batch(n, w, _p(a), _p(np.ascontiguousarray(b)), _p(c), _p(ok))
    ok = ok.astype(bool)
    ref = orc.dxmul(arith, a, b)
    assert ok.mean() > 0.5
    assert np.array_equal(c[:, ok].view(np.uint64), ref[:, ok].view(np.uint64))


@pytest.mark.parametrize("arith,w", [("qtw", 3), ("qdw", 2), ("qqw", 4)])
def test_pow2_product_matches_printed_dxmul(shim, orc, arith, w):
    """mwi::pow2_product, the device's FP64 x MW shortcut for power-of-two
    entries, against the oracle's printed product bit for bit: a = +-1 (a sign
    flip per word, valid for subnormal words too) and other powers of two, with
    zero words of either sign, subnormal lower words and words near the range
    edges; non-finite words must decline."""
    rng = np.random.default_rng(41 + w)
    n = 200_000
    a = rng.choice([1.0, -1.0], n)
    m = rng.integers(0, 4, n)
    a[m == 1] = np.exp2(rng.integers(-60, 61, int((m == 1).sum())).astype(float)) * rng.choice([-1.0, 1.0], int((m == 1).sum()))
    a[m == 2] = rng.uniform(1, 2, int((m == 2).sum()))           # not a power of two: declined
    b = np.empty((w, n))
    b[0] = rng.uniform(-2, 2, n) * np.exp2(rng.integers(-300, 300, n))
    for k in range(1, w):
        b[k] = b[k - 1] * rng.uniform(-1, 1, n) * 2.0 ** -53
    z = rng.integers(0, 9, n)
    b[1, z == 1] = 0.0
    b[1, z == 2] = -0.0
    b[w - 1, z == 3] = -0.0
    b[0, z == 4] = -0.0
    b[w - 1, z == 5] = 3e-310 * rng.choice([-1.0, 1.0], int((z == 5).sum()))   # subnormal lower word
    b[:, z == 6] *= 2.0 ** 900                                    # near overflow after scaling
    b[rng.integers(0, w), z == 7] = np.inf
    b[rng.integers(0, w), z == 8] = np.nan
    c = np.zeros((w, n))
    ok = np.zeros(n, dtype=np.int32)
    shim.pow2_product_batch(n, w, _p(a), _p(np.ascontiguousarray(b)), _p(c), _p(ok))
    ok = ok.astype(bool)
    pm1 = np.abs(a) == 1.0
    finite = np.all(np.isfinite(b), axis=0)
    assert np.array_equal(ok[pm1], finite[pm1])                   # +-1: every finite b is taken
    assert not ok[m == 2].any()
    ref = orc.dxmul(arith, a, b)
    assert ok.mean() > 0.5
    assert np.array_equal(c[:, ok].view(np.uint64), ref[:, ok].view(np.uint64))
