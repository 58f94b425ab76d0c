"""Exact-rational helpers for pinning the oracle (no FP64 solver arithmetic here).

Multi-word values are read as the exact rational sum of their words; error
bounds are then checked in exact arithmetic with ``fractions.Fraction``.
"""
from __future__ import annotations

import math
import random
from fractions import Fraction

import numpy as np

U = Fraction(1, 2 ** 53)      # unit round-off of FP64 (Sec. III)


def val(words) -> Fraction:
    return sum((Fraction(float(w)) for w in words), Fraction(0))


def col(arr, i):
    """Words of element i of a (w, n) SoA array."""
    return [float(arr[k, i]) for k in range(arr.shape[0])]


def split(v: Fraction, w: int) -> list[float]:
    """Nearest-rounding expansion: word k = fl(v - sum of the previous words)."""
    out = []
    rem = v
    for _ in range(w):
        x = float(rem)          # correctly rounded conversion of a rational
        out.append(x)
        rem -= Fraction(x)
    return out


def rand_value(rng: random.Random, bits: int = 220, emin: int = -30, emax: int = 30,
               signed: bool = True) -> Fraction:
    m = rng.getrandbits(bits) | (1 << (bits - 1))
    e = rng.randint(emin, emax)
    v = Fraction(m, 1 << bits) * Fraction(2) ** e
    if signed and rng.random() < 0.5:
        v = -v
    return v


def rand_mw(rng: random.Random, n: int, w: int, **kw) -> np.ndarray:
    """(w, n) array of nearest-rounding expansions of random ~220-bit values."""
    out = np.empty((w, n))
    for i in range(n):
        out[:, i] = split(rand_value(rng, **kw), w)
    return out


def rel_err(approx: Fraction, exact: Fraction) -> Fraction:
    if exact == 0:
        return abs(approx)
    return abs(approx - exact) / abs(exact)


def ulp(x: float) -> float:
    return math.ulp(x)


def dense_fraction(A) -> list[list[Fraction]]:
    """Dense exact copy of a CSR matrix (entries are FP64, hence exact rationals)."""
    M = [[Fraction(0)] * A.n for _ in range(A.n)]
    for i in range(A.n):
        for k in range(int(A.row_ptr[i]), int(A.row_ptr[i + 1])):
            M[i][int(A.col[k])] = Fraction(float(A.val[k]))
    return M


def solve_exact(M, b) -> list[Fraction]:
    """Gaussian elimination in exact rationals (SPD, so no pivoting needed)."""
    n = len(M)
    A = [row[:] + [Fraction(float(b[i]))] for i, row in enumerate(M)]
    for k in range(n):
        piv = A[k][k]
        for i in range(k + 1, n):
            if A[i][k] != 0:
                f = A[i][k] / piv
                for j in range(k, n + 1):
                    A[i][j] -= f * A[k][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = A[i][n] - sum(A[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / A[i][i]
    return x


def cg_exact(M, b, iters: int):
    """Textbook CG (x0 = 0) in exact rationals; returns the list of iterates x_1..x_k
    and residual norms squared rho_1..rho_k."""
    n = len(M)
    x = [Fraction(0)] * n
    r = [Fraction(float(v)) for v in b]
    p = r[:]
    rho = sum(v * v for v in r)
    xs, rhos = [], []
    for _ in range(iters):
        q = [sum(M[i][j] * p[j] for j in range(n) if M[i][j] != 0) for i in range(n)]
        alpha = rho / sum(p[i] * q[i] for i in range(n))
        x = [x[i] + alpha * p[i] for i in range(n)]
        r = [r[i] - alpha * q[i] for i in range(n)]
        rho1 = sum(v * v for v in r)
        xs.append(x[:])
        rhos.append(rho1)
        if rho1 == 0:
            break
        beta = rho1 / rho
        p = [r[i] + beta * p[i] for i in range(n)]
        rho = rho1
    return xs, rhos


def fnorm(v) -> float:
    import mpmath
    mpmath.mp.prec = 400
    return float(mpmath.sqrt(sum(mpmath.mpf(x.numerator) / x.denominator * mpmath.mpf(x.numerator) / x.denominator
                                 for x in v)))


def pcg_exact(M, b, w, iters: int):
    """Textbook preconditioned CG (x0 = 0, M^-1 = diag(w)) in exact rationals;
    w holds FP64 numbers, taken exactly.  Returns the iterates x_1..x_k and
    the squared residual norms r_k^T r_k."""
    n = len(M)
    wf = [Fraction(float(v)) for v in w]
    x = [Fraction(0)] * n
    r = [Fraction(float(v)) for v in b]
    z = [wf[i] * r[i] for i in range(n)]
    p = z[:]
    rho = sum(r[i] * z[i] for i in range(n))
    xs, rrs = [], []
    for _ in range(iters):
        q = [sum(M[i][j] * p[j] for j in range(n) if M[i][j] != 0) for i in range(n)]
        alpha = rho / sum(p[i] * q[i] for i in range(n))
        x = [x[i] + alpha * p[i] for i in range(n)]
        r = [r[i] - alpha * q[i] for i in range(n)]
        z = [wf[i] * r[i] for i in range(n)]
        rho1 = sum(r[i] * z[i] for i in range(n))
        xs.append(x[:])
        rrs.append(sum(v * v for v in r))
        if rho1 == 0:
            break
        beta = rho1 / rho
        p = [z[i] + beta * p[i] for i in range(n)]
        rho = rho1
    return xs, rrs


def bicgstab_exact(M, b, iters: int):
    """Textbook BiCGStab (x0 = 0, shadow residual r0) in exact rationals.
    Returns the iterates x_1..x_k (stops early when s or r becomes zero)."""
    n = len(M)

    def matvec(v):
        return [sum(M[i][j] * v[j] for j in range(n) if M[i][j] != 0) for i in range(n)]

    def dot(u, v):
        return sum(u[i] * v[i] for i in range(n))

    x = [Fraction(0)] * n
    r = [Fraction(float(v)) for v in b]
    rh = r[:]
    rho = dot(rh, r)
    p = v = None
    rho_prev = alpha = omega = None
    xs = []
    for k in range(iters):
        if k == 0:
            p = r[:]
        else:
            beta = (rho / rho_prev) * (alpha / omega)
            p = [r[i] + beta * (p[i] - omega * v[i]) for i in range(n)]
        v = matvec(p)
        alpha = rho / dot(rh, v)
        s = [r[i] - alpha * v[i] for i in range(n)]
        if all(e == 0 for e in s):
            xs.append([x[i] + alpha * p[i] for i in range(n)])
            break
        t = matvec(s)
        omega = dot(t, s) / dot(t, t)
        x = [x[i] + alpha * p[i] + omega * s[i] for i in range(n)]
        r = [s[i] - omega * t[i] for i in range(n)]
        xs.append(x[:])
        rho_prev, rho = rho, dot(rh, r)
        if all(e == 0 for e in r):
            break
    return xs
