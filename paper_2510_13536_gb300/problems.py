"""Seeded synthetic SPD systems in CSR form.

This module builds the inputs that both the CUDA solver and the CPU oracle
consume.  It holds none of the solver's arithmetic: it only lays out sparsity
patterns, draws seeded random coefficients and right-hand sides, and forms
``b = A·1`` where that product is exact by construction (integer stencils,
dyadic weights), which is how the paper builds systems with the known exact
solution ``x* = 1`` (Sec. V-A).

The paper evaluates on SuiteSparse matrices (Table 1) that are not available
here; the generators below are shape analogues of that workload (n of order
10^6, 7 to 1000 nonzeros per row, SPD, stored as general CSR as in Sec. IV-B).

Every generator is deterministic given its seed.  Random numbers come from
``numpy.random.Generator(PCG64(seed))``; uniform doubles are ``random()``,
i.e. ``(u64 >> 11) * 2**-53``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR", "laplacian_2d", "laplacian_3d", "power_law_laplacian", "diffusion_2d",
    "random_spd_small", "rhs_uniform", "rhs_normal", "rhs_ones_exact", "batch_specs",
    "SEED_BASE",
]

# Seeds are SEED_BASE + workload number (1..5), so each workload has its own stream.
SEED_BASE = 20251013


@dataclasses.dataclass
class CSR:
    """A square sparse matrix in compressed-sparse-row form.

    ``row_ptr`` is int64[n+1], ``col`` int32[nnz] (ascending within a row),
    ``val`` float64[nnz].  Symmetric matrices are stored in full (general)
    form, as the paper does (Sec. IV-B).
    """

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            d[i, self.col[s:e]] = self.val[s:e]
        return d

    def with_values(self, val: np.ndarray) -> "CSR":
        return CSR(self.n, self.row_ptr, self.col, np.ascontiguousarray(val, dtype=np.float64), self.name)


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray, name: str) -> CSR:
    """Sort COO triplets by (row, col) and compress; duplicates must not occur."""
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate entries in COO input")
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr, cols.astype(np.int32), vals.astype(np.float64), name)


def _stencil(dims: tuple[int, ...], diag: float, shift: float, name: str) -> CSR:
    """(2d+1)-point Dirichlet Laplacian on a regular grid, row-major (last axis fastest).

    Diagonal ``2·d + shift``, off-diagonals ``-1``.  Entries are generated
    directly in row order, columns ascending, without a sort.
    """
    nd = len(dims)
    n = int(np.prod(dims))
    strides = [int(np.prod(dims[k + 1:])) for k in range(nd)]
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for k in range(nd):
        coords.append(rem // strides[k])
        rem = rem % strides[k]
    # Neighbour offsets in ascending column order: -s0, -s1, ..., -1, 0, +1, ..., +s0
    offs = [-s for s in strides] + [0] + [s for s in reversed(strides)]
    axes = list(range(nd)) + [None] + list(reversed(range(nd)))
    sgn = [-1] * nd + [0] + [1] * nd
    valid = []
    for off, ax, sg in zip(offs, axes, sgn):
        if ax is None:
            valid.append(np.ones(n, dtype=bool))
        else:
            c = coords[ax] + sg
            valid.append((c >= 0) & (c < dims[ax]))
    valid = np.stack(valid, axis=1)                    # [n, 2d+1]
    colmat = idx[:, None] + np.array(offs, dtype=np.int64)[None, :]
    valmat = np.full(valid.shape, -1.0)
    valmat[:, nd] = diag + shift
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = colmat[valid].astype(np.int32)
    val = valmat[valid].astype(np.float64)
    return CSR(n, row_ptr, col, val, name)


def laplacian_2d(m: int, shift: float = 0.0) -> CSR:
    """5-point Dirichlet Laplacian on an m×m grid (n = m², diagonal 4 + shift)."""
    return _stencil((m, m), 4.0, shift, f"lap2d_{m}")


def laplacian_3d(m: int, shift: float = 0.0) -> CSR:
    """7-point Dirichlet Laplacian on an m×m×m grid (n = m³, diagonal 6 + shift)."""
    return _stencil((m, m, m), 6.0, shift, f"lap3d_{m}")


def _truncated_power_law_mean(gamma: float, dmin: float, dmax: float) -> float:
    # Mean of the continuous density ∝ d^-gamma on [dmin, dmax].
    a = 1.0 - gamma
    b = 2.0 - gamma
    z = (dmax ** a - dmin ** a) / a
    m = (dmax ** b - dmin ** b) / b
    return m / z


def power_law_laplacian(n: int, seed: int, mean_deg: float = 30.0, max_deg: float = 1000.0,
                        sigma: float = 2.0, dmin: float = 5.0, shift: float = 1e-8,
                        dyadic: bool = False) -> CSR:
    """Weighted Laplacian of a Chung–Lu power-law graph plus ``shift·I``.

    Expected degrees follow a power law on [dmin, max_deg] whose exponent is
    fitted (bisection) so that the mean is ``mean_deg``.  About
    ``n·mean_deg/2`` edges are drawn with endpoints proportional to the
    expected degrees; self-loops are dropped and repeated pairs merged.  Edge
    weights are lognormal(0, sigma).  Node labels are a random permutation, so
    high-degree rows are spread over the index range.

    ``dyadic=True`` builds the exact-solution twin: weights rounded to the
    2^-20 grid and the shift replaced by 2^-27 (≈7.5e-9), so that every row
    sum is exact and ``b = A·1 = 2^-27·1`` holds without rounding.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = 1.05, 4.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if _truncated_power_law_mean(mid, dmin, max_deg) > mean_deg:
            lo = mid
        else:
            hi = mid
    gamma = 0.5 * (lo + hi)
    # Inverse-CDF sampling of the truncated power law.
    u = rng.random(n)
    a = 1.0 - gamma
    wdeg = (dmin ** a + u * (max_deg ** a - dmin ** a)) ** (1.0 / a)
    wdeg = rng.permutation(wdeg)
    m_edges = int(round(n * mean_deg / 2.0))
    cdf = np.cumsum(wdeg)
    cdf /= cdf[-1]
    src = np.searchsorted(cdf, rng.random(m_edges), side="right")
    dst = np.searchsorted(cdf, rng.random(m_edges), side="right")
    src = np.minimum(src, n - 1)
    dst = np.minimum(dst, n - 1)
    keep = src != dst
    lo_e = np.minimum(src[keep], dst[keep]).astype(np.int64)
    hi_e = np.maximum(src[keep], dst[keep]).astype(np.int64)
    key = np.unique(lo_e * n + hi_e)
    ei, ej = key // n, key % n
    w = rng.lognormal(0.0, sigma, size=key.size)
    if dyadic:
        w = np.maximum(np.round(w * 2.0 ** 20), 1.0) * 2.0 ** -20
        shift = 2.0 ** -27
    deg = np.bincount(ei, weights=w, minlength=n) + np.bincount(ej, weights=w, minlength=n)
    diag = deg + shift
    rows = np.concatenate([ei, ej, np.arange(n)])
    cols = np.concatenate([ej, ei, np.arange(n)])
    vals = np.concatenate([-w, -w, diag])
    A = _from_coo(n, rows, cols, vals, f"powerlaw_{n}{'_dyadic' if dyadic else ''}")
    if dyadic:
        # Row sums must be exact: recompute them in a second order and compare.
        b = rhs_ones_exact(A)
        if not np.all(b == 2.0 ** -27):
            raise AssertionError("dyadic power-law twin lost exactness")
    return A


def _on_grid(v: np.ndarray, e: int = 20) -> np.ndarray:
    """Round to the 2^-e grid (at least one grid step)."""
    return np.maximum(np.round(v * 2.0 ** e), 1.0) * 2.0 ** -e


def diffusion_2d(m: int, seed: int, sigma: float = 1.0, dyadic: bool = False) -> CSR:
    """Cell-centred variable-coefficient diffusion on an m×m grid, 5-point.

    Cell coefficients θ are lognormal(0, sigma).  An interior face between
    cells c and c' has coefficient 2θθ'/(θ+θ') (harmonic mean); a boundary face
    is a Dirichlet face with coefficient θ of its cell.  Row c holds
    ``sum of its face coefficients`` on the diagonal and ``-coefficient`` for
    each interior neighbour, so A is symmetric, irreducibly diagonally
    dominant and SPD.  ``dyadic=True`` rounds every face coefficient to the
    2^-20 grid first, so that the diagonal sums, and A·x for x of ±1, are exact.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.lognormal(0.0, sigma, size=(m, m))
    hx = 2.0 * theta[:, 1:] * theta[:, :-1] / (theta[:, 1:] + theta[:, :-1])   # faces (y, x+1/2)
    hy = 2.0 * theta[1:, :] * theta[:-1, :] / (theta[1:, :] + theta[:-1, :])   # faces (y+1/2, x)
    if dyadic:
        hx, hy, theta = _on_grid(hx), _on_grid(hy), _on_grid(theta)
    diag = np.zeros((m, m))
    diag[:, 1:] += hx
    diag[:, :-1] += hx
    diag[1:, :] += hy
    diag[:-1, :] += hy
    diag[:, 0] += theta[:, 0]
    diag[:, -1] += theta[:, -1]
    diag[0, :] += theta[0, :]
    diag[-1, :] += theta[-1, :]
    n = m * m
    idx = np.arange(n).reshape(m, m)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [diag.ravel()]
    # x-faces
    rows += [idx[:, :-1].ravel(), idx[:, 1:].ravel()]
    cols += [idx[:, 1:].ravel(), idx[:, :-1].ravel()]
    vals += [-hx.ravel(), -hx.ravel()]
    # y-faces
    rows += [idx[:-1, :].ravel(), idx[1:, :].ravel()]
    cols += [idx[1:, :].ravel(), idx[:-1, :].ravel()]
    vals += [-hy.ravel(), -hy.ravel()]
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), f"diffusion2d_{m}")


def convection_diffusion_2d(m: int, beta: float = 1.0, shift: float = 0.0) -> CSR:
    """Nonsymmetric 2-D convection-diffusion on an m x m grid: the 5-point
    Laplacian plus first-order upwind convection with velocity (1, 1), scaled
    so that each row gains ``beta`` on the diagonal and on its west and south
    couplings (``beta`` = mesh Peclet number).  Row (y, x): diagonal
    4 + 2 beta + shift, west -1 - beta, south -1 - beta, east and north -1,
    couplings across the Dirichlet boundary dropped.  A nonsingular M-matrix;
    dyadic beta keeps every entry, and A x for x of +-1, exact."""
    n = m * m
    idx = np.arange(n).reshape(m, m)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 4.0 + 2.0 * beta + shift)]
    for (dy, dx), w in (((0, -1), -1.0 - beta), ((-1, 0), -1.0 - beta), ((0, 1), -1.0), ((1, 0), -1.0)):
        ys, xs = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        ok = (ys + dy >= 0) & (ys + dy < m) & (xs + dx >= 0) & (xs + dx < m)
        rows.append(idx[ok])
        cols.append(idx[(ys + dy)[ok], (xs + dx)[ok]])
        vals.append(np.full(int(ok.sum()), w))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     f"convdiff2d_{m}_{beta:g}")


def random_spd_small(n: int, seed: int, density: float = 0.3, shift_exp: int = -6) -> CSR:
    """Small SPD matrix with dyadic entries (tests with a dense exact solve).

    A random graph Laplacian with integer weights 1..8 plus a diagonal shift
    of ``k·2**shift_exp`` (k in 1..4) per row: irreducibly diagonally
    dominant, hence SPD, with every entry exactly representable so that
    rational arithmetic sees the same matrix.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < density or j == i + 1:
                w = float(rng.integers(1, 9))
                rows += [i, j]
                cols += [j, i]
                vals += [-w, -w]
                diag[i] += w
                diag[j] += w
    diag += rng.integers(1, 5, size=n) * 2.0 ** shift_exp
    rows += list(range(n))
    cols += list(range(n))
    vals += list(diag)
    return _from_coo(n, np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64),
                     np.array(vals), f"spd_small_{n}_{seed}")


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """b_i = 2U - 1 with U uniform on [0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 2.0 * rng.random(n) - 1.0


def rhs_normal(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


def rhs_ones_exact(A: CSR) -> np.ndarray:
    """b = A·1 as exact row sums (exact set-up value, not solver arithmetic).

    Uses ``math.fsum`` per row, which returns the correctly rounded sum; the
    generators above only call this where that sum is representable, so the
    result is exact and ``x* = 1`` solves ``A x = b`` exactly.
    """
    out = np.empty(A.n)
    rp, v = A.row_ptr, A.val
    lens = np.diff(rp)
    # Fast path: integer entries below 2^20 in rows shorter than 2^20 have all
    # partial sums below 2^40, so plain float64 summation is exact.
    if v.size and np.all(v == np.round(v)) and np.max(np.abs(v)) < 2.0 ** 20 and lens.max() < 2 ** 20:
        out[:] = 0.0
        nz = lens > 0
        out[nz] = np.add.reduceat(v, rp[:-1][nz])
        return out
    for i in range(A.n):
        out[i] = math.fsum(v[rp[i]:rp[i + 1]].tolist())
    return out


def batch_specs(nsys: int, seed: int, nmin: int = 1000, nmax: int = 200000):
    """Specifications of a batch of independent Laplacian systems.

    Each system: size U[nmin, nmax]; a 2-D 5-point (m = round(√n)) or a 3-D
    7-point (m = round(∛n)) Dirichlet Laplacian by a fair coin; a diagonal
    shift log-uniform in [1e-6, 1e-2]; arithmetic QDW or QTW by a fair coin;
    b = 2U - 1 with its own seed.  Returns a list of dicts (kind, m, shift,
    arith, rhs_seed); build them with :func:`build_batch_system`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for s in range(nsys):
        nn = int(rng.integers(nmin, nmax + 1))
        three_d = bool(rng.random() < 0.5)
        m = int(round(nn ** (1.0 / 3.0))) if three_d else int(round(math.sqrt(nn)))
        shift = float(10.0 ** rng.uniform(-6.0, -2.0))
        arith = "qtw" if rng.random() < 0.5 else "qdw"
        specs.append(dict(kind="3d" if three_d else "2d", m=m, shift=shift, arith=arith,
                          rhs_seed=seed * 1000 + s))
    return specs


def build_batch_system(spec) -> tuple[CSR, np.ndarray]:
    A = laplacian_3d(spec["m"], spec["shift"]) if spec["kind"] == "3d" else laplacian_2d(spec["m"], spec["shift"])
    return A, rhs_uniform(A.n, spec["rhs_seed"])


# ---------------------------------------------------------------------------
# Named workloads (the five configurations the solver is measured on).
# ---------------------------------------------------------------------------
WORKLOADS = {
    "c1": "2-D Poisson 5-point, 64x64 (n=4096), b = A*1, x0 = 0, tol 1e-12, maxit 2000",
    "c2": "3-D Poisson 7-point, 128^3 (n=2,097,152), b = 2U-1, x0 = 0, tol 1e-14, maxit 20000",
    "c2_twin": "3-D Poisson 7-point, 128^3, b = A*1 (x* = 1), x0 = 0, tol 1e-14, maxit 20000",
    "c3": "power-law graph Laplacian n=1e6, mean degree 30, max 1000, weights lognormal(0,2), +1e-8 I, b ~ N(0,1)",
    "c3_twin": "dyadic power-law twin n=1e6 (weights on 2^-20 grid, shift 2^-27), b = A x* exactly, x* random +-1",
    "c5": "2-D variable-coefficient diffusion 512x512, theta lognormal(0,1), b, w ~ N(0,1)",
}


def workload(name: str):
    """(A, b, tol, maxit) of a named workload; see WORKLOADS."""
    if name == "c1":
        A = laplacian_2d(64)
        return A, rhs_ones_exact(A), 1e-12, 2000
    if name == "c2":
        A = laplacian_3d(128)
        return A, rhs_uniform(A.n, SEED_BASE + 2), 1e-14, 20000
    if name == "c2_twin":
        A = laplacian_3d(128)
        return A, rhs_ones_exact(A), 1e-14, 20000
    if name == "c3":
        A = power_law_laplacian(1_000_000, SEED_BASE + 3)
        return A, rhs_normal(A.n, SEED_BASE + 3 + 100), 1e-14, 20000
    if name == "c3_twin":
        # x* = 1 is an eigenvector of a shifted Laplacian (CG would finish in one
        # step), so the exact solution is a seeded random sign vector instead.
        A = power_law_laplacian(1_000_000, SEED_BASE + 3, dyadic=True)
        xs = random_signs(A.n, SEED_BASE + 3 + 200)
        return A, matvec_exact(A, xs), 1e-14, 20000
    if name == "c5":
        A = diffusion_2d(512, SEED_BASE + 5)
        return A, rhs_normal(A.n, SEED_BASE + 5 + 100), 1e-20, 20000
    raise KeyError(name)


def matvec_grid_exact(A: CSR, x: np.ndarray, e: int = 20) -> np.ndarray:
    """b = A x for entries on the 2^-e grid and x of ±1, summed in FP64.

    Every product is a multiple of 2^-e, so a row sum is exact when the sum
    of the products' magnitudes stays below 2^(53-e); that is checked."""
    prod = A.val * x[A.col]
    if not np.all(np.round(prod * 2.0 ** e) == prod * 2.0 ** e):
        raise ValueError("entries are not on the 2^-e grid")
    starts = A.row_ptr[:-1]
    nonempty = A.row_ptr[1:] > starts
    mag = np.zeros(A.n)
    out = np.zeros(A.n)
    if A.nnz:
        mag[nonempty] = np.add.reduceat(np.abs(prod), starts[nonempty])
        out[nonempty] = np.add.reduceat(prod, starts[nonempty])
    if np.any(mag >= 2.0 ** (53 - e)):
        raise ValueError("row sums could round")
    return out


NORM_SYSTEMS = {
    "norm_poisson": "3-D Poisson 7-point 128^3, x* random +-1, b = A x* (integers, exact)",
    "norm_diffusion": "2-D diffusion 256^2, theta lognormal(0,1), coefficients on the 2^-20 grid, "
                      "x* random +-1, b = A x* (exact)",
}


def exact_solution_system(name: str):
    """(A, b, x*) with b = A x* exactly, for the normalisation-policy sweep."""
    if name == "norm_poisson":
        A = laplacian_3d(128)
        xs = random_signs(A.n, SEED_BASE + 6)
    elif name == "norm_diffusion":
        A = diffusion_2d(256, SEED_BASE + 7, dyadic=True)
        xs = random_signs(A.n, SEED_BASE + 7 + 200)
    else:
        raise KeyError(name)
    return A, matvec_grid_exact(A, xs), xs


def random_signs(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(np.array([-1.0, 1.0]), size=n)


def matvec_exact(A: CSR, x: np.ndarray) -> np.ndarray:
    """b = A x as correctly rounded row sums (math.fsum); exact when every
    product a_ij x_j is exact and the row sum is representable (dyadic entries,
    x of +-1), as for the power-law twin.  Set-up value, not solver arithmetic."""
    out = np.empty(A.n)
    prod = A.val * x[A.col]
    rp = A.row_ptr
    for i in range(A.n):
        out[i] = math.fsum(prod[rp[i]:rp[i + 1]].tolist())
    return out


def c5_loss_weights(n: int) -> np.ndarray:
    """w of the loss L = w^T x of the differentiable-solve workload."""
    return rhs_normal(n, SEED_BASE + 5 + 200)
