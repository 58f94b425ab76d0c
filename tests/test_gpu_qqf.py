"""QQF and QF (four FP32 words, scaled CG) on the CUDA path vs the oracle, bit for bit.

The word algebra (add, mul, FP64 x QQF through the exact three-word split,
division, VecSum4, collapse), the SpMV and dot, and the solver on the CUDA
graph and on host-launched kernels, including right-hand sides far outside
FP32's range (the power-of-two scaling of r and p) and the special cases.
Every test runs for QQF and for QF (QQF renormalised after every operation),
except the QQF breakdown and its QF counterpart.
"""
import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["qqf", "qf"])
def ar(request):
    return request.param


@pytest.fixture(scope="module")
def mw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_13536_gb300 import build, solver
    build.build()
    return solver


def same_bits(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    if not np.array_equal(na, nb):
        return False
    return np.array_equal(a.view(np.uint64)[~na], b.view(np.uint64)[~nb])


def dev(x, dtype=np.float64):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=dtype), device="cuda")


def rand_qqf(rng, n, emin=-20, emax=20):
    """(4, n) FP32 expansions with non-overlapping words (float64 holding FP32 values)."""
    w = np.empty((4, n), dtype=np.float32)
    w[0] = (rng.uniform(1, 2, n) * rng.choice([-1, 1], n) * 2.0 ** rng.integers(emin, emax, n)).astype(np.float32)
    for k in range(1, 4):
        w[k] = (w[k - 1].astype(np.float64) * 2.0 ** -24 * rng.uniform(-1, 1, n)).astype(np.float32)
    return w.astype(np.float64)


def test_word_ops_bit_exact(mw, orc, ar):
    rng = np.random.default_rng(61)
    n = 5000
    a, b = rand_qqf(rng, n), rand_qqf(rng, n)
    b[:, :7] = 0.0
    b[0, :7] = [1.0, -1.0, 2.0 ** -60, 3.0, 0.5, 2.0 ** 60, 1.5]
    for op in ("add", "mul", "div"):
        g = mw.word_op(op, ar, dev(a, np.float32), dev(b, np.float32)).cpu().numpy()
        assert g.dtype == np.float32 and g.shape == (4, n)
        assert same_bits(g, getattr(orc, op)(ar, a, b)), op
    g = mw.word_op("normalize", ar, dev(a, np.float32)).cpu().numpy()
    assert same_bits(g, orc.normalize(ar, a))
    g = mw.word_op("collapse", ar, dev(a, np.float32)).cpu().numpy()
    assert same_bits(g, orc.collapse(ar, a))
    # FP64 x QQF over the split's fast range, its edges and the rounding path.
    s = rng.uniform(1, 2, n) * rng.choice([-1, 1], n) * 2.0 ** rng.integers(-100, 128, n)
    s[:12] = [0.0, -0.0, 5e-310, -3.3e-320, 2.0 ** -97, -2.0 ** -97 * 1.75, 2.0 ** -98, 1.3 * 2.0 ** -100,
              -7.1e-35, 2.0 ** 127 * 1.999, 1.0, -1.0]
    g = mw.word_op("dxmul", ar, dev(s), dev(b, np.float32)).cpu().numpy()
    assert same_bits(g, orc.dxmul(ar, s, b))


def test_pow2_product_bit_exact(mw, orc, ar):
    """FP64 x QQF with power-of-two entries, which the device reduces to four
    exact FP32 scalings when every product is a normal number: against the
    full product of the oracle, over zero lower words of either sign,
    subnormal words, products that leave FP32's normal range and entries at
    and beyond the edges of that range."""
    rng = np.random.default_rng(64)
    n = 6000
    b = rand_qqf(rng, n, emin=-140, emax=127)
    z = rng.integers(0, 8, n)
    for k in range(1, 4):                                   # zero lower words, both signs
        m = z == k
        b[k:, m] = 0.0
        b[k, m & (rng.integers(0, 2, n) == 1)] = -0.0
    b[0, z == 4] = rng.choice([0.0, -0.0], int((z == 4).sum()))
    sub = z == 5                                            # a subnormal lower word
    b[3, sub] = np.float32(1e-42) * rng.choice([-1, 1], int(sub.sum()))
    e = rng.integers(-140, 140, n)
    s = rng.choice([-1.0, 1.0], n) * 2.0 ** e.astype(np.float64)
    s[:10] = [1.0, -1.0, 2.0 ** -126, -2.0 ** -127, 2.0 ** 127, 2.0 ** 128, -2.0 ** -97, 2.0 ** -98, 0.5, 4.0]
    s[10:20] = [1.0, -1.0, 1.0, -1.0, 2.0, 1.0, -1.0, 0.25, 1.0, -1.0]   # non-finite words of b below
    b[:, 10:20] = 1.0
    b[0, 10], b[1, 11], b[2, 12], b[3, 13], b[1, 14] = np.inf, -np.inf, np.nan, np.inf, np.nan
    b[0, 15], b[3, 16], b[1, 17] = -np.inf, np.nan, np.inf
    g = mw.word_op("dxmul", ar, dev(s), dev(b, np.float32)).cpu().numpy()
    assert same_bits(g, orc.dxmul(ar, s, b))


def test_spmv_and_dot(mw, orc, ar):
    rng = np.random.default_rng(62)
    for A, plan in ((P.power_law_laplacian(4000, seed=3, mean_deg=12, max_deg=300), None),
                    (P.laplacian_3d(16, 1e-3), (2, 256, 37))):
        M = mw.CSRMatrix.from_csr(A)
        if plan:
            M.plan = plan
        p = rand_qqf(rng, A.n, -3, 3)
        q = mw.spmv(M, ar, dev(p, np.float32)).cpu().numpy()
        assert same_bits(q, orc.spmv(ar, A, p, V=M.plan[0])), A.name
    u, v = rand_qqf(rng, 70001, -4, 4), rand_qqf(rng, 70001, -4, 4)
    for G in (1, 37, 456):
        g = mw.dot(ar, dev(u, np.float32), dev(v, np.float32), G)
        assert same_bits(g, orc.dot(ar, u, v, R=256, G=G)), G


def _check(mw, orc, M, A, b, tol, maxit, tag, x0=None, ar="qqf"):
    r = mw.solve(M, dev(b), ar, tol, maxit, history=True, x0=None if x0 is None else dev(x0, np.float32))
    xo, ito, rro, sto, ho = orc.cg(ar, A, b, x0=x0, tol=tol, maxit=maxit, plan=M.plan, history=True)
    assert (r.iters, r.status) == (ito, sto), (tag, r.iters, ito, r.status, sto)
    assert same_bits(np.array([r.relres]), np.array([rro])), (tag, r.relres, rro)
    assert r.x.dtype.is_floating_point and r.x.shape == (4, A.n)
    assert same_bits(r.x.cpu().numpy(), xo), tag
    if r.iters:
        assert same_bits(r.history.cpu().numpy(), ho), tag
    return r


def test_cg_graph_path(mw, orc, ar):
    for A, seed, tol, maxit in ((P.laplacian_3d(24, 1e-3), 71, 1e-22, 300),
                                (P.diffusion_2d(90, 3), 72, 1e-20, 800),
                                (P.power_law_laplacian(5000, seed=7, mean_deg=12, max_deg=300), 73, 1e-20, 300)):
        b = P.rhs_uniform(A.n, seed)
        M = mw.CSRMatrix.from_csr(A)
        r = _check(mw, orc, M, A, b, tol, maxit, A.name, ar=ar)
        assert r.iters > 20
        M.plan = (2, 256, 37)
        _check(mw, orc, M, A, b, tol, maxit, A.name + " V=2", ar=ar)


def test_breakdown_on_cancelling_power_law(mw, orc):
    """QQF's known failure: on a 2000-node power-law graph Laplacian whose rows
    cancel strongly, its ~96 bits run out and p^T q loses its sign near
    iteration 800.  The GPU takes the breakdown path at the oracle's iteration,
    with the oracle's residual and solution bits."""
    A = P.power_law_laplacian(2000, seed=7, mean_deg=12, max_deg=300)
    b = P.rhs_uniform(A.n, 32)
    M = mw.CSRMatrix.from_csr(A)
    r = _check(mw, orc, M, A, b, 1e-14, 2000, "power-law 2000")
    assert r.status == 2 and r.iters > 700, (r.status, r.iters)


def test_qf_converges_where_qqf_breaks_down(mw, orc):
    """The same system in QF (every result renormalised): it converges, with
    the oracle's iteration count, residual and solution bits."""
    A = P.power_law_laplacian(2000, seed=7, mean_deg=12, max_deg=300)
    b = P.rhs_uniform(A.n, 32)
    M = mw.CSRMatrix.from_csr(A)
    r = _check(mw, orc, M, A, b, 1e-14, 4000, "power-law 2000", ar="qf")
    assert r.status == 0, (r.status, r.iters)


def test_eager_launches(mw, orc, ar, monkeypatch):
    monkeypatch.setenv("MWCG_EAGER", "1")
    A = P.diffusion_2d(60, 4)
    b = P.rhs_uniform(A.n, 74)
    M = mw.CSRMatrix.from_csr(A)
    _check(mw, orc, M, A, b, 1e-20, 400, "eager", ar=ar)


def test_small_systems_one_cluster(mw, orc, ar):
    """Systems small enough for the one-cluster launch (plan G = the cluster
    size): the cluster solve of the scaled iteration, CG and Jacobi PCG, equals
    the oracle in that plan, history included."""
    for A in (P.laplacian_2d(40), P.laplacian_2d(5), P.random_spd_small(9, seed=3)):
        b = P.rhs_uniform(A.n, 75)
        M = mw.CSRMatrix.from_csr(A)
        _check(mw, orc, M, A, b, 1e-22, 400, A.name, ar=ar)
        M.preconditioner = "jacobi"
        _check_pcg(mw, orc, M, A, b, 1e-22, 400, A.name + " pcg", ar)


def test_scaling_far_outside_fp32_range(mw, orc, ar):
    """b 2^k with |k| > 126: E0 takes the FP64 route of the word scaling;
    the iterations, residuals and history equal the unscaled problem's while
    x (unscaled FP32 words) stays in FP32's range.  At k = -300 the whole
    solution is below FP32's normal range and at k = +300 it overflows at the
    first update: the solve then reports MWCG_OUT_OF_RANGE (4), not success."""
    A = P.laplacian_3d(20, 1e-3)
    b = P.rhs_uniform(A.n, 76)
    M = mw.CSRMatrix.from_csr(A)
    r0 = _check(mw, orc, M, A, b, 1e-22, 300, "k=0", ar=ar)
    assert r0.status == 0
    for k in (-300, -40, 90):
        r = _check(mw, orc, M, A, b * 2.0 ** k, 1e-22, 300, f"k={k}", ar=ar)
        assert (r.iters, r.relres) == (r0.iters, r0.relres), k
        assert same_bits(r.history.cpu().numpy(), r0.history.cpu().numpy()), k
        assert r.status == (4 if k == -300 else 0), (k, r.status)
    r = _check(mw, orc, M, A, b * 2.0 ** 300, 1e-22, 300, "k=300", ar=ar)
    assert (r.status, r.iters) == (4, 1)
    assert same_bits(r.history.cpu().numpy(), r0.history.cpu().numpy()[:1])


def test_nonzero_x0_and_limits(mw, orc, ar):
    A = P.diffusion_2d(50, 6)
    b = P.rhs_uniform(A.n, 77)
    M = mw.CSRMatrix.from_csr(A)
    rng = np.random.default_rng(78)
    x0 = rand_qqf(rng, A.n, -2, 2)
    _check(mw, orc, M, A, b, 1e-20, 500, "x0", x0=x0, ar=ar)
    _check(mw, orc, M, A, b, 1e-300, 7, "maxit", ar=ar)
    _check(mw, orc, M, A, b, 0.0, 3, "tol 0", ar=ar)


def test_special_cases(mw, orc, ar):
    A = P.laplacian_2d(30)
    M = mw.CSRMatrix.from_csr(A)
    r = mw.solve(M, dev(np.zeros(A.n)), ar, 1e-10, 50, x0=dev(np.ones((4, A.n)), np.float32))
    assert (r.iters, r.status, r.relres) == (0, 0, 0.0) and np.all(r.x.cpu().numpy() == 0)
    b = P.matvec_exact(A, np.ones(A.n))
    x0 = np.zeros((4, A.n))
    x0[0] = 1.0
    r = mw.solve(M, dev(b), ar, 1e-10, 50, x0=dev(x0, np.float32))       # r0 = 0 exactly
    assert (r.iters, r.status, r.relres) == (0, 0, 0.0) and np.array_equal(r.x.cpu().numpy(), x0)
    r = mw.solve(M, dev(b), ar, 1e-10, 0)
    xo, ito, rro, sto = orc.cg(ar, A, b, tol=1e-10, maxit=0, plan=M.plan)
    assert (r.iters, r.status) == (ito, sto) == (0, 1) and r.relres == rro
    one = P.CSR(1, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([3.0]))
    M1 = mw.CSRMatrix.from_csr(one)
    _check(mw, orc, M1, one, np.array([1.0]), 1e-30, 5, "n=1", ar=ar)
    E = P.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    r = mw.solve(mw.CSRMatrix.from_csr(E), dev(np.zeros(0)), ar, 1e-10, 10)
    assert (r.iters, r.status, r.relres) == (0, 0, 0.0) and tuple(r.x.shape) == (4, 0)


def test_host_buffers(mw, orc, ar):
    A = P.diffusion_2d(40, 8)
    b = P.rhs_uniform(A.n, 79)
    M = mw.CSRMatrix.from_csr(A)
    x, it, rr, st = mw.solve_host(M, b, ar, 1e-20, 400)
    xo, ito, rro, sto = orc.cg(ar, A, b, tol=1e-20, maxit=400, plan=M.plan)
    assert (it, st) == (ito, sto) and x.dtype == np.float32 and same_bits(x, xo)


def test_adjoint_bit_exact(mw, orc, ar):
    """lambda (the scaled CG on dL/dx), g_b = collapse(lambda) and
    g_val = -collapse(lambda_i x_j) equal the oracle's bit for bit, through the
    C ABI and through autograd."""
    import torch
    A = P.diffusion_2d(48, 9)
    b = P.rhs_uniform(A.n, 81)
    w = np.random.default_rng(82).standard_normal(A.n)
    M = mw.CSRMatrix.from_csr(A)
    r = mw.solve(M, dev(b), ar, 1e-20, 2000)
    xo, ito, _, sto = orc.cg(ar, A, b, tol=1e-20, maxit=2000, plan=M.plan)
    assert (r.iters, r.status) == (ito, sto) == (ito, 0) and same_bits(r.x.cpu().numpy(), xo)
    g_b, g_val, it, rr, st = mw.adjoint(M, r.x, dev(w), ar, 1e-20, 2000)
    ob, ov, lam, oit, orr, ost = orc.adjoint(ar, A, xo, w, 1e-20, 2000, plan=M.plan)
    assert (it, st) == (oit, ost) and st == 0
    assert same_bits(np.array([rr]), np.array([orr]))
    assert same_bits(g_b.cpu().numpy(), ob) and same_bits(g_val.cpu().numpy(), ov)
    vals = torch.tensor(A.val, dtype=torch.float64, device="cuda", requires_grad=True)
    bb = torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True)
    x = mw.solve_differentiable(M, vals, bb, ar, 1e-20, 2000)
    (x * dev(w)).sum().backward()
    assert same_bits(vals.grad.cpu().numpy(), ov) and same_bits(bb.grad.cpu().numpy(), ob)


def _check_pcg(mw, orc, M, A, b, tol, maxit, tag, ar):
    r = mw.solve(M, dev(b), ar, tol, maxit, history=True)
    xo, ito, rro, sto, ho = orc.cg(ar, A, b, tol=tol, maxit=maxit, plan=M.plan, precond="jacobi", history=True)
    assert (r.iters, r.status) == (ito, sto), (tag, r.iters, ito, r.status, sto)
    assert same_bits(np.array([r.relres]), np.array([rro])), tag
    assert same_bits(r.x.cpu().numpy(), xo), tag
    if r.iters:
        assert same_bits(r.history.cpu().numpy(), ho), tag
    return r


def test_jacobi_pcg_bit_exact(mw, orc, ar, monkeypatch):
    """Jacobi PCG in FP32 words (the scaled iteration, z~ = w (x) r~ into q,
    the shift and the stop test from the FP64 residual sum) equals the
    oracle's bit for bit: iterations, status, residual history and x, on the
    graph and on host-launched kernels; a bad diagonal gives status 3."""
    cases = ((P.diffusion_2d(48, 9), 83, 1e-20, 2000),
             (P.power_law_laplacian(3000, seed=7, mean_deg=12, max_deg=300), 84, 1e-14, 3000),
             (P.laplacian_3d(24, 1e-3), 85, 1e-22, 300))
    for A, seed, tol, maxit in cases:
        b = P.rhs_uniform(A.n, seed)
        M = mw.CSRMatrix.from_csr(A)
        M.preconditioner = "jacobi"
        r = _check_pcg(mw, orc, M, A, b, tol, maxit, A.name, ar)
        assert r.iters > 10
    A, seed, tol, maxit = cases[0]
    b = P.rhs_uniform(A.n, seed)
    monkeypatch.setenv("MWCG_EAGER", "1")
    M = mw.CSRMatrix.from_csr(A)
    M.preconditioner = "jacobi"
    _check_pcg(mw, orc, M, A, b, tol, maxit, "eager", ar)
    monkeypatch.delenv("MWCG_EAGER")
    B = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    B.val[[k for k in range(B.row_ptr[7], B.row_ptr[8]) if B.col[k] == 7][0]] = -1.0
    MB = mw.CSRMatrix.from_csr(B)
    MB.preconditioner = "jacobi"
    r = mw.solve(MB, dev(b), ar, tol, maxit)
    assert (r.status, r.iters) == (3, 0)


def test_jacobi_pcg_adjoint_bit_exact(mw, orc, ar):
    A = P.diffusion_2d(40, 10)
    b = P.rhs_uniform(A.n, 86)
    w = np.random.default_rng(87).standard_normal(A.n)
    M = mw.CSRMatrix.from_csr(A)
    M.preconditioner = "jacobi"
    r = mw.solve(M, dev(b), ar, 1e-20, 2000)
    assert r.status == 0
    g_b, g_val, it, rr, st = mw.adjoint(M, r.x, dev(w), ar, 1e-20, 2000)
    ob, ov, lam, oit, orr, ost = orc.adjoint(ar, A, r.x.cpu().numpy().astype(np.float64), w, 1e-20, 2000,
                                             plan=M.plan, precond="jacobi")
    assert (it, st) == (oit, ost) == (oit, 0)
    assert same_bits(g_b.cpu().numpy(), ob) and same_bits(g_val.cpu().numpy(), ov)


def test_batched_bit_exact(mw, orc, ar):
    """The persistent batched kernel runs QQF / QF with the scaled iteration:
    every system equals the oracle's solve in plan {V, 256, cluster size}, bit
    for bit, beside a DW system of the same batch (another word group, launched
    concurrently): CG and Jacobi PCG, b = 0, a maxit stop, a breakdown (QQF on
    the cancelling power-law graph) and x leaving FP32's range (status 4)."""
    import torch
    rng = np.random.default_rng(91)
    specs = []                        # (A, b, arith, tol, maxit, preconditioner)
    for k in range(10):
        kind = k % 3
        if kind == 0:
            A = P.laplacian_2d(int(rng.integers(5, 60)), float(10 ** rng.uniform(-6, -2)))
        elif kind == 1:
            A = P.laplacian_3d(int(rng.integers(3, 22)), float(10 ** rng.uniform(-6, -2)))
        else:
            A = P.diffusion_2d(int(rng.integers(5, 40)), seed=k)
        specs.append((A, P.rhs_uniform(A.n, 200 + k), ar, 1e-20, 3000, "jacobi" if k % 2 else None))
    specs.append((P.laplacian_2d(30), P.rhs_uniform(900, 5), "dw", 1e-20, 3000, None))
    specs.append((P.laplacian_2d(10), np.zeros(100), ar, 1e-12, 100, None))
    specs.append((P.laplacian_2d(12), P.rhs_uniform(144, 7), ar, 1e-30, 4, None))
    specs.append((P.power_law_laplacian(3000, seed=7, mean_deg=12, max_deg=300), P.rhs_uniform(3000, 84), ar,
                  1e-14, 3000, "jacobi"))
    specs.append((P.laplacian_2d(16), P.rhs_uniform(256, 9) * 2.0 ** 300, ar, 1e-20, 500, None))
    Ms = []
    for A, b, a, tol, maxit, pc in specs:
        M = mw.CSRMatrix.from_csr(A)
        if pc:
            M.preconditioner = pc
        Ms.append(M)
    bs = [torch.as_tensor(sp[1], device="cuda") for sp in specs]
    res = mw.solve_batched(Ms, bs, [sp[2] for sp in specs], [sp[3] for sp in specs], [sp[4] for sp in specs])
    C = mw.batched_cluster_size()
    statuses = set()
    for (A, b, a, tol, maxit, pc), M, r in zip(specs, Ms, res):
        V = M.plan_for(a)[0]
        xo, ito, rro, sto = orc.cg(a, A, b, tol=tol, maxit=maxit, plan=(V, 256, C), precond=pc)
        assert (r.iters, r.status) == (ito, sto), (A.name, a, pc, r.iters, ito, r.status, sto)
        assert same_bits(np.array([r.relres]), np.array([rro])), (A.name, a, pc)
        assert same_bits(r.x.cpu().numpy(), xo), (A.name, a, pc)
        statuses.add(sto)
    assert {0, 1, 4} <= statuses and (2 in statuses) == (ar == "qqf")


def test_bicgstab_bit_exact(mw, orc, ar, monkeypatch):
    """BiCGStab in FP32 words (r, p, v, s, t at 2^E, the shadow residual at
    2^E0; the generic p update and SpMV kernels, the scaled init, s and x / r
    kernels) equals the oracle's scaled BiCGStab bit for bit: iterations,
    status, residual history and x, on the graph and on host-launched kernels,
    for nonsymmetric convection-diffusion systems, the early exit (A = 2I),
    a breakdown (a rotation), b = 0, maxit = 0 and x leaving FP32's range."""
    def check(M, A, b, tol, maxit, tag):
        r = mw.solve_bicgstab(M, dev(b), ar, tol, maxit, history=True)
        xo, ito, rro, sto, ho = orc.bicgstab(ar, A, b, tol=tol, maxit=maxit, plan=M.plan, history=True)
        assert (r.iters, r.status) == (ito, sto), (tag, r.iters, ito, r.status, sto)
        assert same_bits(np.array([r.relres]), np.array([rro])), tag
        assert same_bits(r.x.cpu().numpy(), xo), tag
        if r.iters:
            assert same_bits(r.history.cpu().numpy(), ho), tag
        return r
    for A, seed, tol in ((P.convection_diffusion_2d(48, 2.0), 91, 1e-22),
                         (P.convection_diffusion_2d(90, 8.0), 92, 1e-14)):
        b = P.rhs_uniform(A.n, seed)
        M = mw.CSRMatrix.from_csr(A)
        assert check(M, A, b, tol, 3000, A.name).iters > 10
    A = P.convection_diffusion_2d(48, 2.0)
    b = P.rhs_uniform(A.n, 91)
    monkeypatch.setenv("MWCG_EAGER", "1")
    check(mw.CSRMatrix.from_csr(A), A, b, 1e-22, 3000, "eager")
    monkeypatch.delenv("MWCG_EAGER")
    n = 300
    D = P.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    r = check(mw.CSRMatrix.from_csr(D), D, P.rhs_uniform(n, 93), 1e-30, 5, "2I")
    assert (r.status, r.iters) == (0, 1)
    R = P.CSR(2, np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32), np.array([1.0, -1.0]))
    assert check(mw.CSRMatrix.from_csr(R), R, np.array([1.0, 0.0]), 1e-30, 5, "rotation").status == 2
    C = P.convection_diffusion_2d(16, 1.0)
    MC = mw.CSRMatrix.from_csr(C)
    check(MC, C, np.zeros(C.n), 1e-12, 50, "b = 0")
    check(MC, C, P.rhs_uniform(C.n, 94), 1e-12, 0, "maxit 0")
    assert check(MC, C, P.rhs_uniform(C.n, 95) * 2.0 ** 300, 1e-22, 2000, "2^300").status == 4
