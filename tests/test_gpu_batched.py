"""Batched persistent solve vs the CPU oracle (needs a GB300).

Every system of a mixed batch (all arithmetics, ragged sizes, an empty
system, a zero right-hand side, irregular rows) must equal, bit for bit, the
oracle's solve in the mirrored order of plan {V, 256, cluster size}; and the
batched results must agree with one-by-one mwcg_solve calls to the
arithmetic's accuracy.
"""
import numpy as np
import pytest

from paper_2510_13536_gb300 import problems as P

pytestmark = pytest.mark.gpu
ARITHS = ["fp64", "dw", "qdw", "tw", "qtw", "qdw_nn", "qtw_nn", "qw", "qqw", "qqw_nn"]


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
    na, nb = np.isnan(a), np.isnan(b)
    return a.shape == b.shape and np.array_equal(na, nb) and np.array_equal(a.view(np.uint64)[~na],
                                                                             b.view(np.uint64)[~nb])


def _batch():
    rng = np.random.default_rng(3)
    systems = []
    for k in range(21):
        kind = k % 4
        if kind == 0:
            A = P.laplacian_2d(int(rng.integers(3, 60)), float(10 ** rng.uniform(-6, -2)))
        elif kind == 1:
            A = P.laplacian_3d(int(rng.integers(2, 22)), float(10 ** rng.uniform(-6, -2)))
        elif kind == 2:
            A = P.power_law_laplacian(int(rng.integers(300, 4000)), seed=int(k), mean_deg=10, max_deg=150)
        else:
            A = P.diffusion_2d(int(rng.integers(4, 40)), seed=int(k))
        b = P.rhs_uniform(A.n, 100 + k)
        systems.append((A, b, ARITHS[k % len(ARITHS)], 1e-11, 3000))
    systems.append((P.laplacian_2d(10), np.zeros(100), "qtw", 1e-12, 100))            # b = 0
    systems.append((P.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)), np.zeros(0), "dw",
                    1e-12, 100))                                                   # empty system
    systems.append((P.laplacian_2d(12), P.rhs_uniform(144, 7), "qdw", 1e-30, 4))    # stops at maxit
    return systems


def test_batched_bit_exact_against_oracle(mw, orc):
    import torch
    systems = _batch()
    Ms = [mw.CSRMatrix.from_csr(A) for A, *_ in systems]
    bs = [torch.as_tensor(b, device="cuda") for _, b, *_ in systems]
    res = mw.solve_batched(Ms, bs, [s[2] for s in systems], [s[3] for s in systems], [s[4] for s in systems])
    C = mw.batched_cluster_size()
    for (A, b, ar, tol, maxit), M, r in zip(systems, Ms, res):
        V = M.plan[0]
        xo, ito, rro, sto = orc.cg(ar, A, b, tol=tol, maxit=maxit, plan=(V, 256, C))
        assert (r.iters, r.status) == (ito, sto), (A.name, ar)
        assert same_bits(np.array([r.relres]), np.array([rro])), (A.name, ar)
        assert same_bits(r.x.cpu().numpy(), xo), (A.name, ar)


def test_batched_matches_sequential_accuracy(mw):
    import torch
    specs = P.batch_specs(24, seed=P.SEED_BASE + 4, nmin=1000, nmax=20000)
    systems = [P.build_batch_system(s) for s in specs]
    Ms = [mw.CSRMatrix.from_csr(A) for A, _ in systems]
    bs = [torch.as_tensor(b, device="cuda") for _, b in systems]
    ar = [s["arith"] for s in specs]
    res = mw.solve_batched(Ms, bs, ar, 1e-14, 20000)
    for M, b, a, r in zip(Ms, bs, ar, res):
        r1 = mw.solve(M, b, a, 1e-14, 20000)
        assert r.status == r1.status == 0
        assert abs(r.iters - r1.iters) <= max(3, r1.iters // 50)
        x, x1 = mw.collapse(r.x), mw.collapse(r1.x)
        assert float(torch.linalg.norm(x - x1) / torch.linalg.norm(x1)) < 1e-9
