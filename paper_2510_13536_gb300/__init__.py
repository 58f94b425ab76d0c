"""Multi-word-arithmetic Conjugate Gradient for NVIDIA GB300 (sm_103a).

CG on a sparse SPD FP64 CSR system carried out in FP64, DW, QDW, TW or QTW
arithmetic (Mukunoki and Ozaki, "Sparse Iterative Solvers Using High-Precision
Arithmetic with Quasi Multi-Word Algorithms").  Every step of the solve runs
in the hand-written CUDA kernels of ``libmwcg.so`` behind the C ABI declared in
``include/mwcg.h``; this package is the thin Python binding over it.

``problems`` (seeded synthetic systems) imports without the library; the
solver API (``solver``) loads ``libmwcg.so`` and raises if it is absent.
"""

_SOLVER_NAMES = ("CSRMatrix", "SolveResult", "solve", "solve_host", "solve_batched", "adjoint", "spmv", "dot",
                 "word_op", "collapse", "words", "arith_id", "MWCGSolve", "solve_differentiable")


def __getattr__(name):
    if name in _SOLVER_NAMES:
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
