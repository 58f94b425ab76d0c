"""Multi-word-arithmetic Conjugate Gradient for NVIDIA GB300 (sm_103a).

CG on a sparse SPD FP64 CSR system carried out in FP64, DW, QDW, TW or QTW
arithmetic (Mukunoki and Ozaki, "Sparse Iterative Solvers Using High-Precision
Arithmetic with Quasi Multi-Word Algorithms").  Every step of the solve runs
in the hand-written CUDA kernels of ``libmwcg.so`` behind the C ABI declared in
``include/mwcg.h``; this package is the thin Python binding over it.
"""
