/*
 * mwcg.h -- C ABI of the GB300 (sm_103a) multi-word-arithmetic CG solver.
 *
 * The solver runs the Conjugate Gradient method (Algorithm 1 of Mukunoki and
 * Ozaki, "Sparse Iterative Solvers Using High-Precision Arithmetic with Quasi
 * Multi-Word Algorithms") on a sparse symmetric positive definite matrix
 * stored as FP64 CSR, with every vector and scalar of the iteration held in
 * one of five arithmetics built from FP64 words (Sec. III): FP64, DW
 * (double-word), QDW (quasi double-word), TW (triple-word) and QTW (quasi
 * triple-word), plus the unnormalised quasi variants of Sec. V-B3.  A and b
 * are FP64 (Sec. IV-C); the stopping residual is computed in FP64 (Sec.
 * IV-C); the quasi arithmetics normalise r once per iteration after its AXPY
 * (Sec. IV-D).
 *
 * Conventions for every function:
 *  - Multi-word vectors are structure of arrays: a vector of n elements in an
 *    arithmetic with w words (mwcg_words) is a double[w*n] with word k of
 *    element i at [k*n + i]; word 0 is the leading word.  MWCG_QQF's four
 *    FP32 words fill two 8-byte slots per element instead: slot k (k = 0, 1)
 *    of element i, at [k*n + i], holds words 2k and 2k+1 as two consecutive
 *    floats (word 2k at the lower address); mwcg_words returns 2 for it.
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary (preferably pinned) host memory.
 *  - Work is ordered on the caller's CUDA stream (`stream`, a cudaStream_t;
 *    NULL is the legacy default stream).  Functions that return results on
 *    the host synchronise that stream once before returning.
 *  - Return codes: MWCG_OK (0) or a positive solver status, or a negative
 *    error code; mwcg_last_error() then gives a message (thread-local).
 *  - A matrix handle owns its device copy of the matrix and the solver
 *    workspace.  One solve at a time per handle (the workspace is shared);
 *    distinct handles may be used concurrently.
 *  - The reduction kernels opt in to more than 48 KB of dynamic shared memory
 *    (needed only by four-word arithmetics with plans of more than 945
 *    blocks) on the device that is current at the library's first call.
 */
#ifndef MWCG_H
#define MWCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetics (Sec. III).  *_NN: quasi arithmetic without the per-iteration
 * normalisation of r (Sec. V-B3, "CG-QDW-NN", "CG-QTW-NN").  QW and QQW
 * (four words, about 212 bits) are listed in Sec. I without algorithms; here
 * QQW continues QTW's Algorithms 7-10 one level down (VecSum4 normalises it)
 * and QW is every QQW operation followed by a renormalisation to four
 * non-overlapping words.
 * QQF (four FP32 words, about 96 bits; Sec. II notes FP32-word arithmetic
 * where FP64 is missing, Sec. VI processors with little FP64) runs QQW's
 * sequences on FP32 words and operations.  FP64 inputs (the matrix values,
 * b) enter through an exact split into three FP32 words (exact for
 * 2^-97 <= |a| < 2^128, correctly rounded pieces otherwise).  Its CG keeps r
 * and p scaled by a power of two 2^E so that FP32's exponent range follows
 * the shrinking residual (x is unscaled, so its values must lie within
 * FP32's range, |x_i| >= 2^-54 or so for full precision).  QQF supports
 * mwcg_solve, mwcg_solve_history, mwcg_solve_host, mwcg_spmv, mwcg_dot,
 * mwcg_word_op (op 5 collapses its words to FP64) and mwcg_profile_kernels;
 * the normalisation policy does not apply to it (r is normalised every
 * iteration).  It has CG, Jacobi PCG (mwcg_set_preconditioner), BiCGStab,
 * the batched solve, the adjoint and mwcg_dot_noalloc, each with the scaled
 * iteration.
 * A solve whose x leaves FP32's range returns MWCG_OUT_OF_RANGE.
 * QF is QQF with every addition and product (FP64 x QF included) followed
 * by VecSum4, the non-quasi counterpart of QQF as DW is of QDW: on strongly
 * cancelling rows its precision stays relative to the result.  It has QQF's
 * storage, entry points, scaled CG and limits. */
typedef enum {
  MWCG_FP64 = 0,
  MWCG_DW = 1,
  MWCG_QDW = 2,
  MWCG_TW = 3,
  MWCG_QTW = 4,
  MWCG_QDW_NN = 5,
  MWCG_QTW_NN = 6,
  MWCG_QW = 7,
  MWCG_QQW = 8,
  MWCG_QQW_NN = 9,
  MWCG_QQF = 10,
  MWCG_QF = 11
} mwcg_arith;

/* Solver status (>= 0) and error codes (< 0). */
enum {
  MWCG_OK = 0,              /* converged: relres < tol                                  */
  MWCG_NOT_CONVERGED = 1,   /* maxit iterations done without reaching tol               */
  MWCG_BREAKDOWN = 2,       /* collapse(p^T q) not > 0, or a non-finite residual        */
  MWCG_BAD_PRECONDITIONER = 3, /* Jacobi: a diagonal entry missing, <= 0 or not finite; x0 untouched */
  MWCG_OUT_OF_RANGE = 4,    /* QQF, QF: x left FP32's range -- a leading word of x not finite after an   */
                            /* update, or every one below 2^-126 when the solve ends (x is invalid)  */
  MWCG_ERR_ARG = -1,        /* invalid argument (sizes, pointers, CSR structure, plan)  */
  MWCG_ERR_CUDA = -2,       /* a CUDA runtime call failed                               */
  MWCG_ERR_GUARD = -3,      /* device loop guard tripped (internal consistency failure) */
  MWCG_ERR_NOMEM = -4       /* device allocation failed                                 */
};

/* Summation plan of the kernels.  It fixes the order of every FP64 operation
 * and hence the result bits:
 *   V  lanes per CSR row in the SpMV (1, 2, 4, 8, 16 or 32); lane l of a row
 *      owns entries row_start + l + jV and the V lane sums are combined by a
 *      pairwise tree;
 *   T  threads per block (fixed at 256);
 *   G  blocks (1..1024); rows are cut into tiles of T/V (SpMV) or T (vector
 *      kernels) rows, tile t belongs to block t mod G, each block slot sums
 *      its rows across the block's tiles in increasing order, then slots and
 *      blocks are combined by pairwise trees.
 * Automatic plans (the autotuner; the paper fixes no order, Sec. IV-B):
 * mwcg_create_csr derives, per arithmetic, a plan from the row-length
 * distribution with an FP64-instruction cost model (V; G = one resident wave
 * of 3 blocks per SM, or the one-cluster size for small systems).  At the
 * first call in an arithmetic the SpMV is timed under the model's best lane
 * counts (at most three, each within twice the best model cost) on a
 * synthetic vector with every word populated; another lane count replaces
 * the model's only when it is at least 4% faster.  The result is cached per
 * handle and arithmetic.  Because a measurement can decide V, and V the
 * summation order, pin a plan with mwcg_set_plan where results must be
 * reproducible bit for bit across processes or GPUs. */
typedef struct {
  int32_t V;
  int32_t T;
  int32_t G;
} mwcg_plan;

typedef struct mwcg_csr mwcg_csr;

/* Number of 8-byte slots per element of a vector in an arithmetic (its FP64
 * words, 1 to 4; 2 for the four FP32 words of MWCG_QQF and MWCG_QF), or -1
 * if unknown. */
int mwcg_words(int arith);

/* Message of the last error on this thread ("" if none).  Owned by the
 * library, valid until the next call on this thread. */
const char* mwcg_last_error(void);

/* Copy a CSR matrix to the device and build its solver handle.
 *   n        rows = columns (n >= 0);
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz;
 *   col      int32[nnz], 0 <= col < n (any order within a row);
 *   val      double[nnz], finite;
 *   ptrs_on_device  0: the three arrays are host memory, 1: device memory;
 *   out      receives the handle (caller frees it with mwcg_destroy_csr).
 * The structure is validated; violations return MWCG_ERR_ARG, the message
 * naming the first bad row_ptr entry, or the first entry k whose column or
 * value is invalid (the column reported first).  row_ptr is checked on the
 * host (device row_ptr is copied back, 8 (n+1) bytes); device col / val are
 * checked on the device after the copy, with no host copy of the entries.
 * Symmetry is not checked: the paper
 * stores symmetric matrices in general form (Sec. IV-B) and so does the
 * caller.  The arrays are copied; the caller keeps ownership of them. */
int mwcg_create_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    int ptrs_on_device, void* stream, mwcg_csr** out);

/* Release a handle and its device memory (NULL is ignored). */
void mwcg_destroy_csr(mwcg_csr* A);

/* Replace the values of A (same sparsity pattern); val is double[nnz] on the
 * host (on_device = 0) or device (1).  Non-finite values: MWCG_ERR_ARG (the
 * message names the first one) and A keeps its values.  Device values are
 * checked on the device and copied device to device (no host copy of the
 * values); the call synchronises `stream`. */
int mwcg_update_values(mwcg_csr* A, const double* val, int on_device, void* stream);

int64_t mwcg_n(const mwcg_csr* A);
int64_t mwcg_nnz(const mwcg_csr* A);
/* The plan of the handle's last call (before any call: the pinned plan, or
 * the automatic QTW plan). */
int mwcg_get_plan(const mwcg_csr* A, mwcg_plan* out);
/* Pin a plan for every arithmetic (V power of two in 1..32, T = 256, G in
 * 1..1024; MWCG_ERR_ARG otherwise).  plan = NULL returns to the automatic
 * plans. */
int mwcg_set_plan(mwcg_csr* A, const mwcg_plan* plan);
/* The plan a call in `arith` uses: the pinned plan, or the arithmetic's
 * automatic plan, timed first (on `stream`, synchronised) if this is the
 * handle's first call in that arithmetic.  spmv_ms (optional, double[6]):
 * the measured SpMV time in ms for V = 1, 2, 4, ..., 32, 0 where not timed
 * (all 0 for a pinned plan or a system too small to time). */
int mwcg_get_plan_for(mwcg_csr* A, int arith, void* stream, mwcg_plan* out, double* spmv_ms);

/* Normalisation policy of the quasi arithmetics (QDW, QTW), per matrix handle.
 * Sec. IV-D normalises the residual r once per iteration, right after its
 * AXPY (Algorithm 1 line 8), and Sec. VI leaves the frequency and placement
 * of normalisation open; this generalises it.  On CG iteration it (1-based)
 * with every > 0 and it % every == 0, each place in mask is normalised with
 * the arithmetic's normalisation (QuickTwoSum for QDW, VecSum3 for QTW):
 *   MWCG_NORM_R    r_i after its AXPY (line 8)             -- the default
 *   MWCG_NORM_X    x_i after its AXPY (line 7)
 *   MWCG_NORM_P    p_i after its update (line 14)
 *   MWCG_NORM_Q    q_i = (A p)_i once its row is complete (line 5), before
 *                  it enters p^T q
 *   MWCG_NORM_SUM  the SpMV row's running sum after every addition into it
 *                  (each lane's accumulation and each lane-tree combine)
 * every = 0 never normalises (bit-identical to MWCG_QDW_NN / MWCG_QTW_NN).
 * The default is every = 1, mask = MWCG_NORM_R.  DW, TW and FP64 results are
 * unaffected (their operations are normalised or single-word), as are the NN
 * arithmetics (never normalised).  The policy applies to every later solve on
 * the handle (mwcg_solve*, mwcg_adjoint, mwcg_solve_batched).
 * Errors: every < 0 or unknown mask bits -> MWCG_ERR_ARG (policy unchanged). */
#define MWCG_NORM_R 1u
#define MWCG_NORM_X 2u
#define MWCG_NORM_P 4u
#define MWCG_NORM_Q 8u
#define MWCG_NORM_SUM 16u
int mwcg_set_normalization(mwcg_csr* A, int32_t every, uint32_t mask);
int mwcg_get_normalization(const mwcg_csr* A, int32_t* every, uint32_t* mask);

/* Preconditioner of every later solve on the handle (mwcg_solve*,
 * mwcg_adjoint, mwcg_solve_batched).  The paper's solver is unpreconditioned
 * CG (Algorithm 1; Sec. VI names preconditioning as future work):
 *   MWCG_PREC_NONE    Algorithm 1 (the default);
 *   MWCG_PREC_JACOBI  preconditioned CG with M^-1 = diag(w), w_i = fl(1/a_ii)
 *                     in FP64 (the preconditioner is FP64 like A): z = w (x) r
 *                     is the arithmetic's FP64 x multi-word product,
 *                     rho = r^T z in the arithmetic, p = z + beta p.  The
 *                     stopping residual stays FP64 (Sec. IV-C):
 *                     sqrt(sum_i collapse(r_i)^2) / ||b||_2, summed in FP64 in
 *                     the plan's order.  The normalisation policy applies as
 *                     in CG.  w is built on the device at the first solve
 *                     after this call or after mwcg_update_values; a diagonal
 *                     entry that is missing, not positive or not finite makes
 *                     the solve return MWCG_BAD_PRECONDITIONER with x0 untouched.
 *                     MWCG_QQF / MWCG_QF run it with the scaled iteration of
 *                     their CG (r~ = 2^-E r, z~ = w (x) r~, p~ = z~ + (beta~ 2^s) p~),
 *                     the shift taken from the FP64 residual sum.
 * Errors: unknown kind -> MWCG_ERR_ARG. */
#define MWCG_PREC_NONE 0
#define MWCG_PREC_JACOBI 1
int mwcg_set_preconditioner(mwcg_csr* A, int kind);
int mwcg_get_preconditioner(const mwcg_csr* A, int* kind);

/* Solve A x = b by BiCGStab in the given arithmetic, for nonsymmetric A (an
 * extension: the paper's solver is CG, and Sec. VI names other iterative
 * methods as future work).  The textbook recurrence (van der Vorst) with
 * shadow residual rh = r0:
 *   rho = rh^T r; p = r (first pass) or r (+) beta*(p (+) (-omega)*v);
 *   v = A p; alpha = rho / rh^T v; s = r (+) (-alpha)*v;
 *   stop with x (+)= alpha*p if ||s|| / ||b|| < tol; t = A s;
 *   omega = t^T s / t^T t; x = (x (+) alpha*p) (+) omega*s; r = s (+) (-omega)*t;
 *   beta = (rho' / rho) * (alpha / omega).
 * Every vector and scalar is in the arithmetic; the quasi arithmetics
 * normalise both residual AXPYs (s and r) every iteration; the stopping
 * residuals are FP64, sqrt(sum_i collapse(.)^2) / ||b||_2 (Sec. IV-C).
 * Arguments, x0, hist (optional device double[maxit], the FP64 relative
 * residual after each iteration) and the results are as for
 * mwcg_solve_history.  Returns MWCG_OK, MWCG_NOT_CONVERGED, MWCG_BREAKDOWN
 * (collapse of rho, rh^T v or t^T t zero or not finite, omega's collapse zero,
 * or a non-finite residual) or an error.  The handle's preconditioner and
 * normalisation policy apply to CG only; BiCGStab has no batched form.
 * MWCG_QQF / MWCG_QF run it scaled: r, p, v, s, t at 2^E and the shadow
 * residual at 2^E0, alpha and omega unscaled, x += (alpha 2^E) p~ +
 * (omega 2^E) s~, r~ shifted by 2^-sh after its AXPY (sh from the FP64 sum of
 * the r~ it replaces), beta~ = (rho~'/rho~)(alpha/omega); x in the packed FP32
 * layout, MWCG_OUT_OF_RANGE as in mwcg_solve. */
int mwcg_solve_bicgstab(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, double* hist,
                        void* stream, int32_t* iters_out, double* relres_out);

/* Solve A x = b by CG in the given arithmetic (Algorithm 1).
 *   b        device double[n];
 *   x        device double[w*n] (w = mwcg_words(arith)): x0 on entry, the
 *            multi-word solution on return;
 *   tol      stop when sqrt(collapse(r^T r)) / ||b||_2 < tol (FP64, Sec. IV-C);
 *   maxit    iteration limit, 0 <= maxit <= 2^30 (0 returns x0 with status 1);
 *   iters_out, relres_out (host, may be NULL): iterations done (the pass that
 *            stops counts) and the last relative residual.
 * Returns MWCG_OK, MWCG_NOT_CONVERGED, MWCG_BREAKDOWN or an error.  b = 0
 * gives x = 0 and zero iterations; an exact x0 (r0 = 0) zero iterations.
 * The whole solve (initialisation and the loop) is one CUDA graph launch
 * whose loop is a device-side while node; the stream is synchronised once
 * at the end to read the iteration count and residual. */
int mwcg_solve(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, void* stream,
               int32_t* iters_out, double* relres_out);

/* mwcg_solve with host buffers: b_host double[n], x_host double[w*n] (x0 in,
 * solution out).  The copies to and from the device are part of the call. */
int mwcg_solve_host(mwcg_csr* A, const double* b_host, double* x_host, int arith, double tol, int32_t maxit,
                    void* stream, int32_t* iters_out, double* relres_out);

/* Like mwcg_solve, and also writes the FP64 relative residual after every
 * iteration to hist (device double[maxit]); entries past the last iteration
 * are left untouched. */
int mwcg_solve_history(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit,
                       double* hist, void* stream, int32_t* iters_out, double* relres_out);

/* Solve many independent systems in one persistent kernel launch.
 *   nsys             number of systems (>= 0);
 *   A[s]             distinct handles (a handle repeated in one batch is
 *                    MWCG_ERR_ARG: each system uses its handle's workspace);
 *   b[s], x[s]       device pointers as in mwcg_solve (x[s] holds
 *                    mwcg_words(arith[s]) * n_s doubles, x0 on entry);
 *   arith[s], tol[s], maxit[s]  per system (host arrays);
 *   iters_out[s], relres_out[s], status_out[s]  host arrays (may be NULL).
 * Workers are thread-block clusters of mwcg_batched_cluster_size() CTAs that
 * take systems from a device queue (largest first) and run each solve to its
 * end; a system's summation order, and so its result bits, equal those of
 * mwcg_solve with plan {V of its handle, 256, mwcg_batched_cluster_size()}.
 * Every arithmetic is accepted, QQF and QF with their scaled iteration (x[s]
 * in the packed FP32 layout; status MWCG_OUT_OF_RANGE as in mwcg_solve), and
 * a handle's Jacobi preconditioner applies to its system.
 * Returns MWCG_OK when the launch succeeded (per-system outcomes are in
 * status_out), or an error. */
int mwcg_solve_batched(int32_t nsys, mwcg_csr* const* A, const double* const* b, double* const* x,
                       const int32_t* arith, const double* tol, const int32_t* maxit, void* stream,
                       int32_t* iters_out, double* relres_out, int32_t* status_out);

/* Number of CTAs per worker cluster used by mwcg_solve_batched. */
int mwcg_batched_cluster_size(void);

/* Adjoint of a solve, for L with dL/dx = gx (device double[n]):
 *   lambda = CG(A, gx) in the same arithmetic from lambda0 = 0 (A symmetric,
 *   so A^T lambda = gx is solved with the forward kernels);
 *   g_b[i]   = collapse(lambda_i)                (device double[n], may be NULL);
 *   g_val[k] = -collapse(lambda_row(k) * x_col(k)) (device double[nnz], may be NULL),
 *              the product taken in the arithmetic;
 *   x        device double[w*n], the forward solution (only it is needed;
 *            MWCG_QQF / MWCG_QF: its packed FP32 words, as mwcg_solve returns
 *            them, and lambda is solved with the same scaled CG).
 * Every arithmetic has an adjoint.  Returns the status of the adjoint solve
 * (as mwcg_solve) or an error. */
int mwcg_adjoint(mwcg_csr* A, const double* x, const double* gx, int arith, double tol, int32_t maxit, void* stream,
                 double* g_b, double* g_val, int32_t* iters_out, double* relres_out);

/* q = A p in the arithmetic, with the handle's plan (p, q device double[w*n]). */
int mwcg_spmv(mwcg_csr* A, int arith, const double* p, double* q, void* stream);

/* u^T v in the arithmetic over n elements (u, v device double[w*n]) with
 * tiles of 256 rows over G blocks (1..1024); out: host double[w], one word
 * per double (host double[4] holding the four FP32 words for MWCG_QQF). */
int mwcg_dot(int arith, int64_t n, const double* u, const double* v, int32_t G, void* stream, double* out);

/* Capacity, in blocks, of the fixed scratch array of mwcg_dot_noalloc. */
#define MWCG_DOT_NOALLOC_MAX_G 1024

/* mwcg_dot without any device allocation.  The paper has no counterpart: this
 * is a library-level variant for callers that must not allocate device memory
 * -- mwcg_dot calls cudaMalloc and cudaFree on every call, and cudaFree
 * synchronises the whole device, which stalls the other streams of a
 * latency-critical pipeline; code that runs under a fixed device-memory
 * budget or a pooled allocator may also be forbidden hidden allocations.
 * Here the block partials and the ticket counter live in a fixed array
 * compiled into the library (MWCG_DOT_NOALLOC_MAX_G blocks of 12 doubles plus
 * one counter block, about 99 KB, held by every GPU that loads the library
 * until the process exits).  The function calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   arith    0..11 (MWCG_FP64 .. MWCG_QF); any other value returns MWCG_ERR_ARG;
 *   n, u, v, G  as in mwcg_dot (u, v device double[w*n], w = mwcg_words; for
 *            MWCG_QQF / MWCG_QF the packed FP32 layout); G in
 *            1..MWCG_DOT_NOALLOC_MAX_G, larger G returns MWCG_ERR_ARG;
 *   out      device double[w] (caller-owned; double[4], one FP32 word per
 *            double, for MWCG_QQF / MWCG_QF), written in stream order; the
 *            function does not synchronise the stream.
 * The result bits equal mwcg_dot's for the same arguments.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, so make the first call on each device before any
 * stream capture.  All calls share the one array: its counter is cleared at
 * the start of every call and the partials are rewritten, so calls that
 * overlap on the GPU (concurrent streams or threads) race and must be
 * serialised by the caller. */
int mwcg_dot_noalloc(int arith, int64_t n, const double* u, const double* v, int32_t G, void* stream, double* out);

/* Element-wise word operations on device arrays of n elements:
 *   op 0 add c = a + b; 1 mul c = a * b; 2 dxmul c = a (FP64, double[n]) * b;
 *   3 div c = a / b; 4 normalize c = the arithmetic's normalisation of a
 *   (QuickTwoSum for QDW, VecSum3 for QTW, VecSum4 for QQW and QQF,
 *   identity otherwise);
 *   5 collapse c (double[n]) = a summed lowest word first. */
int mwcg_word_op(int op, int arith, int64_t n, const double* a, const double* b, double* c, void* stream);

/* Time the solver's kernels one by one: runs the initialisation and then
 * `niters` CG iterations of A x = b in the arithmetic without the CUDA graph
 * (each kernel launched on `stream` between CUDA events; the stop test is
 * disabled so exactly niters iterations run), and writes the mean duration in
 * milliseconds of the SpMV + p^T q kernel, the x/r update + r^T r kernel and
 * the p update kernel to ms_out[0..2] (host double[3]).  x (device
 * double[w*n]) is overwritten.  niters in 2..100000. */
int mwcg_profile_kernels(mwcg_csr* A, const double* b, double* x, int arith, int32_t niters, void* stream,
                         double* ms_out);

/* Throughput probe for the roofline denominators: runs an FP64 FMA (kind 0),
 * FP64 add (kind 1), 32-bit integer add/xor (kind 2), FP64 add issued as an
 * FMA with multiplier 1 (kind 3) or FP64 multiply (kind 4) loop on every SM with
 * eight independent chains per thread and writes the best of three runs in
 * operations per second (FMA = one operation) to *ops_per_s (host).
 * scratch: device buffer of at least SMs * 8 * 256 * 8 bytes (overwritten). */
int mwcg_probe_peak(int kind, void* scratch, int64_t scratch_bytes, void* stream, double* ops_per_s);

/* x64[i] = collapse of element i of the w-word vector xw (device arrays). */
int mwcg_collapse(const double* xw, int32_t w, int64_t n, double* x64, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MWCG_H */
