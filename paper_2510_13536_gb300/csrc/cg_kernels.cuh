// CG kernels for one arithmetic (template parameter A from mw_device.cuh).
//
// One CG iteration (Algorithm 1) is three kernels:
//   k_spmv   q = A p (line 5) fused with p^T q (line 6); the last block to
//            finish reduces the block partials, divides alpha = rho / p^T q
//            and tests for breakdown.
//   k_update x += alpha p, r -= alpha q (lines 7-8), normalisation of r for
//            the quasi arithmetics (Sec. IV-D), r^T r (line 9); the last block
//            forms the FP64 relative residual (Sec. IV-C), applies the stop
//            test (line 10), beta = rho' / rho (line 13) and sets the CUDA
//            graph's loop condition.
//   k_pupdate p = r + beta p (line 14).
// plus k_init (line 1-2 and ||b||) and k_zero_x.  All of them read the
// per-solve scalars from a DevState in device memory, so one instantiated
// CUDA graph serves every call on the same matrix.
//
// Summation order (must match the CPU oracle's mirrored mode bit for bit),
// a function of the plan {V lanes per row, T threads per block, G blocks}:
//   row i of the SpMV: lane l of the row's V-lane group owns entries
//     row_start + l + jV and sums their products left to right from its first
//     product; lanes are combined by the pairwise tree.
//   dots: rows are cut into tiles of R = T/V (SpMV) or R = T (vector kernels)
//     rows; tile t belongs to block t mod G; slot s of a block adds the leaves
//     of row t*R+s of its tiles in increasing t; the R slots, then the G
//     blocks, are combined by the pairwise tree (level h pairs slot s with
//     s+h for s a multiple of 2h; absent entries skipped).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "mw_device.cuh"

namespace mwk {

constexpr int TPB = 256;                  // threads per block of every kernel
// Block partials of the grid reductions: PART doubles per block -- the
// multi-word value in [0, W), its presence at PRES, FP64 value k at FV + k
// with its presence at FP + k.
constexpr int PART = 12, PRES = 4, FV = 5, FP = 7;
// Dynamic shared memory the last-block reductions need for G blocks of a
// w-word arithmetic: grid_reduce uses G (8 w + 4) bytes, grid_reduce_mix with
// two FP64 values G (8 w + 19); one size serves every reduction kernel.
inline size_t red_smem(int G, int w) { return (size_t)G * (8 * w + 20); }
// Tiles interleaved per thread (A::ILP; never changes the summation order).
// Measured on GB300: the multi-word kernels are fastest with 1; FP64, which is
// memory bound, needs several rows' loads in flight per thread.
constexpr int NWARP = TPB / 32;

enum { ST_CONVERGED = 0, ST_MAXIT = 1, ST_BREAKDOWN = 2, ST_GUARD = 3, ST_RANGE = 4 };

// Per-solve state in device memory.  Written by the host before a launch
// (b, x, tol, maxit, hist) and by the kernels (everything else).
struct DevState {
  const double* b;          // f64[n]
  double* x;                // f64[w][n], x0 in, solution out
  double* hist;             // optional f64[maxit] relative-residual history, or null
  double tol;
  int32_t maxit;
  int32_t pad0;
  double rho[4];             // multi-word scalars, up to four words
  double alpha[4];
  double beta[4];
  double bnorm;
  double relres;
  int32_t iters;
  int32_t status;
  int32_t done;
  int32_t zero_x;
  uint32_t counter;         // last-block election
  uint32_t guard;           // loop passes seen by block 0 of k_spmv (hang guard)
  int32_t norm_every;       // normalisation policy (quasi arithmetics): every k iterations, 0 never
  uint32_t norm_mask;       // NORM_* places
  double omega[4];          // BiCGStab: omega
  int32_t early;            // BiCGStab: ||s|| met the tolerance (x += alpha p ends the solve)
  uint32_t xmax_bits;       // QQF: largest |leading word of x| of this iteration, as FP32 bits
  int32_t q_e;              // QQF: the scaling exponent E (r = 2^E r~)
  int32_t q_s;              // QQF: the shift applied by this iteration's update
  int32_t q_s_next;         // QQF: the shift the next update applies
  int32_t pad1;
};

// Normalisation places (an extension of Sec. IV-D, which normalises r after
// its AXPY once per iteration and leaves frequency and placement open).  On
// iteration it (1-based) with every > 0 and it % every == 0 the masked places
// are normalised with A::normalize (QuickTwoSum for QDW, VecSum3 for QTW; the
// other arithmetics' normalize is the identity):
//   NORM_R   r_i after its AXPY (Algorithm 1 line 8; the default policy {1, R})
//   NORM_X   x_i after its AXPY (line 7)
//   NORM_P   p_i after its update (line 14)
//   NORM_Q   q_i = (A p)_i once the row is complete, before the p^T q leaf
//   NORM_SUM the SpMV row's running sum after every addition into it (each
//            lane's accumulation and each lane-tree combine)
enum : uint32_t { NORM_R = 1, NORM_X = 2, NORM_P = 4, NORM_Q = 8, NORM_SUM = 16, NORM_ALL = 31 };
__host__ __device__ __forceinline__ uint32_t norm_at(int32_t every, uint32_t mask, int it) {
  return (every > 0 && it % every == 0) ? mask : 0u;
}

struct Csr {
  const int64_t* __restrict__ rp;
  const int32_t* __restrict__ col;
  const double* __restrict__ val;
  int64_t n;
};

struct Work {
  double* r;                // f64[w][n]
  double* p;
  double* q;
  double* part;             // f64[G][4] block partials
  DevState* st;
  unsigned long long cond;  // cudaGraphConditionalHandle, valid if has_cond
  int has_cond;
  int V;                    // lanes per row in the SpMV
  int G;                    // blocks
  const double* w;          // Jacobi weights fl(1/a_ii) (preconditioned CG), else null
};

template <class A>
__device__ __forceinline__ typename A::T ld(const double* __restrict__ v, int64_t n, int64_t i) {
  typename A::T t;
#pragma unroll
  for (int k = 0; k < A::W; ++k) t.w[k] = v[k * n + i];
  return t;
}
template <class A>
__device__ __forceinline__ void st(double* __restrict__ v, int64_t n, int64_t i, const typename A::T& t) {
#pragma unroll
  for (int k = 0; k < A::W; ++k) v[k * n + i] = t.w[k];
}
template <class A>
__device__ __forceinline__ typename A::T shfl_down(const typename A::T& v, int off) {
  typename A::T o;
#pragma unroll
  for (int k = 0; k < A::W; ++k) o.w[k] = __shfl_down_sync(0xffffffffu, v.w[k], off);
  return o;
}
// Combine step of the pairwise tree with presence flags.
template <class A>
__device__ __forceinline__ void combine(typename A::T& v, bool& pv, const typename A::T& o, bool po) {
  if (po) {
    if (pv) v = A::add(v, o);
    else { v = o; pv = true; }
  }
}

__device__ __forceinline__ void set_cond(const Work& W, unsigned v) {
  if (W.has_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)W.cond, v);
}

// Pairwise tree over the R = TPB/V slots of a block; slot s lives in thread
// s*V.  Returns the block value in thread 0 (and its presence).
template <class A>
__device__ __forceinline__ void block_tree(typename A::T& v, bool& pv, int V) {
  __shared__ typename A::T sv[NWARP];
  __shared__ int sp[NWARP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int spw = 32 / V;                  // slots per warp
  const int s_in_warp = lane / V;
  for (int h = 1; h < spw; h <<= 1) {
    typename A::T o = shfl_down<A>(v, h * V);
    bool po = __shfl_down_sync(0xffffffffu, (int)pv, h * V) != 0;
    if ((lane % V) == 0 && (s_in_warp % (2 * h)) == 0 && s_in_warp + h < spw) combine<A>(v, pv, o, po);
  }
  if (lane == 0) { sv[warp] = v; sp[warp] = pv ? 1 : 0; }
  __syncthreads();
  if (warp == 0) {
    typename A::T x = (lane < NWARP) ? sv[lane] : A::zero();
    bool px = (lane < NWARP) ? (sp[lane] != 0) : false;
    for (int h = 1; h < NWARP; h <<= 1) {
      typename A::T o = shfl_down<A>(x, h);
      bool po = __shfl_down_sync(0xffffffffu, (int)px, h) != 0;
      if ((lane % (2 * h)) == 0 && lane + h < NWARP) combine<A>(x, px, o, po);
    }
    if (lane == 0) { v = x; pv = px; }
  }
  __syncthreads();
}

// Each block stores its value; the block that finishes last (atomic ticket)
// reduces the G values by the pairwise tree and returns true in every thread
// of that block, with the result in thread 0's `out`.
template <class A, int OFF>
__device__ __forceinline__ bool grid_reduce(const Work& W, const typename A::T& v, bool pv, typename A::T& out,
                                            bool& pout) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    double* dst = W.part + (size_t)blockIdx.x * PART + OFF;
#pragma unroll
    for (int k = 0; k < A::W; ++k) dst[k] = v.w[k];
    dst[PRES] = pv ? 1.0 : 0.0;
    __threadfence();
    unsigned t = atomicAdd(&W.st->counter, 1u);
    am_last = (t == (unsigned)(gridDim.x - 1));
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  // Pairwise tree over the G block values, in shared memory.
  extern __shared__ double dyn[];
  typename A::T* sv = reinterpret_cast<typename A::T*>(dyn);
  int* spf = reinterpret_cast<int*>(sv + gridDim.x);
  const int G = gridDim.x;
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    const double* src = W.part + (size_t)b * PART + OFF;
    typename A::T t;
#pragma unroll
    for (int k = 0; k < A::W; ++k) t.w[k] = __ldcg(src + k);
    sv[b] = t;
    spf[b] = __ldcg(src + PRES) != 0.0 ? 1 : 0;
  }
  __syncthreads();
  for (int h = 1; h < G; h <<= 1) {
    for (int s = 2 * h * threadIdx.x; s + h < G; s += 2 * h * blockDim.x) {
      typename A::T a = sv[s];
      bool pa = spf[s] != 0;
      combine<A>(a, pa, sv[s + h], spf[s + h] != 0);
      sv[s] = a;
      spf[s] = pa ? 1 : 0;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out = sv[0];
    pout = spf[0] != 0;
  }
  return true;
}

// As grid_reduce, for one multi-word value and NF = 1 or 2 FP64 values under
// one election.  Needs G * (8 W + 8 NF + 1 + NF) <= G * 51 bytes of dynamic
// shared memory.
template <class A, int NF>
__device__ __forceinline__ bool grid_reduce_mix(const Work& W, const typename A::T& v, bool pv, const double* f,
                                                const bool* pf, typename A::T& out, bool& pout, double* fout,
                                                bool* pfout) {
  using T = typename A::T;
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    double* dst = W.part + (size_t)blockIdx.x * PART;
#pragma unroll
    for (int k = 0; k < A::W; ++k) dst[k] = v.w[k];
    dst[PRES] = pv ? 1.0 : 0.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      dst[FV + k] = f[k];
      dst[FP + k] = pf[k] ? 1.0 : 0.0;
    }
    __threadfence();
    unsigned tk = atomicAdd(&W.st->counter, 1u);
    am_last = (tk == (unsigned)(gridDim.x - 1));
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  extern __shared__ double dyn[];
  const int G = gridDim.x;
  T* sv = reinterpret_cast<T*>(dyn);
  double* sf = reinterpret_cast<double*>(sv + G);          // [NF][G]
  unsigned char* sp = reinterpret_cast<unsigned char*>(sf + NF * G);   // presence [1 + NF][G]
  for (int bk = threadIdx.x; bk < G; bk += blockDim.x) {
    const double* src = W.part + (size_t)bk * PART;
    T tv;
#pragma unroll
    for (int k = 0; k < A::W; ++k) tv.w[k] = __ldcg(src + k);
    sv[bk] = tv;
    sp[bk] = __ldcg(src + PRES) != 0.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      sf[k * G + bk] = __ldcg(src + FV + k);
      sp[(1 + k) * G + bk] = __ldcg(src + FP + k) != 0.0;
    }
  }
  __syncthreads();
  for (int h = 1; h < G; h <<= 1) {
    for (int s2 = 2 * h * threadIdx.x; s2 + h < G; s2 += 2 * h * blockDim.x) {
      T a = sv[s2];
      bool pa = sp[s2] != 0;
      combine<A>(a, pa, sv[s2 + h], sp[s2 + h] != 0);
      sv[s2] = a;
      sp[s2] = pa;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        mw::MW<1> c{{sf[k * G + s2]}};
        bool pc = sp[(1 + k) * G + s2] != 0;
        combine<mw::FP64>(c, pc, mw::MW<1>{{sf[k * G + s2 + h]}}, sp[(1 + k) * G + s2 + h] != 0);
        sf[k * G + s2] = c.w[0];
        sp[(1 + k) * G + s2] = pc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out = sv[0];
    pout = sp[0] != 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      fout[k] = sf[k * G];
      pfout[k] = sp[(1 + k) * G] != 0;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// q = A p (mode 1, fused with p^T q and the alpha step) or q = A x0 (mode 0).
// ---------------------------------------------------------------------------
// The alpha step (Algorithm 1 line 6): the block's slots of p^T q by the
// pairwise tree, the grid's block values by the last block to finish, then
// alpha = rho / p^T q and the breakdown test, in that block's thread 0.
template <class A>
__device__ __forceinline__ void spmv_alpha(const Work& W, typename A::T acc, bool pacc, int V) {
  using T = typename A::T;
  DevState* S = W.st;
  block_tree<A>(acc, pacc, V);
  T tot;
  bool ptot = false;
  if (!grid_reduce<A, 0>(W, acc, pacc, tot, ptot)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!ptot) tot = A::zero();
    S->iters += 1;
    double pq = A::collapse(tot);
    // Breakdown: collapse(p^T q) not > 0 (NaN included) or not finite.
    if (!(pq > 0.0) || !isfinite(pq)) {
      S->status = ST_BREAKDOWN;
      S->done = 1;
      set_cond(W, 0);
    } else {
      T rho;
#pragma unroll
      for (int k = 0; k < A::W; ++k) rho.w[k] = S->rho[k];
      T al = A::div(rho, tot);
#pragma unroll
      for (int k = 0; k < A::W; ++k) S->alpha[k] = al.w[k];
    }
  }
}

// Entries kk[u], kk[u] + V, ... < ke[u] of the interleaved rows added into
// sum[u] left to right; NS: normalise the running sum after every addition.
// With A::CHUNK > 1 the loads of A::CHUNK entries of every interleaved row are
// issued before the first multiply-add (more loads in flight per thread); the
// products are still added in entry order.
template <class A, bool NS>
__device__ __forceinline__ void row_accumulate(const Csr& M, const double* __restrict__ p, int64_t n, int V,
                                               typename A::T* sum, int64_t* kk, const int64_t* ke) {
  using T = typename A::T;
  if constexpr (A::CHUNK == 1) {
    for (;;) {
      bool more = false;
#pragma unroll
      for (int u = 0; u < A::ILP_SPMV; ++u) {
        if (kk[u] < ke[u]) {
          sum[u] = A::dxmuladd(sum[u], M.val[kk[u]], ld<A>(p, n, M.col[kk[u]]));
          if constexpr (NS) A::normalize(sum[u]);
          kk[u] += V;
        }
        more = more || (kk[u] < ke[u]);
      }
      if (!more) break;
    }
  } else {
    for (;;) {
      bool more = false;
      double va[A::ILP_SPMV][A::CHUNK];
      T pv[A::ILP_SPMV][A::CHUNK];
#pragma unroll
      for (int u = 0; u < A::ILP_SPMV; ++u) {
#pragma unroll
        for (int c = 0; c < A::CHUNK; ++c) {
          const int64_t k = kk[u] + (int64_t)c * V;
          va[u][c] = 0.0;
          if (k < ke[u]) { va[u][c] = M.val[k]; pv[u][c] = ld<A>(p, n, M.col[k]); }
        }
      }
#pragma unroll
      for (int u = 0; u < A::ILP_SPMV; ++u) {
#pragma unroll
        for (int c = 0; c < A::CHUNK; ++c) {
          if (kk[u] < ke[u]) {
            sum[u] = A::dxmuladd(sum[u], va[u][c], pv[u][c]);
            if constexpr (NS) A::normalize(sum[u]);
            kk[u] += V;
          }
        }
        more = more || (kk[u] < ke[u]);
      }
      if (!more) break;
    }
  }
}

// POL: the instantiation that follows the handle's normalisation policy
// (DevState norm_every / norm_mask).  The default instantiation implements
// the default policy {1, NORM_R} with no tests at all: it never normalises
// in the SpMV, and k_update normalises r on every iteration.
template <class A, bool POL = false>
__global__ void __launch_bounds__(TPB, A::MINB) k_spmv(Csr M, Work W, int mode) {
  using T = typename A::T;
  DevState* S = W.st;
  if (mode == 1 && S->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(W, 0);
    return;
  }
  // Hang guard, independent of the last-block elections: the loop can run at
  // most maxit passes, so a pass number above maxit + 1 means an election was
  // lost; stop the loop with an error status.
  if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned g = ++S->guard;
    if (g > (unsigned)S->maxit + 1u) {
      S->status = ST_GUARD;
      S->done = 1;
      set_cond(W, 0);
    }
  }
  const double* __restrict__ p = (mode == 1) ? W.p : S->x;
  double* __restrict__ q = W.q;
  const int64_t n = M.n;
  const int V = W.V;
  // This iteration's normalisations (the init SpMV, mode 0, has none).  Every
  // block reads iters before its ticket; the last block increments it after.
  const uint32_t nm = (POL && mode == 1) ? norm_at(S->norm_every, S->norm_mask, S->iters + 1) : 0u;
  const bool nsum = POL && (nm & NORM_SUM);
  const int R = TPB / V;
  const int lane_in_row = threadIdx.x % V;
  const int slot = threadIdx.x / V;
  const int64_t ntiles = (n + R - 1) / R;
  T acc = A::zero();
  bool pacc = false;
  // A::ILP_SPMV tiles (t, t+G, ...) per pass: their rows' chains are independent,
  // so interleaving them hides latency; the dot leaves are still added in
  // increasing tile order, so the summation order is unchanged.
  for (int64_t t = blockIdx.x; t < ntiles; t += (int64_t)A::ILP_SPMV * gridDim.x) {
    T sum[A::ILP_SPMV];
    bool ps[A::ILP_SPMV];
    int64_t row[A::ILP_SPMV], kk[A::ILP_SPMV], ke[A::ILP_SPMV], len[A::ILP_SPMV];
#pragma unroll
    for (int u = 0; u < A::ILP_SPMV; ++u) {
      const int64_t tu = t + (int64_t)u * gridDim.x;
      row[u] = tu * R + slot;
      int64_t k0 = 0, k1 = 0;
      if (tu < ntiles && row[u] < n) { k0 = M.rp[row[u]]; k1 = M.rp[row[u] + 1]; }
      len[u] = k1 - k0;
      kk[u] = k0 + lane_in_row;
      ke[u] = k1;
      sum[u] = A::zero();
      ps[u] = false;
      if (kk[u] < ke[u]) {
        sum[u] = A::dxmul(M.val[kk[u]], ld<A>(p, n, M.col[kk[u]]));
        ps[u] = true;
        kk[u] += V;
      }
    }
    // The normalising loop is a separate copy (a test inside the loop would be
    // if-converted and cost every entry the normalisation's issue slots).
    if (nsum) row_accumulate<A, true>(M, p, n, V, sum, kk, ke);
    else row_accumulate<A, false>(M, p, n, V, sum, kk, ke);
#pragma unroll
    for (int u = 0; u < A::ILP_SPMV; ++u) {
      // Pairwise tree over the V lanes of the row (groups are aligned in the warp).
      for (int h = 1; h < V; h <<= 1) {
        T o = shfl_down<A>(sum[u], h);
        bool po = (lane_in_row % (2 * h)) == 0 && lane_in_row + h < len[u];
        if constexpr (POL) {
          // A combine into a present lane is an addition: normalise it.
          const bool add = po && ps[u];
          if (po) combine<A>(sum[u], ps[u], o, true);
          if (add && nsum) A::normalize(sum[u]);
        } else {
          if (po) combine<A>(sum[u], ps[u], o, true);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < A::ILP_SPMV; ++u) {
      const int64_t tu = t + (int64_t)u * gridDim.x;
      if (lane_in_row == 0 && tu < ntiles && row[u] < n) {
        if (!ps[u]) sum[u] = A::zero();
        if constexpr (POL) {
          if (nm & NORM_Q) A::normalize(sum[u]);
        }
        st<A>(q, n, row[u], sum[u]);
        if (mode == 1) {
          T leaf = A::mul(ld<A>(p, n, row[u]), sum[u]);
          if (pacc) acc = A::add(acc, leaf);
          else { acc = leaf; pacc = true; }
        }
      }
    }
  }
  if (mode != 1) return;
  spmv_alpha<A>(W, acc, pacc, V);
}

// ---------------------------------------------------------------------------
// r0 = (b,0,..) + (-(A x0)), p0 = r0, rho0 = r0^T r0, ||b||^2 (FP64).
// ---------------------------------------------------------------------------
// Initialisation (Algorithm 1 lines 1-2): r0 = (b, 0, ..) (+) -(A x0) with
// A x0 in q, p0 = r0, rho0 = r0^T r0, ||b||_2 in FP64; the last block sets
// the scalars and the stop flags.  PREC (Jacobi-preconditioned CG):
// z0 = w (x) r0, p0 = z0, rho0 = r0^T z0, and the FP64 residual norm from
// the collapsed r0 (the stopping residual stays FP64, Sec. IV-C).
template <class A, bool PREC = false>
__global__ void __launch_bounds__(TPB) k_init(Csr M, Work W) {
  using T = typename A::T;
  DevState* S = W.st;
  const int64_t n = M.n;
  const double* __restrict__ b = S->b;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T acc = A::zero();
  bool pacc = false;
  constexpr int NF = PREC ? 2 : 1;
  mw::MW<1> fa[NF];                       // [0] b^T b, [1] sum of collapse(r)^2
  bool pf[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) { fa[k].w[0] = 0.0; pf[k] = false; }
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      double bi = b[i];
      T ri = A::add(A::from(bi), mw::neg<A>(ld<A>(W.q, n, i)));
      st<A>(W.r, n, i, ri);
      T leaf;
      if constexpr (PREC) {
        const T zi = A::dxmul(W.w[i], ri);
        st<A>(W.p, n, i, zi);
        leaf = A::mul(ri, zi);
        const double c = A::collapse(ri);
        mw::MW<1> lc{{mw::dmul(c, c)}};
        if (pf[1]) fa[1] = mw::FP64::add(fa[1], lc);
        else { fa[1] = lc; pf[1] = true; }
      } else {
        st<A>(W.p, n, i, ri);
        leaf = A::mul(ri, ri);
      }
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      mw::MW<1> lb{{mw::dmul(bi, bi)}};
      if (pf[0]) fa[0] = mw::FP64::add(fa[0], lb);
      else { fa[0] = lb; pf[0] = true; }
    }
  }
  block_tree<A>(acc, pacc, 1);
#pragma unroll
  for (int k = 0; k < NF; ++k) block_tree<mw::FP64>(fa[k], pf[k], 1);
  double fv[NF], fo[NF];
  bool pfo[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) fv[k] = fa[k].w[0];
  T rho;
  bool prho = false;
  if (!grid_reduce_mix<A, NF>(W, acc, pacc, fv, pf, rho, prho, fo, pfo)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!prho) rho = A::zero();
    double bnorm = __dsqrt_rn(pfo[0] ? fo[0] : 0.0);
    S->bnorm = bnorm;
    S->iters = 0;
    S->status = ST_CONVERGED;
    S->done = 0;
    S->zero_x = 0;
#pragma unroll
    for (int k = 0; k < A::W; ++k) S->rho[k] = rho.w[k];
    if (bnorm == 0.0) {
      S->relres = 0.0;
      S->done = 1;
      S->zero_x = 1;
    } else {
      bool rzero = true;
#pragma unroll
      for (int k = 0; k < A::W; ++k) rzero = rzero && !mw::nonzero(rho.w[k]);
      if constexpr (PREC) S->relres = __ddiv_rn(__dsqrt_rn(pfo[NF - 1] ? fo[NF - 1] : 0.0), bnorm);
      else S->relres = __ddiv_rn(__dsqrt_rn(A::collapse(rho)), bnorm);
      if (rzero) {
        S->relres = 0.0;
        S->done = 1;
      } else if (S->maxit <= 0) {
        S->status = ST_MAXIT;
        S->done = 1;
      }
    }
  }
}

// x = 0 when ||b|| = 0.
template <int Wd>
__global__ void __launch_bounds__(TPB) k_zero_x(Csr M, Work W) {
  DevState* S = W.st;
  if (!S->zero_x) return;
  const int64_t total = (int64_t)Wd * M.n;
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < total; i += (int64_t)gridDim.x * TPB) S->x[i] = 0.0;
}

// One row per thread and tile: x += alpha p, r += (-alpha) q (normalised where
// NX / NR say), and the r^T r leaf added into the thread's slot.
// PREC: also z = w (x) r, stored over q (dead once r is updated), the leaf
// r_i z_i, and the FP64 leaf collapse(r_i)^2 added into (rr, prr).
template <class A, bool NX, bool NR, bool PREC>
__device__ __forceinline__ void update_rows(const Csr& M, const Work& W, double* __restrict__ x,
                                            const typename A::T& al, const typename A::T& mal,
                                            typename A::T& acc, bool& pacc, mw::MW<1>& rr, bool& prr) {
  using T = typename A::T;
  const int64_t n = M.n;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      T xi = A::muladd(ld<A>(x, n, i), al, ld<A>(W.p, n, i));
      if constexpr (NX) A::normalize(xi);
      st<A>(x, n, i, xi);
      T ri = A::muladd(ld<A>(W.r, n, i), mal, ld<A>(W.q, n, i));
      if constexpr (NR) A::normalize(ri);
      st<A>(W.r, n, i, ri);
      T leaf;
      if constexpr (PREC) {
        const T zi = A::dxmul(W.w[i], ri);
        st<A>(W.q, n, i, zi);
        leaf = A::mul(ri, zi);
        const double c = A::collapse(ri);
        mw::MW<1> lc{{mw::dmul(c, c)}};
        if (prr) rr = mw::FP64::add(rr, lc);
        else { rr = lc; prr = true; }
      } else {
        leaf = A::mul(ri, ri);
      }
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
    }
  }
}

// ---------------------------------------------------------------------------
// x += alpha p; r += (-alpha) q; normalise r; rho' = r^T r; stop test; beta.
// POL as for k_spmv: the default instantiation normalises r every iteration.
// PREC (Jacobi-preconditioned CG): z = w (x) r into q, rho' = r^T z, and the
// stopping residual from the FP64 sum of collapse(r_i)^2.
// ---------------------------------------------------------------------------
template <class A, bool POL = false, bool PREC = false>
__global__ void __launch_bounds__(TPB, A::MINB) k_update(Csr M, Work W) {
  using T = typename A::T;
  DevState* S = W.st;
  if (S->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(W, 0);
    return;
  }
  const int64_t n = M.n;
  double* __restrict__ x = S->x;
  T al, mal;
#pragma unroll
  for (int k = 0; k < A::W; ++k) al.w[k] = S->alpha[k];
  mal = mw::neg<A>(al);
  const int64_t ntiles = (n + TPB - 1) / TPB;
  const uint32_t nm = POL ? norm_at(S->norm_every, S->norm_mask, S->iters) : (uint32_t)NORM_R;
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> rr{{0.0}};
  bool prr = false;
  if constexpr (A::ILP == 1) {
    // One loop copy per combination of the x / r normalisations (see
    // row_accumulate); the default instantiation has only {r}.
    if constexpr (!POL) {
      update_rows<A, false, true, PREC>(M, W, x, al, mal, acc, pacc, rr, prr);
    } else {
      switch (((nm & NORM_X) ? 1 : 0) | ((nm & NORM_R) ? 2 : 0)) {
        case 0: update_rows<A, false, false, PREC>(M, W, x, al, mal, acc, pacc, rr, prr); break;
        case 1: update_rows<A, true, false, PREC>(M, W, x, al, mal, acc, pacc, rr, prr); break;
        case 2: update_rows<A, false, true, PREC>(M, W, x, al, mal, acc, pacc, rr, prr); break;
        default: update_rows<A, true, true, PREC>(M, W, x, al, mal, acc, pacc, rr, prr); break;
      }
    }
  } else {
    for (int64_t t = blockIdx.x; t < ntiles; t += (int64_t)A::ILP * gridDim.x) {
      T leaf[A::ILP], xs[A::ILP], ps_[A::ILP], rs[A::ILP], qs[A::ILP];
      bool valid[A::ILP];
      int64_t idx[A::ILP];
      // All loads first (several rows' loads in flight), then compute, then store.
#pragma unroll
      for (int u = 0; u < A::ILP; ++u) {
        const int64_t tu = t + (int64_t)u * gridDim.x;
        idx[u] = tu * TPB + threadIdx.x;
        valid[u] = tu < ntiles && idx[u] < n;
        if (valid[u]) {
          xs[u] = ld<A>(x, n, idx[u]);
          ps_[u] = ld<A>(W.p, n, idx[u]);
          rs[u] = ld<A>(W.r, n, idx[u]);
          qs[u] = ld<A>(W.q, n, idx[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < A::ILP; ++u) {
        leaf[u] = A::zero();
        if (valid[u]) {
          xs[u] = A::muladd(xs[u], al, ps_[u]);
          if (nm & NORM_X) A::normalize(xs[u]);
          rs[u] = A::muladd(rs[u], mal, qs[u]);
          if (nm & NORM_R) A::normalize(rs[u]);
          if constexpr (PREC) {
            qs[u] = A::dxmul(W.w[idx[u]], rs[u]);       // z, stored over q
            leaf[u] = A::mul(rs[u], qs[u]);
          } else {
            leaf[u] = A::mul(rs[u], rs[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < A::ILP; ++u) {
        if (valid[u]) {
          st<A>(x, n, idx[u], xs[u]);
          st<A>(W.r, n, idx[u], rs[u]);
          if constexpr (PREC) st<A>(W.q, n, idx[u], qs[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < A::ILP; ++u) {
        if (valid[u]) {
          if (pacc) acc = A::add(acc, leaf[u]);
          else { acc = leaf[u]; pacc = true; }
          if constexpr (PREC) {
            const double c = A::collapse(rs[u]);
            mw::MW<1> lc{{mw::dmul(c, c)}};
            if (prr) rr = mw::FP64::add(rr, lc);
            else { rr = lc; prr = true; }
          }
        }
      }
    }
  }
  block_tree<A>(acc, pacc, 1);
  T tot;
  bool ptot = false;
  double rrt = 0.0;
  if constexpr (PREC) {
    block_tree<mw::FP64>(rr, prr, 1);
    double fo[1];
    bool pfo[1];
    if (!grid_reduce_mix<A, 1>(W, acc, pacc, &rr.w[0], &prr, tot, ptot, fo, pfo)) return;
    if (threadIdx.x == 0) rrt = pfo[0] ? fo[0] : 0.0;
  } else {
    if (!grid_reduce<A, 0>(W, acc, pacc, tot, ptot)) return;
  }
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!ptot) tot = A::zero();
    const double relres = PREC ? __ddiv_rn(__dsqrt_rn(rrt), S->bnorm)
                               : __ddiv_rn(__dsqrt_rn(A::collapse(tot)), S->bnorm);
    S->relres = relres;
    const int it = S->iters;
    if (S->hist) S->hist[it - 1] = relres;
    unsigned cont = 0;
    if (relres < S->tol) {
      S->status = ST_CONVERGED;
      S->done = 1;
    } else if (!isfinite(relres)) {
      S->status = ST_BREAKDOWN;
      S->done = 1;
    } else if (it >= S->maxit) {
      S->status = ST_MAXIT;
      S->done = 1;
    } else {
      T rho;
#pragma unroll
      for (int k = 0; k < A::W; ++k) rho.w[k] = S->rho[k];
      T be = A::div(tot, rho);
#pragma unroll
      for (int k = 0; k < A::W; ++k) { S->beta[k] = be.w[k]; S->rho[k] = tot.w[k]; }
      cont = 1;
    }
    set_cond(W, cont);
  }
}

// p = r + beta p (POL: normalise p where the policy says so; PREC: p = z +
// beta p, z held in q).
template <class A, bool POL = false, bool PREC = false>
__global__ void __launch_bounds__(TPB, A::MINB) k_pupdate(Csr M, Work W) {
  using T = typename A::T;
  DevState* S = W.st;
  if (S->done) return;
  const int64_t n = M.n;
  T be;
#pragma unroll
  for (int k = 0; k < A::W; ++k) be.w[k] = S->beta[k];
  const int64_t stride = (int64_t)gridDim.x * TPB;
  const double* __restrict__ src = PREC ? W.q : W.r;
  const bool np_ = POL && (norm_at(S->norm_every, S->norm_mask, S->iters) & NORM_P) != 0;
  if constexpr (A::ILP == 1) {
    if (np_) {                // separate loop copies, as in row_accumulate
      for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += stride) {
        T pi = A::muladd(ld<A>(src, n, i), be, ld<A>(W.p, n, i));
        A::normalize(pi);
        st<A>(W.p, n, i, pi);
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += stride)
        st<A>(W.p, n, i, A::muladd(ld<A>(src, n, i), be, ld<A>(W.p, n, i)));
    }
  } else {
    for (int64_t i0 = (int64_t)blockIdx.x * TPB + threadIdx.x; i0 < n; i0 += (int64_t)A::ILP * stride) {
      T rr[A::ILP], pp[A::ILP];
#pragma unroll
      for (int u = 0; u < A::ILP; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < n) { rr[u] = ld<A>(src, n, i); pp[u] = ld<A>(W.p, n, i); }
      }
#pragma unroll
      for (int u = 0; u < A::ILP; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < n) {
          T pi = A::muladd(rr[u], be, pp[u]);
          if (np_) A::normalize(pi);
          st<A>(W.p, n, i, pi);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Gradient of the values: g_k = -collapse(lambda_row(k) * x_col(k)).
// ---------------------------------------------------------------------------
template <class A>
__global__ void __launch_bounds__(TPB) k_grad_values(Csr M, const double* __restrict__ lam,
                                                    const double* __restrict__ x, double* __restrict__ g) {
  const int64_t n = M.n;
  // One warp per row, lanes over the row's entries.
  const int64_t warps = (int64_t)gridDim.x * NWARP;
  const int lane = threadIdx.x & 31;
  for (int64_t row = (int64_t)blockIdx.x * NWARP + (threadIdx.x >> 5); row < n; row += warps) {
    typename A::T li = ld<A>(lam, n, row);
    for (int64_t k = M.rp[row] + lane; k < M.rp[row + 1]; k += 32)
      g[k] = mw::dneg(A::collapse(A::mul(li, ld<A>(x, n, M.col[k]))));
  }
}

// Collapse to FP64, lowest word first.
template <class A>
__global__ void __launch_bounds__(TPB) k_collapse(const double* __restrict__ xw, int64_t n, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB)
    y[i] = A::collapse(ld<A>(xw, n, i));
}

// Stand-alone dot u^T v (tiles of TPB rows, G = gridDim.x blocks); result to out[0..W-1].
template <class A>
__global__ void __launch_bounds__(TPB) k_dot(const double* __restrict__ u, const double* __restrict__ v, int64_t n,
                                             Work W, double* out) {
  using T = typename A::T;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T acc = A::zero();
  bool pacc = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      T leaf = A::mul(ld<A>(u, n, i), ld<A>(v, n, i));
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
    }
  }
  block_tree<A>(acc, pacc, 1);
  T tot;
  bool ptot = false;
  if (!grid_reduce<A, 0>(W, acc, pacc, tot, ptot)) return;
  if (threadIdx.x == 0) {
    W.st->counter = 0;
    if (!ptot) tot = A::zero();
#pragma unroll
    for (int k = 0; k < A::W; ++k) out[k] = tot.w[k];
  }
}

// Element-wise word operations (bit-exactness checks of the word algebra).
enum WordOp { OP_ADD = 0, OP_MUL = 1, OP_DXMUL = 2, OP_DIV = 3, OP_NORMALIZE = 4, OP_COLLAPSE = 5 };
template <class A>
__global__ void __launch_bounds__(TPB) k_word_op(int op, int64_t n, const double* __restrict__ a,
                                                 const double* __restrict__ b, double* __restrict__ c) {
  using T = typename A::T;
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    switch (op) {
      case OP_ADD: st<A>(c, n, i, A::add(ld<A>(a, n, i), ld<A>(b, n, i))); break;
      case OP_MUL: st<A>(c, n, i, A::mul(ld<A>(a, n, i), ld<A>(b, n, i))); break;
      case OP_DXMUL: st<A>(c, n, i, A::dxmul(a[i], ld<A>(b, n, i))); break;
      case OP_DIV: st<A>(c, n, i, A::div(ld<A>(a, n, i), ld<A>(b, n, i))); break;
      case OP_NORMALIZE: { T t = ld<A>(a, n, i); A::normalize(t); st<A>(c, n, i, t); } break;
      case OP_COLLAPSE: c[i] = A::collapse(ld<A>(a, n, i)); break;
      default: break;
    }
  }
}

// Kernel table of one arithmetic, used by the host runtime.
struct KernelTable {
  int words;
  int minb;                 // blocks per SM the loop kernels are compiled for (the plan's G = minb x SMs)
  const void* spmv;
  const void* spmv_pol;     // the three loop kernels under a non-default normalisation policy
  const void* update_pol;
  const void* pupdate_pol;
  const void* init_pcg;     // Jacobi-preconditioned CG: init, update and p update,
  const void* update_pcg;   // default policy / any policy
  const void* pupdate_pcg;
  const void* update_pcg_pol;
  const void* pupdate_pcg_pol;
  const void* init;
  const void* zero_x;
  const void* update;
  const void* pupdate;
  const void* grad_values;
  const void* collapse;
  const void* dot;
  const void* word_op;
};

// AS: the arithmetic type used by the SpMV kernel (the same arithmetic, possibly
// with another pipe-balancing policy; every policy gives the same bits).
template <class A, class AS = A>
KernelTable make_table() {
  KernelTable t;
  t.words = A::W;
  t.minb = A::MINB;
  t.spmv = (const void*)&k_spmv<AS>;
  t.init_pcg = (const void*)&k_init<A, true>;
  t.update_pcg = (const void*)&k_update<A, false, true>;
  t.pupdate_pcg = (const void*)&k_pupdate<A, false, true>;
  if constexpr (A::NORMALISES) {
    t.spmv_pol = (const void*)&k_spmv<AS, true>;
    t.update_pol = (const void*)&k_update<A, true>;
    t.pupdate_pol = (const void*)&k_pupdate<A, true>;
    t.update_pcg_pol = (const void*)&k_update<A, true, true>;
    t.pupdate_pcg_pol = (const void*)&k_pupdate<A, true, true>;
  } else {                  // the policy cannot change these arithmetics' results
    t.spmv_pol = t.spmv;
    t.update_pol = t.update;
    t.pupdate_pol = t.pupdate;
    t.update_pcg_pol = t.update_pcg;
    t.pupdate_pcg_pol = t.pupdate_pcg;
  }
  t.init = (const void*)&k_init<A>;
  t.zero_x = (const void*)&k_zero_x<A::W>;
  t.update = (const void*)&k_update<A>;
  t.pupdate = (const void*)&k_pupdate<A>;
  t.grad_values = (const void*)&k_grad_values<A>;
  t.collapse = (const void*)&k_collapse<A>;
  t.dot = (const void*)&k_dot<A>;
  t.word_op = (const void*)&k_word_op<A>;
  return t;
}

}  // namespace mwk
