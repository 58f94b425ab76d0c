// BiCGStab kernels for one arithmetic (an extension for nonsymmetric systems;
// the paper's solver is CG, Algorithm 1, and Sec. VI names other iterative
// methods as future work).
//
// One iteration of the textbook recurrence (van der Vorst), shadow residual
// rh = r0, is five kernels:
//   k_bi_p      p = r (first pass) or p = r (+) beta*(p (+) (-omega)*v)
//   k_bi_spmv<0> v = A p fused with rh^T v; last block: alpha = rho / rh^T v
//   k_bi_s      s = r (+) (-alpha)*v (normalised for the quasi arithmetics),
//               FP64 ||s||; last block: the early exit when ||s|| / ||b|| < tol
//   k_bi_spmv<1> t = A s fused with t^T s and t^T t; last block: omega
//   k_bi_xr     x = (x (+) alpha*p) (+) omega*s, r = s (+) (-omega)*t
//               (normalised), rho' = rh^T r, FP64 ||r||; last block: stop test,
//               beta = (rho' / rho) * (alpha / omega)
// plus k_bi_init (r0, rh = r0, rho0, ||b||, ||r0||) after the CG SpMV of x0.
// Vectors: r, p (the CG workspace), v (the CG q), rh, s, t (BiWork).  The
// summation order is the CG kernels' (SpMV tiles of T/V rows for the fused
// SpMV dots, vector tiles of T rows otherwise), so the CPU oracle's mirrored
// BiCGStab gives the same bits.  The stopping residuals are FP64 (Sec. IV-C):
// sqrt(sum collapse(.)^2) / ||b||.
#pragma once
#include "cg_kernels.cuh"

namespace mwk {

struct BiWork {
  Work w;                   // r, p, q (= v), partials, state, graph condition, plan
  double* rh;               // shadow residual, f64[w][n]
  double* s;
  double* t;
};

template <class A>
__device__ __forceinline__ bool bad_scalar(const typename A::T& t) {
  const double c = A::collapse(t);
  return c == 0.0 || !isfinite(c);
}

template <class A>
__device__ __forceinline__ void load_scalar(const double* src, typename A::T& t) {
#pragma unroll
  for (int k = 0; k < A::W; ++k) t.w[k] = src[k];
}
template <class A>
__device__ __forceinline__ void store_scalar(double* dst, const typename A::T& t) {
#pragma unroll
  for (int k = 0; k < A::W; ++k) dst[k] = t.w[k];
}

// FP64 leaf collapse(x)^2 added into (acc, pacc).
template <class A>
__device__ __forceinline__ void add_sq(mw::MW<1>& acc, bool& pacc, const typename A::T& x) {
  const double c = A::collapse(x);
  mw::MW<1> l{{mw::dmul(c, c)}};
  if (pacc) acc = mw::FP64::add(acc, l);
  else { acc = l; pacc = true; }
}

// One pairwise-tree pass over the G block partials of a multi-word value at
// slots [off, off + W) with its presence at poff; the result lands in thread
// 0's (out, pout).
template <class A>
__device__ __forceinline__ void tree_pass(const Work& W, int off, int poff, typename A::T* sv, unsigned char* sp,
                                          typename A::T& out, bool& pout) {
  using T = typename A::T;
  const int G = gridDim.x;
  for (int bk = threadIdx.x; bk < G; bk += blockDim.x) {
    const double* src = W.part + (size_t)bk * PART;
    T tv;
#pragma unroll
    for (int k = 0; k < A::W; ++k) tv.w[k] = __ldcg(src + off + k);
    sv[bk] = tv;
    sp[bk] = __ldcg(src + poff) != 0.0;
  }
  __syncthreads();
  for (int h = 1; h < G; h <<= 1) {
    for (int s2 = 2 * h * threadIdx.x; s2 + h < G; s2 += 2 * h * blockDim.x) {
      T x = sv[s2];
      bool px = sp[s2] != 0;
      combine<A>(x, px, sv[s2 + h], sp[s2 + h] != 0);
      sv[s2] = x;
      sp[s2] = px;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out = sv[0];
    pout = sp[0] != 0;
  }
  __syncthreads();
}

// Two multi-word values reduced by the pairwise tree under one election: the
// first in partial slots [0, W) (presence PRES), the second in [FV, FV + W)
// (presence PART - 1).  The two trees run one after the other in the same
// G * (8 W + 1) bytes of dynamic shared memory.
template <class A>
__device__ __forceinline__ bool grid_reduce_two(const Work& W, const typename A::T& a, bool pa,
                                                const typename A::T& b, bool pb, typename A::T& oa, bool& poa,
                                                typename A::T& ob, bool& pob) {
  using T = typename A::T;
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    double* dst = W.part + (size_t)blockIdx.x * PART;
#pragma unroll
    for (int k = 0; k < A::W; ++k) { dst[k] = a.w[k]; dst[FV + k] = b.w[k]; }
    dst[PRES] = pa ? 1.0 : 0.0;
    dst[PART - 1] = pb ? 1.0 : 0.0;
    __threadfence();
    unsigned tk = atomicAdd(&W.st->counter, 1u);
    am_last = (tk == (unsigned)(gridDim.x - 1));
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  extern __shared__ double dyn[];
  T* sv = reinterpret_cast<T*>(dyn);
  unsigned char* sp = reinterpret_cast<unsigned char*>(sv + gridDim.x);
  tree_pass<A>(W, 0, PRES, sv, sp, oa, poa);
  tree_pass<A>(W, FV, PART - 1, sv, sp, ob, pob);
  return true;
}

// r0 = (b, 0, ..) (+) -(A x0) with A x0 in v (the CG SpMV, mode 0); rh = r0;
// rho0 = rh^T r0; ||b||_2 and ||r0||_2 in FP64.
template <class A>
__global__ void __launch_bounds__(TPB) k_bi_init(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  const int64_t n = M.n;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> fa[2] = {{{0.0}}, {{0.0}}};
  bool pf[2] = {false, false};
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const double bi = S->b[i];
      const T ri = A::add(A::from(bi), mw::neg<A>(ld<A>(W.q, n, i)));
      st<A>(W.r, n, i, ri);
      st<A>(B.rh, n, i, ri);
      const T leaf = A::mul(ri, ri);
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      mw::MW<1> lb{{mw::dmul(bi, bi)}};
      if (pf[0]) fa[0] = mw::FP64::add(fa[0], lb);
      else { fa[0] = lb; pf[0] = true; }
      add_sq<A>(fa[1], pf[1], ri);
    }
  }
  block_tree<A>(acc, pacc, 1);
  block_tree<mw::FP64>(fa[0], pf[0], 1);
  block_tree<mw::FP64>(fa[1], pf[1], 1);
  const double fv[2] = {fa[0].w[0], fa[1].w[0]};
  double fo[2];
  bool pfo[2];
  T rho;
  bool prho = false;
  if (!grid_reduce_mix<A, 2>(W, acc, pacc, fv, pf, rho, prho, fo, pfo)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!prho) rho = A::zero();
    const double bnorm = __dsqrt_rn(pfo[0] ? fo[0] : 0.0);
    S->bnorm = bnorm;
    S->iters = 0;
    S->status = ST_CONVERGED;
    S->done = 0;
    S->zero_x = 0;
    S->early = 0;
    store_scalar<A>(S->rho, rho);
    if (bnorm == 0.0) {
      S->relres = 0.0;
      S->done = 1;
      S->zero_x = 1;
    } else {
      bool rzero = true;
#pragma unroll
      for (int k = 0; k < A::W; ++k) rzero = rzero && !mw::nonzero(rho.w[k]);
      S->relres = __ddiv_rn(__dsqrt_rn(pfo[1] ? fo[1] : 0.0), bnorm);
      if (rzero) {
        S->relres = 0.0;
        S->done = 1;
      } else if (S->maxit <= 0) {
        S->status = ST_MAXIT;
        S->done = 1;
      } else if (bad_scalar<A>(rho)) {
        S->status = ST_BREAKDOWN;
        S->done = 1;
      }
    }
  }
}

// p = r on the first pass, else p = r (+) beta*(p (+) (-omega)*v).
template <class A>
__global__ void __launch_bounds__(TPB, A::MINB) k_bi_p(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  if (S->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(W, 0);
    return;
  }
  // Hang guard (as in k_spmv): more passes than maxit + 1 means a lost election.
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned g = ++S->guard;
    if (g > (unsigned)S->maxit + 1u) {
      S->status = ST_GUARD;
      S->done = 1;
      set_cond(W, 0);
    }
  }
  const int64_t n = M.n;
  const int64_t stride = (int64_t)gridDim.x * TPB;
  if (S->iters == 0) {
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += stride) st<A>(W.p, n, i, ld<A>(W.r, n, i));
    return;
  }
  T be, om;
  load_scalar<A>(S->beta, be);
  load_scalar<A>(S->omega, om);
  const T mom = mw::neg<A>(om);
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += stride) {
    const T tmp = A::muladd(ld<A>(W.p, n, i), mom, ld<A>(W.q, n, i));
    st<A>(W.p, n, i, A::muladd(ld<A>(W.r, n, i), be, tmp));
  }
}

// WHICH 0: v = A p, rh^T v, alpha.  WHICH 1: t = A s, t^T s and t^T t, omega.
template <class A, int WHICH>
__global__ void __launch_bounds__(TPB, A::MINB) k_bi_spmv(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  if (S->done || (WHICH == 1 && S->early)) return;
  const double* __restrict__ x = WHICH ? B.s : W.p;
  double* __restrict__ y = WHICH ? B.t : W.q;
  const int64_t n = M.n;
  const int V = W.V;
  const int R = TPB / V;
  const int lane_in_row = threadIdx.x % V;
  const int slot = threadIdx.x / V;
  const int64_t ntiles = (n + R - 1) / R;
  T a1 = A::zero(), a2 = A::zero();
  bool p1 = false, p2 = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t row = t * R + slot;
    int64_t k0 = 0, k1 = 0;
    if (row < n) { k0 = M.rp[row]; k1 = M.rp[row + 1]; }
    const int64_t len = k1 - k0;
    T sum = A::zero();
    bool ps = false;
    int64_t k = k0 + lane_in_row;
    if (k < k1) {
      sum = A::dxmul(M.val[k], ld<A>(x, n, M.col[k]));
      ps = true;
      for (k += V; k < k1; k += V) sum = A::dxmuladd(sum, M.val[k], ld<A>(x, n, M.col[k]));
    }
    for (int h = 1; h < V; h <<= 1) {
      T o = shfl_down<A>(sum, h);
      bool po = (lane_in_row % (2 * h)) == 0 && lane_in_row + h < len;
      if (po) combine<A>(sum, ps, o, true);
    }
    if (lane_in_row == 0 && row < n) {
      if (!ps) sum = A::zero();
      st<A>(y, n, row, sum);
      if (WHICH == 0) {
        const T l = A::mul(ld<A>(B.rh, n, row), sum);
        if (p1) a1 = A::add(a1, l);
        else { a1 = l; p1 = true; }
      } else {
        const T l1 = A::mul(sum, ld<A>(B.s, n, row));
        const T l2 = A::mul(sum, sum);
        if (p1) a1 = A::add(a1, l1);
        else { a1 = l1; p1 = true; }
        if (p2) a2 = A::add(a2, l2);
        else { a2 = l2; p2 = true; }
      }
    }
  }
  block_tree<A>(a1, p1, V);
  if (WHICH == 0) {
    T tot;
    bool ptot = false;
    if (!grid_reduce<A, 0>(W, a1, p1, tot, ptot)) return;
    if (threadIdx.x == 0) {
      S->counter = 0;
      if (!ptot) tot = A::zero();
      S->iters += 1;
      if (bad_scalar<A>(tot)) {
        S->status = ST_BREAKDOWN;
        S->done = 1;
        set_cond(W, 0);
      } else {
        T rho;
        load_scalar<A>(S->rho, rho);
        store_scalar<A>(S->alpha, A::div(rho, tot));
      }
    }
  } else {
    block_tree<A>(a2, p2, V);
    T ts, tt;
    bool pts = false, ptt = false;
    if (!grid_reduce_two<A>(W, a1, p1, a2, p2, ts, pts, tt, ptt)) return;
    if (threadIdx.x == 0) {
      S->counter = 0;
      if (!pts) ts = A::zero();
      if (!ptt) tt = A::zero();
      if (bad_scalar<A>(tt)) {
        S->status = ST_BREAKDOWN;
        S->done = 1;
        set_cond(W, 0);
      } else {
        store_scalar<A>(S->omega, A::div(ts, tt));
      }
    }
  }
}

// s = r (+) (-alpha)*v, normalised; FP64 ||s||; the early exit.
template <class A>
__global__ void __launch_bounds__(TPB, A::MINB) k_bi_s(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  if (S->done) return;
  const int64_t n = M.n;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T al;
  load_scalar<A>(S->alpha, al);
  const T mal = mw::neg<A>(al);
  mw::MW<1> acc{{0.0}};
  bool pacc = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      T si = A::muladd(ld<A>(W.r, n, i), mal, ld<A>(W.q, n, i));
      A::normalize(si);
      st<A>(B.s, n, i, si);
      add_sq<A>(acc, pacc, si);
    }
  }
  block_tree<mw::FP64>(acc, pacc, 1);
  mw::MW<1> tot;
  bool ptot = false;
  if (!grid_reduce<mw::FP64, 0>(W, acc, pacc, tot, ptot)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    const double rs = __ddiv_rn(__dsqrt_rn(ptot ? tot.w[0] : 0.0), S->bnorm);
    if (rs < S->tol) {
      S->early = 1;
      S->relres = rs;
      if (S->hist) S->hist[S->iters - 1] = rs;
    }
  }
}

// x = (x (+) alpha*p) (+) omega*s; r = s (+) (-omega)*t, normalised;
// rho' = rh^T r; FP64 ||r||; stop test; beta.  On the early exit: x = x (+)
// alpha*p only, and the last block ends the loop.
template <class A>
__global__ void __launch_bounds__(TPB, A::MINB) k_bi_xr(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  if (S->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(W, 0);
    return;
  }
  const int64_t n = M.n;
  double* __restrict__ x = S->x;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T al, om;
  load_scalar<A>(S->alpha, al);
  load_scalar<A>(S->omega, om);
  if (S->early) {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) st<A>(x, n, i, A::muladd(ld<A>(x, n, i), al, ld<A>(W.p, n, i)));
    }
    // Every block has written its rows before the last one ends the loop.
    mw::MW<1> z{{0.0}}, tot;
    bool ptot = false;
    if (!grid_reduce<mw::FP64, 0>(W, z, false, tot, ptot)) return;
    if (threadIdx.x == 0) {
      S->counter = 0;
      S->status = ST_CONVERGED;
      S->done = 1;
      set_cond(W, 0);
    }
    return;
  }
  const T mom = mw::neg<A>(om);
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> rr{{0.0}};
  bool prr = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const T si = ld<A>(B.s, n, i);
      st<A>(x, n, i, A::muladd(A::muladd(ld<A>(x, n, i), al, ld<A>(W.p, n, i)), om, si));
      T ri = A::muladd(si, mom, ld<A>(B.t, n, i));
      A::normalize(ri);
      st<A>(W.r, n, i, ri);
      const T leaf = A::mul(ld<A>(B.rh, n, i), ri);
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      add_sq<A>(rr, prr, ri);
    }
  }
  block_tree<A>(acc, pacc, 1);
  block_tree<mw::FP64>(rr, prr, 1);
  T rho1;
  bool prho = false;
  double fo[1];
  bool pfo[1];
  if (!grid_reduce_mix<A, 1>(W, acc, pacc, &rr.w[0], &prr, rho1, prho, fo, pfo)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!prho) rho1 = A::zero();
    const double relres = __ddiv_rn(__dsqrt_rn(pfo[0] ? fo[0] : 0.0), S->bnorm);
    S->relres = relres;
    const int it = S->iters;
    if (S->hist) S->hist[it - 1] = relres;
    unsigned cont = 0;
    if (relres < S->tol) {
      S->status = ST_CONVERGED;
      S->done = 1;
    } else if (!isfinite(relres) || A::collapse(om) == 0.0) {
      S->status = ST_BREAKDOWN;
      S->done = 1;
    } else if (it >= S->maxit) {
      S->status = ST_MAXIT;
      S->done = 1;
    } else if (bad_scalar<A>(rho1)) {          // the next pass's rho
      S->status = ST_BREAKDOWN;
      S->done = 1;
    } else {
      T rho;
      load_scalar<A>(S->rho, rho);
      store_scalar<A>(S->beta, A::mul(A::div(rho1, rho), A::div(al, om)));
      store_scalar<A>(S->rho, rho1);
      cont = 1;
    }
    set_cond(W, cont);
  }
}

struct BiTable {
  const void* init;
  const void* p;
  const void* spmv_v;
  const void* s;
  const void* spmv_t;
  const void* xr;
};

template <class A>
BiTable make_bitable() {
  BiTable t;
  t.init = (const void*)&k_bi_init<A>;
  t.p = (const void*)&k_bi_p<A>;
  t.spmv_v = (const void*)&k_bi_spmv<A, 0>;
  t.s = (const void*)&k_bi_s<A>;
  t.spmv_t = (const void*)&k_bi_spmv<A, 1>;
  t.xr = (const void*)&k_bi_xr<A>;
  return t;
}

}  // namespace mwk
