// BiCGStab in QQF / QF (four FP32 words) with the power-of-two scaling of
// cg_float.cuh.  r, p, v, s and t are held at 2^E (r = 2^E r~, ...), the
// shadow residual at 2^E0 (rh~ = r~0).  rho = rh^T r and rh^T v carry the
// same factor 2^(E0+E), so alpha = rho~ / rh~^T v~ and omega = t~^T s~ / t~^T t~
// are the unscaled values and the generic k_bi_p and k_bi_spmv apply as they
// are; three kernels differ from bicg_kernels.cuh's:
//   k_bi_init_qqf  r~0 = split3(b 2^-E0) (+) 2^-E0 (-(A x0)), rh~ = r~0,
//                  rho~0, the FP64 residual 2^E0 sqrt(sum collapse(r~)^2)/||b||
//                  (E0 and ||b|| from k_qqf_bnorm, which runs before it)
//   k_bi_s_qqf     s~ = normalise(r~ + (-alpha) v~); the early exit on
//                  2^E sqrt(sum collapse(s~)^2) / ||b||
//   k_bi_xr_qqf    x = (x + (alpha 2^E) p~) + (omega 2^E) s~;
//                  r~' = 2^-sh normalise(s~ + (-omega) t~), E' = E + sh;
//                  rho~' = rh~^T r~'; the stop test on 2^E' sqrt(...) / ||b||;
//                  beta~ = (rho~' / rho~)(alpha / omega), so that
//                  p~' = r~' + beta~ (p~ + (-omega) v~) is at 2^E' (k_bi_p)
// The shift sh of an iteration is taken from the FP64 sum of the r~ it
// replaces, clamped as in CG; the range of x is tested as in k_qqf_update
// (after every x update, the early exit's included).  The same sequence as the
// oracle's scaled BiCGStab, bit for bit.
#pragma once
#include "bicg_kernels.cuh"
#include "cg_float.cuh"

namespace mwk {

// Largest |x_i0| bits of the block's rows into the solve's atomic maximum
// (before the block's ticket; the reductions fence).
__device__ __forceinline__ void qqf_xmax(DevState* S, uint32_t xb) {
  __shared__ uint32_t sxb[NWARP];
  xb = __reduce_max_sync(0xFFFFFFFFu, xb);
  if ((threadIdx.x & 31) == 0) sxb[threadIdx.x >> 5] = xb;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < NWARP; ++k) m = max(m, sxb[k]);
    atomicMax(&S->xmax_bits, m);
  }
}

template <class A>
__global__ void __launch_bounds__(TPB) k_bi_init_qqf(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  const int64_t n = M.n;
  const int E = qqf_E(S);
  const double sb = mw::pow2d(-E);
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> rr{{0.0}};
  bool prr = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const T ri = A::add(A::from(__dmul_rn(S->b[i], sb)), A::scale(A::neg(ld<A>(W.q, n, i)), -E));
      st<A>(W.r, n, i, ri);
      st<A>(B.rh, n, i, ri);
      const T leaf = A::mul(ri, ri);
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      add_sq<A>(rr, prr, ri);
    }
  }
  block_tree<A>(acc, pacc, 1);
  block_tree<mw::FP64>(rr, prr, 1);
  T rho;
  bool prho = false;
  double fo[1];
  bool pfo[1];
  if (!grid_reduce_mix<A, 1>(W, acc, pacc, &rr.w[0], &prr, rho, prho, fo, pfo)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!prho) rho = A::zero();
    const double bnorm = S->bnorm;
    const double c = pfo[0] ? fo[0] : 0.0;
    S->iters = 0;
    S->status = ST_CONVERGED;
    S->done = 0;
    S->zero_x = 0;
    S->early = 0;
    S->xmax_bits = 0;
    store_scalar<A>(S->rho, rho);
    if (bnorm == 0.0) {
      S->relres = 0.0;
      S->done = 1;
      S->zero_x = 1;
    } else {
      bool rzero = true;
#pragma unroll
      for (int k = 0; k < A::W; ++k) rzero = rzero && (rho.w[k] == 0.0f);
      S->relres = __ddiv_rn(__dmul_rn(__dsqrt_rn(c), mw::pow2d(E)), bnorm);
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
    qqf_set_scale(S, E, 0, clamp_shift(scale_exp(c, n), E));
  }
}

template <class A>
__global__ void __launch_bounds__(TPB, A::MINB) k_bi_s_qqf(Csr M, BiWork B) {
  using T = typename A::T;
  const Work& W = B.w;
  DevState* S = W.st;
  if (S->done) return;
  const int64_t n = M.n;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T al;
  load_scalar<A>(S->alpha, al);
  const T mal = A::neg(al);
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
    const double rs = __ddiv_rn(__dmul_rn(__dsqrt_rn(ptot ? tot.w[0] : 0.0), mw::pow2d(qqf_E(S))), S->bnorm);
    if (rs < S->tol) {
      S->early = 1;
      S->relres = rs;
      if (S->hist) S->hist[S->iters - 1] = rs;
    }
  }
}

template <class A>
__global__ void __launch_bounds__(TPB, A::MINB) k_bi_xr_qqf(Csr M, BiWork B) {
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
  const int E = qqf_E(S), sh = qqf_next_shift(S);
  T al, om;
  load_scalar<A>(S->alpha, al);
  load_scalar<A>(S->omega, om);
  const T ca = A::scale(al, E);
  uint32_t xb = 0;                 // largest |x_i0| bits of this thread's rows
  if (S->early) {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) {
        const T xn = A::muladd(ld<A>(x, n, i), ca, ld<A>(W.p, n, i));
        st<A>(x, n, i, xn);
        xb = max(xb, __float_as_uint(xn.w[0]) & 0x7FFFFFFFu);
      }
    }
    qqf_xmax(S, xb);
    // Every block has written its rows before the last one ends the loop.
    mw::MW<1> z{{0.0}}, tot;
    bool ptot = false;
    if (!grid_reduce<mw::FP64, 0>(W, z, false, tot, ptot)) return;
    if (threadIdx.x == 0) {
      S->counter = 0;
      const uint32_t xm = atomicOr(&S->xmax_bits, 0u);
      S->xmax_bits = 0;
      S->status = (xm >= 0x7F800000u || xm < 0x00800000u) ? ST_RANGE : ST_CONVERGED;
      S->done = 1;
      set_cond(W, 0);
    }
    return;
  }
  const T co = A::scale(om, E);
  const T mom = A::neg(om);
  const float ps = mw::pow2f(-sh);
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> rr{{0.0}};
  bool prr = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const T si = ld<A>(B.s, n, i);
      const T xn = A::muladd(A::muladd(ld<A>(x, n, i), ca, ld<A>(W.p, n, i)), co, si);
      st<A>(x, n, i, xn);
      xb = max(xb, __float_as_uint(xn.w[0]) & 0x7FFFFFFFu);
      T ri = A::muladd(si, mom, ld<A>(B.t, n, i));
      A::normalize(ri);
#pragma unroll
      for (int j = 0; j < A::W; ++j) ri.w[j] = mw::fmul(ri.w[j], ps);
      st<A>(W.r, n, i, ri);
      const T leaf = A::mul(ld<A>(B.rh, n, i), ri);
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      add_sq<A>(rr, prr, ri);
    }
  }
  qqf_xmax(S, xb);
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
    const uint32_t xm = atomicOr(&S->xmax_bits, 0u);
    S->xmax_bits = 0;
    const bool x_nonfinite = xm >= 0x7F800000u, x_under = xm < 0x00800000u;
    const int En = E + sh;
    const double c = pfo[0] ? fo[0] : 0.0;
    const double relres = __ddiv_rn(__dmul_rn(__dsqrt_rn(c), mw::pow2d(En)), S->bnorm);
    S->relres = relres;
    const int it = S->iters;
    if (S->hist) S->hist[it - 1] = relres;
    unsigned cont = 0;
    if (x_nonfinite) {
      S->status = ST_RANGE;
      S->done = 1;
    } else if (relres < S->tol) {
      S->status = x_under ? ST_RANGE : ST_CONVERGED;
      S->done = 1;
    } else if (!isfinite(relres) || A::collapse(om) == 0.0) {
      S->status = ST_BREAKDOWN;
      S->done = 1;
    } else if (it >= S->maxit) {
      S->status = x_under ? ST_RANGE : ST_MAXIT;
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
    qqf_set_scale(S, En, sh, clamp_shift(scale_exp(c, n), En));
    set_cond(W, cont);
  }
}

template <class A>
BiTable make_bitable_qqf() {
  BiTable t;
  t.init = (const void*)&k_bi_init_qqf<A>;
  t.p = (const void*)&k_bi_p<A>;
  t.spmv_v = (const void*)&k_bi_spmv<A, 0>;
  t.s = (const void*)&k_bi_s_qqf<A>;
  t.spmv_t = (const void*)&k_bi_spmv<A, 1>;
  t.xr = (const void*)&k_bi_xr_qqf<A>;
  return t;
}

}  // namespace mwk
