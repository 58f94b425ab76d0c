// CG in QQF (four FP32 words, mw_float.cuh) with power-of-two scaling.
//
// FP32's exponent stops at 2^-126 (2^-149 subnormal): the lower words of a
// residual near 1e-14 |b|, and of the squares in r^T r, would underflow.  The
// solver therefore keeps r = 2^E r~ and p = 2^E p~ with one integer exponent
// E chosen so that r~ has a root mean square near one; x is
// unscaled.  With rho~ = r~^T r~, pi~ = p~^T q~ and q~ = A p~ (Algorithm 1
// rewritten for the scaled vectors):
//   alpha~ = rho~ / pi~                       (k_spmv, unchanged)
//   x     += (alpha~ 2^E) p~
//   r~'    = 2^-s normalise(r~ + (-alpha~) q~),  E' = E + s
//   rho~'  = r~'^T r~',  ||r|| = 2^E' sqrt(rho~')
//   beta~  = rho~' / rho~,  p~' = r~' + (beta~ 2^s) p~
// The shift s of an iteration is fixed before it, from the rho~ of the r~ it
// updates: floor((ilogb(rho~) - ilogb(n)) / 2), the floor of log2 of the root
// mean square, clamped to [-100, 100] and so that |E + s| <= 1000.  E0 is the
// same function of ||b||^2 (k_qqf_bnorm, a pass before the init), and
// r~0 = split3(b_i 2^-E0) (+) 2^-E0 (-(A x0)).  Every scaled word is one
// correctly rounded multiplication by a power of two.
//
// The kernels keep the plan's summation order (the vector kernels' tiles of
// TPB rows over G blocks) and the stop tests of cg_kernels.cuh.  E, the shift
// applied by this iteration's update and the shift the next update applies
// are kept in the DevState (q_e, q_s, q_s_next).
#pragma once
#include "cg_kernels.cuh"
#include "mw_float.cuh"

namespace mwk {

// Packed storage of QQF vectors: slot k of element i, at k n + i, holds words
// 2k and 2k+1 as a float2 (explicit specialisations of cg_kernels.cuh's
// loads and stores, so every generic kernel reads and writes the packed form).
template <>
__device__ __forceinline__ mw::QQF::T ld<mw::QQF>(const double* __restrict__ v, int64_t n, int64_t i) {
  const float2* __restrict__ f = reinterpret_cast<const float2*>(v);
  const float2 u0 = f[i], u1 = f[n + i];
  return mw::QQF::T{{u0.x, u0.y, u1.x, u1.y}};
}
template <>
__device__ __forceinline__ void st<mw::QQF>(double* __restrict__ v, int64_t n, int64_t i, const mw::QQF::T& t) {
  float2* __restrict__ f = reinterpret_cast<float2*>(v);
  f[i] = make_float2(t.w[0], t.w[1]);
  f[n + i] = make_float2(t.w[2], t.w[3]);
}
template <>
__device__ __forceinline__ mw::QF::T ld<mw::QF>(const double* __restrict__ v, int64_t n, int64_t i) {
  return ld<mw::QQF>(v, n, i);
}
template <>
__device__ __forceinline__ void st<mw::QF>(double* __restrict__ v, int64_t n, int64_t i, const mw::QF::T& t) {
  st<mw::QQF>(v, n, i, t);
}
constexpr int kQqfSlots = 2;          // 8-byte slots per element

__device__ __forceinline__ int qqf_E(const DevState* S) { return S->q_e; }
__device__ __forceinline__ int qqf_shift(const DevState* S) { return S->q_s; }
__device__ __forceinline__ int qqf_next_shift(const DevState* S) { return S->q_s_next; }
__device__ __forceinline__ void qqf_set_scale(DevState* S, int E, int s, int s_next) {
  S->q_e = E;
  S->q_s = s;
  S->q_s_next = s_next;
}

// ilogb of a positive finite FP64 value, from the bits.
__device__ __forceinline__ int ilogb_pos(double c) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(c);
  const int e = (int)(u >> 52);
  return e != 0 ? e - 1023 : -1011 - __clzll((long long)u);
}
__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }
// floor(log2) of the root mean square of a vector whose squares sum to c.
__device__ __forceinline__ int scale_exp(double c, int64_t n) {
  if (!(c > 0.0) || !isfinite(c)) return 0;
  return floor_half(ilogb_pos(c) - ilogb_pos((double)n));
}
__device__ __forceinline__ int clamp_shift(int t, int E) {
  const int lo = max(-100, -1000 - E), hi = min(100, 1000 - E);
  return min(hi, max(lo, t));
}
template <class A>
__device__ __forceinline__ typename A::T load_scalar_f(const double* s) {
  typename A::T t;
#pragma unroll
  for (int k = 0; k < A::W; ++k) t.w[k] = (float)s[k];
  return t;
}

// ||b||_2^2 in FP64 in the init's order; sets ||b|| and E0.
template <class A>
__global__ void __launch_bounds__(TPB) k_qqf_bnorm(Csr M, Work W) {
  DevState* S = W.st;
  const int64_t n = M.n;
  const double* __restrict__ b = S->b;
  const int64_t ntiles = (n + TPB - 1) / TPB;
  mw::MW<1> acc{{0.0}};
  bool pacc = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const mw::MW<1> l{{mw::dmul(b[i], b[i])}};
      if (pacc) acc = mw::FP64::add(acc, l);
      else { acc = l; pacc = true; }
    }
  }
  block_tree<mw::FP64>(acc, pacc, 1);
  mw::MW<1> tot;
  bool ptot = false;
  if (!grid_reduce<mw::FP64, 0>(W, acc, pacc, tot, ptot)) return;
  if (threadIdx.x == 0) {
    S->counter = 0;
    const double bb = ptot ? tot.w[0] : 0.0;
    S->bnorm = __dsqrt_rn(bb);
    qqf_set_scale(S, scale_exp(bb, n), 0, 0);
  }
}

// r~0 = split3(b 2^-E0) (+) 2^-E0 (-(A x0)) with A x0 in q, p~0 = r~0,
// rho~0 = r~0^T r~0; the last block sets the scalars and the stop flags.
// PREC (Jacobi-preconditioned CG): z~0 = w (x) r~0 into q, p~0 = z~0,
// rho~0 = r~0^T z~0, and the residual norm and the shift from the FP64 sum
// of collapse(r~_i)^2.
template <class A, bool PREC = false>
__global__ void __launch_bounds__(TPB) k_qqf_init(Csr M, Work W) {
  using T = typename A::T;
  DevState* S = W.st;
  const int64_t n = M.n;
  const double* __restrict__ b = S->b;
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
      const T ri = A::add(A::from(__dmul_rn(b[i], sb)), A::scale(A::neg(ld<A>(W.q, n, i)), -E));
      st<A>(W.r, n, i, ri);
      T leaf;
      if constexpr (PREC) {
        const T zi = A::dxmul(W.w[i], ri);
        st<A>(W.q, n, i, zi);
        st<A>(W.p, n, i, zi);
        leaf = A::mul(ri, zi);
        const double c = A::collapse(ri);
        const mw::MW<1> lc{{mw::dmul(c, c)}};
        if (prr) rr = mw::FP64::add(rr, lc);
        else { rr = lc; prr = true; }
      } else {
        st<A>(W.p, n, i, ri);
        leaf = A::mul(ri, ri);
      }
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
    }
  }
  block_tree<A>(acc, pacc, 1);
  T rho;
  bool prho = false;
  double rrt = 0.0;
  if constexpr (PREC) {
    block_tree<mw::FP64>(rr, prr, 1);
    double fo[1];
    bool pfo[1];
    if (!grid_reduce_mix<A, 1>(W, acc, pacc, &rr.w[0], &prr, rho, prho, fo, pfo)) return;
    if (threadIdx.x == 0) rrt = pfo[0] ? fo[0] : 0.0;
  } else {
    if (!grid_reduce<A, 0>(W, acc, pacc, rho, prho)) return;
  }
  if (threadIdx.x == 0) {
    S->counter = 0;
    if (!prho) rho = A::zero();
    const double bnorm = S->bnorm;
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
      for (int k = 0; k < A::W; ++k) rzero = rzero && (rho.w[k] == 0.0f);
      const double c = PREC ? rrt : A::collapse(rho);
      S->relres = __ddiv_rn(__dmul_rn(__dsqrt_rn(c), mw::pow2d(E)), bnorm);
      if (rzero) {
        S->relres = 0.0;
        S->done = 1;
      } else if (S->maxit <= 0) {
        S->status = ST_MAXIT;
        S->done = 1;
      }
    }
    qqf_set_scale(S, E, 0, clamp_shift(scale_exp(PREC ? rrt : A::collapse(rho), n), E));
  }
}

// x += (alpha~ 2^E) p~; r~ = 2^-s normalise(r~ + (-alpha~) q~); rho~' = r~^T r~;
// the stop test on 2^(E+s) sqrt(rho~') / ||b||; beta~; the next shift.
// Range of x (unscaled FP32 words): the largest |leading word| of the new x is
// reduced by an atomic maximum of its bits (an order-free reduction); a value
// that is not finite ends the solve with ST_RANGE, and so does a solve that
// would end converged or at maxit with every leading word below 2^-126.
// PREC: z~ = w (x) r~ into q, rho~' = r~^T z~, and the stop test and the next
// shift on the FP64 sum of collapse(r~_i)^2 (the order of pcg_jacobi's).
template <class A, bool PREC = false>
__global__ void __launch_bounds__(TPB, A::MINB) k_qqf_update(Csr M, Work W) {
  using T = typename A::T;
  DevState* S = W.st;
  if (S->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(W, 0);
    return;
  }
  const int64_t n = M.n;
  double* __restrict__ x = S->x;
  const int E = qqf_E(S), s = qqf_next_shift(S);
  const T al = load_scalar_f<A>(S->alpha);
  const T cx = A::scale(al, E);
  const T mal = A::neg(al);
  const float ps = mw::pow2f(-s);
  const int64_t ntiles = (n + TPB - 1) / TPB;
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> rr{{0.0}};
  bool prr = false;
  uint32_t xb = 0;                 // largest |x_i0| bits of this thread's rows (NaN and inf above finite)
  // A::ILP tiles (t, t + G, ...) per pass, all loads first: the kernel is bound
  // by memory latency.  Each slot still adds its leaves in increasing tile
  // order, so the summation order is that of one tile per pass.
  for (int64_t t = blockIdx.x; t < ntiles; t += (int64_t)A::ILP * gridDim.x) {
    T xs[A::ILP], ps_[A::ILP], rs[A::ILP], qs[A::ILP];
    int64_t idx[A::ILP];
    bool valid[A::ILP];
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
      if (valid[u]) {
        const T xn = A::muladd(xs[u], cx, ps_[u]);
        st<A>(x, n, idx[u], xn);
        xb = max(xb, __float_as_uint(xn.w[0]) & 0x7FFFFFFFu);
        T ri = A::muladd(rs[u], mal, qs[u]);
        A::renorm(ri);
#pragma unroll
        for (int j = 0; j < A::W; ++j) ri.w[j] = mw::fmul(ri.w[j], ps);
        st<A>(W.r, n, idx[u], ri);
        T leaf;
        if constexpr (PREC) {
          const T zi = A::dxmul(W.w[idx[u]], ri);
          st<A>(W.q, n, idx[u], zi);
          leaf = A::mul(ri, zi);
          const double c = A::collapse(ri);
          const mw::MW<1> lc{{mw::dmul(c, c)}};
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
  {
    __shared__ uint32_t sxb[NWARP];
    xb = __reduce_max_sync(0xFFFFFFFFu, xb);
    if ((threadIdx.x & 31) == 0) sxb[threadIdx.x >> 5] = xb;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t m = 0;
#pragma unroll
      for (int k = 0; k < NWARP; ++k) m = max(m, sxb[k]);
      atomicMax(&S->xmax_bits, m);     // before the block's ticket (grid_reduce fences)
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
    const uint32_t xm = atomicOr(&S->xmax_bits, 0u);
    S->xmax_bits = 0;
    const bool x_nonfinite = xm >= 0x7F800000u, x_under = xm < 0x00800000u;
    const int En = E + s;
    const double c = PREC ? rrt : A::collapse(tot);
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
    } else if (!isfinite(relres)) {
      S->status = ST_BREAKDOWN;
      S->done = 1;
    } else if (it >= S->maxit) {
      S->status = x_under ? ST_RANGE : ST_MAXIT;
      S->done = 1;
    } else {
      const T rho = load_scalar_f<A>(S->rho);
      const T be = A::div(tot, rho);
#pragma unroll
      for (int k = 0; k < A::W; ++k) { S->beta[k] = be.w[k]; S->rho[k] = tot.w[k]; }
      cont = 1;
    }
    qqf_set_scale(S, En, s, clamp_shift(scale_exp(c, n), En));
    set_cond(W, cont);
  }
}

// p~ = r~ + (beta~ 2^s) p~ (PREC: p~ = z~ + (beta~ 2^s) p~, z~ in q).
template <class A, bool PREC = false>
__global__ void __launch_bounds__(TPB, A::MINB) k_qqf_pupdate(Csr M, Work W) {
  using T = typename A::T;
  DevState* S = W.st;
  if (S->done) return;
  const int64_t n = M.n;
  const double* __restrict__ src = PREC ? W.q : W.r;
  const T cp = A::scale(load_scalar_f<A>(S->beta), qqf_shift(S));
  const int64_t stride = (int64_t)gridDim.x * TPB;
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
      if (i < n) st<A>(W.p, n, i, A::muladd(rr[u], cp, pp[u]));
    }
  }
}

// The kernel table of QQF or QF (A): CG and Jacobi PCG with the fixed
// normalisation policy (r every iteration), and the adjoint's gradient;
// vectors of two 8-byte slots.  Its init is preceded by k_qqf_bnorm
// (qqf_init_pre in inst_qqf.cu).
template <class A>
inline KernelTable make_table_qqf() {
  KernelTable t{};
  t.words = kQqfSlots;
  t.minb = A::MINB;
  t.spmv = (const void*)&k_spmv<A>;
  t.spmv_pol = t.spmv;
  t.init = (const void*)&k_qqf_init<A>;
  t.update = (const void*)&k_qqf_update<A>;
  t.pupdate = (const void*)&k_qqf_pupdate<A>;
  t.update_pol = t.update;
  t.pupdate_pol = t.pupdate;
  t.init_pcg = (const void*)&k_qqf_init<A, true>;
  t.update_pcg = (const void*)&k_qqf_update<A, true>;
  t.pupdate_pcg = (const void*)&k_qqf_pupdate<A, true>;
  t.update_pcg_pol = t.update_pcg;
  t.pupdate_pcg_pol = t.pupdate_pcg;
  t.zero_x = (const void*)&k_zero_x<kQqfSlots>;
  t.grad_values = (const void*)&k_grad_values<A>;
  t.collapse = (const void*)&k_collapse<A>;
  t.dot = (const void*)&k_dot<A>;
  t.word_op = (const void*)&k_word_op<A>;
  return t;
}

}  // namespace mwk
