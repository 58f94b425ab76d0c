// Batched CG in QQF / QF (four FP32 words): the scaled iteration of
// cg_float.cuh run by one thread-block cluster per system.  Each step is the
// one of the single-system kernels (k_qqf_bnorm, k_qqf_init, k_spmv,
// k_qqf_update, k_qqf_pupdate) with the cluster's C CTAs in place of G
// blocks and cluster barriers in place of the last-block elections, so every
// bit of the result equals mwcg_solve's with plan {V, 256, C}.
#pragma once
#include "batched.cuh"
#include "cg_float.cuh"

namespace mwb {

// Slot index (past the reduction's fields) of a CTA's largest |x_i0| bits.
constexpr int kXmaxSlot = 9;

// PREC: Jacobi-preconditioned CG (z~ = w (x) r~ kept in q, rho~ = r~^T z~,
// the stop test and the shift from the FP64 sum of collapse(r~_i)^2).
template <class A, bool PREC = false>
__device__ void solve_cluster_qqf(const ClusterCtx& cc, Slots* slots, Sys& S) {
  using T = typename A::T;
  const int64_t n = S.n;
  const int V = S.V;
  const int R = TPB / V;
  const int lane_in_row = threadIdx.x % V;
  const int slot = threadIdx.x / V;
  const int64_t ntiles_s = (n + R - 1) / R;
  const int64_t ntiles_v = (n + TPB - 1) / TPB;
  const int rank = cc.rank, C = cc.C;
  int buf = 0;

  // q = A p, fused with p^T q when dot (no normalisation policy in QQF).
  auto spmv = [&](const double* __restrict__ p, bool dot, T& acc, bool& pacc) {
    for (int64_t t = rank; t < ntiles_s; t += C) {
      const int64_t row = t * R + slot;
      int64_t k0 = 0, k1 = 0;
      if (row < n) { k0 = S.rp[row]; k1 = S.rp[row + 1]; }
      const int64_t len = k1 - k0;
      T sum = A::zero();
      bool ps = false;
      int64_t k = k0 + lane_in_row;
      if (k < k1) {
        sum = A::dxmul(S.val[k], mwk::ld<A>(p, n, S.col[k]));
        ps = true;
        for (k += V; k < k1; k += V) sum = A::dxmuladd(sum, S.val[k], mwk::ld<A>(p, n, S.col[k]));
      }
      for (int h = 1; h < V; h <<= 1) {
        T o = mwk::shfl_down<A>(sum, h);
        const bool po = (lane_in_row % (2 * h)) == 0 && lane_in_row + h < len;
        if (po) mwk::combine<A>(sum, ps, o, true);
      }
      if (lane_in_row == 0 && row < n) {
        if (!ps) sum = A::zero();
        mwk::st<A>(S.q, n, row, sum);
        if (dot) {
          const T leaf = A::mul(mwk::ld<A>(p, n, row), sum);
          if (pacc) acc = A::add(acc, leaf);
          else { acc = leaf; pacc = true; }
        }
      }
    }
  };

  // Scalars broadcast from each CTA's thread 0 (every CTA computes them from
  // the same reduced inputs): alpha~ at [SA, SA + 4), beta~ at [SB, SB + 4),
  // the relative residual at SR; flags: [0] stop, [1] status, [2] next shift.
  constexpr int SA = 0, SB = 4, SR = 8;
  __shared__ double s_sc[SR + 1];
  __shared__ int s_flag[3];
  __shared__ uint32_t s_xb[mwk::NWARP];

  // ---- ||b||_2^2 in FP64 (k_qqf_bnorm's order) and E0
  mw::MW<1> bb{{0.0}};
  bool pbb = false;
  for (int64_t t = rank; t < ntiles_v; t += C) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const mw::MW<1> l{{mw::dmul(S.b[i], S.b[i])}};
      if (pbb) bb = mw::FP64::add(bb, l);
      else { bb = l; pbb = true; }
    }
  }
  mwk::block_tree<mw::FP64>(bb, pbb, 1);
  bool pbn;
  const mw::MW<1> bbt = cluster_reduce<mw::FP64>(cc, slots, buf, bb, pbb, pbn);
  buf ^= 1;
  const double bb2 = pbn ? bbt.w[0] : 0.0;
  const double bnorm = __dsqrt_rn(bb2);
  int E = mwk::scale_exp(bb2, n);
  int iters = 0, status = mwk::ST_CONVERGED;
  double relres = 0.0;
  if (bnorm == 0.0) {                 // b = 0: x = 0, converged
    for (int64_t i = (int64_t)rank * TPB + threadIdx.x; i < (int64_t)mwk::kQqfSlots * n; i += (int64_t)C * TPB)
      S.x[i] = 0.0;
    if (rank == 0 && threadIdx.x == 0) {
      S.iters = 0;
      S.status = mwk::ST_CONVERGED;
      S.relres = 0.0;
    }
    cc.cl.sync();
    return;
  }

  // ---- r~0 = split3(b 2^-E0) (+) 2^-E0 (-(A x0)), p~0 = r~0 (PREC: z~0), rho~0
  {
    T dummy = A::zero();
    bool pd = false;
    spmv(S.x, false, dummy, pd);
  }
  cc.cl.sync();                       // q = A x0 complete in global memory
  const double sb = mw::pow2d(-E);
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> rr{{0.0}};
  bool prr = false;
  for (int64_t t = rank; t < ntiles_v; t += C) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const T ri = A::add(A::from(__dmul_rn(S.b[i], sb)), A::scale(A::neg(mwk::ld<A>(S.q, n, i)), -E));
      mwk::st<A>(S.r, n, i, ri);
      T leaf;
      if constexpr (PREC) {
        const T zi = A::dxmul(S.w[i], ri);
        mwk::st<A>(S.p, n, i, zi);
        leaf = A::mul(ri, zi);
        const double c = A::collapse(ri);
        const mw::MW<1> lc{{mw::dmul(c, c)}};
        if (prr) rr = mw::FP64::add(rr, lc);
        else { rr = lc; prr = true; }
      } else {
        mwk::st<A>(S.p, n, i, ri);
        leaf = A::mul(ri, ri);
      }
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
    }
  }
  mwk::block_tree<A>(acc, pacc, 1);
  if constexpr (PREC) mwk::block_tree<mw::FP64>(rr, prr, 1);
  bool prho, prrs = false;
  double rrs = 0.0;
  T rho = cluster_reduce<A, PREC ? 1 : 0>(cc, slots, buf, acc, pacc, prho, &rrs, &prrs, rr.w[0], prr);
  buf ^= 1;
  if (!prho) rho = A::zero();
  if (threadIdx.x == 0) {
    bool rzero = true;
#pragma unroll
    for (int k = 0; k < A::W; ++k) rzero = rzero && (rho.w[k] == 0.0f);
    const double c = PREC ? (prrs ? rrs : 0.0) : A::collapse(rho);
    double rr0 = __ddiv_rn(__dmul_rn(__dsqrt_rn(c), mw::pow2d(E)), bnorm);
    int fl = 0, st0 = mwk::ST_CONVERGED;
    if (rzero) { rr0 = 0.0; fl = 1; }
    else if (S.maxit <= 0) { st0 = mwk::ST_MAXIT; fl = 1; }
    s_sc[SR] = rr0;
    s_flag[0] = fl;
    s_flag[1] = st0;
    s_flag[2] = mwk::clamp_shift(mwk::scale_exp(c, n), E);
  }
  __syncthreads();
  relres = s_sc[SR];
  status = s_flag[1];
  bool done = s_flag[0] != 0;
  int s = s_flag[2];

  // ---- iterations; every CTA holds the same scalars and decisions.
  while (!done) {
    cc.cl.sync();                     // p~ (and r~, x) complete before the gathers
    acc = A::zero();
    pacc = false;
    spmv(S.p, true, acc, pacc);
    mwk::block_tree<A>(acc, pacc, V);
    bool ppq;
    T pq = cluster_reduce<A>(cc, slots, buf, acc, pacc, ppq);
    buf ^= 1;
    ++iters;
    __syncthreads();                  // everyone has read s_sc / s_flag of the previous step
    if (threadIdx.x == 0) {
      if (!ppq) pq = A::zero();
      const double pqc = A::collapse(pq);
      const bool brk = !(pqc > 0.0) || !isfinite(pqc);
      s_flag[0] = brk ? 1 : 0;
      if (!brk) {
        const T a1 = A::div(rho, pq);
#pragma unroll
        for (int k = 0; k < A::W; ++k) s_sc[SA + k] = a1.w[k];
      }
    }
    __syncthreads();
    if (s_flag[0]) { status = mwk::ST_BREAKDOWN; break; }
    T al;
#pragma unroll
    for (int k = 0; k < A::W; ++k) al.w[k] = (float)s_sc[SA + k];
    const T cx = A::scale(al, E);
    const T mal = A::neg(al);
    const float ps = mw::pow2f(-s);
    acc = A::zero();
    pacc = false;
    rr = mw::MW<1>{{0.0}};
    prr = false;
    uint32_t xb = 0;                  // largest |x_i0| bits of this thread's rows
    for (int64_t t = rank; t < ntiles_v; t += C) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) {
        const T xn = A::muladd(mwk::ld<A>(S.x, n, i), cx, mwk::ld<A>(S.p, n, i));
        mwk::st<A>(S.x, n, i, xn);
        xb = max(xb, __float_as_uint(xn.w[0]) & 0x7FFFFFFFu);
        T ri = A::muladd(mwk::ld<A>(S.r, n, i), mal, mwk::ld<A>(S.q, n, i));
        A::renorm(ri);
#pragma unroll
        for (int j = 0; j < A::W; ++j) ri.w[j] = mw::fmul(ri.w[j], ps);
        mwk::st<A>(S.r, n, i, ri);
        T leaf;
        if constexpr (PREC) {
          const T zi = A::dxmul(S.w[i], ri);      // z~ over q (this CTA's rows only)
          mwk::st<A>(S.q, n, i, zi);
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
    // The CTA's largest |x_i0| rides in the reduction's buffer: written before
    // its cluster barrier, read by every CTA after it (the buffer is not
    // written again before the next two barriers).
    xb = __reduce_max_sync(0xFFFFFFFFu, xb);
    if ((threadIdx.x & 31) == 0) s_xb[threadIdx.x >> 5] = xb;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t m = 0;
#pragma unroll
      for (int k = 0; k < mwk::NWARP; ++k) m = max(m, s_xb[k]);
      slots->v[buf][kXmaxSlot] = (double)m;
    }
    mwk::block_tree<A>(acc, pacc, 1);
    if constexpr (PREC) mwk::block_tree<mw::FP64>(rr, prr, 1);
    const int ub = buf;
    bool prho1, prqs = false;
    double rqs = 0.0;
    T rho1 = cluster_reduce<A, PREC ? 1 : 0>(cc, slots, buf, acc, pacc, prho1, &rqs, &prqs, rr.w[0], prr);
    buf ^= 1;
    if (!prho1) rho1 = A::zero();
    __syncthreads();
    const int En = E + s;
    if (threadIdx.x == 0) {
      uint32_t xm = 0;
      for (int k = 0; k < C; ++k) xm = max(xm, (uint32_t)cc.cl.map_shared_rank(slots, k)->v[ub][kXmaxSlot]);
      const bool x_nonfinite = xm >= 0x7F800000u, x_under = xm < 0x00800000u;
      const double c = PREC ? (prqs ? rqs : 0.0) : A::collapse(rho1);
      const double rrn = __ddiv_rn(__dmul_rn(__dsqrt_rn(c), mw::pow2d(En)), bnorm);
      if (S.hist && rank == 0) S.hist[iters - 1] = rrn;
      int fl = 1, st = mwk::ST_CONVERGED;
      if (x_nonfinite) st = mwk::ST_RANGE;
      else if (rrn < S.tol) st = x_under ? mwk::ST_RANGE : mwk::ST_CONVERGED;
      else if (!isfinite(rrn)) st = mwk::ST_BREAKDOWN;
      else if (iters >= S.maxit) st = x_under ? mwk::ST_RANGE : mwk::ST_MAXIT;
      else {
        fl = 0;
        const T be = A::div(rho1, rho);
#pragma unroll
        for (int k = 0; k < A::W; ++k) s_sc[SB + k] = be.w[k];
      }
      s_sc[SR] = rrn;
      s_flag[0] = fl;
      s_flag[1] = st;
      s_flag[2] = mwk::clamp_shift(mwk::scale_exp(c, n), En);
    }
    __syncthreads();
    relres = s_sc[SR];
    if (s_flag[0]) { status = s_flag[1]; break; }
    T be;
#pragma unroll
    for (int k = 0; k < A::W; ++k) be.w[k] = (float)s_sc[SB + k];
    const T cp = A::scale(be, s);
    rho = rho1;
    E = En;
    s = s_flag[2];
    // p~ = r~ + (beta~ 2^s) p~ (PREC: z~ + (beta~ 2^s) p~) on this CTA's rows.
    const double* __restrict__ src = PREC ? S.q : S.r;
    for (int64_t t = rank; t < ntiles_v; t += C) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) mwk::st<A>(S.p, n, i, A::muladd(mwk::ld<A>(src, n, i), cp, mwk::ld<A>(S.p, n, i)));
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    S.iters = iters;
    S.status = status;
    S.relres = relres;
  }
  cc.cl.sync();                       // x, outputs complete; slots free for the next system
}

}  // namespace mwb
