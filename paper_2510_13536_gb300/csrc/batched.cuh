// Batched CG: many independent systems in one persistent kernel launch.
//
// Each worker is a thread-block cluster of C CTAs (one per SM).  A worker
// takes the next system from a device queue (systems sorted by decreasing
// cost on the host), runs the whole CG solve of Algorithm 1 for it with the
// cluster's CTAs, and takes the next one.  Within a solve the CTAs split the
// rows exactly as mwcg_solve's G = C blocks do (tile t -> CTA t mod C), so the
// summation order, and hence every bit of the result, equals mwcg_solve with
// plan {V, 256, C}.  Grid-wide steps of the single-system path (last-block
// reductions, kernel boundaries) become cluster barriers: a CTA writes its
// block partial to its shared memory, the cluster synchronises, and every CTA
// reads the C partials through distributed shared memory and reduces them in
// the same pairwise order, so all CTAs hold identical scalars and take
// identical control-flow decisions (which keeps the barrier counts equal).
// Partial buffers alternate between two slots so that a fast CTA never
// overwrites a value a slower CTA is still reading.
#pragma once
#include <cooperative_groups.h>
#include "cg_kernels.cuh"

namespace mwb {

namespace cgx = cooperative_groups;
using mwk::TPB;

struct Sys {
  const int64_t* rp;
  const int32_t* col;
  const double* val;
  int64_t n;
  const double* b;
  double* x;
  double* r;
  double* p;
  double* q;
  double tol;
  int32_t maxit;
  int32_t arith;
  int32_t V;
  int32_t iters;    // out
  int32_t status;   // out
  int32_t pad;
  double relres;    // out
};

struct ClusterCtx {
  cgx::cluster_group cl;
  int rank;
  int C;
};

// Partial slots in shared memory: [2 buffers][8 doubles] (3 words, presence,
// FP64 value, presence).
struct Slots {
  double v[2][8];
};

// Reduce per-CTA values across the cluster: every CTA returns the same result.
template <class A>
__device__ __forceinline__ typename A::T cluster_reduce(const ClusterCtx& cc, Slots* slots, int buf,
                                                        const typename A::T& v, bool pv, bool& pout,
                                                        double* fp64 = nullptr, bool* pfp64 = nullptr,
                                                        double fv = 0.0, bool pf = false) {
  using T = typename A::T;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < A::W; ++k) slots->v[buf][k] = v.w[k];
    slots->v[buf][3] = pv ? 1.0 : 0.0;
    slots->v[buf][4] = fv;
    slots->v[buf][7] = pf ? 1.0 : 0.0;
  }
  cc.cl.sync();
  __shared__ T sv[32];
  __shared__ int sp[32];
  __shared__ double sf[32];
  __shared__ int spf[32];
  // Gather the C values (C <= 32) into this CTA's shared memory, then tree.
  if (threadIdx.x < (unsigned)cc.C) {
    Slots* rs = cc.cl.map_shared_rank(slots, (int)threadIdx.x);
    T t;
#pragma unroll
    for (int k = 0; k < A::W; ++k) t.w[k] = rs->v[buf][k];
    sv[threadIdx.x] = t;
    sp[threadIdx.x] = rs->v[buf][3] != 0.0;
    sf[threadIdx.x] = rs->v[buf][4];
    spf[threadIdx.x] = rs->v[buf][7] != 0.0;
  }
  __syncthreads();
  __shared__ T res;
  __shared__ int pres;
  __shared__ double resf;
  __shared__ int presf;
  if (threadIdx.x == 0) {
    const int C = cc.C;
    for (int h = 1; h < C; h <<= 1) {
      for (int s = 0; s + h < C; s += 2 * h) {
        T a = sv[s];
        bool pa = sp[s] != 0;
        mwk::combine<A>(a, pa, sv[s + h], sp[s + h] != 0);
        sv[s] = a;
        sp[s] = pa;
        mw::MW<1> c{{sf[s]}};
        bool pc = spf[s] != 0;
        mwk::combine<mw::FP64>(c, pc, mw::MW<1>{{sf[s + h]}}, spf[s + h] != 0);
        sf[s] = c.w[0];
        spf[s] = pc;
      }
    }
    res = sv[0];
    pres = sp[0];
    resf = sf[0];
    presf = spf[0];
  }
  __syncthreads();
  pout = pres != 0;
  if (fp64) *fp64 = resf;
  if (pfp64) *pfp64 = presf != 0;
  return res;
}

template <class A>
__device__ void solve_cluster(const ClusterCtx& cc, Slots* slots, Sys& S) {
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

  // q = A p (mode 0: p = x0, no dot) or fused with p^T q (mode 1).
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
        bool po = (lane_in_row % (2 * h)) == 0 && lane_in_row + h < len;
        if (po) mwk::combine<A>(sum, ps, o, true);
      }
      if (lane_in_row == 0 && row < n) {
        if (!ps) sum = A::zero();
        mwk::st<A>(S.q, n, row, sum);
        if (dot) {
          T leaf = A::mul(mwk::ld<A>(p, n, row), sum);
          if (pacc) acc = A::add(acc, leaf);
          else { acc = leaf; pacc = true; }
        }
      }
    }
  };

  // ---- initialisation
  {
    T dummy = A::zero();
    bool pd = false;
    spmv(S.x, false, dummy, pd);
  }
  cc.cl.sync();                       // q = A x0 complete in global memory
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> bb{{0.0}};
  bool pbb = false;
  for (int64_t t = rank; t < ntiles_v; t += C) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const double bi = S.b[i];
      T ri = A::add(A::from(bi), mw::neg<A>(mwk::ld<A>(S.q, n, i)));
      mwk::st<A>(S.r, n, i, ri);
      mwk::st<A>(S.p, n, i, ri);
      T leaf = A::mul(ri, ri);
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      mw::MW<1> lb{{mw::dmul(bi, bi)}};
      if (pbb) bb = mw::FP64::add(bb, lb);
      else { bb = lb; pbb = true; }
    }
  }
  mwk::block_tree<A>(acc, pacc, 1);
  mwk::block_tree<mw::FP64>(bb, pbb, 1);
  bool prho, pbn;
  double bn2;
  T rho = cluster_reduce<A>(cc, slots, buf, acc, pacc, prho, &bn2, &pbn, bb.w[0], pbb);
  buf ^= 1;
  if (!prho) rho = A::zero();
  const double bnorm = __dsqrt_rn(pbn ? bn2 : 0.0);
  int iters = 0, status = mwk::ST_CONVERGED;
  double relres = 0.0;
  bool done = false;
  if (bnorm == 0.0) {
    for (int64_t i = (int64_t)rank * TPB + threadIdx.x; i < (int64_t)A::W * n; i += (int64_t)C * TPB) S.x[i] = 0.0;
    done = true;
  } else {
    bool rzero = true;
#pragma unroll
    for (int k = 0; k < A::W; ++k) rzero = rzero && !mw::nonzero(rho.w[k]);
    relres = __ddiv_rn(__dsqrt_rn(A::collapse(rho)), bnorm);
    if (rzero) { relres = 0.0; done = true; }
    else if (S.maxit <= 0) { status = mwk::ST_MAXIT; done = true; }
  }

  // ---- CG iterations; every CTA holds the same scalars and decisions.
  while (!done) {
    cc.cl.sync();                     // p (and r, x) complete before the gathers
    acc = A::zero();
    pacc = false;
    spmv(S.p, true, acc, pacc);
    mwk::block_tree<A>(acc, pacc, V);
    bool ppq;
    T pq = cluster_reduce<A>(cc, slots, buf, acc, pacc, ppq);
    buf ^= 1;
    if (!ppq) pq = A::zero();
    ++iters;
    const double pqc = A::collapse(pq);
    if (!(pqc > 0.0) || !isfinite(pqc)) { status = mwk::ST_BREAKDOWN; break; }
    const T al = A::div(rho, pq);
    const T mal = mw::neg<A>(al);
    acc = A::zero();
    pacc = false;
    for (int64_t t = rank; t < ntiles_v; t += C) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) {
        mwk::st<A>(S.x, n, i, A::muladd(mwk::ld<A>(S.x, n, i), al, mwk::ld<A>(S.p, n, i)));
        T ri = A::muladd(mwk::ld<A>(S.r, n, i), mal, mwk::ld<A>(S.q, n, i));
        A::normalize(ri);
        mwk::st<A>(S.r, n, i, ri);
        T leaf = A::mul(ri, ri);
        if (pacc) acc = A::add(acc, leaf);
        else { acc = leaf; pacc = true; }
      }
    }
    mwk::block_tree<A>(acc, pacc, 1);
    bool prr;
    T rho1 = cluster_reduce<A>(cc, slots, buf, acc, pacc, prr);
    buf ^= 1;
    if (!prr) rho1 = A::zero();
    relres = __ddiv_rn(__dsqrt_rn(A::collapse(rho1)), bnorm);
    if (relres < S.tol) { status = mwk::ST_CONVERGED; break; }
    if (!isfinite(relres)) { status = mwk::ST_BREAKDOWN; break; }
    if (iters >= S.maxit) { status = mwk::ST_MAXIT; break; }
    const T be = A::div(rho1, rho);
    rho = rho1;
    // p = r + beta p on this CTA's rows (the update tiles).
    for (int64_t t = rank; t < ntiles_v; t += C) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) mwk::st<A>(S.p, n, i, A::muladd(mwk::ld<A>(S.r, n, i), be, mwk::ld<A>(S.p, n, i)));
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
