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
  double* hist;     // optional per-iteration FP64 relative residual, or null
  int32_t norm_every;   // normalisation policy (mwk::norm_at)
  uint32_t norm_mask;
  const double* w;      // Jacobi weights (preconditioned CG), or null
};

struct ClusterCtx {
  cgx::cluster_group cl;
  int rank;
  int C;
};

// Partial slots in shared memory: [2 buffers][mwk::PART doubles] in the
// layout of the grid reductions (words, presence, two FP64 values and their
// presences).
struct Slots {
  double v[2][mwk::PART];
};

// Reduce per-CTA values across the cluster: every CTA returns the same result.
// NF = 0, 1 or 2 FP64 values ride along (fv/pf into fp64/pfp64, fv2/pf2
// into fp64_2/pfp64_2), reduced by the same tree; NF is a compile-time
// count so that the reductions of the loop carry only what they need.
template <class A, int NF = 0>
__device__ __forceinline__ typename A::T cluster_reduce(const ClusterCtx& cc, Slots* slots, int buf,
                                                        const typename A::T& v, bool pv, bool& pout,
                                                        double* fp64 = nullptr, bool* pfp64 = nullptr,
                                                        double fv = 0.0, bool pf = false,
                                                        double* fp64_2 = nullptr, bool* pfp64_2 = nullptr,
                                                        double fv2 = 0.0, bool pf2 = false) {
  using T = typename A::T;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < A::W; ++k) slots->v[buf][k] = v.w[k];
    slots->v[buf][mwk::PRES] = pv ? 1.0 : 0.0;
    if (NF >= 1) {
      slots->v[buf][mwk::FV] = fv;
      slots->v[buf][mwk::FP] = pf ? 1.0 : 0.0;
    }
    if (NF >= 2) {
      slots->v[buf][mwk::FV + 1] = fv2;
      slots->v[buf][mwk::FP + 1] = pf2 ? 1.0 : 0.0;
    }
  }
  cc.cl.sync();
  __shared__ T sv[32];
  __shared__ int sp[32];
  __shared__ double sf[32];
  __shared__ int spf[32];
  __shared__ double sf2[32];
  __shared__ int spf2[32];
  // Gather the C values (C <= 32) into this CTA's shared memory, then tree.
  if (threadIdx.x < (unsigned)cc.C) {
    Slots* rs = cc.cl.map_shared_rank(slots, (int)threadIdx.x);
    T t;
#pragma unroll
    for (int k = 0; k < A::W; ++k) t.w[k] = rs->v[buf][k];
    sv[threadIdx.x] = t;
    sp[threadIdx.x] = rs->v[buf][mwk::PRES] != 0.0;
    if (NF >= 1) {
      sf[threadIdx.x] = rs->v[buf][mwk::FV];
      spf[threadIdx.x] = rs->v[buf][mwk::FP] != 0.0;
    }
    if (NF >= 2) {
      sf2[threadIdx.x] = rs->v[buf][mwk::FV + 1];
      spf2[threadIdx.x] = rs->v[buf][mwk::FP + 1] != 0.0;
    }
  }
  __syncthreads();
  __shared__ T res;
  __shared__ int pres;
  __shared__ double resf, resf2;
  __shared__ int presf, presf2;
  // Pairwise tree over the C values in warp 0: level h combines lane s with
  // lane s+h for s a multiple of 2h (the same order as a sequential tree, at
  // log2(C) dependent steps instead of C-1).
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int C = cc.C;
    T a = (lane < C) ? sv[lane] : A::zero();
    bool pa = (lane < C) ? (sp[lane] != 0) : false;
    mw::MW<1> c{{(NF >= 1 && lane < C) ? sf[lane] : 0.0}};
    bool pc = (NF >= 1 && lane < C) ? (spf[lane] != 0) : false;
    mw::MW<1> c2{{(NF >= 2 && lane < C) ? sf2[lane] : 0.0}};
    bool pc2 = (NF >= 2 && lane < C) ? (spf2[lane] != 0) : false;
    for (int h = 1; h < C; h <<= 1) {
      T o = mwk::shfl_down<A>(a, h);
      bool po = __shfl_down_sync(0xffffffffu, (int)pa, h) != 0;
      mw::MW<1> oc{{0.0}}, oc2{{0.0}};
      bool poc = false, poc2 = false;
      if (NF >= 1) {
        oc = mwk::shfl_down<mw::FP64>(c, h);
        poc = __shfl_down_sync(0xffffffffu, (int)pc, h) != 0;
      }
      if (NF >= 2) {
        oc2 = mwk::shfl_down<mw::FP64>(c2, h);
        poc2 = __shfl_down_sync(0xffffffffu, (int)pc2, h) != 0;
      }
      if ((lane % (2 * h)) == 0 && lane + h < C) {
        mwk::combine<A>(a, pa, o, po);
        if (NF >= 1) mwk::combine<mw::FP64>(c, pc, oc, poc);
        if (NF >= 2) mwk::combine<mw::FP64>(c2, pc2, oc2, poc2);
      }
    }
    if (lane == 0) {
      res = a;
      pres = pa;
      resf = c.w[0];
      presf = pc;
      resf2 = c2.w[0];
      presf2 = pc2;
    }
  }
  __syncthreads();
  pout = pres != 0;
  if (fp64) *fp64 = resf;
  if (pfp64) *pfp64 = presf != 0;
  if (fp64_2) *fp64_2 = resf2;
  if (pfp64_2) *pfp64_2 = presf2 != 0;
  return res;
}

// PREC: Jacobi-preconditioned CG (z = w (x) r kept in q, rho = r^T z, FP64
// stopping residual from the collapsed r), as k_init / k_update / k_pupdate.
template <class A, bool PREC = false>
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

  // q = A p (mode 0: p = x0, no dot) or fused with p^T q (mode 1); nm: the
  // iteration's normalisation places (NORM_SUM, NORM_Q apply here).
  auto spmv = [&](const double* __restrict__ p, bool dot, T& acc, bool& pacc, uint32_t nm) {
    const bool nsum = (nm & mwk::NORM_SUM) != 0;
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
        for (k += V; k < k1; k += V) {
          sum = A::dxmuladd(sum, S.val[k], mwk::ld<A>(p, n, S.col[k]));
          if (nsum) A::normalize(sum);
        }
      }
      for (int h = 1; h < V; h <<= 1) {
        T o = mwk::shfl_down<A>(sum, h);
        bool po = (lane_in_row % (2 * h)) == 0 && lane_in_row + h < len;
        const bool add = po && ps;
        if (po) mwk::combine<A>(sum, ps, o, true);
        if (add && nsum) A::normalize(sum);
      }
      if (lane_in_row == 0 && row < n) {
        if (!ps) sum = A::zero();
        if (nm & mwk::NORM_Q) A::normalize(sum);
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
    spmv(S.x, false, dummy, pd, 0u);
  }
  cc.cl.sync();                       // q = A x0 complete in global memory
  T acc = A::zero();
  bool pacc = false;
  mw::MW<1> bb{{0.0}}, rr{{0.0}};
  bool pbb = false, prr = false;
  for (int64_t t = rank; t < ntiles_v; t += C) {
    const int64_t i = t * TPB + threadIdx.x;
    if (i < n) {
      const double bi = S.b[i];
      T ri = A::add(A::from(bi), mw::neg<A>(mwk::ld<A>(S.q, n, i)));
      mwk::st<A>(S.r, n, i, ri);
      T leaf;
      if constexpr (PREC) {
        const T zi = A::dxmul(S.w[i], ri);
        mwk::st<A>(S.p, n, i, zi);
        leaf = A::mul(ri, zi);
        const double c = A::collapse(ri);
        mw::MW<1> lc{{mw::dmul(c, c)}};
        if (prr) rr = mw::FP64::add(rr, lc);
        else { rr = lc; prr = true; }
      } else {
        mwk::st<A>(S.p, n, i, ri);
        leaf = A::mul(ri, ri);
      }
      if (pacc) acc = A::add(acc, leaf);
      else { acc = leaf; pacc = true; }
      mw::MW<1> lb{{mw::dmul(bi, bi)}};
      if (pbb) bb = mw::FP64::add(bb, lb);
      else { bb = lb; pbb = true; }
    }
  }
  mwk::block_tree<A>(acc, pacc, 1);
  mwk::block_tree<mw::FP64>(bb, pbb, 1);
  if constexpr (PREC) mwk::block_tree<mw::FP64>(rr, prr, 1);
  bool prho, pbn, prrs = false;
  double bn2, rrs = 0.0;
  T rho = cluster_reduce<A, PREC ? 2 : 1>(cc, slots, buf, acc, pacc, prho, &bn2, &pbn, bb.w[0], pbb, &rrs, &prrs,
                                          rr.w[0], prr);
  buf ^= 1;
  // Scalar steps run on one thread per CTA (the FP64 pipe is shared by the
  // whole SM) and are broadcast through shared memory.  Every CTA's thread 0
  // computes them from the same inputs, so all CTAs agree.
  // Broadcast scalars: [0] ||b|| then the relative residual, alpha at
  // [SA, SA + W), beta at [SB, SB + W), the iteration's residual at SR.
  constexpr int SA = 1, SB = SA + 4, SR = SB + 4;
  __shared__ double s_sc[SR + 1];
  __shared__ int s_flag[2];
  if (threadIdx.x == 0) {
    if (!prho) rho = A::zero();
    const double bnorm0 = __dsqrt_rn(pbn ? bn2 : 0.0);
    int fl = 0;                        // 0 run, 1 zero x and stop, 2 stop
    double rr0 = 0.0;
    int st0 = mwk::ST_CONVERGED;
    if (bnorm0 == 0.0) {
      fl = 1;
    } else {
      bool rzero = true;
#pragma unroll
      for (int k = 0; k < A::W; ++k) rzero = rzero && !mw::nonzero(rho.w[k]);
      rr0 = PREC ? __ddiv_rn(__dsqrt_rn(prrs ? rrs : 0.0), bnorm0)
                 : __ddiv_rn(__dsqrt_rn(A::collapse(rho)), bnorm0);
      if (rzero) { rr0 = 0.0; fl = 2; }
      else if (S.maxit <= 0) { st0 = mwk::ST_MAXIT; fl = 2; }
    }
    s_sc[0] = bnorm0;
    s_sc[SR] = rr0;
    s_flag[0] = fl;
    s_flag[1] = st0;
  }
  __syncthreads();
  const double bnorm = s_sc[0];
  int iters = 0, status = s_flag[1];
  double relres = s_sc[SR];
  bool done = s_flag[0] != 0;
  if (s_flag[0] == 1) {
    for (int64_t i = (int64_t)rank * TPB + threadIdx.x; i < (int64_t)A::W * n; i += (int64_t)C * TPB) S.x[i] = 0.0;
  }
  if (!prho) rho = A::zero();

  // ---- CG iterations; every CTA holds the same scalars and decisions.
  while (!done) {
    cc.cl.sync();                     // p (and r, x) complete before the gathers
    acc = A::zero();
    pacc = false;
    const uint32_t nm = mwk::norm_at(S.norm_every, S.norm_mask, iters + 1);
    spmv(S.p, true, acc, pacc, nm);
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
    for (int k = 0; k < A::W; ++k) al.w[k] = s_sc[SA + k];
    const T mal = mw::neg<A>(al);
    acc = A::zero();
    pacc = false;
    mw::MW<1> rq{{0.0}};
    bool prq = false;
    for (int64_t t = rank; t < ntiles_v; t += C) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) {
        T xi = A::muladd(mwk::ld<A>(S.x, n, i), al, mwk::ld<A>(S.p, n, i));
        if (nm & mwk::NORM_X) A::normalize(xi);
        mwk::st<A>(S.x, n, i, xi);
        T ri = A::muladd(mwk::ld<A>(S.r, n, i), mal, mwk::ld<A>(S.q, n, i));
        if (nm & mwk::NORM_R) A::normalize(ri);
        mwk::st<A>(S.r, n, i, ri);
        T leaf;
        if constexpr (PREC) {
          const T zi = A::dxmul(S.w[i], ri);      // z over q (this CTA's rows only)
          mwk::st<A>(S.q, n, i, zi);
          leaf = A::mul(ri, zi);
          const double c = A::collapse(ri);
          mw::MW<1> lc{{mw::dmul(c, c)}};
          if (prq) rq = mw::FP64::add(rq, lc);
          else { rq = lc; prq = true; }
        } else {
          leaf = A::mul(ri, ri);
        }
        if (pacc) acc = A::add(acc, leaf);
        else { acc = leaf; pacc = true; }
      }
    }
    mwk::block_tree<A>(acc, pacc, 1);
    if constexpr (PREC) mwk::block_tree<mw::FP64>(rq, prq, 1);
    bool prr, prqs = false;
    double rqs = 0.0;
    T rho1 = cluster_reduce<A, PREC ? 1 : 0>(cc, slots, buf, acc, pacc, prr, &rqs, &prqs, rq.w[0], prq);
    buf ^= 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!prr) rho1 = A::zero();
      const double rr = PREC ? __ddiv_rn(__dsqrt_rn(prqs ? rqs : 0.0), bnorm)
                             : __ddiv_rn(__dsqrt_rn(A::collapse(rho1)), bnorm);
      if (S.hist && rank == 0) S.hist[iters - 1] = rr;
      int fl = 0;
      if (rr < S.tol) fl = 1;
      else if (!isfinite(rr)) fl = 2;
      else if (iters >= S.maxit) fl = 3;
      else {
        const T be = A::div(rho1, rho);
#pragma unroll
        for (int k = 0; k < A::W; ++k) s_sc[SB + k] = be.w[k];
      }
      s_sc[SR] = rr;
      s_flag[0] = fl;
    }
    __syncthreads();
    relres = s_sc[SR];
    if (s_flag[0] == 1) { status = mwk::ST_CONVERGED; break; }
    if (s_flag[0] == 2) { status = mwk::ST_BREAKDOWN; break; }
    if (s_flag[0] == 3) { status = mwk::ST_MAXIT; break; }
    T be;
#pragma unroll
    for (int k = 0; k < A::W; ++k) be.w[k] = s_sc[SB + k];
    if (!prr) rho1 = A::zero();
    rho = rho1;
    // p = r + beta p (PREC: z + beta p) on this CTA's rows (the update tiles).
    const double* __restrict__ src = PREC ? S.q : S.r;
    for (int64_t t = rank; t < ntiles_v; t += C) {
      const int64_t i = t * TPB + threadIdx.x;
      if (i < n) {
        T pi = A::muladd(mwk::ld<A>(src, n, i), be, mwk::ld<A>(S.p, n, i));
        if (nm & mwk::NORM_P) A::normalize(pi);
        mwk::st<A>(S.p, n, i, pi);
      }
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    S.iters = iters;
    S.status = status;
    S.relres = relres;
  }
  cc.cl.sync();                       // x, outputs complete; slots free for the next system
}

// Word groups of the persistent kernel: GRP 0 = FP64, DW, QDW, QDW-NN;
// GRP 1 = TW, QTW, QTW-NN; GRP 2 = QW, QQW, QQW-NN (the four-word
// arithmetics of mw_device4.cuh, included by its translation units); GRP 3 =
// QQF, QF (four FP32 words, the scaled iteration of batched_float.cuh).
inline int word_group(int arith) {
  return (arith == 3 || arith == 4 || arith == 6) ? 1 : (arith >= 10) ? 3 : (arith >= 7) ? 2 : 0;
}

template <bool PREC, int GRP>
__device__ __forceinline__ void solve_any(const ClusterCtx& cc, Slots* slots, Sys& S);

// The persistent kernel: clusters take systems from the queue until it is
// empty.  One instantiation per (PREC, word group), each compiled in its own
// translation unit (batched_k*.cu): a kernel holding every arithmetic's
// solver takes minutes to compile.
template <bool PREC, int GRP>
__global__ void __launch_bounds__(TPB, 2) k_batched(Sys* __restrict__ sys, int nsys, unsigned* queue) {
  __shared__ Slots slots;
  __shared__ int s_next;
  cgx::cluster_group cl = cgx::this_cluster();
  const ClusterCtx cc{cl, (int)cl.block_rank(), (int)cl.num_blocks()};
  for (;;) {
    if (cc.rank == 0 && threadIdx.x == 0) s_next = (int)atomicAdd(queue, 1u);
    cl.sync();
    const int sid = *cl.map_shared_rank(&s_next, 0);
    cl.sync();                               // every CTA has read s_next before it is overwritten
    if (sid >= nsys) break;
    solve_any<PREC, GRP>(cc, &slots, sys[sid]);     // the host groups systems by (PREC, GRP)
  }
}

// Dynamic shared memory that keeps one CTA per SM, used for the one-cluster
// solve of a single small system (its CTAs then spread over as many SMs as
// possible).  Batches run without it: two CTAs per SM (the kernels are
// compiled for 2 blocks per SM, at most 128 registers, no spills) keep twice
// the warps per SM busy (c4, 256 systems: 8.26 s with the pad, 5.14 s without).
constexpr size_t kPadSmem = 120 * 1024;

// Host: run k_batched<PREC, GRP> over n systems already on the device (queue
// zeroed), clusters of `cluster` CTAs: as many clusters as fit at once, at
// most n and, if max_clusters > 0, at most max_clusters.  The translation
// unit that calls it holds that instantiation.
template <bool PREC, int GRP>
cudaError_t run_group(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad, int* nclusters,
                      int max_clusters) {
  const void* kern = (const void*)&k_batched<PREC, GRP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPadSmem);
  if (e == cudaSuccess && cluster > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(TPB);
  cfg.dynamicSmemBytes = pad;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (e == cudaSuccess) {
    cfg.gridDim = dim3(cluster);
    e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
  }
  if (e == cudaSuccess) {
    if (max_clusters > 0 && nc > max_clusters) nc = max_clusters;
    nc = nc < 1 ? 1 : (nc < n ? nc : n);
    cfg.gridDim = dim3(nc * cluster);
    e = cudaLaunchKernelEx(&cfg, k_batched<PREC, GRP>, dsys, n, queue);
  }
  if (nclusters) *nclusters = nc;
  return e;
}

}  // namespace mwb
