// Host runtime and C ABI (include/mwcg.h) of the multi-word CG solver.
//
// A matrix handle owns the device CSR, the solver workspace (r, p, q and the
// block partials), a DevState block and, per arithmetic, an instantiated
// CUDA graph of the whole solve: SpMV of x0, initialisation, and a
// conditional WHILE node whose body is one CG iteration (Algorithm 1, lines
// 5-14).  The loop condition is set on the device by the kernels, so a solve
// is one graph launch plus one small copy of the results back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "mwcg.h"
#include "cg_kernels.cuh"
#include "bicg_kernels.cuh"
#include "batched.cuh"

namespace mwb_host {
int cluster_size();
int small_cluster_size();
cudaError_t launch(mwb::Sys* hsys, int nsys, cudaStream_t s, int cluster, int* clusters_out);
}  // namespace mwb_host

namespace mwcg_precond {
cudaError_t jacobi_weights(const int64_t* rp, const int32_t* col, const double* val, int64_t n, double* w,
                           int* bad, cudaStream_t s);
}  // namespace mwcg_precond

namespace mwk {
KernelTable table_fp64();
KernelTable table_dw();
KernelTable table_qdw();
KernelTable table_qdw_nn();
KernelTable table_tw();
KernelTable table_qtw();
KernelTable table_qtw_nn();
KernelTable table_qw();
KernelTable table_qqw();
KernelTable table_qqw_nn();
KernelTable table_qqf();
KernelTable table_qf();
const void* qqf_init_pre();   // QQF and QF: ||b|| and the first scale, before the init
BiTable bitable_fp64();
BiTable bitable_dw();
BiTable bitable_qdw();
BiTable bitable_tw();
BiTable bitable_qtw();
BiTable bitable_qdw_nn();
BiTable bitable_qtw_nn();
BiTable bitable_qw();
BiTable bitable_qqw();
BiTable bitable_qqw_nn();
BiTable bitable_qqf();
BiTable bitable_qf();
}  // namespace mwk

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? MWCG_ERR_NOMEM : MWCG_ERR_CUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                        \
  } while (0)

constexpr int kNArith = 12;   // MWCG_FP64 .. MWCG_QF
// The FP32-word arithmetics: scaled CG and BiCGStab, packed vectors.
bool fp32_words(int arith) { return arith == MWCG_QQF || arith == MWCG_QF; }
constexpr int kMaxG = 1024;

// Dynamic shared memory of the last-block reductions (mwk::red_smem: 44 KB at
// G = 1024 for w = 3, 52 KB for w = 4, which is above the 48 KB available
// without opting in, so every reduction kernel opts in once, to the largest
// size: the attribute is a cap, and a lower one would refuse launches that
// need the default 48 KB).
using mwk::red_smem;

// Creates the CUDA context with an ordinary runtime call before the kernel
// tables' one-time set-up.  Observed on GB300 (driver 580): when a
// cudaFuncSetAttribute inside that std::call_once was the first call of the
// process to touch the context, the driver crashed the process (SIGSEGV in
// cuKernelGetFunction); with the context created first it never did.
void init_runtime() {
  static std::atomic<int> done{0};
  if (!done.load(std::memory_order_acquire)) {
    cudaFree(nullptr);
    cudaGetLastError();
    done.store(1, std::memory_order_release);
  }
}

const mwk::KernelTable* table(int arith) {
  static mwk::KernelTable t[kNArith];
  static std::once_flag once;
  init_runtime();
  std::call_once(once, [] {
    t[0] = mwk::table_fp64();
    t[1] = mwk::table_dw();
    t[2] = mwk::table_qdw();
    t[3] = mwk::table_tw();
    t[4] = mwk::table_qtw();
    t[5] = mwk::table_qdw_nn();
    t[6] = mwk::table_qtw_nn();
    t[7] = mwk::table_qw();
    t[8] = mwk::table_qqw();
    t[9] = mwk::table_qqw_nn();
    t[10] = mwk::table_qqf();
    t[11] = mwk::table_qf();
    for (auto& k : t)
      for (const void* f : {k.spmv, k.spmv_pol, k.init, k.init_pcg, k.update, k.update_pol, k.update_pcg,
                            k.update_pcg_pol, k.dot})
        if (f) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red_smem(kMaxG, 4));
    cudaGetLastError();
  });
  if (arith < 0 || arith >= kNArith) return nullptr;
  return &t[arith];
}

// Kernel run between the x0 SpMV and the init, or null (QQF only).
const void* init_pre(int arith) { return fp32_words(arith) ? mwk::qqf_init_pre() : nullptr; }

const mwk::BiTable* bitable(int arith) {
  static mwk::BiTable t[kNArith];
  static std::once_flag once;
  init_runtime();
  std::call_once(once, [] {
    t[0] = mwk::bitable_fp64();
    t[1] = mwk::bitable_dw();
    t[2] = mwk::bitable_qdw();
    t[3] = mwk::bitable_tw();
    t[4] = mwk::bitable_qtw();
    t[5] = mwk::bitable_qdw_nn();
    t[6] = mwk::bitable_qtw_nn();
    t[7] = mwk::bitable_qw();
    t[8] = mwk::bitable_qqw();
    t[9] = mwk::bitable_qqw_nn();
    t[10] = mwk::bitable_qqf();
    t[11] = mwk::bitable_qf();
    for (auto& k : t)
      for (const void* f : {k.init, k.spmv_v, k.s, k.spmv_t, k.xr})
        if (f) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red_smem(kMaxG, 4));
    cudaGetLastError();
  });
  if (arith < 0 || arith >= kNArith || !t[arith].init) return nullptr;
  return &t[arith];
}

constexpr int32_t kMaxIt = 1 << 30;



struct GraphCache {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  mwcg_plan plan{0, 0, 0};
  int key = -1;                // kernel selection it was built with (LoopKernels::key)
};

int sm_count_of(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

bool is_pow2_le32(int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32; }

}  // namespace

namespace mwcg_detail {
// Sets the thread's last-error message (used by the other translation units).
int set_error(int code, const char* msg) {
  g_err = msg ? msg : "";
  return code;
}
}  // namespace mwcg_detail

struct mwcg_csr {
  int device = 0;
  int64_t n = 0, nnz = 0;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  mwcg_plan plan{1, 256, 1};
  double* ws = nullptr;        // r, p, q: 3 vectors of up to 4 words
  double* part = nullptr;      // kMaxG * 8
  mwk::DevState* st = nullptr;
  mwk::DevState* h_st = nullptr;   // pinned mirror
  double* lam = nullptr;       // adjoint solution, lazily allocated
  double* hb = nullptr;        // staging for host-buffer solves, lazily allocated
  double* hx = nullptr;
  GraphCache graphs[kNArith];
  GraphCache bigraphs[kNArith];  // BiCGStab
  double* bws = nullptr;         // BiCGStab: rh, s, t (four words each), lazily allocated
  // Plans.  `plan` is the plan of the current call.  A plan set with
  // mwcg_set_plan is pinned for every arithmetic; otherwise each arithmetic
  // has its own automatic plan: the cost model's choice at creation, checked
  // by timing the SpMV under the model's best candidates at the first call in
  // that arithmetic (tune_plan).
  bool pinned = false;
  mwcg_plan pinned_plan{1, 256, 1};
  mwcg_plan auto_plan[kNArith];
  bool tuned[kNArith] = {};
  double tune_ms[kNArith][6] = {};   // SpMV ms per candidate V = 2^j (0: not timed)
  double passes[6] = {}, warps[6] = {};   // row-length statistics of the cost model
  int32_t norm_every = 1;       // normalisation policy of the quasi arithmetics
  uint32_t norm_mask = mwk::NORM_R;
  int prec = MWCG_PREC_NONE;    // preconditioner
  double* w = nullptr;          // Jacobi weights, rebuilt after a value update
  int* w_bad = nullptr;         // device flag of the weights kernel
  int64_t* vbad = nullptr;      // device word of mwcg_update_values' check
  bool w_valid = false;
  bool w_undefined = false;     // a diagonal entry missing, not positive or not finite
};

namespace {

void free_graphs(mwcg_csr* A) {
  for (GraphCache* set : {A->graphs, A->bigraphs})
    for (int k = 0; k < kNArith; ++k) {
      GraphCache& g = set[k];
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      g = GraphCache{};
    }
}

// FP64 operations per SpMV multiply-add and per add, by arithmetic (Sec. III
// counts; TW about 80 and 45 with its branches).  Used only to rank plans.
void op_costs(int arith, double& mac, double& add) {
  switch (arith) {
    case MWCG_FP64: mac = 1; add = 1; break;
    case MWCG_DW: mac = 17; add = 11; break;
    case MWCG_QDW: case MWCG_QDW_NN: mac = 11; add = 8; break;
    case MWCG_TW: mac = 80; add = 45; break;
    case MWCG_QW: mac = 110; add = 60; break;
    case MWCG_QQW: case MWCG_QQW_NN: mac = 70; add = 40; break;
    default: mac = 33; add = 21; break;
  }
}

// Plan model from the row-length sequence.  The multi-word SpMV is bound by
// the FP64 pipe, and a warp instruction costs the same whatever its
// active-lane count, so the cost of V lanes per row is, per warp (32/V
// consecutive rows), the longest row's ceil(len/V) multiply-adds plus
// log2(V) tree adds.  FP64 arithmetic is memory bound: there the cost adds the
// number of 32-lane load rounds, which favours wider rows.  row_stats keeps,
// for V = 2^j, the sum over warps of ceil(max len / V) and the warp count.
void row_stats(const std::vector<int64_t>& len, double* passes, double* warps) {
  const int64_t n = (int64_t)len.size();
  for (int j = 0; j < 6; ++j) {
    const int V = 1 << j, rows_per_warp = 32 / V;
    double ps = 0, ws = 0;
    for (int64_t r0 = 0; r0 < n; r0 += rows_per_warp) {
      int64_t mx = 0;
      for (int64_t r = r0; r < std::min(n, r0 + rows_per_warp); ++r) mx = std::max(mx, len[r]);
      ps += (double)((mx + V - 1) / V);
      ws += 1;
    }
    passes[j] = ps;
    warps[j] = ws;
  }
}
double plan_cost(const double* passes, const double* warps, int j, int arith) {
  double mac, add;
  op_costs(arith, mac, add);
  double c = passes[j] * mac + j * add * warps[j];
  if (arith == MWCG_FP64) c += passes[j] * 2.0;
  return c;
}
// Lane counts 2^j ranked by model cost: the best first (a lane count is
// preferred to a narrower one only when it is 2% cheaper).
std::vector<int> ranked_lanes(const double* passes, const double* warps, int arith) {
  int best = 0;
  double bc = plan_cost(passes, warps, 0, arith);
  for (int j = 1; j < 6; ++j) {
    const double c = plan_cost(passes, warps, j, arith);
    if (c < bc * 0.98) { bc = c; best = j; }
  }
  std::vector<int> order{best};
  std::vector<std::pair<double, int>> rest;
  for (int j = 0; j < 6; ++j)
    if (j != best) rest.push_back({plan_cost(passes, warps, j, arith), j});
  std::sort(rest.begin(), rest.end());
  for (auto& r : rest) order.push_back(r.second);
  return order;
}
mwcg_plan choose_plan(const double* passes, const double* warps, int64_t n, int sms, int arith, int small_cluster,
                      int minb) {
  mwcg_plan p;
  p.V = 1 << ranked_lanes(passes, warps, arith)[0];
  p.T = mwk::TPB;
  const int64_t tiles = (n + mwk::TPB - 1) / mwk::TPB;
  // One resident wave: the kernels' launch bounds keep `minb` blocks of 256
  // threads per SM within the register file (3 for the FP64-word
  // arithmetics, 4 for the FP32-word ones).
  p.G = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)minb * sms, std::min<int64_t>(tiles, kMaxG)));
  // A system of at most `small_cluster` tiles is solved by one thread-block
  // cluster in a single launch (see run_solve).  With G >= tiles every tile is
  // its own block, so G = small_cluster gives the same summation order as
  // G = tiles.
  if (tiles <= small_cluster) p.G = small_cluster;
  return p;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int validate_row_ptr(int64_t n, const int64_t* rp) {
  if (rp[0] != 0) return fail(MWCG_ERR_ARG, "row_ptr[0] = %lld, expected 0", (long long)rp[0]);
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return fail(MWCG_ERR_ARG, "row_ptr decreases at row %lld", (long long)i);
  return MWCG_OK;
}

// The first invalid entry k (column outside [0, n) or value not finite), with
// the column reported before the value.
int entry_error(int64_t k, int32_t c, double v, int64_t n) {
  if (c < 0 || (int64_t)c >= n)
    return fail(MWCG_ERR_ARG, "col[%lld] = %d out of range [0, %lld)", (long long)k, c, (long long)n);
  return fail(MWCG_ERR_ARG, "val[%lld] is not finite", (long long)k);
}

int validate_entries(int64_t n, int64_t nnz, const int32_t* col, const double* val) {
  for (int64_t k = 0; k < nnz; ++k)
    if (col[k] < 0 || (int64_t)col[k] >= n || !std::isfinite(val[k])) return entry_error(k, col[k], val[k], n);
  return MWCG_OK;
}

// Smallest k with col[k] outside [0, n) or val[k] not finite, by an atomic
// minimum (*first starts above any index).
__global__ void k_first_bad_entry(const int32_t* __restrict__ col, const double* __restrict__ val, int64_t nnz,
                                  int64_t n, int64_t* first) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    if (col[k] < 0 || (int64_t)col[k] >= n || !isfinite(val[k]))
      atomicMin(reinterpret_cast<unsigned long long*>(first), (unsigned long long)k);
}

template <class... Args>
int add_kernel(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* dep, size_t ndep, const void* fn,
               int grid, size_t smem, Args... args) {
  void* ptrs[] = {(void*)&args...};
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(mwk::TPB);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = ptrs;
  kp.extra = nullptr;
  CK(cudaGraphAddKernelNode(node, g, dep, ndep, &kp));
  return MWCG_OK;
}

mwk::Csr csr_view(const mwcg_csr* A) { return mwk::Csr{A->rp, A->col, A->val, A->n}; }

mwk::Work work_view(const mwcg_csr* A, unsigned long long cond, int has_cond) {
  const int64_t n = A->n;
  mwk::Work W;
  W.r = A->ws;
  W.p = A->ws + 4 * n;
  W.q = A->ws + 8 * n;
  W.part = A->part;
  W.st = A->st;
  W.cond = cond;
  W.has_cond = has_cond;
  W.V = A->plan.V;
  W.G = A->plan.G;
  W.w = (A->prec == MWCG_PREC_JACOBI) ? A->w : nullptr;
  return W;
}

// The loop kernels: the default instantiations implement the default
// normalisation policy {1, NORM_R} with no run-time tests; any other policy
// runs the instantiations that read it from the DevState.  A Jacobi
// preconditioner selects the PCG init / update / p-update kernels.
struct LoopKernels {
  const void* init;
  const void* spmv;
  const void* update;
  const void* pupdate;
  int key;                     // bit 0: policy kernels, bit 1: preconditioned
};
LoopKernels loop_kernels(const mwcg_csr* A, const mwk::KernelTable* kt) {
  const bool pol = !(A->norm_every == 1 && A->norm_mask == mwk::NORM_R);
  const bool pc = A->prec == MWCG_PREC_JACOBI;
  LoopKernels k;
  k.key = (pol ? 1 : 0) | (pc ? 2 : 0);
  k.init = pc ? kt->init_pcg : kt->init;
  k.spmv = pol ? kt->spmv_pol : kt->spmv;
  if (pc) {
    k.update = pol ? kt->update_pcg_pol : kt->update_pcg;
    k.pupdate = pol ? kt->pupdate_pcg_pol : kt->pupdate_pcg;
  } else {
    k.update = pol ? kt->update_pol : kt->update;
    k.pupdate = pol ? kt->pupdate_pol : kt->pupdate;
  }
  return k;
}

// Build (or reuse) the graph of a whole solve in one arithmetic.
int ensure_graph(mwcg_csr* A, int arith) {
  GraphCache& gc = A->graphs[arith];
  const LoopKernels lk = loop_kernels(A, table(arith));
  if (gc.exec && gc.plan.V == A->plan.V && gc.plan.G == A->plan.G && gc.key == lk.key) return MWCG_OK;
  if (gc.exec) cudaGraphExecDestroy(gc.exec);
  if (gc.graph) cudaGraphDestroy(gc.graph);
  gc = GraphCache{};
  const mwk::KernelTable* kt = table(arith);
  const int G = A->plan.G;
  const size_t smem = red_smem(G, kt->words);
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(MWCG_ERR_CUDA, "cudaGraphConditionalHandleCreate: %s", cudaGetErrorString(e));
  }
  const mwk::Csr M = csr_view(A);
  const mwk::Work W = work_view(A, (unsigned long long)h, 1);
  cudaGraphNode_t n0, n1, n2, nw, b0, b1, b2;
  int rc;
  const int mode0 = 0, mode1 = 1;
  cudaGraphNode_t npre = nullptr;
  const void* pre = init_pre(arith);
  if ((rc = add_kernel(&n0, g, nullptr, 0, kt->spmv, G, smem, M, W, mode0)) ||
      (pre && (rc = add_kernel(&npre, g, &n0, 1, pre, G, smem, M, W))) ||
      (rc = add_kernel(&n1, g, npre ? &npre : &n0, 1, lk.init, G, smem, M, W)) ||
      (rc = add_kernel(&n2, g, &n1, 1, kt->zero_x, G, 0, M, W))) {
    cudaGraphDestroy(g);
    return rc;
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(&nw, g, &n2, nullptr, 1, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(MWCG_ERR_CUDA, "cudaGraphAddNode(while): %s", cudaGetErrorString(e));
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((rc = add_kernel(&b0, body, nullptr, 0, lk.spmv, G, smem, M, W, mode1)) ||
      (rc = add_kernel(&b1, body, &b0, 1, lk.update, G, smem, M, W)) ||
      (rc = add_kernel(&b2, body, &b1, 1, lk.pupdate, G, 0, M, W))) {
    cudaGraphDestroy(g);
    return rc;
  }
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(MWCG_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  gc.graph = g;
  gc.exec = ex;
  gc.plan = A->plan;
  gc.key = lk.key;
  return MWCG_OK;
}

int ensure_ws(mwcg_csr* A) {
  if (A->ws || A->n == 0) return MWCG_OK;
  CK(cudaMalloc(&A->ws, sizeof(double) * 12 * (size_t)A->n));   // r, p, q: up to four words each
  return MWCG_OK;
}

// Smallest k with val[k] not finite, by an atomic minimum (*first starts
// above any index).
__global__ void k_first_nonfinite(const double* __restrict__ val, int64_t nnz, int64_t* first) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(val[k])) atomicMin(reinterpret_cast<unsigned long long*>(first), (unsigned long long)k);
}

// Synthetic SpMV input for plan timing: every word of p populated (a vector
// whose lower words are zero runs faster than the iterates do).  FP64 words:
// word k of element i is +-(1 + h_i 2^-32) 2^(-53 k); FP32 words (packed two
// to a slot): word j is +-(1 + h_i 2^-32) 2^(-24 j); h_i a 32-bit hash of i.
__global__ void k_fill_probe(double* v, int64_t n, int slots, int fp32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ULL;
    h ^= h >> 29;
    const double m = (1.0 + (double)(uint32_t)(h >> 16) * 0x1p-32) * ((h & 1) ? -1.0 : 1.0);
    for (int k = 0; k < slots; ++k) {
      if (fp32) {
        float2 f = make_float2((float)(m * ldexp(1.0, -48 * k)), (float)(m * ldexp(1.0, -48 * k - 24)));
        reinterpret_cast<float2*>(v)[k * n + i] = f;
      } else {
        v[k * n + i] = m * ldexp(1.0, -53 * k);
      }
    }
  }
}

// The plan check of an arithmetic, once per handle: the SpMV (q = A p, the
// kernel that depends on the lane count V) is timed with CUDA events under
// the cost model's candidates (the best and those within twice its cost, at
// most three; same G), two warm launches then three timed; the model's choice
// is kept unless another candidate is at least 4% faster.  Systems small
// enough for the one-cluster solve keep the model's plan.
int tune_plan(mwcg_csr* A, int arith, cudaStream_t s) {
  A->tuned[arith] = true;
  const int64_t n = A->n;
  const int64_t tiles = (n + mwk::TPB - 1) / mwk::TPB;
  const mwcg_plan model = A->auto_plan[arith];
  if (n == 0 || tiles <= mwb_host::small_cluster_size()) return MWCG_OK;
  const std::vector<int> rank = ranked_lanes(A->passes, A->warps, arith);
  const double c0 = plan_cost(A->passes, A->warps, rank[0], arith);
  std::vector<int> cand;
  for (int j : rank)
    if (cand.size() < 3 && plan_cost(A->passes, A->warps, j, arith) <= 2.0 * c0) cand.push_back(j);
  if (cand.size() < 2) return MWCG_OK;
  int rc;
  if ((rc = ensure_ws(A)) != MWCG_OK) return rc;
  const mwk::KernelTable* kt = table(arith);
  double* p = A->ws + 4 * n;
  const bool fp32 = fp32_words(arith);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_fill_probe<<<grid, 256, 0, s>>>(p, n, mwcg_words(arith), fp32 ? 1 : 0);
  CK(cudaGetLastError());
  mwk::DevState* h = A->h_st;
  std::memset(h, 0, sizeof *h);
  h->x = p;                                   // the mode-0 SpMV reads its input from x
  CK(cudaMemcpyAsync(A->st, h, sizeof *h, cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const mwcg_plan saved = A->plan;
  double best_ms = -1;
  int best_j = cand[0];
  cudaError_t ce = cudaSuccess;
  for (size_t c = 0; c < cand.size() && ce == cudaSuccess; ++c) {
    A->plan = mwcg_plan{1 << cand[c], mwk::TPB, model.G};
    mwk::Csr M = csr_view(A);
    mwk::Work W = work_view(A, 0, 0);
    int mode0 = 0;
    void* args[] = {(void*)&M, (void*)&W, (void*)&mode0};
    const size_t smem = red_smem(model.G, kt->words);
    for (int r = 0; r < 5 && ce == cudaSuccess; ++r) {
      if (r == 2) ce = cudaEventRecord(e0, s);
      if (ce == cudaSuccess) ce = cudaLaunchKernel(kt->spmv, dim3(model.G), dim3(mwk::TPB), args, smem, s);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    const double t = ms / 3.0;
    A->tune_ms[arith][cand[c]] = t;
    if (c == 0 || t < 0.96 * best_ms) {      // the model's choice unless beaten by 4%
      best_ms = t;
      best_j = cand[c];
    }
  }
  A->plan = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return fail(MWCG_ERR_CUDA, "plan timing: %s", cudaGetErrorString(ce));
  A->auto_plan[arith].V = 1 << best_j;
  return MWCG_OK;
}

// Set A->plan for a call in `arith`: the pinned plan, or the arithmetic's
// automatic plan (checked by timing at its first call).
int select_plan(mwcg_csr* A, int arith, cudaStream_t s) {
  if (A->pinned) {
    A->plan = A->pinned_plan;
    return MWCG_OK;
  }
  if (!A->tuned[arith]) {
    const int rc = tune_plan(A, arith, s);
    if (rc != MWCG_OK) return rc;
  }
  A->plan = A->auto_plan[arith];
  return MWCG_OK;
}

// Jacobi weights for a preconditioned solve, built on first use after the
// preconditioner was set or the values changed.  *undefined: a diagonal
// entry is missing, not positive or not finite.
int ensure_weights(mwcg_csr* A, cudaStream_t s, bool* undefined) {
  *undefined = false;
  if (A->prec != MWCG_PREC_JACOBI || A->n == 0) return MWCG_OK;
  if (!A->w_valid) {
    if (!A->w) CK(cudaMalloc(&A->w, sizeof(double) * (size_t)A->n));
    if (!A->w_bad) CK(cudaMalloc(&A->w_bad, sizeof(int)));
    CK(cudaMemsetAsync(A->w_bad, 0, sizeof(int), s));
    CK(mwcg_precond::jacobi_weights(A->rp, A->col, A->val, A->n, A->w, A->w_bad, s));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, A->w_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    A->w_undefined = bad != 0;
    A->w_valid = true;
  }
  *undefined = A->w_undefined;
  return MWCG_OK;
}

// MWCG_EAGER=1 in the environment runs the solve without the CUDA graph: the
// host launches the same kernels, 16 iterations at a time, and reads the
// device's stop flag between batches (profilers cannot see kernels inside a
// graph with conditional nodes).
bool eager_mode() {
  const char* e = std::getenv("MWCG_EAGER");
  return e && e[0] == '1';
}

int run_eager(mwcg_csr* A, int arith, cudaStream_t s) {
  const mwk::KernelTable* kt = table(arith);
  mwk::Csr M = csr_view(A);
  mwk::Work W = work_view(A, 0, 0);
  const int G = A->plan.G;
  const size_t smem = red_smem(G, kt->words);
  int mode0 = 0, mode1 = 1;
  void* a_spmv0[] = {(void*)&M, (void*)&W, (void*)&mode0};
  void* a_spmv1[] = {(void*)&M, (void*)&W, (void*)&mode1};
  void* a_mw[] = {(void*)&M, (void*)&W};
  const LoopKernels lk = loop_kernels(A, kt);
  CK(cudaLaunchKernel(kt->spmv, dim3(G), dim3(mwk::TPB), a_spmv0, smem, s));
  if (const void* pre = init_pre(arith)) CK(cudaLaunchKernel(pre, dim3(G), dim3(mwk::TPB), a_mw, smem, s));
  CK(cudaLaunchKernel(lk.init, dim3(G), dim3(mwk::TPB), a_mw, smem, s));
  CK(cudaLaunchKernel(kt->zero_x, dim3(G), dim3(mwk::TPB), a_mw, 0, s));
  mwk::DevState* h = A->h_st;
  const int64_t batches = (int64_t)h->maxit / 16 + 2;
  for (int64_t bt = 0; bt < batches; ++bt) {
    CK(cudaMemcpyAsync(h, A->st, sizeof *h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->done) break;
    for (int i = 0; i < 16; ++i) {
      CK(cudaLaunchKernel(lk.spmv, dim3(G), dim3(mwk::TPB), a_spmv1, smem, s));
      CK(cudaLaunchKernel(lk.update, dim3(G), dim3(mwk::TPB), a_mw, smem, s));
      CK(cudaLaunchKernel(lk.pupdate, dim3(G), dim3(mwk::TPB), a_mw, 0, s));
    }
  }
  return MWCG_OK;
}

// Small systems (at most `small_cluster_size()` tiles of 256 rows, with the
// plan's G equal to that size) run in one persistent launch of one thread-
// block cluster: the same summation order as the graph (plan {V, 256, G}),
// with hardware cluster barriers instead of three kernel launches per
// iteration.
int run_cluster(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, double* hist,
                cudaStream_t s, int32_t* iters_out, double* relres_out) {
  mwb::Sys q{};
  const int64_t n = A->n;
  q.rp = A->rp;
  q.col = A->col;
  q.val = A->val;
  q.n = n;
  q.b = b;
  q.x = x;
  q.r = A->ws;
  q.p = A->ws + 4 * n;
  q.q = A->ws + 8 * n;
  q.tol = tol;
  q.maxit = maxit;
  q.arith = arith;
  q.V = A->plan.V;
  q.hist = hist;
  q.norm_every = A->norm_every;
  q.norm_mask = A->norm_mask;
  q.w = (A->prec == MWCG_PREC_JACOBI) ? A->w : nullptr;
  cudaError_t e = mwb_host::launch(&q, 1, s, A->plan.G, nullptr);
  if (e != cudaSuccess) return fail(MWCG_ERR_CUDA, "cluster solve: %s", cudaGetErrorString(e));
  if (iters_out) *iters_out = q.iters;
  if (relres_out) *relres_out = q.relres;
  return q.status;
}

int run_solve(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, double* hist,
              cudaStream_t s, int32_t* iters_out, double* relres_out) {
  int rc;
  if ((rc = select_plan(A, arith, s)) != MWCG_OK) return rc;
  if (A->prec == MWCG_PREC_JACOBI && !table(arith)->init_pcg)
    return fail(MWCG_ERR_ARG, "arithmetic %d has no preconditioned solver", arith);
  if ((rc = ensure_ws(A)) != MWCG_OK) return rc;
  bool undefined = false;
  if ((rc = ensure_weights(A, s, &undefined)) != MWCG_OK) return rc;
  if (undefined) {                     // x0 untouched, no iteration
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return MWCG_BAD_PRECONDITIONER;
  }
  const int64_t tiles = (A->n + mwk::TPB - 1) / mwk::TPB;
  const int small = mwb_host::small_cluster_size();
  if (!eager_mode() && A->plan.G == small && tiles <= small)
    return run_cluster(A, b, x, arith, tol, maxit, hist, s, iters_out, relres_out);
  const bool eager = eager_mode();
  if (!eager && (rc = ensure_graph(A, arith)) != MWCG_OK) return rc;
  mwk::DevState* h = A->h_st;
  std::memset(h, 0, sizeof *h);
  h->b = b;
  h->x = x;
  h->hist = hist;
  h->tol = tol;
  h->maxit = maxit;
  h->norm_every = A->norm_every;
  h->norm_mask = A->norm_mask;
  CK(cudaMemcpyAsync(A->st, h, sizeof *h, cudaMemcpyHostToDevice, s));
  if (eager) {
    if ((rc = run_eager(A, arith, s)) != MWCG_OK) return rc;
  } else {
    CK(cudaGraphLaunch(A->graphs[arith].exec, s));
  }
  CK(cudaMemcpyAsync(h, A->st, sizeof *h, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (iters_out) *iters_out = h->iters;
  if (relres_out) *relres_out = h->relres;
  if (h->status == mwk::ST_GUARD) return fail(MWCG_ERR_GUARD, "device loop guard tripped");
  return h->status;
}

// ---------------------------------------------------------------------------
// BiCGStab: one CUDA graph per (matrix, arithmetic) -- the x0 SpMV, init and
// zero_x nodes, then a conditional WHILE node over the five loop kernels.
// Small systems run the same graph (there is no single-cluster BiCGStab).
// ---------------------------------------------------------------------------
mwk::BiWork biwork_view(const mwcg_csr* A, unsigned long long cond, int has_cond) {
  const int64_t n = A->n;
  mwk::BiWork B;
  B.w = work_view(A, cond, has_cond);
  B.w.w = nullptr;
  B.rh = A->bws;
  B.s = A->bws + 4 * n;
  B.t = A->bws + 8 * n;
  return B;
}

int ensure_bigraph(mwcg_csr* A, int arith) {
  GraphCache& gc = A->bigraphs[arith];
  if (gc.exec && gc.plan.V == A->plan.V && gc.plan.G == A->plan.G) return MWCG_OK;
  if (gc.exec) cudaGraphExecDestroy(gc.exec);
  if (gc.graph) cudaGraphDestroy(gc.graph);
  gc = GraphCache{};
  const mwk::KernelTable* kt = table(arith);
  const mwk::BiTable* bt = bitable(arith);
  const int G = A->plan.G;
  const size_t smem = red_smem(G, kt->words);
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(MWCG_ERR_CUDA, "cudaGraphConditionalHandleCreate: %s", cudaGetErrorString(e));
  }
  const mwk::Csr M = csr_view(A);
  const mwk::Work W = work_view(A, (unsigned long long)h, 1);
  const mwk::BiWork B = biwork_view(A, (unsigned long long)h, 1);
  cudaGraphNode_t n0, n1, n2, nw, b[5];
  cudaGraphNode_t npre = nullptr;
  int rc;
  const int mode0 = 0;
  const void* pre = init_pre(arith);          // QQF / QF: ||b|| and the first scale
  if ((rc = add_kernel(&n0, g, nullptr, 0, kt->spmv, G, smem, M, W, mode0)) ||
      (pre && (rc = add_kernel(&npre, g, &n0, 1, pre, G, smem, M, W))) ||
      (rc = add_kernel(&n1, g, npre ? &npre : &n0, 1, bt->init, G, smem, M, B)) ||
      (rc = add_kernel(&n2, g, &n1, 1, kt->zero_x, G, 0, M, W))) {
    cudaGraphDestroy(g);
    return rc;
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(&nw, g, &n2, nullptr, 1, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(MWCG_ERR_CUDA, "cudaGraphAddNode(while): %s", cudaGetErrorString(e));
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const void* fns[5] = {bt->p, bt->spmv_v, bt->s, bt->spmv_t, bt->xr};
  const size_t sm[5] = {0, smem, smem, smem, smem};
  for (int k = 0; k < 5; ++k) {
    if ((rc = add_kernel(&b[k], body, k ? &b[k - 1] : nullptr, k ? 1 : 0, fns[k], G, sm[k], M, B))) {
      cudaGraphDestroy(g);
      return rc;
    }
  }
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(MWCG_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  gc.graph = g;
  gc.exec = ex;
  gc.plan = A->plan;
  return MWCG_OK;
}

int run_bicg(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, double* hist,
             cudaStream_t s, int32_t* iters_out, double* relres_out) {
  int rc;
  if ((rc = select_plan(A, arith, s)) != MWCG_OK) return rc;
  if ((rc = ensure_ws(A)) != MWCG_OK) return rc;
  if (!A->bws) CK(cudaMalloc(&A->bws, sizeof(double) * 12 * (size_t)A->n));
  const bool eager = eager_mode();
  if (!eager && (rc = ensure_bigraph(A, arith)) != MWCG_OK) return rc;
  mwk::DevState* h = A->h_st;
  std::memset(h, 0, sizeof *h);
  h->b = b;
  h->x = x;
  h->hist = hist;
  h->tol = tol;
  h->maxit = maxit;
  CK(cudaMemcpyAsync(A->st, h, sizeof *h, cudaMemcpyHostToDevice, s));
  if (eager) {
    const mwk::KernelTable* kt = table(arith);
    const mwk::BiTable* bt = bitable(arith);
    mwk::Csr M = csr_view(A);
    mwk::Work W = work_view(A, 0, 0);
    mwk::BiWork B = biwork_view(A, 0, 0);
    const int G = A->plan.G;
    const size_t smem = red_smem(G, kt->words);
    int mode0 = 0;
    void* a_spmv0[] = {(void*)&M, (void*)&W, (void*)&mode0};
    void* a_w[] = {(void*)&M, (void*)&W};
    void* a_b[] = {(void*)&M, (void*)&B};
    CK(cudaLaunchKernel(kt->spmv, dim3(G), dim3(mwk::TPB), a_spmv0, smem, s));
    if (const void* pre = init_pre(arith)) CK(cudaLaunchKernel(pre, dim3(G), dim3(mwk::TPB), a_w, smem, s));
    CK(cudaLaunchKernel(bt->init, dim3(G), dim3(mwk::TPB), a_b, smem, s));
    CK(cudaLaunchKernel(kt->zero_x, dim3(G), dim3(mwk::TPB), a_w, 0, s));
    const void* fns[5] = {bt->p, bt->spmv_v, bt->s, bt->spmv_t, bt->xr};
    const int64_t batches = (int64_t)maxit / 16 + 2;
    for (int64_t bt_ = 0; bt_ < batches; ++bt_) {
      CK(cudaMemcpyAsync(h, A->st, sizeof *h, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h->done) break;
      for (int i = 0; i < 16; ++i)
        for (int k = 0; k < 5; ++k) CK(cudaLaunchKernel(fns[k], dim3(G), dim3(mwk::TPB), a_b, k ? smem : 0, s));
    }
  } else {
    CK(cudaGraphLaunch(A->bigraphs[arith].exec, s));
  }
  CK(cudaMemcpyAsync(h, A->st, sizeof *h, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (iters_out) *iters_out = h->iters;
  if (relres_out) *relres_out = h->relres;
  if (h->status == mwk::ST_GUARD) return fail(MWCG_ERR_GUARD, "device loop guard tripped");
  return h->status;
}

int check_solve_args(const mwcg_csr* A, const void* b, const void* x, int arith, double tol, int32_t maxit) {
  if (!A) return fail(MWCG_ERR_ARG, "null matrix handle");
  if (!table(arith)) return fail(MWCG_ERR_ARG, "unknown arithmetic %d", arith);
  if (A->n > 0 && (!b || !x)) return fail(MWCG_ERR_ARG, "null b or x");
  if (!(tol >= 0.0) || std::isnan(tol)) return fail(MWCG_ERR_ARG, "tol must be >= 0");
  if (maxit < 0 || maxit > kMaxIt) return fail(MWCG_ERR_ARG, "maxit must be in [0, 2^30]");
  return MWCG_OK;
}

}  // namespace

extern "C" {

int mwcg_words(int arith) {
  static const int w[kNArith] = {1, 2, 2, 3, 3, 2, 3, 4, 4, 4, 2, 2};   // QQF, QF: 4 FP32 words in 2 slots
  return (arith >= 0 && arith < kNArith) ? w[arith] : -1;
}

const char* mwcg_last_error(void) { return g_err.c_str(); }

int mwcg_create_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, int ptrs_on_device,
                    void* stream, mwcg_csr** out) {
  g_err.clear();
  if (!out) return fail(MWCG_ERR_ARG, "null output handle pointer");
  *out = nullptr;
  if (n < 0 || n > (int64_t)INT32_MAX) return fail(MWCG_ERR_ARG, "n = %lld out of range", (long long)n);
  if (!row_ptr) return fail(MWCG_ERR_ARG, "null row_ptr");
  cudaStream_t s = S(stream);
  // Host copies for validation and plan selection.
  std::vector<int64_t> hrp(n + 1);
  if (ptrs_on_device) CK(cudaMemcpy(hrp.data(), row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
  else std::memcpy(hrp.data(), row_ptr, sizeof(int64_t) * (n + 1));
  const int64_t nnz = hrp[n];
  if (nnz < 0 || nnz > ((int64_t)1 << 40)) return fail(MWCG_ERR_ARG, "nnz = %lld out of range", (long long)nnz);
  if (nnz > 0 && (!col || !val)) return fail(MWCG_ERR_ARG, "null col or val");
  int rc = validate_row_ptr(n, hrp.data());
  if (rc != MWCG_OK) return rc;
  // Host entries are checked here; device entries are checked on the device
  // once copied (no host copy of the nnz entries).
  if (!ptrs_on_device && (rc = validate_entries(n, nnz, col, val)) != MWCG_OK) return rc;

  mwcg_csr* A = new mwcg_csr();
  CK(cudaGetDevice(&A->device));
  A->n = n;
  A->nnz = nnz;
  auto cleanup = [&](int code) {
    mwcg_destroy_csr(A);
    return code;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&A->rp, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
      (nnz && (e = cudaMalloc(&A->col, sizeof(int32_t) * nnz)) != cudaSuccess) ||
      (nnz && (e = cudaMalloc(&A->val, sizeof(double) * nnz)) != cudaSuccess) ||
      (e = cudaMalloc(&A->part, sizeof(double) * mwk::PART * kMaxG)) != cudaSuccess ||
      (e = cudaMalloc(&A->st, sizeof(mwk::DevState))) != cudaSuccess ||
      (e = cudaMallocHost(&A->h_st, sizeof(mwk::DevState))) != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? MWCG_ERR_NOMEM : MWCG_ERR_CUDA, "allocation: %s",
                        cudaGetErrorString(e)));
  const cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((e = cudaMemcpyAsync(A->rp, ptrs_on_device ? row_ptr : hrp.data(), sizeof(int64_t) * (n + 1), kind, s)) !=
          cudaSuccess ||
      (nnz && (e = cudaMemcpyAsync(A->col, col, sizeof(int32_t) * nnz, kind, s)) != cudaSuccess) ||
      (nnz && (e = cudaMemcpyAsync(A->val, val, sizeof(double) * nnz, kind, s)) != cudaSuccess) ||
      (e = cudaMemsetAsync(A->st, 0, sizeof(mwk::DevState), s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cleanup(fail(MWCG_ERR_CUDA, "copy to device: %s", cudaGetErrorString(e)));
  if (ptrs_on_device && nnz) {
    int64_t* first = nullptr;
    int64_t bad = 0;
    if ((e = cudaMalloc(&first, sizeof(int64_t))) == cudaSuccess &&
        (e = cudaMemsetAsync(first, 0x7f, sizeof(int64_t), s)) == cudaSuccess) {
      const int grid = (int)std::min<int64_t>((nnz + 255) / 256, 4096);
      k_first_bad_entry<<<grid, 256, 0, s>>>(A->col, A->val, nnz, n, first);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, first, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(first);
    if (e != cudaSuccess) return cleanup(fail(MWCG_ERR_CUDA, "entry check: %s", cudaGetErrorString(e)));
    if (bad < nnz) {
      int32_t c = 0;
      double v = 0.0;
      if ((e = cudaMemcpy(&c, A->col + bad, sizeof c, cudaMemcpyDeviceToHost)) != cudaSuccess ||
          (e = cudaMemcpy(&v, A->val + bad, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cleanup(fail(MWCG_ERR_CUDA, "entry check: %s", cudaGetErrorString(e)));
      return cleanup(entry_error(bad, c, v, n));
    }
  }
  {
    std::vector<int64_t> rowlen(n);
    for (int64_t i = 0; i < n; ++i) rowlen[i] = hrp[i + 1] - hrp[i];
    row_stats(rowlen, A->passes, A->warps);
  }
  const int sms = sm_count_of(A->device), small = mwb_host::small_cluster_size();
  for (int a = 0; a < kNArith; ++a)
    A->auto_plan[a] = choose_plan(A->passes, A->warps, n, sms, a, small, table(a)->minb);
  A->plan = A->auto_plan[MWCG_QTW];
  *out = A;
  return MWCG_OK;
}

void mwcg_destroy_csr(mwcg_csr* A) {
  if (!A) return;
  free_graphs(A);
  cudaFree(A->rp);
  cudaFree(A->col);
  cudaFree(A->val);
  cudaFree(A->ws);
  cudaFree(A->part);
  cudaFree(A->st);
  cudaFree(A->lam);
  cudaFree(A->hb);
  cudaFree(A->hx);
  cudaFree(A->w);
  cudaFree(A->w_bad);
  cudaFree(A->vbad);
  cudaFree(A->bws);
  if (A->h_st) cudaFreeHost(A->h_st);
  delete A;
}

int mwcg_update_values(mwcg_csr* A, const double* val, int on_device, void* stream) {
  g_err.clear();
  if (!A) return fail(MWCG_ERR_ARG, "null matrix handle");
  if (A->nnz == 0) return MWCG_OK;
  if (!val) return fail(MWCG_ERR_ARG, "null val");
  cudaStream_t s = S(stream);
  if (on_device) {
    // Validated on the device (the first non-finite index, if any, comes back
    // as one 8-byte word), then copied device to device: no host round trip
    // of the values, which autograd updates on every step.
    if (!A->vbad) CK(cudaMalloc(&A->vbad, sizeof(int64_t)));
    int64_t* first = A->vbad;
    CK(cudaMemsetAsync(first, 0x7f, sizeof(int64_t), s));
    const int grid = (int)std::min<int64_t>((A->nnz + 255) / 256, 4096);
    k_first_nonfinite<<<grid, 256, 0, s>>>(val, A->nnz, first);
    int64_t bad = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, first, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(MWCG_ERR_CUDA, "value check: %s", cudaGetErrorString(e));
    if (bad < A->nnz) return fail(MWCG_ERR_ARG, "val[%lld] is not finite", (long long)bad);
    CK(cudaMemcpyAsync(A->val, val, sizeof(double) * A->nnz, cudaMemcpyDeviceToDevice, s));
  } else {
    for (int64_t k = 0; k < A->nnz; ++k)
      if (!std::isfinite(val[k])) return fail(MWCG_ERR_ARG, "val[%lld] is not finite", (long long)k);
    CK(cudaMemcpyAsync(A->val, val, sizeof(double) * A->nnz, cudaMemcpyHostToDevice, s));
  }
  CK(cudaStreamSynchronize(s));
  A->w_valid = false;                  // Jacobi weights follow the new diagonal
  return MWCG_OK;
}

int64_t mwcg_n(const mwcg_csr* A) { return A ? A->n : -1; }
int64_t mwcg_nnz(const mwcg_csr* A) { return A ? A->nnz : -1; }

int mwcg_get_plan(const mwcg_csr* A, mwcg_plan* out) {
  if (!A || !out) return fail(MWCG_ERR_ARG, "null argument");
  *out = A->plan;
  return MWCG_OK;
}

int mwcg_set_plan(mwcg_csr* A, const mwcg_plan* p) {
  if (!A) return fail(MWCG_ERR_ARG, "null argument");
  if (!p) {                            // back to the automatic plans
    A->pinned = false;
    A->plan = A->auto_plan[MWCG_QTW];
    return MWCG_OK;
  }
  if (!is_pow2_le32(p->V) || p->T != mwk::TPB || p->G < 1 || p->G > kMaxG)
    return fail(MWCG_ERR_ARG, "invalid plan V=%d T=%d G=%d", p->V, p->T, p->G);
  A->pinned = true;
  A->pinned_plan = *p;
  A->plan = *p;
  return MWCG_OK;
}

int mwcg_get_plan_for(mwcg_csr* A, int arith, void* stream, mwcg_plan* out, double* spmv_ms) {
  g_err.clear();
  if (!A || !out || !table(arith)) return fail(MWCG_ERR_ARG, "bad handle, arithmetic or output");
  const int rc = select_plan(A, arith, S(stream));
  if (rc != MWCG_OK) return rc;
  *out = A->plan;
  if (spmv_ms)
    for (int j = 0; j < 6; ++j) spmv_ms[j] = A->pinned ? 0.0 : A->tune_ms[arith][j];
  return MWCG_OK;
}

int mwcg_set_normalization(mwcg_csr* A, int32_t every, uint32_t mask) {
  if (!A) return fail(MWCG_ERR_ARG, "null matrix handle");
  if (every < 0) return fail(MWCG_ERR_ARG, "every = %d < 0", (int)every);
  if (mask & ~(uint32_t)mwk::NORM_ALL) return fail(MWCG_ERR_ARG, "unknown normalisation bits 0x%x", (unsigned)mask);
  A->norm_every = every;
  A->norm_mask = mask;
  return MWCG_OK;
}

int mwcg_set_preconditioner(mwcg_csr* A, int kind) {
  if (!A) return fail(MWCG_ERR_ARG, "null matrix handle");
  if (kind != MWCG_PREC_NONE && kind != MWCG_PREC_JACOBI) return fail(MWCG_ERR_ARG, "unknown preconditioner %d", kind);
  if (kind != A->prec) A->w_valid = false;
  A->prec = kind;
  return MWCG_OK;
}

int mwcg_get_preconditioner(const mwcg_csr* A, int* kind) {
  if (!A || !kind) return fail(MWCG_ERR_ARG, "null argument");
  *kind = A->prec;
  return MWCG_OK;
}

int mwcg_get_normalization(const mwcg_csr* A, int32_t* every, uint32_t* mask) {
  if (!A || !every || !mask) return fail(MWCG_ERR_ARG, "null argument");
  *every = A->norm_every;
  *mask = A->norm_mask;
  return MWCG_OK;
}

int mwcg_solve_bicgstab(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, double* hist,
                        void* stream, int32_t* iters_out, double* relres_out) {
  g_err.clear();
  int rc = check_solve_args(A, b, x, arith, tol, maxit);
  if (rc != MWCG_OK) return rc;
  if (!bitable(arith)) return fail(MWCG_ERR_ARG, "arithmetic %d has no BiCGStab", arith);
  if (A->n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return MWCG_OK;
  }
  return run_bicg(A, b, x, arith, tol, maxit, hist, S(stream), iters_out, relres_out);
}

int mwcg_solve(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit, void* stream,
               int32_t* iters_out, double* relres_out) {
  return mwcg_solve_history(A, b, x, arith, tol, maxit, nullptr, stream, iters_out, relres_out);
}

int mwcg_solve_history(mwcg_csr* A, const double* b, double* x, int arith, double tol, int32_t maxit,
                       double* hist, void* stream, int32_t* iters_out, double* relres_out) {
  g_err.clear();
  int rc = check_solve_args(A, b, x, arith, tol, maxit);
  if (rc != MWCG_OK) return rc;
  if (A->n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return MWCG_OK;
  }
  return run_solve(A, b, x, arith, tol, maxit, hist, S(stream), iters_out, relres_out);
}

int mwcg_solve_host(mwcg_csr* A, const double* b_host, double* x_host, int arith, double tol, int32_t maxit,
                    void* stream, int32_t* iters_out, double* relres_out) {
  g_err.clear();
  int rc = check_solve_args(A, b_host, x_host, arith, tol, maxit);
  if (rc != MWCG_OK) return rc;
  if (A->n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return MWCG_OK;
  }
  const size_t n = (size_t)A->n;
  const int w = mwcg_words(arith);
  if (!A->hb) CK(cudaMalloc(&A->hb, sizeof(double) * n));
  if (!A->hx) CK(cudaMalloc(&A->hx, sizeof(double) * 4 * n));
  cudaStream_t s = S(stream);
  CK(cudaMemcpyAsync(A->hb, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(A->hx, x_host, sizeof(double) * w * n, cudaMemcpyHostToDevice, s));
  rc = run_solve(A, A->hb, A->hx, arith, tol, maxit, nullptr, s, iters_out, relres_out);
  if (rc < 0) return rc;
  CK(cudaMemcpyAsync(x_host, A->hx, sizeof(double) * w * n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return rc;
}

int mwcg_adjoint(mwcg_csr* A, const double* x, const double* gx, int arith, double tol, int32_t maxit, void* stream,
                 double* g_b, double* g_val, int32_t* iters_out, double* relres_out) {
  g_err.clear();
  int rc = check_solve_args(A, gx, x, arith, tol, maxit);
  if (rc != MWCG_OK) return rc;
  if (!table(arith)->grad_values) return fail(MWCG_ERR_ARG, "arithmetic %d has no adjoint", arith);
  if (A->n == 0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return MWCG_OK;
  }
  cudaStream_t s = S(stream);
  const size_t n = (size_t)A->n;
  if (!A->lam) CK(cudaMalloc(&A->lam, sizeof(double) * 4 * n));
  CK(cudaMemsetAsync(A->lam, 0, sizeof(double) * 4 * n, s));
  rc = run_solve(A, gx, A->lam, arith, tol, maxit, nullptr, s, iters_out, relres_out);
  if (rc < 0 || rc == MWCG_BAD_PRECONDITIONER) return rc;
  const mwk::KernelTable* kt = table(arith);
  const mwk::Csr M = csr_view(A);
  const int G = A->plan.G;
  if (g_b) {
    void* args[] = {(void*)&A->lam, (void*)&A->n, (void*)&g_b};
    CK(cudaLaunchKernel(kt->collapse, dim3(G), dim3(mwk::TPB), args, 0, s));
  }
  if (g_val && A->nnz) {
    const double* lam = A->lam;
    void* args[] = {(void*)&M, (void*)&lam, (void*)&x, (void*)&g_val};
    CK(cudaLaunchKernel(kt->grad_values, dim3(std::max(G, 1)), dim3(mwk::TPB), args, 0, s));
  }
  CK(cudaStreamSynchronize(s));
  return rc;
}

int mwcg_spmv(mwcg_csr* A, int arith, const double* p, double* q, void* stream) {
  g_err.clear();
  if (!A || !table(arith)) return fail(MWCG_ERR_ARG, "bad handle or arithmetic");
  if (A->n == 0) return MWCG_OK;
  if (!p || !q) return fail(MWCG_ERR_ARG, "null p or q");
  cudaStream_t s = S(stream);
  int rc;
  if ((rc = select_plan(A, arith, s)) != MWCG_OK) return rc;
  if ((rc = ensure_ws(A)) != MWCG_OK) return rc;
  mwk::DevState* h = A->h_st;
  std::memset(h, 0, sizeof *h);
  h->x = const_cast<double*>(p);
  CK(cudaMemcpyAsync(A->st, h, sizeof *h, cudaMemcpyHostToDevice, s));
  mwk::Csr M = csr_view(A);
  mwk::Work W = work_view(A, 0, 0);
  W.q = q;
  int mode = 0;
  void* args[] = {(void*)&M, (void*)&W, (void*)&mode};
  CK(cudaLaunchKernel(table(arith)->spmv, dim3(A->plan.G), dim3(mwk::TPB), args,
                      red_smem(A->plan.G, table(arith)->words), s));
  CK(cudaStreamSynchronize(s));
  return MWCG_OK;
}

int mwcg_dot(int arith, int64_t n, const double* u, const double* v, int32_t G, void* stream, double* out) {
  g_err.clear();
  if (!table(arith) || n < 0 || G < 1 || G > kMaxG || !out) return fail(MWCG_ERR_ARG, "bad argument");
  const int w = fp32_words(arith) ? 4 : mwcg_words(arith);      // one word per double
  if (n == 0) {
    for (int k = 0; k < w; ++k) out[k] = 0.0;
    return MWCG_OK;
  }
  if (!u || !v) return fail(MWCG_ERR_ARG, "null u or v");
  cudaStream_t s = S(stream);
  double* part = nullptr;
  mwk::DevState* st = nullptr;
  double* dout = nullptr;
  cudaError_t e = cudaMalloc(&part, sizeof(double) * mwk::PART * G);
  if (e == cudaSuccess) e = cudaMalloc(&st, sizeof(mwk::DevState));
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(mwk::DevState), s);
  if (e == cudaSuccess) {
    mwk::Work W{};
    W.part = part;
    W.st = st;
    W.V = 1;
    W.G = G;
    void* args[] = {(void*)&u, (void*)&v, (void*)&n, (void*)&W, (void*)&dout};
    e = cudaLaunchKernel(table(arith)->dot, dim3(G), dim3(mwk::TPB), args, red_smem(G, table(arith)->words), s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * w, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  cudaFree(st);
  cudaFree(dout);
  if (e != cudaSuccess) return fail(MWCG_ERR_CUDA, "mwcg_dot: %s", cudaGetErrorString(e));
  return MWCG_OK;
}

int mwcg_word_op(int op, int arith, int64_t n, const double* a, const double* b, double* c, void* stream) {
  g_err.clear();
  if (!table(arith) || op < 0 || op > 5 || n < 0) return fail(MWCG_ERR_ARG, "bad argument");
  if (n == 0) return MWCG_OK;
  if (!a || !c || ((op <= 3) && !b)) return fail(MWCG_ERR_ARG, "null operand");
  cudaStream_t s = S(stream);
  const int grid = (int)std::min<int64_t>((n + mwk::TPB - 1) / mwk::TPB, 4096);
  void* args[] = {(void*)&op, (void*)&n, (void*)&a, (void*)&b, (void*)&c};
  CK(cudaLaunchKernel(table(arith)->word_op, dim3(grid), dim3(mwk::TPB), args, 0, s));
  CK(cudaStreamSynchronize(s));
  return MWCG_OK;
}

int mwcg_collapse(const double* xw, int32_t w, int64_t n, double* x64, void* stream) {
  g_err.clear();
  if (w < 1 || w > 4 || n < 0) return fail(MWCG_ERR_ARG, "bad argument");
  if (n == 0) return MWCG_OK;
  if (!xw || !x64) return fail(MWCG_ERR_ARG, "null pointer");
  const int arith = (w == 1) ? MWCG_FP64 : (w == 2) ? MWCG_DW : (w == 3) ? MWCG_QTW : MWCG_QQW;
  const int grid = (int)std::min<int64_t>((n + mwk::TPB - 1) / mwk::TPB, 4096);
  void* args[] = {(void*)&xw, (void*)&n, (void*)&x64};
  CK(cudaLaunchKernel(table(arith)->collapse, dim3(grid), dim3(mwk::TPB), args, 0, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  return MWCG_OK;
}

int mwcg_profile_kernels(mwcg_csr* A, const double* b, double* x, int arith, int32_t niters, void* stream,
                         double* ms_out) {
  g_err.clear();
  int rc = check_solve_args(A, b, x, arith, 0.0, niters);
  if (rc != MWCG_OK) return rc;
  if (niters < 2 || niters > 100000 || !ms_out || A->n == 0) return fail(MWCG_ERR_ARG, "bad profile arguments");
  cudaStream_t s = S(stream);
  if ((rc = select_plan(A, arith, s)) != MWCG_OK) return rc;
  if ((rc = ensure_ws(A)) != MWCG_OK) return rc;
  const mwk::KernelTable* kt = table(arith);
  if (A->prec == MWCG_PREC_JACOBI && !kt->init_pcg)
    return fail(MWCG_ERR_ARG, "arithmetic %d has no preconditioned solver", arith);
  mwk::DevState* h = A->h_st;
  std::memset(h, 0, sizeof *h);
  h->b = b;
  h->x = x;
  h->tol = 0.0;
  h->maxit = niters;
  h->norm_every = A->norm_every;
  h->norm_mask = A->norm_mask;
  CK(cudaMemcpyAsync(A->st, h, sizeof *h, cudaMemcpyHostToDevice, s));
  mwk::Csr M = csr_view(A);
  mwk::Work W = work_view(A, 0, 0);
  const int G = A->plan.G;
  const size_t smem = red_smem(G, kt->words);
  int mode0 = 0, mode1 = 1;
  void* a_spmv0[] = {(void*)&M, (void*)&W, (void*)&mode0};
  void* a_spmv1[] = {(void*)&M, (void*)&W, (void*)&mode1};
  void* a_mw[] = {(void*)&M, (void*)&W};
  const LoopKernels lk = loop_kernels(A, kt);
  CK(cudaLaunchKernel(kt->spmv, dim3(G), dim3(mwk::TPB), a_spmv0, smem, s));
  if (const void* pre = init_pre(arith)) CK(cudaLaunchKernel(pre, dim3(G), dim3(mwk::TPB), a_mw, smem, s));
  CK(cudaLaunchKernel(lk.init, dim3(G), dim3(mwk::TPB), a_mw, smem, s));
  CK(cudaLaunchKernel(kt->zero_x, dim3(G), dim3(mwk::TPB), a_mw, 0, s));
  std::vector<cudaEvent_t> ev(3 * (size_t)niters + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  int err = MWCG_OK;
  cudaError_t ce = cudaEventRecord(ev[0], s);
  for (int i = 0; i < niters && ce == cudaSuccess; ++i) {
    ce = cudaLaunchKernel(lk.spmv, dim3(G), dim3(mwk::TPB), a_spmv1, smem, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * i + 1], s);
    if (ce == cudaSuccess) ce = cudaLaunchKernel(lk.update, dim3(G), dim3(mwk::TPB), a_mw, smem, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * i + 2], s);
    if (ce == cudaSuccess) ce = cudaLaunchKernel(lk.pupdate, dim3(G), dim3(mwk::TPB), a_mw, 0, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * i + 3], s);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) err = fail(MWCG_ERR_CUDA, "profile: %s", cudaGetErrorString(ce));
  double acc[3] = {0, 0, 0};
  if (err == MWCG_OK) {
    // The last p update is skipped by design (the loop has stopped), so it is
    // averaged over the first niters-1 iterations.
    for (int i = 0; i < niters; ++i)
      for (int k = 0; k < 3; ++k) {
        if (k == 2 && i == niters - 1) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[3 * i + k], ev[3 * i + k + 1]);
        acc[k] += ms;
      }
    ms_out[0] = acc[0] / niters;
    ms_out[1] = acc[1] / niters;
    ms_out[2] = acc[2] / (niters - 1);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return err;
}

int mwcg_batched_cluster_size(void) { return mwb_host::cluster_size(); }

int mwcg_solve_batched(int32_t nsys, mwcg_csr* const* A, const double* const* b, double* const* x,
                       const int32_t* arith, const double* tol, const int32_t* maxit, void* stream,
                       int32_t* iters_out, double* relres_out, int32_t* status_out) {
  g_err.clear();
  if (nsys < 0) return fail(MWCG_ERR_ARG, "nsys < 0");
  if (nsys == 0) return MWCG_OK;
  if (!A || !b || !x || !arith || !tol || !maxit) return fail(MWCG_ERR_ARG, "null argument array");
  std::set<const mwcg_csr*> seen;
  for (int s = 0; s < nsys; ++s) {
    int rc = check_solve_args(A[s], b[s], x[s], arith[s], tol[s], maxit[s]);
    if (rc != MWCG_OK) return fail(rc, "system %d: %s", s, g_err.c_str());
    if (!seen.insert(A[s]).second) return fail(MWCG_ERR_ARG, "system %d: matrix handle repeated in the batch", s);
    if ((rc = ensure_ws(A[s])) != MWCG_OK) return rc;
    if ((rc = select_plan(A[s], arith[s], S(stream))) != MWCG_OK) return rc;
  }
  std::vector<mwb::Sys> hs;
  std::vector<int> idx;
  std::vector<double> cost;
  for (int s = 0; s < nsys; ++s) {
    bool undefined = false;
    int rc = ensure_weights(A[s], S(stream), &undefined);
    if (rc != MWCG_OK) return rc;
    if (A[s]->n == 0 || undefined) {   // nothing to do / preconditioner undefined: x0 untouched
      if (iters_out) iters_out[s] = 0;
      if (relres_out) relres_out[s] = 0.0;
      if (status_out) status_out[s] = undefined ? MWCG_BAD_PRECONDITIONER : MWCG_OK;
      continue;
    }
    mwb::Sys q{};
    const int64_t n = A[s]->n;
    q.rp = A[s]->rp;
    q.col = A[s]->col;
    q.val = A[s]->val;
    q.n = n;
    q.b = b[s];
    q.x = x[s];
    q.r = A[s]->ws;
    q.p = A[s]->ws + 4 * n;
    q.q = A[s]->ws + 8 * n;
    q.tol = tol[s];
    q.maxit = maxit[s];
    q.arith = arith[s];
    q.V = A[s]->plan.V;
    q.norm_every = A[s]->norm_every;
    q.norm_mask = A[s]->norm_mask;
    q.w = (A[s]->prec == MWCG_PREC_JACOBI) ? A[s]->w : nullptr;
    double mac, add;
    op_costs(arith[s], mac, add);
    cost.push_back((double)A[s]->nnz * mac + (double)n * 10.0 * add);
    idx.push_back(s);
    hs.push_back(q);
  }
  if (hs.empty()) return MWCG_OK;
  // Largest estimated work first (longest-processing-time order for the queue).
  std::vector<int> order(hs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<mwb::Sys> qs(hs.size());
  for (size_t i = 0; i < order.size(); ++i) qs[i] = hs[order[i]];
  cudaError_t e = mwb_host::launch(qs.data(), (int)qs.size(), S(stream), mwb_host::cluster_size(), nullptr);
  if (e != cudaSuccess) return fail(MWCG_ERR_CUDA, "batched launch: %s", cudaGetErrorString(e));
  for (size_t i = 0; i < order.size(); ++i) {
    const int s = idx[order[i]];
    if (iters_out) iters_out[s] = qs[i].iters;
    if (relres_out) relres_out[s] = qs[i].relres;
    if (status_out) status_out[s] = qs[i].status;
  }
  return MWCG_OK;
}

}  // extern "C"
