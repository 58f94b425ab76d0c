// mwcg_dot_noalloc: the multi-word dot product without any device allocation.
//
// mwcg_dot allocates its block partials, its ticket counter and its result
// buffer with cudaMalloc on every call and frees them with cudaFree.  Some
// callers cannot do that: cudaFree synchronises the whole device (stalling
// every other stream of a latency-critical pipeline), and code that runs under
// a fixed device-memory budget or inside a pooled allocator may be forbidden
// to make hidden allocations.  This entry point keeps its scratch in a fixed
// array inside the library instead (the caller still passes the inputs and
// the output), so it never calls cudaMalloc, cudaFree or any allocating
// library routine.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mwcg.h"
#include "cg_kernels.cuh"

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
}  // namespace mwk

namespace mwcg_detail {
int set_error(int code, const char* msg);
}

namespace {

// Capacity: block partials for up to kNoallocMaxG blocks (mwk::PART = 12
// doubles each) followed by one DevState (ticket counter).  About 99 KB, held
// by every GPU that loads the library until the process exits.
constexpr int kNoallocMaxG = MWCG_DOT_NOALLOC_MAX_G;
constexpr size_t kPartDoubles = (size_t)kNoallocMaxG * mwk::PART;
constexpr size_t kStateDoubles = (sizeof(mwk::DevState) + sizeof(double) - 1) / sizeof(double);

__device__ __align__(256) double g_dot_scratch[kPartDoubles + kStateDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_dev[kMaxDevices] = {};    // device address of g_dot_scratch, per device

const mwk::KernelTable& table_of(int arith) {
  static mwk::KernelTable t[12];
  static std::once_flag once;
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
  });
  return t[arith];
}

int err(int code, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "mwcg_dot_noalloc: %s: %s", what, cudaGetErrorString(e));
  return mwcg_detail::set_error(code, buf);
}

// Device address of the scratch array on the current device.  The host-side
// name g_dot_scratch is only a stand-in, never a device address, so it is
// looked up once per device (with that device current) and cached.
int scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(MWCG_ERR_CUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_dot_noalloc: device index too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_dot_scratch);
    if (e != cudaSuccess) return err(MWCG_ERR_CUDA, "cudaGetSymbolAddress", e);
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return MWCG_OK;
}

}  // namespace

extern "C" int mwcg_dot_noalloc(int arith, int64_t n, const double* u, const double* v, int32_t G, void* stream,
                                double* out) {
  mwcg_detail::set_error(MWCG_OK, "");
  if (arith < 0 || arith > 11) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_dot_noalloc: unknown arithmetic");
  if (n < 0) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_dot_noalloc: n < 0");
  if (G < 1 || G > kNoallocMaxG) {
    char buf[160];
    snprintf(buf, sizeof buf, "mwcg_dot_noalloc: G = %d outside 1..%d (capacity of the static scratch array)", G,
             kNoallocMaxG);
    return mwcg_detail::set_error(MWCG_ERR_ARG, buf);
  }
  if (!out) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_dot_noalloc: null out");
  if (n > 0 && (!u || !v)) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_dot_noalloc: null u or v");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const mwk::KernelTable& kt = table_of(arith);
  if (n == 0) {
    const int outw = arith >= MWCG_QQF ? 4 : kt.words;   // FP32 words: one per double
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * outw, s);
    return e == cudaSuccess ? MWCG_OK : err(MWCG_ERR_CUDA, "cudaMemsetAsync", e);
  }
  double* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc != MWCG_OK) return rc;
  mwk::DevState* st = reinterpret_cast<mwk::DevState*>(base + kPartDoubles);
  // The ticket counter must start at zero; the partials are all rewritten.
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(mwk::DevState), s);
  if (e != cudaSuccess) return err(MWCG_ERR_CUDA, "cudaMemsetAsync", e);
  mwk::Work W{};
  W.part = base;
  W.st = st;
  W.V = 1;
  W.G = G;
  void* args[] = {(void*)&u, (void*)&v, (void*)&n, (void*)&W, (void*)&out};
  e = cudaLaunchKernel(kt.dot, dim3(G), dim3(mwk::TPB), args, mwk::red_smem(G, kt.words), s);
  if (e != cudaSuccess) return err(MWCG_ERR_CUDA, "kernel launch", e);
  return MWCG_OK;
}
