// Pipe-throughput probes used for the roofline denominators (mwcg_probe_peak).
//
// On GB300 the multi-word kernels are bound by the FP64 pipe, so the
// roofline is taken against the FP64 operation rate.  These kernels run eight
// independent dependency chains per thread on every SM and report operations
// per second (FMA counted as one operation).
#include <cuda_runtime.h>

#include <cstdio>

#include "mwcg.h"

namespace mwcg_detail {
int set_error(int code, const char* msg);
}

namespace {

__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int iters, double s) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = __fma_rn(a0, s, s); a1 = __fma_rn(a1, s, s); a2 = __fma_rn(a2, s, s); a3 = __fma_rn(a3, s, s);
    a4 = __fma_rn(a4, s, s); a5 = __fma_rn(a5, s, s); a6 = __fma_rn(a6, s, s); a7 = __fma_rn(a7, s, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void __launch_bounds__(256) k_probe_dadd(double* out, int iters, double s) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = __dadd_rn(a0, s); a1 = __dadd_rn(a1, s); a2 = __dadd_rn(a2, s); a3 = __dadd_rn(a3, s);
    a4 = __dadd_rn(a4, s); a5 = __dadd_rn(a5, s); a6 = __dadd_rn(a6, s); a7 = __dadd_rn(a7, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__constant__ double c_probe_one = 1.0;
// fl(a + b) issued as an FMA whose multiplier (1.0) comes from constant memory,
// so that the compiler cannot turn it back into an addition.
__device__ __forceinline__ double fma_one(double a, double b) { return __fma_rn(a, c_probe_one, b); }

__global__ void __launch_bounds__(256) k_probe_add_as_fma(double* out, int iters, double s) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma_one(a0, s); a1 = fma_one(a1, s); a2 = fma_one(a2, s); a3 = fma_one(a3, s);
    a4 = fma_one(a4, s); a5 = fma_one(a5, s); a6 = fma_one(a6, s); a7 = fma_one(a7, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void __launch_bounds__(256) k_probe_dmul(double* out, int iters, double s) {
  double a0 = threadIdx.x * 1e-3 + 1, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = __dmul_rn(a0, s); a1 = __dmul_rn(a1, s); a2 = __dmul_rn(a2, s); a3 = __dmul_rn(a3, s);
    a4 = __dmul_rn(a4, s); a5 = __dmul_rn(a5, s); a6 = __dmul_rn(a6, s); a7 = __dmul_rn(a7, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void __launch_bounds__(256) k_probe_int(unsigned* out, int iters, unsigned s) {
  unsigned a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
           a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = (a0 ^ s) + a1; a1 = (a1 ^ s) + a2; a2 = (a2 ^ s) + a3; a3 = (a3 ^ s) + a4;
    a4 = (a4 ^ s) + a5; a5 = (a5 ^ s) + a6; a6 = (a6 ^ s) + a7; a7 = (a7 ^ s) + a0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

}  // namespace

extern "C" int mwcg_probe_peak(int kind, void* scratch, int64_t scratch_bytes, void* stream, double* ops_per_s) {
  if (kind < 0 || kind > 4 || !ops_per_s || !scratch) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_probe_peak: bad argument");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  if (scratch_bytes < (int64_t)blocks * threads * 8) return mwcg_detail::set_error(MWCG_ERR_ARG, "mwcg_probe_peak: scratch too small");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int iters = (kind == 2) ? 100000 : 2000;
  const double ops_per_thread = 8.0 * iters * (kind == 2 ? 2.0 : 1.0);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    if (kind == 0) k_probe_dfma<<<blocks, threads, 0, s>>>((double*)scratch, iters, 0.999);
    else if (kind == 1) k_probe_dadd<<<blocks, threads, 0, s>>>((double*)scratch, iters, 1e-9);
    else if (kind == 2) k_probe_int<<<blocks, threads, 0, s>>>((unsigned*)scratch, iters, 12345u);
    else if (kind == 3) k_probe_add_as_fma<<<blocks, threads, 0, s>>>((double*)scratch, iters, 1e-9);
    else k_probe_dmul<<<blocks, threads, 0, s>>>((double*)scratch, iters, 0.9999999);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double rate = ops_per_thread * blocks * threads / (ms * 1e-3);
    if (rate > best) best = rate;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    char buf[200];
    snprintf(buf, sizeof buf, "mwcg_probe_peak: %s", cudaGetErrorString(err));
    return mwcg_detail::set_error(MWCG_ERR_CUDA, buf);
  }
  *ops_per_s = best;
  return MWCG_OK;
}
