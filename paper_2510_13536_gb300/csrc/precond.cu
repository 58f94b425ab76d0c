// Jacobi weights of the preconditioned CG: w_i = fl(1 / a_ii).
//
// One thread per row scans the row for its diagonal entry.  A row without a
// diagonal entry, or with one that is not positive or not finite, leaves the
// preconditioner undefined: w_i is set to 0 and *bad to 1 (the solver then
// returns MWCG_BAD_PRECONDITIONER without iterating).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

__global__ void __launch_bounds__(256) k_jacobi_weights(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                        const double* __restrict__ val, int64_t n,
                                                        double* __restrict__ w, int* __restrict__ bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    bool found = false;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (col[k] == i) {
        d = val[k];
        found = true;
        break;
      }
    }
    if (!found || !(d > 0.0) || !isfinite(d)) {
      w[i] = 0.0;
      *bad = 1;
    } else {
      w[i] = __ddiv_rn(1.0, d);
    }
  }
}

}  // namespace

namespace mwcg_precond {

cudaError_t jacobi_weights(const int64_t* rp, const int32_t* col, const double* val, int64_t n, double* w,
                           int* bad, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks64 = (n + 255) / 256;
  const int blocks = (int)(blocks64 < 4096 ? blocks64 : 4096);
  k_jacobi_weights<<<blocks, 256, 0, s>>>(rp, col, val, n, w, bad);
  return cudaGetLastError();
}

}  // namespace mwcg_precond
