// The persistent batched kernel for Jacobi-preconditioned systems (its own
// translation unit: the kernel instantiates every arithmetic's solver).
#include <cuda_runtime.h>

#include "batched.cuh"

namespace mwb {

cudaError_t run_group_pcg(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters) {
  return run_group<true>(dsys, n, queue, s, cluster, pad, nclusters);
}

}  // namespace mwb
