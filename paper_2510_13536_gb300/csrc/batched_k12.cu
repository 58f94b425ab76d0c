// Persistent batched kernel for word group 2 (QW, QQW, QQW_NN), Jacobi-preconditioned systems.
#include <cuda_runtime.h>

#include "mw_device4.cuh"
#include "batched.cuh"

namespace mwb {

template <>
__device__ __forceinline__ void solve_any<true, 2>(const ClusterCtx& cc, Slots* slots, Sys& S) {
  switch (S.arith) {
    case 7: solve_cluster<mw::QW, true>(cc, slots, S); break;
    case 8: solve_cluster<mw::QQW, true>(cc, slots, S); break;
    default: solve_cluster<mw::QQW_NN, true>(cc, slots, S); break;
  }
}

cudaError_t run_group_12(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters, int max_clusters) {
  return run_group<true, 2>(dsys, n, queue, s, cluster, pad, nclusters, max_clusters);
}

}  // namespace mwb
