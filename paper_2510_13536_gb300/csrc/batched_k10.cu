// Persistent batched kernel for word group 0 (FP64, DW, QDW, QDW_NN), Jacobi-preconditioned systems.
#include <cuda_runtime.h>

#include "batched.cuh"

namespace mwb {

template <>
__device__ __forceinline__ void solve_any<true, 0>(const ClusterCtx& cc, Slots* slots, Sys& S) {
  switch (S.arith) {
    case 0: solve_cluster<mw::FP64, true>(cc, slots, S); break;
    case 1: solve_cluster<mw::DW, true>(cc, slots, S); break;
    case 2: solve_cluster<mw::QDW, true>(cc, slots, S); break;
    default: solve_cluster<mw::QDW_NN, true>(cc, slots, S); break;
  }
}

cudaError_t run_group_10(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters, int max_clusters) {
  return run_group<true, 0>(dsys, n, queue, s, cluster, pad, nclusters, max_clusters);
}

}  // namespace mwb
