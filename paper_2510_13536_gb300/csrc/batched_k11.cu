// Persistent batched kernel for word group 1 (TW, QTW, QTW_NN), Jacobi-preconditioned systems.
#include <cuda_runtime.h>

#include "batched.cuh"

namespace mwb {

template <>
__device__ __forceinline__ void solve_any<true, 1>(const ClusterCtx& cc, Slots* slots, Sys& S) {
  switch (S.arith) {
    case 3: solve_cluster<mw::TW, true>(cc, slots, S); break;
    case 4: solve_cluster<mw::QTW, true>(cc, slots, S); break;
    default: solve_cluster<mw::QTW_NN, true>(cc, slots, S); break;
  }
}

cudaError_t run_group_11(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters, int max_clusters) {
  return run_group<true, 1>(dsys, n, queue, s, cluster, pad, nclusters, max_clusters);
}

}  // namespace mwb
