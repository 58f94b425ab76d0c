// Persistent batched kernel for word group 1 (TW, QTW, QTW_NN), unpreconditioned systems.
#include <cuda_runtime.h>

#include "batched.cuh"

namespace mwb {

template <>
__device__ __forceinline__ void solve_any<false, 1>(const ClusterCtx& cc, Slots* slots, Sys& S) {
  switch (S.arith) {
    case 3: solve_cluster<mw::TW, false>(cc, slots, S); break;
    case 4: solve_cluster<mw::QTW, false>(cc, slots, S); break;
    default: solve_cluster<mw::QTW_NN, false>(cc, slots, S); break;
  }
}

cudaError_t run_group_01(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters, int max_clusters) {
  return run_group<false, 1>(dsys, n, queue, s, cluster, pad, nclusters, max_clusters);
}

}  // namespace mwb
