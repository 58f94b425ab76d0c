// Persistent batched kernel for word group 3 (QQF, QF: four FP32 words), unpreconditioned systems.
#include <cuda_runtime.h>

#include "batched_float.cuh"

namespace mwb {

template <>
__device__ __forceinline__ void solve_any<false, 3>(const ClusterCtx& cc, Slots* slots, Sys& S) {
  if (S.arith == 10) solve_cluster_qqf<mw::QQF, false>(cc, slots, S);
  else solve_cluster_qqf<mw::QF, false>(cc, slots, S);
}

cudaError_t run_group_03(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters, int max_clusters) {
  return run_group<false, 3>(dsys, n, queue, s, cluster, pad, nclusters, max_clusters);
}

}  // namespace mwb
