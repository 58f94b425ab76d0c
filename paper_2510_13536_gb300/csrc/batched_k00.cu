// Persistent batched kernel for word group 0 (FP64, DW, QDW, QDW_NN), unpreconditioned systems.
#include <cuda_runtime.h>

#include "batched.cuh"

namespace mwb {

template <>
__device__ __forceinline__ void solve_any<false, 0>(const ClusterCtx& cc, Slots* slots, Sys& S) {
  switch (S.arith) {
    case 0: solve_cluster<mw::FP64, false>(cc, slots, S); break;
    case 1: solve_cluster<mw::DW, false>(cc, slots, S); break;
    case 2: solve_cluster<mw::QDW, false>(cc, slots, S); break;
    default: solve_cluster<mw::QDW_NN, false>(cc, slots, S); break;
  }
}

cudaError_t run_group_00(Sys* dsys, int n, unsigned* queue, cudaStream_t s, int cluster, size_t pad,
                          int* nclusters, int max_clusters) {
  return run_group<false, 0>(dsys, n, queue, s, cluster, pad, nclusters, max_clusters);
}

// The kernel whose occupancy decides the small-system cluster size.
const void* kernel_00() { return (const void*)&k_batched<false, 0>; }

}  // namespace mwb
