// Persistent batched CG kernel and its launcher (mwcg_solve_batched).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <set>
#include <vector>

#include "batched.cuh"

namespace mwb {

constexpr int kCluster = 8;                 // CTAs per worker cluster (portable maximum)
constexpr size_t kPadSmem = 120 * 1024;     // dynamic shared memory that keeps one CTA per SM

__global__ void __launch_bounds__(TPB, 1) k_batched(Sys* __restrict__ sys, int nsys, unsigned* queue) {
  __shared__ Slots slots;
  __shared__ int s_next;
  cgx::cluster_group cl = cgx::this_cluster();
  const ClusterCtx cc{cl, (int)cl.block_rank(), (int)cl.num_blocks()};
  for (;;) {
    if (cc.rank == 0 && threadIdx.x == 0) s_next = (int)atomicAdd(queue, 1u);
    cl.sync();
    const int sid = *cl.map_shared_rank(&s_next, 0);
    cl.sync();                               // every CTA has read s_next before it is overwritten
    if (sid >= nsys) break;
    Sys& S = sys[sid];
    switch (S.arith) {
      case 0: solve_cluster<mw::FP64>(cc, &slots, S); break;
      case 1: solve_cluster<mw::DW>(cc, &slots, S); break;
      case 2: solve_cluster<mw::QDW>(cc, &slots, S); break;
      case 3: solve_cluster<mw::TW>(cc, &slots, S); break;
      case 4: solve_cluster<mw::QTW>(cc, &slots, S); break;
      case 5: solve_cluster<mw::QDW_NN>(cc, &slots, S); break;
      default: solve_cluster<mw::QTW_NN>(cc, &slots, S); break;
    }
  }
}

}  // namespace mwb

// Host side, called from capi.cu.
namespace mwb_host {

int cluster_size() { return mwb::kCluster; }

namespace {
int g_small_cluster[64] = {};
}

// Largest cluster size (16, else 8) with which one cluster of one-CTA-per-SM
// blocks can be resident on the current device; used for single small
// systems.  Cached per device.
int small_cluster_size() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return mwb::kCluster;
  if (g_small_cluster[dev]) return g_small_cluster[dev];
  int best = mwb::kCluster;
  if (cudaFuncSetAttribute(mwb::k_batched, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(mwb::k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mwb::kPadSmem) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(mwb::TPB);
    cfg.dynamicSmemBytes = mwb::kPadSmem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, mwb::k_batched, &cfg) == cudaSuccess && n >= 1) best = 16;
  }
  cudaGetLastError();
  g_small_cluster[dev] = best;
  return best;
}

// Launch the persistent kernel over `nsys` prepared systems (host array, in
// queue order) with clusters of `cluster` CTAs.  Returns a cudaError_t;
// outputs are copied back into hsys.
cudaError_t launch(mwb::Sys* hsys, int nsys, cudaStream_t s, int cluster, int* clusters_out) {
  // MWCG_BATCH_PAD=0 drops the shared-memory pad that keeps one CTA per SM
  // (clusters may then share SMs); for tuning runs.
  const char* pad_env = std::getenv("MWCG_BATCH_PAD");
  const size_t pad = (pad_env && pad_env[0] == '0') ? 0 : mwb::kPadSmem;
  mwb::Sys* dsys = nullptr;
  unsigned* queue = nullptr;
  cudaError_t e = cudaMalloc(&dsys, sizeof(mwb::Sys) * nsys);
  if (e == cudaSuccess) e = cudaMalloc(&queue, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dsys, hsys, sizeof(mwb::Sys) * nsys, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mwb::k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mwb::kPadSmem);
  if (e == cudaSuccess && cluster > 8)
    e = cudaFuncSetAttribute(mwb::k_batched, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(mwb::TPB);
  cfg.dynamicSmemBytes = pad;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (e == cudaSuccess) {
    cfg.gridDim = dim3(cluster);
    e = cudaOccupancyMaxActiveClusters(&nclusters, mwb::k_batched, &cfg);
  }
  if (e == cudaSuccess) {
    nclusters = std::max(1, std::min(nclusters, nsys));
    cfg.gridDim = dim3(nclusters * cluster);
    int n = nsys;
    e = cudaLaunchKernelEx(&cfg, mwb::k_batched, dsys, n, queue);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hsys, dsys, sizeof(mwb::Sys) * nsys, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dsys);
  cudaFree(queue);
  if (clusters_out) *clusters_out = nclusters;
  return e;
}

}  // namespace mwb_host
