// Persistent batched CG kernel and its launcher (mwcg_solve_batched).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <set>
#include <vector>

#include "batched.cuh"

namespace mwb {

constexpr int kCluster = 8;                 // CTAs per worker cluster (portable maximum)

// Defined in batched_k<PREC><GRP>.cu: run_group<PREC, GRP>, one kernel each.
using RunGroup = cudaError_t (*)(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_00(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_01(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_02(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_10(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_11(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_12(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_03(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
cudaError_t run_group_13(Sys*, int, unsigned*, cudaStream_t, int, size_t, int*, int);
const void* kernel_00();

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
  const void* kern = mwb::kernel_00();
  cudaFree(nullptr);          // the context exists before the attribute calls (see capi.cu)
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mwb::kPadSmem) == cudaSuccess) {
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
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) best = 16;
  }
  cudaGetLastError();
  g_small_cluster[dev] = best;
  return best;
}

// Launch the persistent kernel over `nsys` prepared systems (host array, in
// queue order) with clusters of `cluster` CTAs.  Systems are grouped by
// (preconditioned or not, word group), one kernel instantiation per group,
// every group in queue order.  The groups run concurrently on streams forked
// from `s` and joined back into it: their kernels share no data and never
// wait on one another, so a later group's clusters take SMs as an earlier
// group's clusters finish.  (Splitting the clusters between the groups in
// proportion to their estimated work was measured slower: the estimate cannot
// know the iteration counts.)  A system's result depends only on its own
// plan, not on the grouping.  Returns a cudaError_t; outputs are copied back
// into hsys.
cudaError_t launch(mwb::Sys* hsys, int nsys, cudaStream_t s, int cluster, int* clusters_out) {
  // A single system keeps one CTA per SM (the pad); a batch packs two CTAs of
  // (possibly different) clusters per SM.
  const size_t pad = nsys == 1 ? mwb::kPadSmem : 0;
  constexpr int NG = 8;                      // (preconditioned or not) x four word groups
  static const mwb::RunGroup run[NG] = {mwb::run_group_00, mwb::run_group_01, mwb::run_group_02,
                                        mwb::run_group_03, mwb::run_group_10, mwb::run_group_11,
                                        mwb::run_group_12, mwb::run_group_13};
  std::vector<mwb::Sys> grp[NG];
  std::vector<int> where[NG];
  for (int i = 0; i < nsys; ++i) {
    const int g = (hsys[i].w ? 4 : 0) + mwb::word_group(hsys[i].arith);
    grp[g].push_back(hsys[i]);
    where[g].push_back(i);
  }
  mwb::Sys* dsys = nullptr;
  unsigned* queue = nullptr;
  cudaStream_t gs[NG] = {};
  cudaEvent_t ev[NG + 1] = {};
  cudaError_t e = cudaMalloc(&dsys, sizeof(mwb::Sys) * nsys);
  if (e == cudaSuccess) e = cudaMalloc(&queue, NG * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, NG * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[NG], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[NG], s);                 // fork point
  int nclusters = 0, off = 0, ngroups = 0;
  for (int g = 0; g < NG; ++g) ngroups += grp[g].empty() ? 0 : 1;
  for (int g = 0; g < NG && e == cudaSuccess; ++g) {
    const int n = (int)grp[g].size();
    if (n == 0) continue;
    if (ngroups == 1) {                       // one group (e.g. a single system): the caller's stream
      gs[g] = s;
    } else {
      e = cudaStreamCreateWithFlags(&gs[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(gs[g], ev[NG], 0);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[g], cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dsys + off, grp[g].data(), sizeof(mwb::Sys) * n, cudaMemcpyHostToDevice, gs[g]);
    int nc = 0;
    if (e == cudaSuccess) e = run[g](dsys + off, n, queue + g, gs[g], cluster, pad, &nc, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(grp[g].data(), dsys + off, sizeof(mwb::Sys) * n, cudaMemcpyDeviceToHost, gs[g]);
    if (e == cudaSuccess && gs[g] != s) {
      e = cudaEventRecord(ev[g], gs[g]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[g], 0);       // join
    }
    nclusters = std::max(nclusters, nc);
    off += n;
  }
  const cudaError_t es = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = es;
  for (int g = 0; g <= NG; ++g) {
    if (g < NG && gs[g] && gs[g] != s) cudaStreamDestroy(gs[g]);
    if (ev[g]) cudaEventDestroy(ev[g]);
  }
  if (e == cudaSuccess)
    for (int g = 0; g < NG; ++g)
      for (size_t k = 0; k < grp[g].size(); ++k) hsys[where[g][k]] = grp[g][k];
  cudaFree(dsys);
  cudaFree(queue);
  if (clusters_out) *clusters_out = nclusters;
  return e;
}

}  // namespace mwb_host
