// Mixed-precision constraint solve: the two single-box launch forms of the
// body in mixed_body.cuh (one thread-block cluster for boxes up to 64^3, a
// cooperative grid above).
#include "mixed_body.cuh"

namespace maze {

__global__ void __launch_bounds__(kMixedClusterThreads, 1) k_mixed_cluster(MixedArgs a) {
  extern __shared__ __align__(16) float dsm[];
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;
  ClusterSync s;
  mixed_body(a, s, a.resident ? dsm : nullptr);
}

__global__ void __launch_bounds__(kMixedGridThreads) k_mixed_grid(MixedArgs a) {
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;
  GridSync s;
  s.recs = a.recs;
  s.bar = a.bar;
  s.rec = a.rec;
  mixed_body(a, s, nullptr);
}

size_t resident_bytes_host(const MixedArgs& a, int C) { return resident_bytes(a, C); }

int mixed_cluster_size() {
  // 16 CTAs when the device can co-schedule a 16-CTA cluster of this kernel,
  // else the portable 8
  static int cached = 0;
  if (cached) return cached;
  cudaFuncSetAttribute(k_mixed_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_mixed_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, kResidentSmem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(kMixedClusterThreads);
  cfg.dynamicSmemBytes = kResidentSmem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_mixed_cluster, &cfg) == cudaSuccess && nclusters >= 1)
    cached = 16;
  else
    cached = 8;
  cudaGetLastError();
  return cached;
}

int mixed_grid_blocks(int n_points) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_grid, kMixedGridThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int want = (n_points + kMixedGridThreads - 1) / kMixedGridThreads;
  int cap = sms * per_sm;
  if (cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
  return want < cap ? want : cap;
}

int mixed_grid_regs() {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_mixed_grid) != cudaSuccess) return 64;
  return fa.numRegs;
}

cudaError_t launch_mixed_solve(const MixedArgs& a, int cluster, int blocks, cudaStream_t s, int threads) {
  cudaLaunchConfig_t cfg = {};
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (cluster > 0) {
    cfg.blockDim = dim3(kMixedClusterThreads);
    cfg.gridDim = dim3(cluster);
    cfg.dynamicSmemBytes = a.resident ? resident_bytes(a, cluster) : 0;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mixed_cluster, a);
  }
  cfg.blockDim = dim3(threads > 0 ? threads : kMixedGridThreads);
  cfg.gridDim = dim3(blocks);
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mixed_grid, a);
}

}  // namespace maze
