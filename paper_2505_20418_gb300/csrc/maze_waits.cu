// maze_wait_probe: one of the bounded device-side waits (grid barrier, grid
// reductions) driven to its limit on purpose, so that the give-up path -
// record MAZE_ERR_TIMEOUT, return from every block - can be observed on the
// GPU without a fault: the wait is for a round that no block completes.
#include <string>

#include "maze_internal.cuh"

namespace maze {

namespace {

constexpr int kProbeBlocks = 4;
constexpr int kProbeThreads = 128;

__global__ void __launch_bounds__(kProbeThreads) k_wait_probe(int which, unsigned* bar, LLRec* recs, maze_stats* rec) {
  if (which == 0) {
    // every block adds one arrival, so the counter stops at gridDim.x; this
    // block waits for the second round (2 gridDim.x arrivals)
    unsigned epoch = 1;
    grid_barrier(bar, epoch, rec);
  } else {
    // the last block publishes its record under round 3, the others under
    // round 1 (same record buffer): no block ever sees every record of its round
    const unsigned e = blockIdx.x == gridDim.x - 1 ? 3u : 1u;
    if (which == 1) {
      const double v[1] = {1.0};
      const bool is_max[1] = {false};
      double out[1];
      grid_reduce<1>(v, is_max, recs, e, rec, out);
    } else {
      unsigned long long out = 0;
      grid_reduce_u64(1ull, recs, e, rec, out);
    }
  }
}

}  // namespace

}  // namespace maze

extern "C" maze_status maze_wait_probe(int32_t which, void* cuda_stream, int32_t* status_out) {
  using namespace maze;
  if (which < 0 || which > 2 || !status_out) {
    set_last_error("maze_wait_probe: which must be 0, 1 or 2 and status_out non-NULL");
    return MAZE_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* bar = nullptr;
  LLRec* recs = nullptr;
  maze_stats* rec = nullptr;
  const size_t rec_bytes = 2 * (size_t)kProbeBlocks * 4 * sizeof(LLRec);
  cudaError_t e = cudaMalloc(&bar, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&recs, rec_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&rec, sizeof(maze_stats));
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(recs, 0, rec_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, sizeof(maze_stats), s);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kProbeBlocks);
    cfg.blockDim = dim3(kProbeThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_wait_probe, (int)which, bar, recs, rec);
  }
  maze_stats host = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, rec, sizeof(maze_stats), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bar);
  cudaFree(recs);
  cudaFree(rec);
  if (e != cudaSuccess) {
    set_last_error((std::string("maze_wait_probe: ") + cudaGetErrorString(e)).c_str());
    return MAZE_ERR_CUDA;
  }
  *status_out = host.status;
  return MAZE_OK;
}
