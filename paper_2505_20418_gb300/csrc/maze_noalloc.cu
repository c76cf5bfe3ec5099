// Allocation-free variant of the constraint solve (M y = sigma_p by CG).
//
// Some callers cannot call cudaMalloc: a host framework that owns all device
// memory through its own pool (a raw cudaMalloc outside the pool can fail
// while the pool holds the memory, or fragment it), a latency-critical loop in
// which cudaMalloc's implicit device synchronisation would stall the pipeline,
// or a process that runs under a fixed, audited device-memory budget. This
// entry point serves them: the caller passes sigma_p and y in its own device
// memory and the solver's work vectors live in one file-scope __device__
// array, sized for grids up to kNoAllocMaxN^3, that every GPU loading the
// library holds until process exit. The call allocates nothing.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "maze_internal.cuh"

namespace maze {

namespace {

constexpr int kNoAllocMaxN = 64;
constexpr size_t kNoAllocMaxPts = (size_t)kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN;
constexpr int kNoAllocMaxBlocks = 2048;
// layout in doubles: r, p, Mp [kNoAllocMaxPts each] | partials [2][kNoAllocMaxBlocks][4]
// | status block (a maze_stats record and the barrier counter)
constexpr size_t kOffR = 0;
constexpr size_t kOffP = kNoAllocMaxPts;
constexpr size_t kOffMp = 2 * kNoAllocMaxPts;
constexpr size_t kOffPart = 3 * kNoAllocMaxPts;
constexpr size_t kOffStat = kOffPart + 2 * (size_t)kNoAllocMaxBlocks * 4;
constexpr size_t kStatDoubles = 32;   // maze_stats (104 B) + barrier counter, padded
constexpr size_t kScratchDoubles = kOffStat + kStatDoubles;
static_assert(sizeof(maze_stats) + sizeof(unsigned) <= kStatDoubles * sizeof(double), "status block");

// ~6.4 MB per device, shared by every call of maze_solve_shake_noalloc.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kNoAllocThreads = 256;

__device__ __forceinline__ void na_partial(const double* v, const bool* is_max, int K, double* part) {
  __shared__ double s[kNoAllocThreads / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < K; ++k) {
    const double w = is_max[k] ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0) s[warp][k] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) {
      double acc = s[0][k];
      for (int u = 1; u < kNoAllocThreads / 32; ++u) acc = is_max[k] ? fmax(acc, s[u][k]) : acc + s[u][k];
      part[blockIdx.x * 4 + k] = acc;
    }
  }
}

__device__ __forceinline__ void na_combine(const double* part, const bool* is_max, int K, double* out) {
  __shared__ double s_out[4];
  if (threadIdx.x < 32) {
    for (int k = 0; k < K; ++k) {
      double acc = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
        const double v = __ldcg(&part[b * 4 + k]);
        acc = is_max[k] ? fmax(acc, v) : acc + v;
      }
      acc = is_max[k] ? warp_max(acc) : warp_sum(acc);
      if (threadIdx.x == 0) s_out[k] = acc;
    }
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) out[k] = s_out[k];
  __syncthreads();
}

// CG on M y = sigma from the caller's y (same recurrences and stopping rule as
// the solve inside maze_solve), then y -= mean(y). Work vectors come from the
// static scratch array, named directly in device code.
__global__ void __launch_bounds__(kNoAllocThreads)
k_shake_cg_noalloc(int N, const double* __restrict__ sigma, double* __restrict__ y, double tol, int max_iter) {
  double* r = g_noalloc_scratch + kOffR;
  double* p = g_noalloc_scratch + kOffP;
  double* Mp = g_noalloc_scratch + kOffMp;
  double* part = g_noalloc_scratch + kOffPart;
  maze_stats* rec = reinterpret_cast<maze_stats*>(g_noalloc_scratch + kOffStat);
  unsigned* bar = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(rec) + sizeof(maze_stats));
  const int n = N * N * N;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const size_t pbuf = (size_t)gridDim.x * 4;
  unsigned epoch = 0;
  int red = 0;
  const bool m3[3] = {false, true, false};
  const bool m1[1] = {false};
  const bool m2[2] = {false, true};
  double tot[3];

  auto true_residual = [&](bool store) {
    double rr = 0, ys = 0;
    unsigned long long rmax = 0;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N);
      const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
      const double rv = sigma[m] - My;
      if (store) r[m] = rv;
      rr += rv * rv;
      rmax = max(rmax, abs_bits(rv));
      ys += y[m];
    }
    const double v[3] = {rr, absmax_value(rmax), ys};
    na_partial(v, m3, 3, part + (red & 1) * pbuf);
  };

  true_residual(true);
  if (!grid_barrier(bar, epoch, rec)) return;
  na_combine(part + (red & 1) * pbuf, m3, 3, tot);
  ++red;
  double rho = tot[0], res = tot[1], ysum = tot[2];
  int it = 0;
  bool conv = res < tol, fresh = true, have_ysum = true;
  bool finite = isfinite(res) && isfinite(rho) && isfinite(ysum);
  double beta = 0.0;
  while (!conv && finite && it < max_iter) {
    have_ysum = false;
    for (int m = tid; m < n; m += stride) p[m] = fresh ? r[m] : r[m] + beta * p[m];
    if (!grid_barrier(bar, epoch, rec)) return;
    {
      double pmp = 0;
      for (int m = tid; m < n; m += stride) {
        const Nbr b = neighbours(m, N);
        const double pm = p[m];
        const double mp = (p[b.xm] + p[b.xp]) + (p[b.ym] + p[b.yp]) + (p[b.zm] + p[b.zp]) - 6.0 * pm;
        Mp[m] = mp;
        pmp += pm * mp;
      }
      const double v[1] = {pmp};
      na_partial(v, m1, 1, part + (red & 1) * pbuf);
    }
    if (!grid_barrier(bar, epoch, rec)) return;
    double t1[1];
    na_combine(part + (red & 1) * pbuf, m1, 1, t1);
    ++red;
    if (!isfinite(t1[0])) {
      finite = false;
      break;
    }
    const double alpha = rho / t1[0];
    {
      double rr = 0;
      unsigned long long rmax = 0;
      for (int m = tid; m < n; m += stride) {
        y[m] += alpha * p[m];
        const double rv = r[m] - alpha * Mp[m];
        r[m] = rv;
        rr += rv * rv;
        rmax = max(rmax, abs_bits(rv));
      }
      const double v[2] = {rr, absmax_value(rmax)};
      na_partial(v, m2, 2, part + (red & 1) * pbuf);
    }
    if (!grid_barrier(bar, epoch, rec)) return;
    double t2[2];
    na_combine(part + (red & 1) * pbuf, m2, 2, t2);
    ++red;
    ++it;
    res = t2[1];
    finite = isfinite(res) && isfinite(t2[0]);
    if (!finite) break;
    if (res < tol) {
      true_residual(true);
      if (!grid_barrier(bar, epoch, rec)) return;
      na_combine(part + (red & 1) * pbuf, m3, 3, tot);
      ++red;
      res = tot[1];
      ysum = tot[2];
      have_ysum = true;
      if (!isfinite(res) || !isfinite(ysum) || !isfinite(tot[0])) {
        finite = false;
        break;
      }
      if (res < tol) {
        conv = true;
        break;
      }
      rho = tot[0];
      fresh = true;
      continue;
    }
    beta = t2[0] / rho;
    rho = t2[0];
    fresh = false;
  }
  if (!have_ysum) {
    true_residual(false);
    if (!grid_barrier(bar, epoch, rec)) return;
    na_combine(part + (red & 1) * pbuf, m3, 3, tot);
    ++red;
    res = tot[1];
    ysum = tot[2];
  }
  const double ybar = ysum / (double)n;
  for (int m = tid; m < n; m += stride) y[m] -= ybar;
  if (tid == 0) {
    rec->iters = it;
    rec->resid = res;
    if (rec->status == MAZE_OK) {
      if (!finite || !isfinite(res) || !isfinite(ysum)) rec->status = MAZE_ERR_NONFINITE;
      else if (!(res < tol)) rec->status = MAZE_ERR_NOT_CONVERGED;
    }
  }
}

// Per-device set-up: the device address of the scratch array (host code sees
// only a host-side stand-in for the symbol) and the cooperative grid size.
struct DevSetup {
  bool done = false;
  double* scratch = nullptr;
  int blocks = 0;
};
constexpr int kMaxDevices = 64;
DevSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

maze_status na_fail(maze_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

}  // namespace

}  // namespace maze

extern "C" maze_status maze_solve_shake_noalloc(int32_t grid_N, const double* sigma_p, double* y, double tol,
                                               int32_t max_iter, void* cuda_stream, int32_t* iters,
                                               double* resid_inf) {
  using namespace maze;
  if (!sigma_p || !y) return na_fail(MAZE_ERR_INVALID, "sigma_p and y must be device pointers");
  if ((const void*)sigma_p == (const void*)y)
    return na_fail(MAZE_ERR_INVALID, "sigma_p and y must be distinct buffers (y is overwritten while sigma_p is read)");
  if (grid_N < 8 || grid_N % 2)
    return na_fail(MAZE_ERR_INVALID, "grid_N must be even and >= 8");
  if (grid_N > kNoAllocMaxN)
    return na_fail(MAZE_ERR_INVALID, "maze_solve_shake_noalloc supports grid_N <= " + std::to_string(kNoAllocMaxN) +
                                         " (fixed scratch of 64^3 points); use maze_solve for larger grids");
  if (!(tol > 0) || max_iter < 1) return na_fail(MAZE_ERR_INVALID, "tol must be > 0 and max_iter >= 1");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(MAZE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(MAZE_ERR_CUDA, "device index out of range");
  DevSetup st;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_setup[dev].done) {
      // first call on this device (the device is current): resolve the
      // scratch array's device address and the co-resident grid size
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return na_fail(MAZE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      int sms = 0, per_sm = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shake_cg_noalloc, kNoAllocThreads, 0);
      if (e != cudaSuccess) return na_fail(MAZE_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
      int cap = sms * (per_sm < 1 ? 1 : per_sm);
      g_setup[dev].scratch = static_cast<double*>(ptr);
      g_setup[dev].blocks = cap < kNoAllocMaxBlocks ? cap : kNoAllocMaxBlocks;
      g_setup[dev].done = true;
    }
    st = g_setup[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n = grid_N * grid_N * grid_N;
  int blocks = (n + kNoAllocThreads - 1) / kNoAllocThreads;
  if (blocks > st.blocks) blocks = st.blocks;
  // the status record and barrier counter must start at zero on every call
  e = cudaMemsetAsync(st.scratch + kOffStat, 0, kStatDoubles * sizeof(double), s);
  if (e != cudaSuccess) return na_fail(MAZE_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kNoAllocThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_shake_cg_noalloc, (int)grid_N, sigma_p, y, tol, (int)max_iter);
  if (e != cudaSuccess) return na_fail(MAZE_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  maze_stats rec;
  e = cudaMemcpyAsync(&rec, st.scratch + kOffStat, sizeof(maze_stats), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(MAZE_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
  if (iters) *iters = rec.iters;
  if (resid_inf) *resid_inf = rec.resid;
  if (rec.status == MAZE_ERR_NOT_CONVERGED) return na_fail(MAZE_ERR_NOT_CONVERGED, "constraint solve not converged");
  if (rec.status != MAZE_OK) return na_fail((maze_status)rec.status, "device status " + std::to_string(rec.status));
  return MAZE_OK;
}
