// maze_wait_probe: one of the bounded device-side waits (grid barrier, grid
// reductions) driven to its limit on purpose, so that the give-up path -
// record MAZE_ERR_TIMEOUT, return from every block - can be observed on the
// GPU without a fault: the wait is for a round that no block completes.
//
// maze_convert_probe: the integer-pipe FP32/FP64 conversions the hot kernels
// use, computed beside the conversion instructions for a checker;
// maze_exp_probe: the pair forces' table-driven exponential beside exp();
// maze_df_probe: the double-float exponential and Tosi-Fumi pair of the FP64
// boxes' pair kernel, and the FP64 pair beside them.
#include <string>
#include <vector>

#include "ion_body.cuh"

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

// The integer-pipe conversions of maze_internal.cuh beside the conversion
// instructions, element by element.
__global__ void k_convert_probe(const double* in, int n, float* f_own, float* f_hw, double* d_own, double* d_hw,
                                long long* fl_own, long long* fl_hw, double* q_own, double* q_hw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = in[i];
  f_own[i] = dbl_to_flt(v);
  const float f = __double2float_rn(v);
  f_hw[i] = f;
  d_own[i] = flt_to_dbl(f);
  d_hw[i] = (double)f;
  const bool small = fabs(v) < 4.0e18;
  fl_own[i] = small ? floor_ll(v) : 0;
  fl_hw[i] = small ? (long long)floor(v) : 0;
  const long long k = small ? (long long)(v * 1048576.0) : 0;   // v 2^20 as an integer
  q_own[i] = fix_to_dbl(k, 1075 - 20);
  q_hw[i] = (double)k * (1.0 / 1048576.0);
}

// exp_tab beside exp().
__global__ void k_exp_probe(const double* in, int n, const double* tab, double* own, double* ref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  own[i] = exp_tab(in[i], tab);
  ref[i] = exp(in[i]);
}

// df_exp, tf_pair_df or tf_pair on host doubles split into (hi, lo) floats.
__global__ void k_df_probe(ForceArgs a, int what, const double* in, const int* kind, int n, double* o0, double* o1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = in[i];
  const float xh = dbl_to_flt(x);
  const dfl xd = {xh, dbl_to_flt(x - flt_to_dbl(xh))};
  if (what == 0) {
    const dfl e = df_exp(xd, a.exp2tab_f);
    o0[i] = flt_to_dbl(e.h) + flt_to_dbl(e.l);
  } else if (what == 1) {
    dfl fr, V;
    tf_pair_df(a, kind[i], xd, fr, V);
    o0[i] = flt_to_dbl(fr.h) + flt_to_dbl(fr.l);
    o1[i] = flt_to_dbl(V.h) + flt_to_dbl(V.l);
  } else {
    double fr, V;
    tf_pair(a, kind[i], x, fr, V);
    o0[i] = fr;
    o1[i] = V;
  }
}

}  // namespace

}  // namespace maze

extern "C" maze_status maze_exp_probe(const double* in, int32_t n, double* own, double* ref) {
  using namespace maze;
  if (n < 0 || (n > 0 && (!in || !own || !ref))) {
    set_last_error("maze_exp_probe: n must be >= 0 and every array non-NULL");
    return MAZE_ERR_INVALID;
  }
  if (n == 0) return MAZE_OK;
  const size_t N = (size_t)n;
  double tab[64];
  exp2_table(tab);
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, (3 * N + 64) * 8);
  if (e == cudaSuccess) e = cudaMemcpy(buf, in, N * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(buf + 3 * N, tab, 64 * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_exp_probe<<<(n + 255) / 256, 256>>>(buf, n, buf + 3 * N, buf + N, buf + 2 * N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(own, buf + N, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, buf + 2 * N, N * 8, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_last_error((std::string("maze_exp_probe: ") + cudaGetErrorString(e)).c_str());
    return MAZE_ERR_CUDA;
  }
  return MAZE_OK;
}

extern "C" maze_status maze_convert_probe(const double* in, int32_t n, float* f_own, float* f_hw, double* d_own,
                                          double* d_hw, int64_t* floor_own, int64_t* floor_hw, double* fix_own,
                                          double* fix_hw) {
  using namespace maze;
  if (n < 0 || (n > 0 && (!in || !f_own || !f_hw || !d_own || !d_hw || !floor_own || !floor_hw || !fix_own ||
                          !fix_hw))) {
    set_last_error("maze_convert_probe: n must be >= 0 and every array non-NULL");
    return MAZE_ERR_INVALID;
  }
  if (n == 0) return MAZE_OK;
  char* buf = nullptr;
  const size_t N = (size_t)n;
  const size_t bytes = N * (8 + 4 + 4 + 8 + 8 + 8 + 8 + 8 + 8);
  cudaError_t e = cudaMalloc(&buf, bytes);
  double* d_in = reinterpret_cast<double*>(buf);
  double* dd_own = d_in + N;
  double* dd_hw = dd_own + N;
  double* dq_own = dd_hw + N;
  double* dq_hw = dq_own + N;
  long long* dfl_own = reinterpret_cast<long long*>(dq_hw + N);
  long long* dfl_hw = dfl_own + N;
  float* df_own = reinterpret_cast<float*>(dfl_hw + N);
  float* df_hw = df_own + N;
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, N * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_convert_probe<<<(n + 255) / 256, 256>>>(d_in, n, df_own, df_hw, dd_own, dd_hw, dfl_own, dfl_hw, dq_own, dq_hw);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(f_own, df_own, N * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(f_hw, df_hw, N * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(d_own, dd_own, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(d_hw, dd_hw, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(floor_own, dfl_own, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(floor_hw, dfl_hw, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(fix_own, dq_own, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(fix_hw, dq_hw, N * 8, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_last_error((std::string("maze_convert_probe: ") + cudaGetErrorString(e)).c_str());
    return MAZE_ERR_CUDA;
  }
  return MAZE_OK;
}

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

extern "C" maze_status maze_df_probe(const maze_config* cfg, int32_t what, const double* in, const int32_t* kind,
                                     int32_t n, double* out0, double* out1) {
  using namespace maze;
  if (what < 0 || what > 2 || n < 0 || (n > 0 && (!in || !out0 || (what > 0 && (!cfg || !kind || !out1))))) {
    set_last_error("maze_df_probe: what must be 0, 1 or 2, n >= 0, and the arrays (and cfg for a pair) non-NULL");
    return MAZE_ERR_INVALID;
  }
  if (what > 0)
    for (int32_t i = 0; i < n; ++i)
      if (kind[i] < 0 || kind[i] > 2) {
        set_last_error("maze_df_probe: kind must be 0, 1 or 2");
        return MAZE_ERR_INVALID;
      }
  if (n == 0) return MAZE_OK;
  ForceArgs a = {};
  if (what > 0) fill_pair_consts(*cfg, a);
  std::vector<double> e2(64);
  exp2_table(e2.data());
  std::vector<float2> tab(64);
  for (int j = 0; j < 64; ++j) tab[j] = make_float2((float)e2[j], (float)(e2[j] - (double)(float)e2[j]));
  const size_t N = (size_t)n;
  char* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 64 * 8 + 64 * sizeof(float2) + N * (8 + 4 + 8 + 8));
  double* d_tab = reinterpret_cast<double*>(buf);
  float2* d_tabf = reinterpret_cast<float2*>(d_tab + 64);
  double* d_in = reinterpret_cast<double*>(d_tabf + 64);
  double* d_o0 = d_in + N;
  double* d_o1 = d_o0 + N;
  int* d_kind = reinterpret_cast<int*>(d_o1 + N);
  if (e == cudaSuccess) e = cudaMemcpy(d_tab, e2.data(), 64 * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_tabf, tab.data(), 64 * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, N * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d_kind, 0, N * 4);
  if (e == cudaSuccess && what > 0) e = cudaMemcpy(d_kind, kind, N * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    a.exp2tab = d_tab;
    a.exp2tab_f = d_tabf;
    k_df_probe<<<(n + 255) / 256, 256>>>(a, what, d_in, d_kind, n, d_o0, d_o1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out0, d_o0, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && what > 0) e = cudaMemcpy(out1, d_o1, N * 8, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_last_error((std::string("maze_df_probe: ") + cudaGetErrorString(e)).c_str());
    return MAZE_ERR_CUDA;
  }
  return MAZE_OK;
}
