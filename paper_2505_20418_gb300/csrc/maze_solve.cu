// S4-S6 of the MaZe step in one cooperative persistent kernel:
//   S4  phi_p = 2 phi^k - phi^{k-1},  sigma_p = (h/4pi) M phi_p + q   (Eq. SHAKE)
//   S5  warm-started conjugate gradient on M y = sigma_p               (Eq. SHAKEy, App. B)
//   S6  phi^{k+1} = phi_p - (4pi/h) (y - mean y)                       (Eq. SHAKEPhiFinal)
//
// App. B preconditions CG with J = diag(M) = -6 I. A scalar preconditioner
// cancels out of the CG recurrences (alpha scales by the scalar, the search
// direction by its inverse), so the iterates equal those of plain CG on M,
// which is what runs here; CG needs M definite, and negative-definite M on
// the zero-mean subspace works as well as positive definite.
//
// The stopping test is the paper's residual max_n |(M y - sigma_p)_n|
// (Eq. res_poisson_maze) on the recursive residual, confirmed by one true
// residual; a failed confirmation restarts CG from the true residual.
// Grid-wide synchronisation uses a bounded barrier; every reduction sums the
// block partials in the same fixed order in every block, so all blocks take
// identical decisions and the result is bit-reproducible.
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

namespace {

// Block-level sums of up to 4 values, written as this block's partial.
template <int K>
__device__ __forceinline__ void block_partial(const double (&v)[K], const bool (&is_max)[K], double* part) {
  __shared__ double s[kSolveThreads / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = is_max[k] ? warp_max(v[k]) : warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) s[warp][k] = w[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double acc = s[0][k];
      for (int u = 1; u < kSolveThreads / 32; ++u) acc = is_max[k] ? fmax(acc, s[u][k]) : acc + s[u][k];
      part[blockIdx.x * 4 + k] = acc;
    }
  }
}

// After the barrier: every block combines all partials in the same order.
template <int K>
__device__ __forceinline__ void grid_combine(const double* part, const bool (&is_max)[K], double (&out)[K]) {
  __shared__ double s_out[4];
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double acc = is_max[k] ? 0.0 : 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
        const double v = __ldcg(&part[b * 4 + k]);
        acc = is_max[k] ? fmax(acc, v) : acc + v;
      }
      acc = is_max[k] ? warp_max(acc) : warp_sum(acc);
      if (threadIdx.x == 0) s_out[k] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = s_out[k];
  __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(kSolveThreads) k_cg_solve(SolveArgs a) {
  unsigned epoch = 0;   // barrier count (thread 0)
  int red = 0;          // reduction count: selects the partial buffer
  const int n = a.n, N = a.N;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const size_t pbuf = (size_t)gridDim.x * 4;
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;

  const bool sum3[3] = {false, true, false};     // (r.r, max|r|, sum y)
  const bool sum1[1] = {false};
  const bool sum2[2] = {false, true};

  // ---- S4 and the initial residual r0 = sigma_p - M y0
  {
    double rr = 0, rmax = 0, ys = 0;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N);
      const double q = (double)(long long)a.qfix[m] * kQInv;
      a.qfix[m] = 0ull;
      if (a.q_out) a.q_out[m] = q;
      double php = 0.0, Mphp = 0.0;
      if (!a.zero_phi) {
        const double* pk = a.phi_k;
        const double* pm = a.phi_km1;
        php = 2.0 * pk[m] - pm[m];
        const double nk = (pk[b.xm] + pk[b.xp]) + (pk[b.ym] + pk[b.yp]) + (pk[b.zm] + pk[b.zp]);
        const double nm = (pm[b.xm] + pm[b.xp]) + (pm[b.ym] + pm[b.yp]) + (pm[b.zm] + pm[b.zp]);
        Mphp = 2.0 * nk - nm - 6.0 * php;
      }
      const double sg = a.c_sig * Mphp + q;
      a.phi_out[m] = php;
      a.sigma[m] = sg;
      const double* y = a.y;
      const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
      const double r = sg - My;
      a.r[m] = r;
      rr += r * r;
      rmax = fmax(rmax, fabs(r));
      ys += y[m];
    }
    const double v[3] = {rr, rmax, ys};
    block_partial<3>(v, sum3, a.part + (red & 1) * pbuf);
  }
  if (!grid_barrier(a.bar, epoch, a.rec)) return;
  double tot[3];
  grid_combine<3>(a.part + (red & 1) * pbuf, sum3, tot);
  ++red;
  double rho = tot[0], res = tot[1], ysum = tot[2];
  int it = 0;
  bool conv = res < a.tol;
  bool fresh = true;
  bool have_ysum = true;
  double beta = 0.0;
  bool finite = isfinite(res);

  while (!conv && finite && it < a.max_iter) {
    have_ysum = false;
    // phase A: p = r + beta p
    for (int m = tid; m < n; m += stride) a.p[m] = fresh ? a.r[m] : a.r[m] + beta * a.p[m];
    if (!grid_barrier(a.bar, epoch, a.rec)) return;
    // phase B: Mp and p.Mp
    {
      double pmp = 0;
      const double* p = a.p;
      for (int m = tid; m < n; m += stride) {
        const Nbr b = neighbours(m, N);
        const double pm = p[m];
        const double mp = (p[b.xm] + p[b.xp]) + (p[b.ym] + p[b.yp]) + (p[b.zm] + p[b.zp]) - 6.0 * pm;
        a.Mp[m] = mp;
        pmp += pm * mp;
      }
      const double v[1] = {pmp};
      block_partial<1>(v, sum1, a.part + (red & 1) * pbuf);
    }
    if (!grid_barrier(a.bar, epoch, a.rec)) return;
    double t1[1];
    grid_combine<1>(a.part + (red & 1) * pbuf, sum1, t1);
    ++red;
    const double alpha = rho / t1[0];
    // phase C: y += alpha p, r -= alpha Mp; r.r and max|r|
    {
      double rr = 0, rmax = 0;
      for (int m = tid; m < n; m += stride) {
        a.y[m] += alpha * a.p[m];
        const double r = a.r[m] - alpha * a.Mp[m];
        a.r[m] = r;
        rr += r * r;
        rmax = fmax(rmax, fabs(r));
      }
      const double v[2] = {rr, rmax};
      block_partial<2>(v, sum2, a.part + (red & 1) * pbuf);
    }
    if (!grid_barrier(a.bar, epoch, a.rec)) return;
    double t2[2];
    grid_combine<2>(a.part + (red & 1) * pbuf, sum2, t2);
    ++red;
    ++it;
    res = t2[1];
    finite = isfinite(res) && isfinite(t2[0]);
    if (!finite) break;
    if (res < a.tol) {
      // confirm with the true residual sigma_p - M y (also gives sum y)
      double rr = 0, rmax = 0, ys = 0;
      const double* y = a.y;
      for (int m = tid; m < n; m += stride) {
        const Nbr b = neighbours(m, N);
        const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
        const double r = a.sigma[m] - My;
        a.r[m] = r;
        rr += r * r;
        rmax = fmax(rmax, fabs(r));
        ys += y[m];
      }
      const double v[3] = {rr, rmax, ys};
      block_partial<3>(v, sum3, a.part + (red & 1) * pbuf);
      if (!grid_barrier(a.bar, epoch, a.rec)) return;
      grid_combine<3>(a.part + (red & 1) * pbuf, sum3, tot);
      ++red;
      res = tot[1];
      ysum = tot[2];
      have_ysum = true;
      if (res < a.tol) {
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
    // stopped at max_iter or on a non-finite value: true residual and sum y
    double rr = 0, rmax = 0, ys = 0;
    const double* y = a.y;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N);
      const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
      const double r = a.sigma[m] - My;
      rr += r * r;
      rmax = fmax(rmax, fabs(r));
      ys += y[m];
    }
    const double v[3] = {rr, rmax, ys};
    block_partial<3>(v, sum3, a.part + (red & 1) * pbuf);
    if (!grid_barrier(a.bar, epoch, a.rec)) return;
    grid_combine<3>(a.part + (red & 1) * pbuf, sum3, tot);
    ++red;
    res = tot[1];
    ysum = tot[2];
  }
  // ---- S6: remove the constant mode of y and correct phi
  const double ybar = ysum / (double)n;
  for (int m = tid; m < n; m += stride) {
    const double yv = a.y[m] - ybar;
    a.y[m] = yv;
    a.phi_out[m] = a.phi_out[m] - a.c_phi * yv;
  }
  if (tid == 0) {
    maze_stats* r = a.rec;
    r->iters = it;
    r->resid = res;
    r->total_iters += it;
    if (!isfinite(res)) r->status = MAZE_ERR_NONFINITE;
    else if (!(res < a.tol)) r->status = MAZE_ERR_NOT_CONVERGED;
  }
}

int solve_blocks(int n_points) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_solve, kSolveThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int want = (n_points + kSolveThreads - 1) / kSolveThreads;
  int cap = sms * per_sm;
  return want < cap ? want : cap;
}

cudaError_t launch_cg_solve(const SolveArgs& a, int blocks, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cg_solve, a);
}

}  // namespace maze
