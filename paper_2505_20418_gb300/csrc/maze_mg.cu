// S4-S6 of the MaZe step with the multigrid constraint solver (Sec. III.A), in
// one cooperative persistent kernel:
//   S4  phi_p = 2 phi^k - phi^{k-1},  sigma_p = (h/4pi) M phi_p + q   (Eq. SHAKE)
//   S5  V-cycles on M y = sigma_p from the previous y until
//       max_n |(M y - sigma_p)_n| < tol, the residual checked after every
//       V-cycle (Eqs. SHAKEy, res_poisson_maze)
//   S6  phi^{k+1} = phi_p - (4pi/h)(y - mean y)                          (Eq. SHAKEPhiFinal)
//
// V-cycle on levels l = 0..L-1 (N_l halves while even and above 8), operators of
// Sec. III.A: nu1 red-black Gauss-Seidel sweeps (red = i+j+k even; a point is
// set to (sum of its six neighbours - b)/6), residual r = b - M x, coarse rhs
// 4 * (27-point full weighting of r) (M is h^2-scaled), recursion from a zero
// coarse guess, trilinear prolongation of the coarse correction, nu2 sweeps.
// The coarsest grid (at most 8^3 points) is solved exactly: the paper runs CG
// to convergence there; here the exact zero-mean solution is one product with
// the pseudo-inverse of the circulant coarsest M, a periodic convolution
// kernel g computed once on the host from M's eigenvalues.
//
// Two exact shortcuts of the same arithmetic: the first red half-sweep on a
// coarse level starts from the zero guess, so it needs no neighbour reads;
// the prolongation updates black points only, because the red half-sweep that
// follows overwrites every red point without reading its old value.
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

namespace {

// point of colour c (0 red, 1 black) with half-index h on an N^3 grid (N even)
__device__ __forceinline__ int colour_point(int h, int N, int c, int& i, int& j, int& k) {
  const int half = N >> 1;
  const int row = h / half;
  const int t = h - row * half;
  k = row / N;
  j = row - k * N;
  i = 2 * t + ((j + k + c) & 1);
  return i + N * (j + N * k);
}

__device__ __forceinline__ int wrapi(int a, int N) { return a < 0 ? a + N : (a >= N ? a - N : a); }

template <typename T>
__device__ __forceinline__ T nbr_sum(const T* x, int i, int j, int k, int N) {
  const int NN = N * N;
  const int n = i + N * j + NN * k;
  const int xm = i == 0 ? n + N - 1 : n - 1, xp = i == N - 1 ? n - N + 1 : n + 1;
  const int ym = j == 0 ? n + NN - N : n - N, yp = j == N - 1 ? n - NN + N : n + N;
  const int zm = k == 0 ? n + NN * (N - 1) : n - NN, zp = k == N - 1 ? n - NN * (N - 1) : n + NN;
  return (x[xm] + x[xp]) + (x[ym] + x[yp]) + (x[zm] + x[zp]);
}

}  // namespace

__global__ void __launch_bounds__(kSolveThreads) k_mg_solve(SolveArgs a, MgArgs g) {
  unsigned epoch = 0, bar_epoch = 0;
  const int n = a.n, N0 = a.N;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;
  const bool m2[2] = {true, false};   // (max |r|, sum y)
  double tot[2];

  // ---- S4 and the initial residual of the warm start
  {
    double ys = 0;
    unsigned long long rmax = 0;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N0);
      const double q = (double)(long long)a.qfix[m] * kQInv;
      a.qfix[m] = 0ull;
      if (a.q_out) a.q_out[m] = q;
      double php = 0.0, Mphp = 0.0;
      if (!a.zero_phi) {
        const double* pk = a.phi_k;
        const double* pm = a.phi_km1;
        const double nk = (pk[b.xm] + pk[b.xp]) + (pk[b.ym] + pk[b.yp]) + (pk[b.zm] + pk[b.zp]);
        if (a.static_guess) {
          php = pk[m];
          Mphp = nk - 6.0 * php;
        } else {
          php = 2.0 * pk[m] - pm[m];
          const double nm = (pm[b.xm] + pm[b.xp]) + (pm[b.ym] + pm[b.yp]) + (pm[b.zm] + pm[b.zp]);
          Mphp = 2.0 * nk - nm - 6.0 * php;
        }
      }
      const double sg = a.c_sig * Mphp + q;
      a.phi_out[m] = php;
      a.sigma[m] = sg;
      const double* y = a.y;
      const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
      rmax = max(rmax, abs_bits(sg - My));
      ys += y[m];
    }
    const double v[2] = {absmax_value(rmax), ys};
    if (!grid_reduce<2>(v, m2, a.recs, ++epoch, a.rec, tot)) return;
  }
  double res = tot[0], ysum = tot[1];
  int it = 0;
  bool finite = isfinite(res) && isfinite(ysum);

  while (finite && !(res < a.tol) && it < a.max_iter) {
    // ---- down: smooth, residual, restrict
    for (int l = 0; l < g.L - 1; ++l) {
      const int N = g.Nl[l], NN = N * N, hcount = N * NN / 2;
      double* x = l == 0 ? a.y : g.x + g.off[l];
      const double* b = l == 0 ? a.sigma : g.b + g.off[l];
      for (int s = 0; s < g.nu1; ++s) {
        for (int c = 0; c < 2; ++c) {
          const bool from_zero = (l > 0 && s == 0 && c == 0);
          for (int h = tid; h < hcount; h += stride) {
            int i, j, k;
            const int m = colour_point(h, N, c, i, j, k);
            x[m] = from_zero ? -b[m] * (1.0 / 6.0) : (nbr_sum(x, i, j, k, N) - b[m]) * (1.0 / 6.0);
          }
          if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
        }
      }
      double* r = g.r + g.off[l];
      for (int m = tid; m < N * NN; m += stride) {
        const int k = m / NN, j = (m - k * NN) / N, i = m - k * NN - j * N;
        r[m] = b[m] - (nbr_sum(x, i, j, k, N) - 6.0 * x[m]);
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      const int Nc = g.Nl[l + 1], NNc = Nc * Nc;
      double* bc = g.b + g.off[l + 1];
      for (int m = tid; m < Nc * NNc; m += stride) {
        const int K = m / NNc, J = (m - K * NNc) / Nc, I = m - K * NNc - J * Nc;
        double acc = 0.0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
          const int z = wrapi(2 * K + dz, N);
          const double wz = dz == 0 ? 0.5 : 0.25;
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapi(2 * J + dy, N);
            const double wzy = wz * (dy == 0 ? 0.5 : 0.25);
            const double* row = r + (size_t)z * NN + (size_t)yy * N;
            acc += wzy * (0.25 * row[wrapi(2 * I - 1, N)] + 0.5 * row[2 * I] + 0.25 * row[wrapi(2 * I + 1, N)]);
          }
        }
        bc[m] = 4.0 * acc;
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
    }
    // ---- coarsest: x = g * b (exact zero-mean solve), one warp per point
    {
      const int Nc = g.Nl[g.L - 1], NNc = Nc * Nc, nc3 = Nc * NNc;
      const double* bc = g.b + g.off[g.L - 1];
      double* xc = g.x + g.off[g.L - 1];
      const int lane = threadIdx.x & 31;
      const int wid = tid >> 5, nwarps = stride >> 5;
      for (int p = wid; p < nc3; p += nwarps) {
        const int pk = p / NNc, pj = (p - pk * NNc) / Nc, pi = p - pk * NNc - pj * Nc;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int u = 0;
        for (int q = lane; q < nc3; q += 32, ++u) {
          const int qk = q / NNc, qj = (q - qk * NNc) / Nc, qi = q - qk * NNc - qj * Nc;
          const int d = wrapi(pi - qi, Nc) + Nc * (wrapi(pj - qj, Nc) + Nc * wrapi(pk - qk, Nc));
          acc[u & 3] += g.gker[d] * bc[q];
        }
        long long S;
        int E;
        warp_dsum_fix((acc[0] + acc[1]) + (acc[2] + acc[3]), S, E);
        if (lane == 0) xc[p] = fix_to_dbl(S, E);
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
    }
    // ---- up: prolong (black points), smooth
    for (int l = g.L - 2; l >= 0; --l) {
      const int N = g.Nl[l], NN = N * N, hcount = N * NN / 2;
      const int Nc = g.Nl[l + 1], NNc = Nc * Nc;
      double* x = l == 0 ? a.y : g.x + g.off[l];
      const double* b = l == 0 ? a.sigma : g.b + g.off[l];
      const double* xc = g.x + g.off[l + 1];
      for (int h = tid; h < hcount; h += stride) {
        int i, j, k;
        const int m = colour_point(h, N, 1, i, j, k);
        // trilinear: per axis the coarse index i/2 (even i) or the mean of
        // (i-1)/2 and (i+1)/2 (odd i), periodic
        const int i0 = i >> 1, i1 = (i & 1) ? wrapi(i0 + 1, Nc) : i0;
        const int j0 = j >> 1, j1 = (j & 1) ? wrapi(j0 + 1, Nc) : j0;
        const int k0 = k >> 1, k1 = (k & 1) ? wrapi(k0 + 1, Nc) : k0;
        const double* c0 = xc + (size_t)k0 * NNc;
        const double* c1 = xc + (size_t)k1 * NNc;
        const double e = 0.125 * (((c0[j0 * Nc + i0] + c0[j0 * Nc + i1]) + (c0[j1 * Nc + i0] + c0[j1 * Nc + i1])) +
                                  ((c1[j0 * Nc + i0] + c1[j0 * Nc + i1]) + (c1[j1 * Nc + i0] + c1[j1 * Nc + i1])));
        x[m] += e;
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      for (int s = 0; s < g.nu2; ++s) {
        for (int c = 0; c < 2; ++c) {
          for (int h = tid; h < hcount; h += stride) {
            int i, j, k;
            const int m = colour_point(h, N, c, i, j, k);
            x[m] = (nbr_sum(x, i, j, k, N) - b[m]) * (1.0 / 6.0);
          }
          if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
        }
      }
    }
    ++it;
    // ---- residual check (Eq. res_poisson_maze) and sum y
    {
      double ys = 0;
      unsigned long long rmax = 0;
      const double* y = a.y;
      for (int m = tid; m < n; m += stride) {
        const Nbr b = neighbours(m, N0);
        const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
        rmax = max(rmax, abs_bits(a.sigma[m] - My));
        ys += y[m];
      }
      const double v[2] = {absmax_value(rmax), ys};
      if (!grid_reduce<2>(v, m2, a.recs, ++epoch, a.rec, tot)) return;
      res = tot[0];
      ysum = tot[1];
      finite = isfinite(res) && isfinite(ysum);
    }
  }
  // ---- S6
  const double ybar = ysum * a.inv_n;
  for (int m = tid; m < n; m += stride) {
    const double yv = a.y[m] - ybar;
    a.y[m] = yv;
    a.phi_out[m] = a.phi_out[m] - a.c_phi * yv;
  }
  if (tid == 0) {
    maze_stats* r = a.rec;
    r->iters = it;
    r->resid = res * a.res_scale;
    r->total_iters += it;
    if (!isfinite(res) || !isfinite(ysum)) r->status = MAZE_ERR_NONFINITE;
    else if (!(res < a.tol)) r->status = MAZE_ERR_NOT_CONVERGED;
  }
}

int mg_blocks(int n_points) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_solve, kSolveThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int want = (n_points + kSolveThreads - 1) / kSolveThreads;
  int cap = sms * per_sm;
  if (cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
  return want < cap ? want : cap;
}

cudaError_t launch_mg_solve(const SolveArgs& a, const MgArgs& g, int blocks, cudaStream_t s) {
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
  return cudaLaunchKernelEx(&cfg, k_mg_solve, a, g);
}

}  // namespace maze
