// S4-S6 of the MaZe step with the multigrid constraint solver (Sec. III.A), in
// FP64, in one cooperative persistent kernel:
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
// kernel computed once on the host from M's eigenvalues.
//
// On GB300 the FP64 pipe issues 2 operations per clock per SM (1/64 of the
// FP32 rate), so on large grids this kernel is bound by FP64 arithmetic, not
// by HBM. It spends as few FP64 operations per point as the method allows,
// each an exact restatement of the same arithmetic:
//  * every level stores its right-hand side pre-scaled, bs = -b/6, so a
//    Gauss-Seidel update is the six-neighbour sum and one FMA,
//    x = s/6 + bs, and a residual is 6 (x - bs) - s;
//  * after a black half-sweep the residual at black points is zero (each was
//    just set to make it zero), so the residual that feeds the restriction,
//    and the convergence test after a V-cycle, are formed at red points
//    only, and the 27-point full weighting reads only its 13 red points;
//  * on a coarse level the first red half-sweep from the zero guess is
//    x = bs: the restriction writes it together with the right-hand side;
//  * the prolongation updates black points only (the next red half-sweep
//    overwrites every red point without reading it);
//  * maxima are integer maxima of IEEE bit patterns (no FP64 compare), and
//    the mean of y is formed once, after the last V-cycle.
// Grids of 128^3 points and more run one 1024-thread block per SM, so every
// SM carries the same work; smaller grids, whose phases give each thread
// only a few points, run up to 256 blocks of 256 threads (the work and its
// memory traffic spread over more SMs).
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

namespace {

// Sum of the six periodic neighbours of (i, j, k), in a fixed order. (No
// pointer here is __restrict__: every vector is written in some phase of the
// kernel, so none may be read through the non-coherent read-only path.)
__device__ __forceinline__ double nbr6(const double* x, int i, int j, int k, int N) {
  const int NN = N * N;
  const int n = i + N * j + NN * k;
  const int xm = i == 0 ? n + N - 1 : n - 1, xp = i == N - 1 ? n - N + 1 : n + 1;
  const int ym = j == 0 ? n + NN - N : n - N, yp = j == N - 1 ? n - NN + N : n + N;
  const int zm = k == 0 ? n + NN * (N - 1) : n - NN, zp = k == N - 1 ? n - NN * (N - 1) : n + NN;
  return (x[xm] + x[xp]) + (x[ym] + x[yp]) + (x[zm] + x[zp]);
}

__device__ __forceinline__ int wrapi(int a, int N) { return a < 0 ? a + N : (a >= N ? a - N : a); }

// One red-black half-sweep of colour c on level (N, lg): x = s/6 + bs.
// (Taking two points per round with all loads before the stores measured
// the same: 7.04 against 7.01 ms per 256^3 solve.)
__device__ __forceinline__ void half_sweep(double* x, const double* bs, int N, int lg, int c, int tid, int stride) {
  const int hcount = N * N * (N >> 1);
#pragma unroll 2
  for (int h = tid; h < hcount; h += stride) {
    int i, j, k;
    colour_point(h, N, lg, c, i, j, k);
    const int m = i + N * (j + N * k);
    x[m] = fma(nbr6(x, i, j, k, N), 1.0 / 6.0, bs[m]);
  }
}

}  // namespace

__global__ void __launch_bounds__(kMgThreads, 1) k_mg_solve(SolveArgs a, MgArgs g) {
  unsigned epoch = 0, bar_epoch = 0;
  const int n = a.n, N0 = a.N;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;
  const bool mmax[1] = {true};
  const bool msum[1] = {false};
  double* sig6 = g.b;   // level 0 slot of the right-hand sides: -sigma_p / 6

  // ---- S4 and the residual of the warm start (every point)
  double res;
  {
    unsigned long long rmax = 0;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N0);
      const double sg = shake_rhs(a, m, b);
      sig6[m] = sg * (-1.0 / 6.0);
      const double* y = a.y;
      const double My = fma(-6.0, y[m], (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]));
      rmax = max(rmax, abs_bits(sg - My));
    }
    const double v[1] = {absmax_value(rmax)};
    double t[1];
    if (!grid_reduce<1>(v, mmax, a.recs, ++epoch, a.rec, t)) return;
    res = t[0];
  }
  int it = 0;

  while (isfinite(res) && !(res < a.tol) && it < a.max_iter) {
    // ---- down: smooth, residual at red points, restrict
    for (int l = 0; l < g.L - 1; ++l) {
      const int N = g.Nl[l], lg = g.lg[l];
      double* x = l == 0 ? a.y : g.x + g.off[l];
      const double* bs = g.b + g.off[l];
      for (int s = 0; s < g.nu1; ++s) {
        // on a coarse level the first red half-sweep (x = bs from the zero
        // guess) was written by the restriction
        if (!(l > 0 && s == 0)) {
          half_sweep(x, bs, N, lg, 0, tid, stride);
          if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
        }
        half_sweep(x, bs, N, lg, 1, tid, stride);
        if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      }
      double* r = g.r + g.off[l];
      {
        const int hcount = N * N * (N >> 1);
        for (int h = tid; h < hcount; h += stride) {
          int i, j, k;
          colour_point(h, N, lg, 0, i, j, k);
          const int m = i + N * (j + N * k);
          r[m] = fma(6.0, x[m] - bs[m], -nbr6(x, i, j, k, N));
        }
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      // full weighting from the 13 red points of the 3^3 neighbourhood of
      // fine point (2I, 2J, 2K): the centre (weight 1/8) and the 12 points
      // two of whose offsets are +-1 (weight 1/32); b_c = 4 FW(r) is stored
      // as -b_c/6, and a red coarse point gets its first half-sweep x = bs
      const int Nc = g.Nl[l + 1], NNc = Nc * Nc;
      const bool coarsest = (l + 1 == g.L - 1);
      double* bc = g.b + g.off[l + 1];
      double* xc = g.x + g.off[l + 1];
      const int NN = N * N;
      for (int mc = tid; mc < Nc * NNc; mc += stride) {
        const int K = mc / NNc, J = (mc - K * NNc) / Nc, I = mc - K * NNc - J * Nc;
        const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
        const int im = wrapi(i0 - 1, N), ip = i0 + 1;   // i0 + 1 <= N - 1
        const int jm = wrapi(j0 - 1, N) * N, jp = (j0 + 1) * N, jc = j0 * N;
        const int km = wrapi(k0 - 1, N) * NN, kp = (k0 + 1) * NN, kc = k0 * NN;
        const double s12 = ((r[kc + jm + im] + r[kc + jm + ip]) + (r[kc + jp + im] + r[kc + jp + ip])) +
                           ((r[km + jc + im] + r[km + jc + ip]) + (r[kp + jc + im] + r[kp + jc + ip])) +
                           ((r[km + jm + i0] + r[km + jp + i0]) + (r[kp + jm + i0] + r[kp + jp + i0]));
        const double v = fma(s12, -1.0 / 48.0, r[kc + jc + i0] * (-1.0 / 12.0));
        bc[mc] = v;
        if (!coarsest && ((I + J + K) & 1) == 0) xc[mc] = v;
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
    }
    // ---- coarsest: x = G' * bs (exact zero-mean solve; G' = -6 times the
    // pseudo-inverse kernel, folded on the host), one warp per point
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
          acc[u & 3] = fma(g.gker[d], bc[q], acc[u & 3]);
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
      const int N = g.Nl[l], lg = g.lg[l], hcount = N * N * (N >> 1);
      const int Nc = g.Nl[l + 1], NNc = Nc * Nc;
      double* x = l == 0 ? a.y : g.x + g.off[l];
      const double* bs = g.b + g.off[l];
      const double* xc = g.x + g.off[l + 1];
      for (int h = tid; h < hcount; h += stride) {
        int i, j, k;
        colour_point(h, N, lg, 1, i, j, k);
        // trilinear: per axis the coarse index i/2 (even i) or the mean of
        // (i-1)/2 and (i+1)/2 (odd i), periodic; a black point has one odd
        // coordinate (mean of 2 coarse values) or three (mean of 8)
        const int m = i + N * (j + N * k);
        const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
        const int odd = (i & 1) + (j & 1) + (k & 1);
        double e;
        if (odd == 1) {
          const int c0 = i0 + Nc * (j0 + Nc * k0);
          const int c1 = (i & 1) ? wrapi(i0 + 1, Nc) + Nc * (j0 + Nc * k0)
                       : (j & 1) ? i0 + Nc * (wrapi(j0 + 1, Nc) + Nc * k0)
                                 : i0 + Nc * (j0 + Nc * wrapi(k0 + 1, Nc));
          e = 0.5 * (xc[c0] + xc[c1]);
        } else {
          const int i1 = wrapi(i0 + 1, Nc), j1 = wrapi(j0 + 1, Nc), k1 = wrapi(k0 + 1, Nc);
          const double* c0 = xc + (size_t)k0 * NNc;
          const double* c1 = xc + (size_t)k1 * NNc;
          e = 0.125 * (((c0[j0 * Nc + i0] + c0[j0 * Nc + i1]) + (c0[j1 * Nc + i0] + c0[j1 * Nc + i1])) +
                       ((c1[j0 * Nc + i0] + c1[j0 * Nc + i1]) + (c1[j1 * Nc + i0] + c1[j1 * Nc + i1])));
        }
        x[m] += e;
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      for (int s = 0; s < g.nu2; ++s) {
        for (int c = 0; c < 2; ++c) {
          half_sweep(x, bs, N, lg, c, tid, stride);
          if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
        }
      }
    }
    ++it;
    // ---- convergence test (Eq. res_poisson_maze) at red points: the black
    // residual after the last black half-sweep is zero
    {
      unsigned long long rmax = 0;
      const int N = N0, lg = g.lg[0], hcount = N * N * (N >> 1);
      const double* y = a.y;
#pragma unroll 2
      for (int h = tid; h < hcount; h += stride) {
        int i, j, k;
        colour_point(h, N, lg, 0, i, j, k);
        const int m = i + N * (j + N * k);
        rmax = max(rmax, abs_bits(fma(6.0, y[m] - sig6[m], -nbr6(y, i, j, k, N))));
      }
      const double v[1] = {absmax_value(rmax)};
      double t[1];
      if (!grid_reduce<1>(v, mmax, a.recs, ++epoch, a.rec, t)) return;
      res = t[0];
    }
  }
  // ---- mean of y, then S6
  double ysum;
  {
    double ys = 0.0;
    for (int m = tid; m < n; m += stride) ys += a.y[m];
    const double v[1] = {ys};
    double t[1];
    if (!grid_reduce<1>(v, msum, a.recs, ++epoch, a.rec, t)) return;
    ysum = t[0];
  }
  const double ybar = ysum * a.inv_n;
  for (int m = tid; m < n; m += stride) {
    const double yv = a.y[m] - ybar;
    a.y[m] = yv;
    a.phi_out[m] = fma(-a.c_phi, yv, a.phi_out[m]);
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
  const int threads = mg_threads(n_points);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_solve, threads, 0);
  if (per_sm < 1) per_sm = 1;
  int want = (n_points + threads - 1) / threads;
  int cap = sms * per_sm;
  if (cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
  return want < cap ? want : cap;
}

cudaError_t launch_mg_solve(const SolveArgs& a, const MgArgs& g, int blocks, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(mg_threads(a.n));
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
