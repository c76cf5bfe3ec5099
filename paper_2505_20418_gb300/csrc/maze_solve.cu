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
// An iteration takes two grid rounds (flag-carrying reductions, see
// grid_reduce): the direction update is fused into the stencil pass by
// recomputing p_new at the six neighbours from r and a double-buffered p_old.
// Every reduction combines the block partials in the same fixed order in
// every block, so all blocks take identical decisions and the result is
// bit-reproducible.
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

__global__ void __launch_bounds__(kSolveThreads) k_cg_solve(SolveArgs a) {
  unsigned epoch = 0;   // reduction rounds of this launch
  const int n = a.n, N = a.N;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;

  const bool m3[3] = {false, true, false};     // (r.r, max|r|, sum y)
  const bool m1[1] = {false};
  const bool m2[2] = {false, true};
  double tot[3];

  // ---- S4 and the initial residual r0 = sigma_p - M y0
  {
    double rr = 0, ys = 0;
    unsigned long long rmax = 0;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N);
      const double q = fix_to_dbl((long long)a.qfix[m], 1075 - 50);   // qfix 2^-50, integer ops only
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
      const double r = sg - My;
      a.r[m] = r;
      rr += r * r;
      rmax = max(rmax, abs_bits(r));
      ys += y[m];
    }
    const double v[3] = {rr, absmax_value(rmax), ys};
    if (!grid_reduce<3>(v, m3, a.recs, ++epoch, a.rec, tot)) return;
  }
  double rho = tot[0], res = tot[1], ysum = tot[2];
  int it = 0;
  bool conv = res < a.tol;
  bool fresh = true;
  bool have_ysum = true;
  double beta = 0.0;
  bool finite = isfinite(res) && isfinite(rho) && isfinite(ysum);
  int cur = 0;          // p_old lives in p[cur], p_new goes to p[cur ^ 1]

  while (!conv && finite && it < a.max_iter) {
    have_ysum = false;
    // phase AB: p_new = r + beta p_old, here and at the six neighbours (from
    // r and p_old, which no block writes in this phase), then Mp_new and the
    // partial p_new.Mp_new. One grid round instead of a barrier between the
    // direction update and the stencil.
    double* pn = cur ? a.p : a.p1;
    const double* po = cur ? a.p1 : a.p;
    {
      double pmp = 0;
      const double* r = a.r;
      for (int m = tid; m < n; m += stride) {
        const Nbr b = neighbours(m, N);
        double c0, s6;
        if (fresh) {
          c0 = r[m];
          s6 = (r[b.xm] + r[b.xp]) + (r[b.ym] + r[b.yp]) + (r[b.zm] + r[b.zp]);
        } else {
          c0 = r[m] + beta * po[m];
          s6 = ((r[b.xm] + beta * po[b.xm]) + (r[b.xp] + beta * po[b.xp])) +
               ((r[b.ym] + beta * po[b.ym]) + (r[b.yp] + beta * po[b.yp])) +
               ((r[b.zm] + beta * po[b.zm]) + (r[b.zp] + beta * po[b.zp]));
        }
        const double mp = s6 - 6.0 * c0;
        pn[m] = c0;
        a.Mp[m] = mp;
        pmp += c0 * mp;
      }
      const double v[1] = {pmp};
      double t1[1], alpha;
      const double rho_c = rho;
      if (!grid_reduce<1>(v, m1, a.recs, ++epoch, a.rec, t1,
                          [rho_c](const double* t) { return rho_c * recip_newton(t[0]); }, &alpha))
        return;
      // phase C: y += alpha p_new, r -= alpha Mp; r.r and max|r|
      double rr = 0;
      unsigned long long rmax = 0;
      for (int m = tid; m < n; m += stride) {
        a.y[m] += alpha * pn[m];
        const double rv = a.r[m] - alpha * a.Mp[m];
        a.r[m] = rv;
        rr += rv * rv;
        rmax = max(rmax, abs_bits(rv));
      }
      const double v2[2] = {rr, absmax_value(rmax)};
      double t2[2], beta_new;
      const double rho_old = rho;
      if (!grid_reduce<2>(v2, m2, a.recs, ++epoch, a.rec, t2,
                          [rho_old](const double* t) { return t[0] * recip_newton(rho_old); }, &beta_new))
        return;
      cur ^= 1;
      ++it;
      res = t2[1];
      finite = isfinite(res) && isfinite(t2[0]);
      if (!finite) break;
      if (res < a.tol) {
        // confirm with the true residual sigma_p - M y (also gives sum y)
        double rr3 = 0, ys = 0;
        unsigned long long rmax3 = 0;
        const double* y = a.y;
        for (int m = tid; m < n; m += stride) {
          const Nbr b = neighbours(m, N);
          const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
          const double rv = a.sigma[m] - My;
          a.r[m] = rv;
          rr3 += rv * rv;
          rmax3 = max(rmax3, abs_bits(rv));
          ys += y[m];
        }
        const double v3[3] = {rr3, absmax_value(rmax3), ys};
        if (!grid_reduce<3>(v3, m3, a.recs, ++epoch, a.rec, tot)) return;
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
      beta = beta_new;
      rho = t2[0];
      fresh = false;
    }
  }
  if (!have_ysum) {
    // stopped at max_iter or on a non-finite value: true residual and sum y
    double rr = 0, ys = 0;
    unsigned long long rmax = 0;
    const double* y = a.y;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N);
      const double My = (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]) - 6.0 * y[m];
      const double rv = a.sigma[m] - My;
      rr += rv * rv;
      rmax = max(rmax, abs_bits(rv));
      ys += y[m];
    }
    const double v[3] = {rr, absmax_value(rmax), ys};
    if (!grid_reduce<3>(v, m3, a.recs, ++epoch, a.rec, tot)) return;
    res = tot[1];
    ysum = tot[2];
  }
  // ---- S6: remove the constant mode of y and correct phi
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

int solve_blocks(int n_points) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_solve, kSolveThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int want = (n_points + kSolveThreads - 1) / kSolveThreads;
  int cap = sms * per_sm;
  if (cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
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
