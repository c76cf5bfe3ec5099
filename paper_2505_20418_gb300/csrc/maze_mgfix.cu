// S4-S6 of the MaZe step with the multigrid solver (Sec. III.A) at precision
// MAZE_FP64_FIXMG: FP64 state, and V-cycles that solve for the correction of
// y in exact 64-bit integer arithmetic. One cooperative persistent kernel.
//
// FP64, as in the FP64 kernel: phi, sigma_p, y; S4 (Eq. SHAKE); the residual
// of the warm start r_0 = sigma_p - M y at every point; S6 (Eq.
// SHAKEPhiFinal). The Laplacian of phi_p in S4 is summed exactly in integers
// and rounded once (exact_combination). Integer: the V-cycles solve M E = r_0 for the correction E
// of y (y_final = y + E 2^-F), every value of every level an integer multiple
// of 2^-F. In exact arithmetic this is the FP64 kernel's iteration: red-black
// Gauss-Seidel from y with right-hand side sigma_p, and from E = 0 with
// right-hand side r_0, give the same iterates y + E (the update is affine), and
// so do the restriction, the coarsest solve and the prolongation, which are
// linear. The operators are those of the FP64 kernel: nu1 red-black sweeps,
// 27-point full weighting of the residual (its 13 red points), the exact
// zero-mean coarsest solve by the pseudo-inverse kernel, trilinear
// prolongation, nu2 sweeps, the stopping test max |sigma_p - M y| < tol after
// every V-cycle (Eqs. SHAKEy, res_poisson_maze).
//
// Why: GB300 issues FP64 at 2 operations per clock per SM, and a Gauss-Seidel
// point update costs 6 of them, so the FP64 V-cycle is bound by the FP64 pipe.
// The same update in 64-bit integers (adds and a multiply-high for the
// division by 6) runs on the integer pipes, and the V-cycle becomes bound by
// HBM traffic. y is read and written once, in S6.
//
// Exactness and range:
//  * the stopping test is exact: r = r_0 - M E at red points is formed in
//    integers after each V-cycle, and after the last black half-sweep a black
//    point's residual is the rounding of its division by 6 (at most 3 units),
//    taken as it is made. The only roundings of the result are the FP64
//    operations that make r_0 and y + E 2^-F.
//  * a Gauss-Seidel update divides by 6 rounding half away from zero; the
//    full weighting divides by 8 and the prolongation by 2 or 8, rounding
//    half up: half a unit, 2^-(H+1) of max |r_0|, each.
//  * the scale: F makes max |r_0| 2^F fall in [2^(H-1), 2^H), H = 58 -
//    2 ceil(log2 N). E approximates M^+ r_0 and |M^+|_inf is about 0.048 N^2
//    (the h^2-scaled periodic Laplacian), so corrections stay below 2^54 and
//    six-neighbour sums below 2^57.
//  * once the residual has fallen 20 bits below the scale (solves from a
//    cold start), E is applied to y, the exact residual r_0 - M E at every
//    point becomes the right-hand side, shifted left to the finer scale, and
//    the iteration goes on from E = 0 (a restart: the same iterates).
//  * a coarsest correction of 2^58 units or more (a diverging solve) ends the
//    solve with MAZE_ERR_NONFINITE instead of wrapping around.
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

namespace {

constexpr int kMaxScale = 1000;   // F stays within the range of 2^-F as a double

__device__ __forceinline__ long long shl(long long v, int s) { return (long long)((unsigned long long)v << s); }

__device__ __forceinline__ unsigned long long iabs(long long v) {
  return v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
}

// round(v / 6), half away from zero (|v| < 2^63 - 3).
__device__ __forceinline__ long long div6(long long v) {
  const long long q = (long long)((iabs(v) + 3ull) / 6ull);
  return v < 0 ? -q : q;
}

// round(v / 2^k), half up.
__device__ __forceinline__ long long div2k(long long v, int k) { return (v + (1LL << (k - 1))) >> k; }

// Storage: every level but the coarsest keeps each vector split by colour,
// the red points (i + j + k even) first, then the black, each in half-index
// order h = t + (N/2)(j + N k) with i = 2t + ((j + k + c) & 1); a half-sweep
// then reads only the other colour's array and writes its own, in unit
// stride. The coarsest level (an edge of at most 8, possibly odd) is stored
// in natural order i + N (j + N k).

// (t, j, k) of half-index h on an edge N (lg = log2 N, or -1).
__device__ __forceinline__ void half_decode(int h, int N, int lg, int& t, int& j, int& k) {
  if (lg > 0) {
    const int row = h >> (lg - 1);
    t = h & ((N >> 1) - 1);
    k = row >> lg;
    j = row & (N - 1);
  } else {
    const int hN = N >> 1;
    const int row = h / hN;
    t = h - row * hN;
    k = row / N;
    j = row - k * N;
  }
}

// Index of point (i, j, k) in a level's storage.
__device__ __forceinline__ int store_index(int i, int j, int k, int N, bool split) {
  if (!split) return i + N * (j + N * k);
  return ((i + j + k) & 1) * ((N * N * N) >> 1) + (i >> 1) + (N >> 1) * (j + N * k);
}

// Sum of the six periodic neighbours of the point at half-index h = (t, j, k)
// of parity p (i = 2t + p), all of the other colour, read from that colour's
// array o: the two x-neighbours sit at h and h -+ 1 of o, the others at
// h +- N/2 and h +- N^2/2. A fixed order.
__device__ __forceinline__ long long nbr6s(const long long* o, int h, int t, int j, int k, int p, int N) {
  const int hN = N >> 1, Sy = hN, Sz = hN * N;
  const int hx = p ? (t == hN - 1 ? h - (hN - 1) : h + 1) : (t == 0 ? h + (hN - 1) : h - 1);
  const int ym = j == 0 ? h + (N - 1) * Sy : h - Sy, yp = j == N - 1 ? h - (N - 1) * Sy : h + Sy;
  const int zm = k == 0 ? h + (N - 1) * Sz : h - Sz, zp = k == N - 1 ? h - (N - 1) * Sz : h + Sz;
  return (o[h] + o[hx]) + (o[ym] + o[yp]) + (o[zm] + o[zp]);
}

__device__ __forceinline__ int wrapi(int a, int N) { return a < 0 ? a + N : (a >= N ? a - N : a); }

// round(v 2^(1075 - E)) for a finite v whose exponent field is at most E + 3.
__device__ __forceinline__ long long to_units(double v, int E) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const long long m = e ? (b & 0xfffffffffffffLL) | (1LL << 52) : (b & 0xfffffffffffffLL);
  const int sh = E - (e ? e : 1);
  const long long x = sh <= 0 ? m << (-sh) : (sh >= 62 ? 0 : (m + (1LL << (sh - 1))) >> sh);
  return b < 0 ? -x : x;
}

// sum_k c_k v_k with small integer coefficients, rounded once: every v_k
// rounded to an eighth of an ulp of the largest |v_k| (exact for the values
// within 3 binades of it), the integers summed exactly. A NaN or infinity
// gives NaN.
template <int K>
__device__ __forceinline__ double exact_combination(const double (&v)[K], const int (&c)[K]) {
  int emax = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) emax = max(emax, dbl_exp(v[k]));
  if (emax == 0x7ff) return __longlong_as_double(0x7ff8000000000000LL);
  const int E = emax - 3;
  long long s = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) s += (long long)c[k] * to_units(v[k], E);
  return fix_to_dbl(s, E);
}

// S4 at point m (Eq. SHAKE) as shake_rhs, with the Laplacian of phi_p summed
// exactly on the integer pipe, M phi_p = 2 (s_k - 6 phi^k) - (s_{k-1} -
// 6 phi^{k-1}) over the fourteen values (s the six-neighbour sums); and the
// warm start's M y in FP64 (the two pipes share the work).
__device__ __forceinline__ double shake_rhs_fix(const SolveArgs& a, int m, const Nbr& b, double& My) {
  const double q = fix_to_dbl((long long)a.qfix[m], 1075 - 50);
  a.qfix[m] = 0ull;
  if (a.q_out) a.q_out[m] = q;
  double php = 0.0, Mphp = 0.0;
  if (!a.zero_phi) {
    const double* pk = a.phi_k;
    if (a.static_guess) {
      php = pk[m];
      const double v[7] = {pk[b.xm], pk[b.xp], pk[b.ym], pk[b.yp], pk[b.zm], pk[b.zp], php};
      const int c[7] = {1, 1, 1, 1, 1, 1, -6};
      Mphp = exact_combination(v, c);
    } else {
      const double* pm = a.phi_km1;
      const double v[14] = {pk[b.xm], pk[b.xp], pk[b.ym], pk[b.yp], pk[b.zm], pk[b.zp], pk[m],
                            pm[b.xm], pm[b.xp], pm[b.ym], pm[b.yp], pm[b.zm], pm[b.zp], pm[m]};
      const int c[14] = {2, 2, 2, 2, 2, 2, -12, -1, -1, -1, -1, -1, -1, 6};
      Mphp = exact_combination(v, c);
      php = fma(2.0, v[6], -v[13]);
    }
  }
  const double sg = fma(a.c_sig, Mphp, q);
  a.phi_out[m] = php;
  a.sigma[m] = sg;
  const double* y = a.y;
  My = fma(-6.0, y[m], (y[b.xm] + y[b.xp]) + (y[b.ym] + y[b.yp]) + (y[b.zm] + y[b.zp]));
  return sg;
}

__device__ __forceinline__ longlong2 ld2(const long long* p) { return *reinterpret_cast<const longlong2*>(p); }
__device__ __forceinline__ void st2(long long* p, long long u, long long v) {
  *reinterpret_cast<longlong2*>(p) = make_longlong2(u, v);
}

// Six-neighbour sums s0, s1 of the two same-row points at half-indices h0 and
// h0 + 1 (h0 = (t0, j, k), t0 even, parity p; N a multiple of 4 so that a row
// holds whole pairs), from the other colour's array o with 16-byte loads: the
// pairs at h0, h0 +- N/2 and h0 +- N^2/2, and the one x-neighbour outside the
// pair, o[t0 - 1] (p = 0) or o[t0 + 2] (p = 1), periodic in the row.
__device__ __forceinline__ void nbr6_pair(const long long* o, int h0, int t0, int j, int k, int p, int N, long long& s0,
                                          long long& s1) {
  const int hN = N >> 1, Sz = hN * N;
  const int ym = j == 0 ? h0 + (N - 1) * hN : h0 - hN, yp = j == N - 1 ? h0 - (N - 1) * hN : h0 + hN;
  const int zm = k == 0 ? h0 + (N - 1) * Sz : h0 - Sz, zp = k == N - 1 ? h0 - (N - 1) * Sz : h0 + Sz;
  const longlong2 c = ld2(o + h0), u = ld2(o + ym), v = ld2(o + yp), d = ld2(o + zm), e = ld2(o + zp);
  const long long w = p ? o[t0 == hN - 2 ? h0 - t0 : h0 + 2] : o[t0 == 0 ? h0 + hN - 1 : h0 - 1];
  s0 = (p ? c.x + c.y : w + c.x) + (u.x + v.x) + (d.x + e.x);
  s1 = (p ? c.y + w : c.x + c.y) + (u.y + v.y) + (d.y + e.y);
}

// One red-black half-sweep of colour c on a split level with its red and
// black halves at xr and xb: x = round((s - b) / 6); two points per thread
// and round where the edge is a multiple of 4.
__device__ __forceinline__ void half_sweep_i(long long* xr, long long* xb, const long long* b, int N, int lg, int c,
                                             int tid, int stride) {
  const int half = (N * N * N) >> 1;
  long long* xc = c ? xb : xr;
  const long long* xo = c ? xr : xb;
  const long long* bc = b + c * half;
  if ((N & 3) == 0) {
    const int npair = half >> 1;
#pragma unroll 2
    for (int u = tid; u < npair; u += stride) {
      const int h0 = 2 * u;
      int t0, j, k;
      half_decode(h0, N, lg, t0, j, k);
      long long s0, s1;
      nbr6_pair(xo, h0, t0, j, k, (j + k + c) & 1, N, s0, s1);
      const longlong2 bv = ld2(bc + h0);
      st2(xc + h0, div6(s0 - bv.x), div6(s1 - bv.y));
    }
    return;
  }
#pragma unroll 2
  for (int h = tid; h < half; h += stride) {
    int t, j, k;
    half_decode(h, N, lg, t, j, k);
    xc[h] = div6(nbr6s(xo, h, t, j, k, (j + k + c) & 1, N) - bc[h]);
  }
}

}  // namespace

__global__ void __launch_bounds__(kMgThreads, 1) k_mgfix_solve(SolveArgs a, MgArgs g, int H) {
  unsigned epoch = 0, bar_epoch = 0;
  const int n = a.n, N0 = a.N, lg0 = g.lg[0], half0 = n >> 1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (*a.gate != 0 || a.rec->status != MAZE_OK) return;
  long long* const X = reinterpret_cast<long long*>(g.x);   // corrections, level 0 included
  long long* const B = reinterpret_cast<long long*>(g.b);   // right-hand sides
  long long* const R = reinterpret_cast<long long*>(g.r);   // residuals at red points
  // level 0's red corrections and its red residuals (for the restriction)
  // live in two arrays whose roles swap when the stopping test has already
  // made the next V-cycle's first red half-sweep (below)
  long long* e_red = X;
  long long* r_red0 = R;
  long long* const e_blk = X + half0;
  long long* const b_red = B;
  long long* const b_blk = B + half0;
  double* const y = a.y;

  // ---- S4 and the residual of the warm start (FP64, every point), kept as
  // its bit pattern in the level-0 right-hand side until the scale is known
  double res, ysum0;   // max |r_0|; sum of y before the correction
  {
    const bool mm[2] = {true, false};
    unsigned long long rmax = 0;
    double ys = 0.0;
    for (int m = tid; m < n; m += stride) {
      const Nbr b = neighbours(m, N0);
      double My;
      const double sg = shake_rhs_fix(a, m, b, My);
      const double r0 = sg - My;
      int i, j, k;
      if (lg0 > 0) {
        i = m & (N0 - 1);
        j = (m >> lg0) & (N0 - 1);
        k = m >> (2 * lg0);
      } else {
        k = m / (N0 * N0);
        j = (m - k * N0 * N0) / N0;
        i = m - N0 * (j + N0 * k);
      }
      B[store_index(i, j, k, N0, true)] = __double_as_longlong(r0);
      rmax = max(rmax, abs_bits(r0));
      ys += y[m];
    }
    const double v[2] = {absmax_value(rmax), ys};
    double t[2];
    if (!grid_reduce<2>(v, mm, a.recs, ++epoch, a.rec, t)) return;
    res = t[0];
    ysum0 = t[1];
  }
  // max |r_0| 2^F in [2^(H-1), 2^H)
  int F = H - 1 - (dbl_exp(res) - 1023);
  if (F > kMaxScale) F = kMaxScale;
  int it = 0;
  bool fresh = true;   // E = 0: level 0's first red half-sweep is E = round(-b / 6)
  bool red_done = false;   // the stopping test made the next V-cycle's first red half-sweep
  const bool spec = g.nu1 > 0;   // (the V-cycle starts with a red half-sweep on level 0)
  unsigned long long rmax = 0;
  bool ovf = false;
  double esum = 0.0;   // sum of E (units 2^-F) after the last V-cycle

  while (isfinite(res) && !(res < a.tol) && it < a.max_iter) {
    if (fresh) {
      // ---- level 0, first red half-sweep from E = 0; on the first V-cycle the
      // FP64 residual is first rounded to units of 2^-F (both colours)
      for (int h0 = 2 * tid; h0 < half0; h0 += 2 * stride) {   // (half0 = N0^3 / 2 is a multiple of 4)
        longlong2 bv = ld2(b_red + h0);
        if (it == 0) {
          bv = make_longlong2(round_scaled(__longlong_as_double(bv.x), F), round_scaled(__longlong_as_double(bv.y), F));
          st2(b_red + h0, bv.x, bv.y);
          const longlong2 bb = ld2(b_blk + h0);
          st2(b_blk + h0, round_scaled(__longlong_as_double(bb.x), F), round_scaled(__longlong_as_double(bb.y), F));
        }
        st2(e_red + h0, div6(-bv.x), div6(-bv.y));
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
    }
    // ---- down: smooth, residual at red points, restrict
    for (int l = 0; l < g.L - 1; ++l) {
      const int N = g.Nl[l], lg = g.lg[l], half = (N * N * N) >> 1;
      long long* xr = l ? X + g.off[l] : e_red;
      long long* xb = l ? xr + half : e_blk;
      const long long* b = B + g.off[l];
      for (int t = 0; t < g.nu1; ++t) {
        // a first red half-sweep from a zero guess was written by the step
        // above (level 0, fresh) or by the restriction (coarse levels); on
        // level 0 the previous stopping test may have made it (red_done)
        if (t > 0 || (l == 0 && !fresh && !red_done)) {
          half_sweep_i(xr, xb, b, N, lg, 0, tid, stride);
          if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
        }
        half_sweep_i(xr, xb, b, N, lg, 1, tid, stride);
        if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      }
      long long* r = l ? R + g.off[l] : r_red0;   // red half-indices
      if ((N & 3) == 0) {
#pragma unroll 2
        for (int h0 = 2 * tid; h0 < half; h0 += 2 * stride) {
          int t0, j, k;
          half_decode(h0, N, lg, t0, j, k);
          long long s0, s1;
          nbr6_pair(xb, h0, t0, j, k, (j + k) & 1, N, s0, s1);
          const longlong2 xv = ld2(xr + h0), bv = ld2(b + h0);
          st2(r + h0, bv.x - s0 + 6 * xv.x, bv.y - s1 + 6 * xv.y);
        }
      } else {
#pragma unroll 2
        for (int h = tid; h < half; h += stride) {
          int t, j, k;
          half_decode(h, N, lg, t, j, k);
          r[h] = b[h] - nbr6s(xb, h, t, j, k, (j + k) & 1, N) + 6 * xr[h];
        }
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      // b_c = 4 FW(r) = r_centre / 2 + (sum of the 12 red points two of whose
      // offsets are +-1) / 8, over coarse points in storage order; a red
      // coarse point gets its first half-sweep
      const int Nc = g.Nl[l + 1], lgc = g.lg[l + 1], nc3 = Nc * Nc * Nc;
      const bool coarsest = (l + 1 == g.L - 1);
      long long* bc = B + g.off[l + 1];
      long long* xc = X + g.off[l + 1];
      const int hN = N >> 1, NhN = N * hN;
      for (int q = tid; q < nc3; q += stride) {
        int I, J, K;
        if (coarsest) {
          K = q / (Nc * Nc);
          J = (q - K * Nc * Nc) / Nc;
          I = q - Nc * (J + Nc * K);
        } else {
          const int hc = nc3 >> 1, C = q >= hc ? 1 : 0;
          int T;
          half_decode(q - C * hc, Nc, lgc, T, J, K);
          I = 2 * T + ((J + K + C) & 1);
        }
        // fine red point (i, j, k) at half-index (i >> 1) + (N/2)(j + N k)
        const int t0 = I, tm = wrapi(2 * I - 1, N) >> 1;   // x-offsets 0 and -1 (+1 shares t0)
        const int j0 = 2 * J, jm = wrapi(j0 - 1, N), jp = j0 + 1;
        const int k0 = 2 * K, km = wrapi(k0 - 1, N), kp = k0 + 1;
        const int rj0 = hN * j0, rjm = hN * jm, rjp = hN * jp;
        const int rk0 = NhN * k0, rkm = NhN * km, rkp = NhN * kp;
        const long long s12 = ((r[rk0 + rjm + tm] + r[rk0 + rjm + t0]) + (r[rk0 + rjp + tm] + r[rk0 + rjp + t0])) +
                              ((r[rkm + rj0 + tm] + r[rkm + rj0 + t0]) + (r[rkp + rj0 + tm] + r[rkp + rj0 + t0])) +
                              ((r[rkm + rjm + t0] + r[rkm + rjp + t0]) + (r[rkp + rjm + t0] + r[rkp + rjp + t0]));
        const long long v = div2k(4 * r[rk0 + rj0 + t0] + s12, 3);
        bc[q] = v;
        if (!coarsest && q < (nc3 >> 1)) xc[q] = div6(-v);
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
    }
    // ---- coarsest (natural order): x = M^+ b, the FP64 product with the
    // pseudo-inverse kernel (stored as -6 M^+), exact warp sums, one warp per point
    {
      const int Nc = g.Nl[g.L - 1], NNc = Nc * Nc, nc3 = Nc * NNc;
      const long long* bc = B + g.off[g.L - 1];
      long long* xc = X + g.off[g.L - 1];
      const int lane = threadIdx.x & 31;
      const int wid = tid >> 5, nwarps = stride >> 5;
      for (int p = wid; p < nc3; p += nwarps) {
        const int pk = p / NNc, pj = (p - pk * NNc) / Nc, pi = p - pk * NNc - pj * Nc;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int u = 0;
        for (int q = lane; q < nc3; q += 32, ++u) {
          const int qk = q / NNc, qj = (q - qk * NNc) / Nc, qi = q - qk * NNc - qj * Nc;
          const int d = wrapi(pi - qi, Nc) + Nc * (wrapi(pj - qj, Nc) + Nc * wrapi(pk - qk, Nc));
          acc[u & 3] = fma(g.gker[d], fix_to_dbl(bc[q], 1075), acc[u & 3]);
        }
        long long S;
        int E;
        warp_dsum_fix((acc[0] + acc[1]) + (acc[2] + acc[3]), S, E);
        if (lane == 0) {
          const double v = fix_to_dbl(S, E) * (-1.0 / 6.0);
          const bool big = !(fabs(v) < 0x1p58);
          ovf = ovf || big;
          xc[p] = big ? 0 : round_scaled(v, 0);
        }
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
    }
    // ---- up: prolong (black points), smooth; the last black half-sweep on
    // level 0 also takes the black points' residual (the rounding of the
    // division, at most 3 units) into the stopping test
    for (int l = g.L - 2; l >= 0; --l) {
      const int N = g.Nl[l], lg = g.lg[l], half = (N * N * N) >> 1;
      const int Nc = g.Nl[l + 1];
      const bool csplit = l + 1 < g.L - 1;
      long long* xr = l ? X + g.off[l] : e_red;
      long long* xb = l ? xr + half : e_blk;
      const long long* b = B + g.off[l];
      const long long* xc = X + g.off[l + 1];
      for (int h = tid; h < half; h += stride) {
        int t, j, k;
        half_decode(h, N, lg, t, j, k);
        const int i = 2 * t + ((j + k + 1) & 1);
        const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
        const int odd = (i & 1) + (j & 1) + (k & 1);
        long long e;
        if (odd == 1) {
          const int c0 = store_index(i0, j0, k0, Nc, csplit);
          const int c1 = (i & 1) ? store_index(wrapi(i0 + 1, Nc), j0, k0, Nc, csplit)
                       : (j & 1) ? store_index(i0, wrapi(j0 + 1, Nc), k0, Nc, csplit)
                                 : store_index(i0, j0, wrapi(k0 + 1, Nc), Nc, csplit);
          e = div2k(xc[c0] + xc[c1], 1);
        } else {
          const int i1 = wrapi(i0 + 1, Nc), j1 = wrapi(j0 + 1, Nc), k1 = wrapi(k0 + 1, Nc);
          e = div2k(((xc[store_index(i0, j0, k0, Nc, csplit)] + xc[store_index(i1, j0, k0, Nc, csplit)]) +
                     (xc[store_index(i0, j1, k0, Nc, csplit)] + xc[store_index(i1, j1, k0, Nc, csplit)])) +
                        ((xc[store_index(i0, j0, k1, Nc, csplit)] + xc[store_index(i1, j0, k1, Nc, csplit)]) +
                         (xc[store_index(i0, j1, k1, Nc, csplit)] + xc[store_index(i1, j1, k1, Nc, csplit)])),
                    3);
        }
        xb[h] += e;
      }
      if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      for (int t = 0; t < g.nu2; ++t) {
        half_sweep_i(xr, xb, b, N, lg, 0, tid, stride);
        if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
        if (l == 0 && t == g.nu2 - 1) {
          if ((N & 3) == 0) {
#pragma unroll 2
            for (int h0 = 2 * tid; h0 < half; h0 += 2 * stride) {
              int t0, j, k;
              half_decode(h0, N, lg, t0, j, k);
              long long s0, s1;
              nbr6_pair(xr, h0, t0, j, k, (j + k + 1) & 1, N, s0, s1);
              const longlong2 bv = ld2(b + half + h0);
              const long long v0 = s0 - bv.x, v1 = s1 - bv.y;
              const long long e0 = div6(v0), e1 = div6(v1);
              st2(xb + h0, e0, e1);
              rmax = max(rmax, max(iabs(6 * e0 - v0), iabs(6 * e1 - v1)));
            }
          } else {
#pragma unroll 2
            for (int h = tid; h < half; h += stride) {
              int tt, j, k;
              half_decode(h, N, lg, tt, j, k);
              const long long v = nbr6s(xr, h, tt, j, k, (j + k + 1) & 1, N) - b[half + h];
              const long long ev = div6(v);
              xb[h] = ev;
              rmax = max(rmax, iabs(6 * ev - v));
            }
          }
        } else {
          half_sweep_i(xr, xb, b, N, lg, 1, tid, stride);
        }
        if (!grid_barrier(a.bar, bar_epoch, a.rec)) return;
      }
    }
    ++it;
    fresh = false;
    // ---- the stopping test (Eq. res_poisson_maze) on max |r|, r = b - M E at
    // red points (exact)
    // (and the sum of E, exact per thread: at most 2 half0 / threads terms below 2^54)
    // The same pass also makes the red half-sweep that the next V-cycle
    // would start with (it reads the same black neighbours and right-hand
    // side) into the spare red array; if the solve goes on, the two red
    // arrays swap roles and the next V-cycle skips that half-sweep. The
    // iterates are unchanged; a pass and a grid barrier per V-cycle go.
    {
      long long es = 0;
      if ((N0 & 3) == 0) {
#pragma unroll 2
        for (int h0 = 2 * tid; h0 < half0; h0 += 2 * stride) {
          int t0, j, k;
          half_decode(h0, N0, lg0, t0, j, k);
          long long s0, s1;
          nbr6_pair(e_blk, h0, t0, j, k, (j + k) & 1, N0, s0, s1);
          const longlong2 er = ld2(e_red + h0), eb = ld2(e_blk + h0), bv = ld2(b_red + h0);
          rmax = max(rmax, max(iabs(bv.x - s0 + 6 * er.x), iabs(bv.y - s1 + 6 * er.y)));
          es += (er.x + er.y) + (eb.x + eb.y);
          if (spec) st2(r_red0 + h0, div6(s0 - bv.x), div6(s1 - bv.y));
        }
      } else {
#pragma unroll 2
        for (int h = tid; h < half0; h += stride) {
          int t, j, k;
          half_decode(h, N0, lg0, t, j, k);
          const long long s0 = nbr6s(e_blk, h, t, j, k, (j + k) & 1, N0);
          rmax = max(rmax, iabs(b_red[h] - s0 + 6 * e_red[h]));
          es += e_red[h] + e_blk[h];
          if (spec) r_red0[h] = div6(s0 - b_red[h]);
        }
      }
      const double v[3] = {fix_to_dbl((long long)rmax, 1075), ovf ? 1.0 : 0.0, fix_to_dbl(es, 1075)};
      const bool mm[3] = {true, true, false};
      double t[3];
      if (!grid_reduce<3>(v, mm, a.recs, ++epoch, a.rec, t)) return;
      rmax = 0;
      esum = t[2];
      if (t[1] != 0.0) {
        res = __longlong_as_double(0x7ff0000000000000LL);   // overflow: reported as non-finite
        break;
      }
      res = t[0] * __longlong_as_double((long long)(1023 - F) << 52);
      // a residual 20 bits below the scale (a solve from a cold start): apply E
      // to y, keep the exact residual r = b - M E at every point as the new
      // right-hand side, rescaled, and start again from E = 0
      const int sft = t[0] > 0.0 ? (H - 1) - (dbl_exp(t[0]) - 1023) : 0;
      red_done = false;
      if (!(res < a.tol) && it < a.max_iter && !(sft >= 20 && F + sft <= kMaxScale) && spec) {
        // the solve goes on without a restart: the red half-sweep above is
        // the next V-cycle's first (all threads take the same decision)
        long long* const tmp = e_red;
        e_red = r_red0;
        r_red0 = tmp;
        red_done = true;
      }
      if (!(res < a.tol) && it < a.max_iter && sft >= 20 && F + sft <= kMaxScale) {
        const int E = 1075 - F;
        double ys = 0.0;
        for (int h = tid; h < half0; h += stride) {
          int t0, j, k;
          half_decode(h, N0, lg0, t0, j, k);
          const int p = (j + k) & 1;
          const long long er = e_red[h], eb = e_blk[h];
          const long long rr = b_red[h] - nbr6s(e_blk, h, t0, j, k, p, N0) + 6 * er;
          const long long rb = b_blk[h] - nbr6s(e_red, h, t0, j, k, 1 - p, N0) + 6 * eb;
          b_red[h] = shl(rr, sft);
          b_blk[h] = shl(rb, sft);
          double2* yp = reinterpret_cast<double2*>(y + 2 * t0 + N0 * (j + N0 * k));
          double2 yv = *yp;
          const double dr = fix_to_dbl(er, E), db = fix_to_dbl(eb, E);
          yv.x += p ? db : dr;
          yv.y += p ? dr : db;
          *yp = yv;
          ys += yv.x + yv.y;
        }
        const double v1[1] = {ys};
        const bool ms[1] = {false};
        double t1[1];
        if (!grid_reduce<1>(v1, ms, a.recs, ++epoch, a.rec, t1)) return;   // (also the barrier before E = 0)
        ysum0 = t1[0];
        F += sft;
        fresh = true;
      }
    }
  }
  // (the last grid reduction above orders every write of E before S6's reads)
  // ---- y + E 2^-F (after a V-cycle since the last restart) and S6; the mean
  // of y from the sums; half-index h covers the points i = 2t, 2t + 1 of its row
  const bool apply = it > 0 && !fresh;
  const int Ey = 1075 - F;
  const double ysum = apply ? ysum0 + esum * __longlong_as_double((long long)(1023 - F) << 52) : ysum0;
  const double ybar = ysum * a.inv_n;
  for (int h = tid; h < half0; h += stride) {
    int t0, j, k;
    half_decode(h, N0, lg0, t0, j, k);
    const int p = (j + k) & 1;
    const int m = 2 * t0 + N0 * (j + N0 * k);
    double2 yv = *reinterpret_cast<const double2*>(y + m);
    if (apply) {
      const double dr = fix_to_dbl(e_red[h], Ey), db = fix_to_dbl(e_blk[h], Ey);
      yv.x += p ? db : dr;
      yv.y += p ? dr : db;
    }
    yv.x -= ybar;
    yv.y -= ybar;
    *reinterpret_cast<double2*>(y + m) = yv;
    double2 ph = *reinterpret_cast<const double2*>(a.phi_out + m);
    ph.x = fma(-a.c_phi, yv.x, ph.x);
    ph.y = fma(-a.c_phi, yv.y, ph.y);
    *reinterpret_cast<double2*>(a.phi_out + m) = ph;
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

// Registers per thread of the solve kernel (for sharing SMs with another kernel).
int mgfix_regs() {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_mgfix_solve) != cudaSuccess) return 64;
  return fa.numRegs;
}

// H of the fixed-point scale for a finest edge N: 58 - 2 ceil(log2 N).
int mgfix_headroom(int N) {
  int c = 0;
  while ((1 << c) < N) ++c;
  return 58 - 2 * c;
}

int mgfix_blocks(int n_points) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = mg_threads(n_points);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mgfix_solve, threads, 0);
  if (per_sm < 1) per_sm = 1;
  int want = (n_points + threads - 1) / threads;
  int cap = sms * per_sm;
  if (cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
  return want < cap ? want : cap;
}

// threads = 0: mg_threads(n); otherwise that many per block (at most
// kMgThreads; fewer leave room on each SM for a kernel that runs beside).
cudaError_t launch_mgfix_solve(const SolveArgs& a, const MgArgs& g, int blocks, int threads, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads > 0 ? threads : mg_threads(a.n));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mgfix_solve, a, g, mgfix_headroom(a.N));
}

}  // namespace maze
