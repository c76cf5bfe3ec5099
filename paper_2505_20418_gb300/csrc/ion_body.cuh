// Device bodies of the ion-side steps of a MaZe step, shared by the
// single-box kernels (maze_ions.cu) and the batched step kernel:
//   S1 half kick + drift, S3 charge spreading (Eq. A11 weights), S2 cell list,
//   S7 gather of Eq. F_nostra, S8 Tosi-Fumi pairs, S9 half kick and energies.
#pragma once
#include <math.h>

#include "maze_internal.cuh"
#include "df_arith.cuh"

namespace maze {

// B-spline weights of one axis for an ion at grid coordinate u (Sec. II.A).
// The support starts at node floor(u) - (P/2 - 1); t = u - floor(u).
// P = 2: linear B-spline (1 - t, t).
// P = 4: cubic B-spline ((1-t)^3, 3t^3 - 6t^2 + 4, -3t^3 + 3t^2 + 3t + 1, t^3) / 6.
// Split u into the first support node and the fractional offset t.
__device__ __forceinline__ int axis_split(double u, int P, int N, double& t) {
  const long long fl = floor_ll(u);   // (integer pipe; |u| < 2N)
  t = u - fix_to_dbl(fl, 1075);
  int first = (int)fl - (P / 2 - 1);
  if (first < 0) first += N;
  if (first >= N) first -= N;
  return first;
}

// The P weights at fractional offset t (R = double, or float in mixed mode);
// for P = 2 the two unused slots are zero.
template <typename R>
__device__ __forceinline__ void bspline_weights(R t, int P, R* w) {
  if (P == 2) {
    w[0] = R(1) - t;
    w[1] = t;
    w[2] = R(0);
    w[3] = R(0);
  } else {
    const R t2 = t * t, t3 = t2 * t;
    const R s = R(1) - t;
    const R sixth = R(1) / R(6);
    w[0] = s * s * s * sixth;
    w[1] = (R(3) * t3 - R(6) * t2 + R(4)) * sixth;
    w[2] = (R(-3) * t3 + R(3) * t2 + R(3) * t + R(1)) * sixth;
    w[3] = t3 * sixth;
  }
}

// d w_a / dt of the weights above (the estimator of Eq. F_Benoit); for
// P = 4: (-(1-t)^2, 3t^2 - 4t, -3t^2 + 2t + 1, t^2) / 2, for P = 2: (-1, 1).
template <typename R>
__device__ __forceinline__ void bspline_dweights(R t, int P, R* d) {
  if (P == 2) {
    d[0] = R(-1);
    d[1] = R(1);
    d[2] = R(0);
    d[3] = R(0);
  } else {
    const R s = R(1) - t;
    const R half = R(1) / R(2);
    d[0] = -s * s * half;
    d[1] = (R(3) * t * t - R(4) * t) * half;
    d[2] = (R(-3) * t * t + R(2) * t + R(1)) * half;
    d[3] = t * t * half;
  }
}

__device__ __forceinline__ int wrap_idx(int a, int N) { return a >= N ? a - N : a; }

// Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC 2011): each
// round multiplies words 0 and 2 by the Philox constants, mixes the high and
// low halves of the products with words 1 and 3 and the round key; the key
// advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// OVRVO's O step for ion i (Sivak, Chodera, Crooks 2013): v <- a v + sd xi,
// three standard normals by the Box-Muller transform of the four uniforms
// u = (x + 1/2) 2^-32 of one Philox block with counter (i, step, stage, 0).
__device__ __forceinline__ void o_step(const LangevinArgs& o, int i, int t, unsigned step, unsigned stage,
                                       double& vx, double& vy, double& vz) {
  const uint4 x = philox4x32_10(make_uint4((unsigned)i, step, stage, 0u), o.key0, o.key1);
  const double s32 = 2.3283064365386963e-10;   // 2^-32
  const double u0 = ((double)x.x + 0.5) * s32, u1 = ((double)x.y + 0.5) * s32;
  const double u2 = ((double)x.z + 0.5) * s32, u3 = ((double)x.w + 0.5) * s32;
  const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
  double s1, c1, s3, c3;
  sincospi(2.0 * u1, &s1, &c1);
  sincospi(2.0 * u3, &s3, &c3);
  const double sd = t ? o.sd1 : o.sd0;
  vx = o.a * vx + sd * (r01 * c1);
  vy = o.a * vy + sd * (r01 * s1);
  vz = o.a * vz + sd * (r23 * c3);
}

// A position wrapped into [0, L) exactly as maze_set wraps it on the host
// (the same operations: an in-box value unchanged, else x - L floor(x / L)).
__device__ __forceinline__ double wrap_set(double x, double L) {
  if (x >= 0.0 && x < L) return x;
  x -= L * floor(x / L);
  if (x < 0.0) x += L;
  if (x >= L) x = 0.0;
  return x;
}

__device__ __forceinline__ double wrap_pos(double x, double L, double inv_L) {
  const long long k = floor_ll(x * inv_L);   // (integer pipe; 0 for a position already in the box)
  if (k != 0) x -= L * fix_to_dbl(k, 1075);
  if (x < 0.0) x += L;
  if (x >= L) x -= L;
  return x;
}

// S1 for ion i: Verlet half kick and drift (when a.do_move), the FP32 copy,
// the cell count and the B-spline weights of the new position (stored: the
// spread and the gather of the same step reuse them).
__device__ __forceinline__ void move_ion(const IonArgs& a, int i) {
  const int N = a.N, P = a.P;
  {
    // (maze_step_io's exchange: this step's positions and velocities straight
    // from the caller's pinned [n][3] arrays, or the context's stage; the
    // positions wrapped as maze_set wraps them)
    const double* pin = a.io ? a.io->pos_in + 3 * (size_t)i : nullptr;
    const double* vin = a.io ? a.io->vel_in + 3 * (size_t)i : nullptr;
    double x = pin ? wrap_set(pin[0], a.L) : a.pos[i], y = pin ? wrap_set(pin[1], a.L) : a.pos[a.n + i],
           z = pin ? wrap_set(pin[2], a.L) : a.pos[2 * a.n + i];
    const int t = a.type[i];
    if (pin && !a.do_move) {
      a.pos[i] = x;
      a.pos[a.n + i] = y;
      a.pos[2 * a.n + i] = z;
      a.vel[i] = vin[0];
      a.vel[a.n + i] = vin[1];
      a.vel[2 * a.n + i] = vin[2];
    }
    if (a.do_move) {
      const double kick = t ? a.kick1 : a.kick0;
      double vx = vin ? vin[0] : a.vel[i], vy = vin ? vin[1] : a.vel[a.n + i], vz = vin ? vin[2] : a.vel[2 * a.n + i];
      if (a.ou.on) o_step(a.ou, i, t, (unsigned)a.rec->step, 0u, vx, vy, vz);
      vx += kick * a.force[i];
      vy += kick * a.force[a.n + i];
      vz += kick * a.force[2 * a.n + i];
      a.vel[i] = vx;
      a.vel[a.n + i] = vy;
      a.vel[2 * a.n + i] = vz;
      x = wrap_pos(x + a.dt * vx, a.L, a.inv_L);
      y = wrap_pos(y + a.dt * vy, a.L, a.inv_L);
      z = wrap_pos(z + a.dt * vz, a.L, a.inv_L);
      a.pos[i] = x;
      a.pos[a.n + i] = y;
      a.pos[2 * a.n + i] = z;
    }
    // every index below comes from a position in [0, L): a position that is
    // not (NaN, or so large that the wrap lost it) is replaced by the box
    // origin and the step is marked non-finite, so no index can leave its
    // array and the next step does not run
    if (!(x >= 0.0 && x < a.L && y >= 0.0 && y < a.L && z >= 0.0 && z < a.L)) {
      x = y = z = 0.0;
      atomicCAS(&a.rec->status, MAZE_OK, MAZE_ERR_NONFINITE);
    }
    const double Q = t ? a.charge1 : a.charge0;
    a.pos32[i] = make_float4(dbl_to_flt(x), dbl_to_flt(y), dbl_to_flt(z), dbl_to_flt(Q));
    int cx = 0, cy = 0, cz = 0;
    if (a.nc >= 3) {
      const double cs = a.cell_scale;
      cx = min((int)floor_ll(x * cs), a.nc - 1);   // (x >= 0: floor = truncation)
      cy = min((int)floor_ll(y * cs), a.nc - 1);
      cz = min((int)floor_ll(z * cs), a.nc - 1);
      const int c = cx + a.nc * (cy + a.nc * cz);
      a.cell_of[i] = c;
      atomicAdd(&a.cell_count[c], 1);
    }
    if (a.rel_hi) {
      // position relative to the own cell's corner as a (hi, lo) float pair:
      // pair displacements then need no FP64 arithmetic (mixed precision)
      const double rx = x - cx * a.cell_len, ry = y - cy * a.cell_len, rz = z - cz * a.cell_len;
      const float hx = dbl_to_flt(rx), hy = dbl_to_flt(ry), hz = dbl_to_flt(rz);
      a.rel_hi[i] = make_float4(hx, hy, hz, dbl_to_flt(Q));
      a.rel_lo[i] = make_float4(dbl_to_flt(rx - flt_to_dbl(hx)), dbl_to_flt(ry - flt_to_dbl(hy)),
                                dbl_to_flt(rz - flt_to_dbl(hz)), (float)t);
    }
    double tx, ty, tz;
    const int fx = axis_split(x * a.inv_h, P, N, tx);
    const int fy = axis_split(y * a.inv_h, P, N, ty);
    const int fz = axis_split(z * a.inv_h, P, N, tz);
    if (a.wbuf32) {
      // mixed precision: FP32 weights from the exact fractional offsets
      float w[12];
      bspline_weights<float>(dbl_to_flt(tx), P, w);
      bspline_weights<float>(dbl_to_flt(ty), P, w + 4);
      bspline_weights<float>(dbl_to_flt(tz), P, w + 8);
      float4* gw = reinterpret_cast<float4*>(a.wbuf32 + (size_t)i * 12);
      gw[0] = make_float4(w[0], w[1], w[2], w[3]);
      gw[1] = make_float4(w[4], w[5], w[6], w[7]);
      gw[2] = make_float4(w[8], w[9], w[10], w[11]);
      if (a.wdbuf32) {
        bspline_dweights<float>(dbl_to_flt(tx), P, w);
        bspline_dweights<float>(dbl_to_flt(ty), P, w + 4);
        bspline_dweights<float>(dbl_to_flt(tz), P, w + 8);
        float4* gd = reinterpret_cast<float4*>(a.wdbuf32 + (size_t)i * 12);
        gd[0] = make_float4(w[0], w[1], w[2], w[3]);
        gd[1] = make_float4(w[4], w[5], w[6], w[7]);
        gd[2] = make_float4(w[8], w[9], w[10], w[11]);
      }
    } else {
      double w[12];
      bspline_weights<double>(tx, P, w);
      bspline_weights<double>(ty, P, w + 4);
      bspline_weights<double>(tz, P, w + 8);
      double* gw = a.wbuf + (size_t)i * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) gw[k] = w[k];
      if (a.wdbuf) {
        bspline_dweights<double>(tx, P, w);
        bspline_dweights<double>(ty, P, w + 4);
        bspline_dweights<double>(tz, P, w + 8);
        double* gd = a.wdbuf + (size_t)i * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) gd[k] = w[k];
      }
    }
    a.wbase[i] = make_int4(fx, fy, fz, 0);
  }
}


// S3: q_n += Q W(r - r_n), W = w_x w_y w_z over the P^3 support, one warp per
// ion (lane l takes support points l and l+32), fixed-point atomics. The
// ion's contributions are made to sum exactly to Q 2^50 (the rounding
// remainder, found with an exact warp integer sum, goes to support point 0),
// so a neutral system stays exactly neutral on the grid: the periodic M has
// no inverse on the constant mode, and a rounding net charge would put a floor
// under the constraint residual.
__device__ __forceinline__ void spread_ion(const IonArgs& a, int i, int lane) {
  const int N = a.N, P = a.P, P3 = P * P * P;
  const int4 b = a.wbase[i];
  const double Q = a.type[i] ? a.charge1 : a.charge0;
  long long v[2] = {0, 0};
  int idx[2] = {-1, -1};
  // P is 2 or 4: support index sidx = ia + P (ib + P ic) by shifts; a lane's
  // two points (sidx = lane, lane + 32) share ia and ib, so the FP64 product
  // Q w_a w_b is formed once per lane
  const int lp = P == 4 ? 2 : 1;
  const int ia = lane & (P - 1), ib = (lane >> lp) & (P - 1);
  double qab = 0.0;
  if (!a.wbuf32) {
    const double* w = a.wbuf + (size_t)i * 12;
    qab = Q * w[ia] * w[4 + ib];
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int sidx = lane + 32 * u;
    if (sidx >= P3) continue;
    const int ic = sidx >> (2 * lp);
    if (a.wbuf32) {
      // mixed precision: FP32 products
      const float* w = a.wbuf32 + (size_t)i * 12;
      v[u] = round_scaled_f(dbl_to_flt(Q) * w[8 + ic] * w[4 + ib] * w[ia], 50);   // 2^50 = kQScale
    } else {
      v[u] = round_scaled(qab * a.wbuf[(size_t)i * 12 + 8 + ic], 50);   // 2^50 = kQScale
    }
    const int ix = wrap_idx(b.x + ia, N), iy = wrap_idx(b.y + ib, N), iz = wrap_idx(b.z + ic, N);
    idx[u] = (int)(((size_t)iz * N + iy) * N + ix);
  }
  const long long total = warp_isum(v[0] + v[1]);
  if (lane == 0) v[0] += round_scaled(Q, 50) - total;   // (Q 2^50 exactly, on the integer pipe)
#pragma unroll
  for (int u = 0; u < 2; ++u)
    if (idx[u] >= 0) atomicAdd(&a.qfix[idx[u]], (unsigned long long)v[u]);
}

// S2: cell list. One block scans the counts (and clears them for the next
// step), ions claim slots, then each cell sorts its slots by ion index so the
// pair sums run in a fixed order.

// Exclusive scan of the cell counts by one block of up to 1024 threads.
__device__ __forceinline__ void cell_scan_block(const CellArgs& a) {
  __shared__ int s_part[1024];
  const int T = blockDim.x;
  const int chunk = (a.ncell + T - 1) / T;
  const int lo = min(threadIdx.x * chunk, a.ncell), hi = min(lo + chunk, a.ncell);
  int sum = 0;
  for (int c = lo; c < hi; ++c) sum += a.cell_count[c];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan over the per-thread sums
  for (int o = 1; o < T; o <<= 1) {
    const int v = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s_part[threadIdx.x] - sum;
  for (int c = lo; c < hi; ++c) {
    a.cell_start[c] = run;
    a.cursor[c] = run;
    run += a.cell_count[c];
    a.cell_count[c] = 0;
  }
  if (threadIdx.x == T - 1) a.cell_start[a.ncell] = s_part[T - 1];
  __syncthreads();
}

__device__ __forceinline__ void cell_fill_ion(const CellArgs& a, int i) {
  const int slot = atomicAdd(&a.cursor[a.cell_of[i]], 1);
  a.cell_ions[slot] = i;
}

// One warp sorts cell c: each slot's rank among the cell's (distinct) ion
// indices gives its sorted position (``ids``: kSortCap ints of shared memory).
// Cells larger than that fall back to an insertion sort by lane 0.
constexpr int kSortCap = 256;
__device__ __forceinline__ void cell_sort_one(const CellArgs& a, int c, int lane, int* ids) {
  const int lo = a.cell_start[c], hi = a.cell_start[c + 1], m = hi - lo;
  if (m == 0) return;
  if (m > kSortCap) {
    if (lane == 0)
      for (int u = lo + 1; u < hi; ++u) {
        const int v = a.cell_ions[u];
        int w = u - 1;
        while (w >= lo && a.cell_ions[w] > v) {
          a.cell_ions[w + 1] = a.cell_ions[w];
          --w;
        }
        a.cell_ions[w + 1] = v;
      }
    __syncwarp();
    for (int u = lo + lane; u < hi; u += 32) {
      const int v = a.cell_ions[u];
      a.pos_sorted[u] = a.pos32[v];
      if (a.rel_hi) {
        a.rel_hi_sorted[u] = a.rel_hi[v];
        a.rel_lo_sorted[u] = a.rel_lo[v];
      }
    }
    __syncwarp();
    return;
  }
  for (int u = lane; u < m; u += 32) ids[u] = a.cell_ions[lo + u];
  __syncwarp();
  for (int u = lane; u < m; u += 32) {
    const int v = ids[u];
    int rank = 0;
    for (int k = 0; k < m; ++k) rank += ids[k] < v;
    a.cell_ions[lo + rank] = v;
    a.pos_sorted[lo + rank] = a.pos32[v];
    if (a.rel_hi) {
      a.rel_hi_sorted[lo + rank] = a.rel_hi[v];
      a.rel_lo_sorted[lo + rank] = a.rel_lo[v];
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void tf_pair(const ForceArgs& a, int kind, double r2, double& fr, double& V) {
  // V = A exp(B (s - r)) - C r^-6 - D r^-8 - V(r_c);  fr = -(dV/dr) / r.
  // 1/r from an FP32 seed y0 (relative error e0 below ~2^-22) by one step of
  // Halley's (third-order) iteration for the reciprocal square root:
  // e = 1 - r2 y0^2, y = y0 (1 + e/2 + 3e^2/8); the error falls to ~e0^3, below
  // FP64 rounding. y0^2 is exact in FP64 (a 24-bit significand squared), so no
  // FP64 square root, division or conversion is needed: 5 FP64 operations.
  const double y0 = flt_to_dbl(rsqrtf(dbl_to_flt(r2)));   // conversions on the integer pipe
  const double e = fma(-r2, y0 * y0, 1.0);
  const double ir = fma(y0, e * fma(e, 0.375, 0.5), y0);
  const double r = r2 * ir;
  const double ir2 = ir * ir;
  const double ir4 = ir2 * ir2;
  const double ir6 = ir4 * ir2;
  const double ir8 = ir4 * ir4;
  const double ex = exp_tab(fma(-a.B, r, a.Ec[kind]), a.exp2tab);   // A exp(B (s - r))
  V = ex - fma(a.C[kind], ir6, fma(a.D[kind], ir8, a.Vc[kind]));
  fr = fma(a.B * ex, ir, -ir8 * fma(a.D8[kind], ir2, a.C6[kind]));   // B ex / r - 6C r^-8 - 8D r^-10
}

__device__ __forceinline__ dfl f2df(float2 v) { return {v.x, v.y}; }

// tf_pair in double-float arithmetic on the FP32 pipe (FP64 boxes of the
// once-per-pair kernel): the same quantities from the squared distance r2 as
// a (hi, lo) pair, to ~1e-13 of the terms' magnitudes. 1/r from the FP32
// reciprocal square root of r2's hi part, one FP32 Newton step (y0 within an
// ulp or two, so that the correction below is small and its roundings
// negligible), then one Halley step with e = 1 - r2 y0^2 formed exactly (y0^2
// and r2.h y0^2 as exact products; 1 - r2.h y0^2 is exact, the two lie
// within a factor of 2): y = y0 + y0 e (1/2 + 3e/8); the repulsion
// exp(Ec - B r) by df_exp; V and fr as in tf_pair.
__device__ __forceinline__ void tf_pair_df(const ForceArgs& a, int kind, dfl r2, dfl& fr, dfl& V) {
  const PairDf& k = a.pdf;
  float y0 = rsqrtf(r2.h);
  y0 = __fmul_rn(y0, __fmaf_rn(-0.5f, __fmul_rn(__fmul_rn(r2.h, y0), y0), 1.5f));
  const dfl y2 = df_two_prod(y0, y0);
  const dfl b = df_two_prod(r2.h, y2.h);
  const float bl = __fmaf_rn(r2.l, y2.h, __fmaf_rn(r2.h, y2.l, b.l));
  const float e = __fsub_rn(__fsub_rn(1.f, b.h), bl);
  const dfl ir = df_fast_sum(y0, __fmul_rn(y0, __fmul_rn(e, __fmaf_rn(e, 0.375f, 0.5f))));
  const dfl r = df_mul(r2, ir);
  const dfl ir2 = df_sqr(ir);
  const dfl ir4 = df_sqr(ir2);
  const dfl ir6 = df_mul(ir4, ir2);
  const dfl ir8 = df_sqr(ir4);
  const dfl ex = df_exp(df_add(f2df(k.Ec[kind]), df_neg(df_mul(f2df(k.B), r))), a.exp2tab_f);   // A exp(B (s - r))
  V = df_add(ex, df_neg(df_add(df_mul(f2df(k.C[kind]), ir6), df_add(df_mul(f2df(k.D[kind]), ir8), f2df(k.Vc[kind])))));
  // B ex / r - r^-8 (6C + 8D r^-2)
  fr = df_add(df_mul(df_mul(f2df(k.B), ex), ir),
              df_neg(df_mul(ir8, df_add(df_mul(f2df(k.D8[kind]), ir2), f2df(k.C6[kind])))));
}

// round((h + l) 2^40) as a 64-bit integer for a normalised pair (within one
// unit: each part rounds once). h 2^40 by round_scaled_f; l (|l| <= ulp(h)/2)
// below 2^-18 by the FP32 rounding trick, fma(l, 2^40, 1.5 2^23) leaving the
// nearest integer in the low mantissa bits (2 operations instead of ~15),
// else by round_scaled_f too.
__device__ __forceinline__ long long df_fix40(dfl v) {
  long long lo;
  if (fabsf(v.l) < 0x1p-18f) lo = __float_as_int(__fmaf_rn(v.l, 0x1p40f, 0x1.8p23f)) - 0x4b400000;
  else lo = round_scaled_f(v.l, 40);
  return round_scaled_f(v.h, 40) + lo;
}

// Per-lane pair sums (FP64 mode uses the doubles, mixed the floats).
struct PairSum {
  double fx = 0, fy = 0, fz = 0, v = 0;
  float fxf = 0.f, fyf = 0.f, fzf = 0.f, vf = 0.f;
};

// Tosi-Fumi pair (i, j): minimum image from the FP32 shift and the exact FP64
// displacement, exact cutoff test, FP64 (or FP32 in mixed mode) arithmetic.
__device__ __forceinline__ void pair_add(const ForceArgs& a, int ti, double x, double y, double z, float4 pi32,
                                         int tj, float4 pj, double xj, double yj, double zj, PairSum& ps) {
  const float iL = a.inv_Lf;
  const float sx = rintf((pj.x - pi32.x) * iL), sy = rintf((pj.y - pi32.y) * iL), sz = rintf((pj.z - pi32.z) * iL);
  const double ddx = (xj - x) - flt_to_dbl(sx) * a.L;
  const double ddy = (yj - y) - flt_to_dbl(sy) * a.L;
  const double ddz = (zj - z) - flt_to_dbl(sz) * a.L;
  const int kind = ti + tj;
  const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
  if (r2 >= a.rc2) return;
  double fr, V;
  tf_pair(a, kind, r2, fr, V);
  ps.fx -= fr * ddx;
  ps.fy -= fr * ddy;
  ps.fz -= fr * ddz;
  ps.v += V;
}

// (rj + off) - ri for positions and offset given as hi + lo float pairs,
// each addition made error-free by Knuth's TwoSum: the FP32 result carries
// the displacement to ~1e-7 relative, without FP64 arithmetic.
__device__ __forceinline__ float disp_df(float rih, float ril, float rjh, float rjl, float offh, float offl) {
  const float s = __fadd_rn(rjh, offh);
  const float bb = __fsub_rn(s, rjh);
  const float e1 = __fadd_rn(__fsub_rn(rjh, __fsub_rn(s, bb)), __fsub_rn(offh, bb));
  const float d = __fsub_rn(s, rih);
  const float cc = __fsub_rn(d, s);
  const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(d, cc)), __fsub_rn(-rih, cc));
  return __fadd_rn(d, __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(__fadd_rn(rjl, offl), ril)));
}

// Mixed-precision Tosi-Fumi pair from an FP32 displacement.
__device__ __forceinline__ void pair_f(const ForceArgs& a, int kind, float dx, float dy, float dz, PairSum& ps) {
  const float r2 = dx * dx + dy * dy + dz * dz;
  if (r2 >= a.rc2f) return;
  const float ir = rsqrtf(r2);
  const float r = r2 * ir;
  const float ir2 = ir * ir;
  const float ir6 = ir2 * ir2 * ir2;
  const float ir8 = ir6 * ir2;
  const float ex = a.Af[kind] * expf(a.Bf * (a.sf[kind] - r));
  const float V = ex - a.Cf[kind] * ir6 - a.Df[kind] * ir8 - a.Vcf[kind];
  const float fr = a.Bf * ex * ir - 6.f * a.Cf[kind] * ir8 - 8.f * a.Df[kind] * ir8 * ir2;
  ps.fxf -= fr * dx;
  ps.fyf -= fr * dy;
  ps.fzf -= fr * dz;
  ps.vf += V;
}

// Warp sum of a PairSum into FP64 totals (every lane gets them).
__device__ __forceinline__ void pair_total(const ForceArgs& a, PairSum& ps, double& fx, double& fy, double& fz, double& v) {
  if (a.mixed) {
    for (int o = 16; o > 0; o >>= 1) {
      ps.fxf += __shfl_xor_sync(0xffffffffu, ps.fxf, o);
      ps.fyf += __shfl_xor_sync(0xffffffffu, ps.fyf, o);
      ps.fzf += __shfl_xor_sync(0xffffffffu, ps.fzf, o);
      ps.vf += __shfl_xor_sync(0xffffffffu, ps.vf, o);
    }
    fx = ps.fxf;
    fy = ps.fyf;
    fz = ps.fzf;
    v = ps.vf;
  } else {
    fx = warp_sum(ps.fx);
    fy = warp_sum(ps.fy);
    fz = warp_sum(ps.fz);
    v = warp_sum(ps.v);
  }
}

// FP32 pre-filter: minimum-image distance below the cutoff plus a margin.
__device__ __forceinline__ bool pair_filter(const ForceArgs& a, float4 pi32, float4 pj) {
  const float Lf = a.Lf;
  float dx = pj.x - pi32.x, dy = pj.y - pi32.y, dz = pj.z - pi32.z;
  dx -= rintf(dx * a.inv_Lf) * Lf;
  dy -= rintf(dy * a.inv_Lf) * Lf;
  dz -= rintf(dz * a.inv_Lf) * Lf;
  return dx * dx + dy * dy + dz * dz < a.rc2_filter;
}

// S7 for ion i, one warp: Eq. F_nostra, F = -k_e Q sum_n W (phi_{n+e} -
// phi_{n-e}) / 2h with the weights k_move stored for this position, and
// sum_n W phi_n for the discrete energy. Every lane gets the sums.
__device__ __forceinline__ void gather_el(const ForceArgs& a, int i, int lane, double& gx, double& gy, double& gz,
                                          double& vd) {
  const int N = a.N, P = a.P;
  const int4 first = a.wbase[i];
  const int P3 = P * P * P;
  gx = gy = gz = vd = 0;
  // P is 2 or 4: support index sidx = ia + P (ib + P ic) by shifts; grid
  // indices fit 32 bits (N <= 1024)
  const int lp = P == 4 ? 2 : 1;
  const int NN = N * N;
  if (a.gradw) {
    // Eq. F_Benoit: sum_n grad W phi_n; returned as 2 sum_n (dW/dt) phi_n so
    // that the common prefactor -k_e Q / 2h gives -k_e Q sum_n grad W phi_n
    if (a.mixed) {
      const float* w = a.wbuf32 + (size_t)i * 12;
      const float* d = a.wdbuf32 + (size_t)i * 12;
      const float2* f = reinterpret_cast<const float2*>(a.phi);
      float sx = 0.f, sy = 0.f, sz = 0.f, s0 = 0.f;
      for (int sidx = lane; sidx < P3; sidx += 32) {
        const int ia = sidx & (P - 1), ib = (sidx >> lp) & (P - 1), ic = sidx >> (2 * lp);
        const int ix = wrap_idx(first.x + ia, N), iy = wrap_idx(first.y + ib, N), iz = wrap_idx(first.z + ic, N);
        const float2 c0 = f[iz * NN + iy * N + ix];
        const float ph = c0.x + c0.y;
        const float wyz = w[4 + ib] * w[8 + ic];
        sx += d[ia] * wyz * ph;
        sy += w[ia] * d[4 + ib] * w[8 + ic] * ph;
        sz += w[ia] * w[4 + ib] * d[8 + ic] * ph;
        s0 += w[ia] * wyz * ph;
      }
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      }
      gx = 2.0 * flt_to_dbl(sx);
      gy = 2.0 * flt_to_dbl(sy);
      gz = 2.0 * flt_to_dbl(sz);
      vd = s0;
    } else {
      const double* w = a.wbuf + (size_t)i * 12;
      const double* d = a.wdbuf + (size_t)i * 12;
      for (int sidx = lane; sidx < P3; sidx += 32) {
        const int ia = sidx & (P - 1), ib = (sidx >> lp) & (P - 1), ic = sidx >> (2 * lp);
        const int ix = wrap_idx(first.x + ia, N), iy = wrap_idx(first.y + ib, N), iz = wrap_idx(first.z + ic, N);
        const int at = iz * NN + iy * N + ix;
        double ph;
        if (a.phi_df) {
          const float2 c0 = reinterpret_cast<const float2*>(a.phi)[at];
          ph = flt_to_dbl(c0.x) + flt_to_dbl(c0.y);
        } else {
          ph = a.phi[at];
        }
        const double wyz = w[4 + ib] * w[8 + ic];
        gx += d[ia] * wyz * ph;
        gy += w[ia] * d[4 + ib] * w[8 + ic] * ph;
        gz += w[ia] * w[4 + ib] * d[8 + ic] * ph;
        vd += w[ia] * wyz * ph;
      }
      gx = 2.0 * warp_sum(gx);
      gy = 2.0 * warp_sum(gy);
      gz = 2.0 * warp_sum(gz);
      vd = warp_sum(vd);
    }
    return;
  }
  if (a.mixed) {
    // mixed precision: FP32 weights, differences of the double-float
    // potential in FP32, FP32 sums
    const float* w = a.wbuf32 + (size_t)i * 12;
    const float2* f = reinterpret_cast<const float2*>(a.phi);
    float sx = 0.f, sy = 0.f, sz = 0.f, s0 = 0.f;
    for (int sidx = lane; sidx < P3; sidx += 32) {
      const int ia = sidx & (P - 1), ib = (sidx >> lp) & (P - 1), ic = sidx >> (2 * lp);
      const int ix = wrap_idx(first.x + ia, N), iy = wrap_idx(first.y + ib, N), iz = wrap_idx(first.z + ic, N);
      const float wt = w[ia] * w[4 + ib] * w[8 + ic];
      const int row = iz * NN + iy * N;
      const float2 xp = f[row + (ix == N - 1 ? 0 : ix + 1)], xm = f[row + (ix == 0 ? N - 1 : ix - 1)];
      const float2 yp = f[iz * NN + (iy == N - 1 ? 0 : iy + 1) * N + ix];
      const float2 ym = f[iz * NN + (iy == 0 ? N - 1 : iy - 1) * N + ix];
      const float2 zp = f[(iz == N - 1 ? 0 : iz + 1) * NN + iy * N + ix];
      const float2 zm = f[(iz == 0 ? N - 1 : iz - 1) * NN + iy * N + ix];
      const float2 c0 = f[row + ix];
      sx += wt * ((xp.x - xm.x) + (xp.y - xm.y));
      sy += wt * ((yp.x - ym.x) + (yp.y - ym.y));
      sz += wt * ((zp.x - zm.x) + (zp.y - zm.y));
      s0 += wt * (c0.x + c0.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    }
    gx = sx;
    gy = sy;
    gz = sz;
    vd = s0;
  } else {
    const double* w = a.wbuf + (size_t)i * 12;
    // a lane's support points (sidx = lane, lane + 32) share ia and ib: the
    // FP64 product w_a w_b once per lane (the same association as before)
    const int ia = lane & (P - 1), ib = (lane >> lp) & (P - 1);
    const double wab = w[ia] * w[4 + ib];
    for (int sidx = lane; sidx < P3; sidx += 32) {
      const int ic = sidx >> (2 * lp);
      const int ix = wrap_idx(first.x + ia, N), iy = wrap_idx(first.y + ib, N), iz = wrap_idx(first.z + ic, N);
      const double wt = wab * w[8 + ic];
      const int row = iz * NN + iy * N;
      const int ixp = row + (ix == N - 1 ? 0 : ix + 1), ixm = row + (ix == 0 ? N - 1 : ix - 1);
      const int iyp = iz * NN + (iy == N - 1 ? 0 : iy + 1) * N + ix;
      const int iym = iz * NN + (iy == 0 ? N - 1 : iy - 1) * N + ix;
      const int izp = (iz == N - 1 ? 0 : iz + 1) * NN + iy * N + ix;
      const int izm = (iz == 0 ? N - 1 : iz - 1) * NN + iy * N + ix;
      double px, py, pz, p0;
      if (a.phi_df) {
        // double-float potential: differences of the (hi, lo) pairs in FP32
        const float2* f = reinterpret_cast<const float2*>(a.phi);
        const float2 xp = f[ixp], xm = f[ixm], yp = f[iyp], ym = f[iym], zp = f[izp], zm = f[izm], c0 = f[row + ix];
        px = flt_to_dbl((xp.x - xm.x) + (xp.y - xm.y));
        py = flt_to_dbl((yp.x - ym.x) + (yp.y - ym.y));
        pz = flt_to_dbl((zp.x - zm.x) + (zp.y - zm.y));
        p0 = flt_to_dbl(c0.x) + flt_to_dbl(c0.y);
      } else {
        const double* ph = a.phi;
        px = ph[ixp] - ph[ixm];
        py = ph[iyp] - ph[iym];
        pz = ph[izp] - ph[izm];
        p0 = ph[row + ix];
      }
      gx += wt * px;
      gy += wt * py;
      gz += wt * pz;
      vd += wt * p0;
    }
    // warp totals as exact integer sums on the integer pipe (an FP64
    // shuffle tree would cost 20 FP64 operations per lane and ion)
    gx = warp_dsum(gx);
    gy = warp_dsum(gy);
    gz = warp_dsum(gz);
    vd = warp_dsum(vd);
  }
}

// S9 for ion i (one lane): total force, second half kick, V_work increment
// (Eq. E_nostra, trapezoid rule), and the ion's energy / momentum terms
// 0 KE, 1 V_TF (pairs counted twice), 2 1/2 phi.q, 3 dV_work, 4-6 momentum.
__device__ __forceinline__ void finish_ion(const ForceArgs& a, int i, double gx, double gy, double gz, double vd,
                                           double ftx, double fty, double ftz, double vtf, double (&acc)[7]) {
  const int n = a.n;
  const int t = a.type[i];
  const double Q = t ? a.charge1 : a.charge0;
  const double fe = -MAZE_KE_EV_ANGSTROM * Q * a.inv_2h;
  const double Fex = fe * gx, Fey = fe * gy, Fez = fe * gz;
  const double Fx = Fex + ftx, Fy = Fey + fty, Fz = Fez + ftz;
  double vx = a.vel[i], vy = a.vel[n + i], vz = a.vel[2 * n + i];
  const double m = t ? a.mass1 : a.mass0;
  double dw = 0.0;
  if (a.do_kick) {
    // dV_work = -1/2 (F_el^k + F_el^{k+1}) . dt v_half
    const double ox = a.force_el[i], oy = a.force_el[n + i], oz = a.force_el[2 * n + i];
    dw = -0.5 * a.dt * ((ox + Fex) * vx + (oy + Fey) * vy + (oz + Fez) * vz);
    const double kick = t ? a.kick1 : a.kick0;
    vx += kick * Fx;
    vy += kick * Fy;
    vz += kick * Fz;
    if (a.ou.on) o_step(a.ou, i, t, (unsigned)a.rec->step, 1u, vx, vy, vz);
    a.vel[i] = vx;
    a.vel[n + i] = vy;
    a.vel[2 * n + i] = vz;
  }
  a.force[i] = Fx;
  a.force[n + i] = Fy;
  a.force[2 * n + i] = Fz;
  a.force_el[i] = Fex;
  a.force_el[n + i] = Fey;
  a.force_el[2 * n + i] = Fez;
  acc[0] += a.ke_coef * m * (vx * vx + vy * vy + vz * vz);
  acc[1] += 0.5 * vtf;
  acc[2] += 0.5 * MAZE_KE_EV_ANGSTROM * Q * vd;
  acc[3] += dw;
  acc[4] += m * vx;
  acc[5] += m * vy;
  acc[6] += m * vz;
}

// a step whose solve hit max_iter still completes (forces, energies, step
// count); any other error stops the step
__device__ __forceinline__ bool forces_live(const ForceArgs& a) {
  const int st0 = a.rec->status;
  return *a.gate == 0 && (st0 == MAZE_OK || st0 == MAZE_ERR_NOT_CONVERGED);
}

// S7 + S8 for ion i, one warp: the gather of Eq. F_nostra and the Tosi-Fumi
// pair sums over candidates from global memory (the cell list, or all ions),
// filter survivors queued in ``q`` (64 ints of shared memory per warp) and
// evaluated 32 at a time. Every lane returns r = (gx, gy, gz, vd, Fx, Fy, Fz,
// V_TF). Mixed precision takes this path only for boxes without cells, where
// the (hi, lo) coordinates are relative to the box corner.
__device__ __forceinline__ void forces_ion_warp(const ForceArgs& a, int i, int lane, int* q, double (&r)[8]) {
  const int n = a.n;
  const double x = a.pos[i], y = a.pos[n + i], z = a.pos[2 * n + i];
  const int t = a.type[i];
  double gx, gy, gz, vd;
  gather_el(a, i, lane, gx, gy, gz, vd);
  const float4 pi32 = a.pos32[i];
  float4 rih = make_float4(0.f, 0.f, 0.f, 0.f), ril = rih;
  if (a.mixed) {
    rih = a.rel_hi[i];
    ril = a.rel_lo[i];
  }
  int qn = 0;
  PairSum ps;
  auto eval = [&](int j2) {
    if (a.mixed) {
      // box-relative hi/lo coordinates, minimum image -s L as hi/lo
      const float4 jh = a.rel_hi[j2], jl = a.rel_lo[j2];
      const float sx = rintf((jh.x - rih.x) * a.inv_Lf), sy = rintf((jh.y - rih.y) * a.inv_Lf),
                  sz = rintf((jh.z - rih.z) * a.inv_Lf);
      const float dx = disp_df(rih.x, ril.x, jh.x, jl.x, -sx * a.L_h, -sx * a.L_l);
      const float dy = disp_df(rih.y, ril.y, jh.y, jl.y, -sy * a.L_h, -sy * a.L_l);
      const float dz = disp_df(rih.z, ril.z, jh.z, jl.z, -sz * a.L_h, -sz * a.L_l);
      pair_f(a, t + (int)jl.w, dx, dy, dz, ps);
    } else {
      pair_add(a, t, x, y, z, pi32, a.type[j2], a.pos32[j2], a.pos[j2], a.pos[n + j2], a.pos[2 * n + j2], ps);
    }
  };
  auto offer = [&](int j, float4 pj, bool valid) {
    const bool pass = valid && j != i && pair_filter(a, pi32, pj);
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if (pass) q[qn + __popc(m & ((1u << lane) - 1u))] = j;
    qn += __popc(m);
    __syncwarp();
    if (qn >= 32) {
      eval(q[lane]);
      __syncwarp();
      if (lane < qn - 32) q[lane] = q[32 + lane];
      __syncwarp();
      qn -= 32;
    }
  };
  // candidate slots [lo, hi) in chunks of 32, the next chunk's loads issued
  // before the current chunk is filtered
  auto scan = [&](int lo, int hi, const int* ids, const float4* pp) {
    int u = lo + lane;
    bool v = u < hi;
    int j = v ? (ids ? ids[u] : u) : -1;
    float4 pj = v ? pp[u] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int u0 = lo; u0 < hi; u0 += 32) {
      const int un = u0 + 32 + lane;
      const bool vn = un < hi;
      const int jn = vn ? (ids ? ids[un] : un) : -1;
      const float4 pn = vn ? pp[un] : make_float4(0.f, 0.f, 0.f, 0.f);
      offer(j, pj, v);
      j = jn;
      pj = pn;
      v = vn;
    }
  };
  if (a.nc >= 3) {
    const int nc = a.nc, R = a.reach, S = 2 * R + 1, NB = S * S * S;
    const int c = a.cell_of[i];
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    for (int base = 0; base < NB; base += 32) {
      int rlo = 0, rhi = 0;
      const int t = base + lane;
      if (t < NB) {
        const int dx = t % S - R, dy = (t / S) % S - R, dz = t / (S * S) - R;
        const int cc = (cx + dx + nc) % nc + nc * ((cy + dy + nc) % nc + nc * ((cz + dz + nc) % nc));
        rlo = a.cell_start[cc];
        rhi = a.cell_start[cc + 1];
      }
      const int cnt = min(32, NB - base);
      for (int tt = 0; tt < cnt; ++tt) {
        const int lo = __shfl_sync(0xffffffffu, rlo, tt), hi = __shfl_sync(0xffffffffu, rhi, tt);
        scan(lo, hi, a.cell_ions, a.pos_sorted);
      }
    }
  } else {
    scan(0, n, nullptr, a.pos32);
  }
  if (lane < qn) eval(q[lane]);
  double ftx, fty, ftz, vtf;
  pair_total(a, ps, ftx, fty, ftz, vtf);
  r[0] = gx;
  r[1] = gy;
  r[2] = gz;
  r[3] = vd;
  r[4] = ftx;
  r[5] = fty;
  r[6] = ftz;
  r[7] = vtf;
}

// S7 + S8 for the ions of slice s (of ``split``) of cell c, one block of kW
// warps: the candidates of the (2 reach + 1)^3 neighbour cells are staged in
// shared memory in chunks; each warp takes ions of the slice, queues filter survivors and
// evaluates them 32 at a time. Pair sums per ion accumulate in shared memory
// in chunk order, so the result does not depend on kW or the slicing. FP64
// mode stages FP64 positions; mixed precision stages the cell-relative hi/lo
// floats with the neighbour cell's offset folded in, so displacements are
// exact FP32 sums. The slice's ions are finished one per thread into acc.
constexpr int kPairChunk = 864;
constexpr int kCellGroup = 64;
constexpr int kMaxNbr = 125;   // (2 reach + 1)^3 for reach <= 2
template <int kW>
struct CellSmem {
  float4 p[kPairChunk];                          // FP32 position (filter) / hi part
  __align__(16) double xyz[3][kPairChunk];       // FP64 positions; mixed: lo parts in rows 0-1
  int j[kPairChunk];
  int lo[kMaxNbr], cum[kMaxNbr + 1];
  double f[kCellGroup][8];                       // pair sums, then gather sums
  int queue[kW][2 * 64];                         // one 64-entry queue per ion a warp filters at once
};

// Mixed precision: the warp's home ions g0 + G tk + (0..G-1) for tasks tk =
// warp, warp + kW, ... each filtered against every staged candidate of the
// chunk with one candidate load per lane and one ballot per ion; per ion the
// queue, the 32-pair batches and the pair sums are those of the one-ion
// loop, so the result does not depend on G. q: G queues of 64 entries.
template <int G>
__device__ __forceinline__ void scan_ions_mixed(const ForceArgs& a, const float4* sp, const float4* sl, const int* sj,
                                                int* q, int g0, int gn, int len, int warp, int kW, int lane,
                                                double (*f)[8]) {
  for (int tk = warp; G * tk < gn; tk += kW) {
    float4 ph[G], pl[G];
    int ty[G], self[G], qn[G];
    bool has[G];
    PairSum ps[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      has[u] = G * tk + u < gn;
      const int sl_ = g0 + (has[u] ? G * tk + u : G * tk);
      ph[u] = a.rel_hi_sorted[sl_];
      pl[u] = a.rel_lo_sorted[sl_];
      ty[u] = a.type[a.cell_ions[sl_]];
      self[u] = sl_;
      qn[u] = 0;
    }
    auto evalm = [&](int u, int e2) {
      const float4 h = sp[e2], l = sl[e2];
      const float dx = disp_df(ph[u].x, pl[u].x, h.x, l.x, 0.f, 0.f);
      const float dy = disp_df(ph[u].y, pl[u].y, h.y, l.y, 0.f, 0.f);
      const float dz = disp_df(ph[u].z, pl[u].z, h.z, l.z, 0.f, 0.f);
      pair_f(a, ty[u] + (int)l.w, dx, dy, dz, ps[u]);
    };
    for (int e0 = 0; e0 < len; e0 += 32) {
      const int e = e0 + lane;
      const bool in = e < len;
      const int je = in ? sj[e] : -1;
      const float4 h = in ? sp[e] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < G; ++u) {
        bool pass = false;
        if (in && has[u] && je != self[u]) {
          const float dx = h.x - ph[u].x, dy = h.y - ph[u].y, dz = h.z - ph[u].z;
          pass = dx * dx + dy * dy + dz * dz < a.rc2_filter;
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) q[64 * u + qn[u] + __popc(m & ((1u << lane) - 1u))] = e;
        qn[u] += __popc(m);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < G; ++u)
        if (qn[u] >= 32) {
          evalm(u, q[64 * u + lane]);
          __syncwarp();
          if (lane < qn[u] - 32) q[64 * u + lane] = q[64 * u + 32 + lane];
          __syncwarp();
          qn[u] -= 32;
        }
    }
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (lane < qn[u]) evalm(u, q[64 * u + lane]);
    __syncwarp();
#pragma unroll
    for (int u = 0; u < G; ++u) {
      double fx, fy, fz, v;
      pair_total(a, ps[u], fx, fy, fz, v);
      if (lane == 0 && has[u]) {
        double* r = f[G * tk + u];
        r[4] += fx;
        r[5] += fy;
        r[6] += fz;
        r[7] += v;
      }
    }
  }
}

// kPairsOnly: S8 alone (the pair sums of each ion to a.pair_out, 4 doubles
// per ion: force x, y, z and energy); the gather and the finishing then run
// in k_gather_finish, with the same per-ion arithmetic.
template <int kW, bool kPairsOnly = false>
__device__ __forceinline__ void forces_cell_slice(const ForceArgs& a, int c, int s, int split, CellSmem<kW>& sm,
                                                  double (&acc)[7]) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int n = a.n, nc = a.nc, R = a.reach, S = 2 * R + 1, NB = S * S * S;
  __syncthreads();   // the previous slice's readers of sm are done
  const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
  for (int t = threadIdx.x; t < NB; t += blockDim.x) {
    const int dx = t % S - R, dy = (t / S) % S - R, dz = t / (S * S) - R;
    const int cc = (cx + dx + nc) % nc + nc * ((cy + dy + nc) % nc + nc * ((cz + dz + nc) % nc));
    sm.lo[t] = a.cell_start[cc];
    sm.cum[t + 1] = a.cell_start[cc + 1] - a.cell_start[cc];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.cum[0] = 0;
    for (int t = 0; t < NB; ++t) sm.cum[t + 1] += sm.cum[t];
  }
  __syncthreads();
  const int total = sm.cum[NB];
  const int c0 = a.cell_start[c], cn = a.cell_start[c + 1] - c0;
  const int per = (cn + split - 1) / split;
  const int clo = c0 + min(cn, s * per), chi = c0 + min(cn, (s + 1) * per);
  float4* s_l = reinterpret_cast<float4*>(&sm.xyz[0][0]);   // mixed: lo parts (+ type in w)
  for (int g0 = clo; g0 < chi; g0 += kCellGroup) {
    const int gn = min(kCellGroup, chi - g0);
    for (int e = threadIdx.x; e < gn * 8; e += blockDim.x) sm.f[e >> 3][e & 7] = 0.0;
    for (int ch0 = 0; ch0 < total; ch0 += kPairChunk) {
      const int len = min(kPairChunk, total - ch0);
      __syncthreads();
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int tt = ch0 + e;
        // neighbour cell k of candidate tt: the last k with cum[k] <= tt
        int k = 0;
        for (int step = 64; step > 0; step >>= 1)
          if (k + step < NB && sm.cum[k + step] <= tt) k += step;
        const int slot = sm.lo[k] + (tt - sm.cum[k]);
        if (a.mixed) {
          // neighbour offset (dx, dy, dz) * cell_len folded into hi/lo
          // (reach 1, the usual case: constant divisors)
          const int kx = S == 3 ? k % 3 : k % S, ky = S == 3 ? (k / 3) % 3 : (k / S) % S,
                    kz = S == 3 ? k / 9 : k / (S * S);
          const float ox = (float)(kx - R), oy = (float)(ky - R), oz = (float)(kz - R);
          const float4 h = a.rel_hi_sorted[slot], l = a.rel_lo_sorted[slot];
          float4 hh, ll;
          // TwoSum of each coordinate with the offset's hi part
          const float sx = __fadd_rn(h.x, ox * a.cell_len_h), sy = __fadd_rn(h.y, oy * a.cell_len_h),
                      sz = __fadd_rn(h.z, oz * a.cell_len_h);
          const float bx = __fsub_rn(sx, h.x), by = __fsub_rn(sy, h.y), bz = __fsub_rn(sz, h.z);
          const float ex = __fadd_rn(__fsub_rn(h.x, __fsub_rn(sx, bx)), __fsub_rn(ox * a.cell_len_h, bx));
          const float ey = __fadd_rn(__fsub_rn(h.y, __fsub_rn(sy, by)), __fsub_rn(oy * a.cell_len_h, by));
          const float ez = __fadd_rn(__fsub_rn(h.z, __fsub_rn(sz, bz)), __fsub_rn(oz * a.cell_len_h, bz));
          hh = make_float4(sx, sy, sz, h.w);
          ll = make_float4(__fadd_rn(ex, __fadd_rn(l.x, ox * a.cell_len_l)), __fadd_rn(ey, __fadd_rn(l.y, oy * a.cell_len_l)),
                           __fadd_rn(ez, __fadd_rn(l.z, oz * a.cell_len_l)), l.w);
          sm.p[e] = hh;
          s_l[e] = ll;
          sm.j[e] = slot;
        } else {
          const int j = a.cell_ions[slot];
          sm.j[e] = j;
          sm.p[e] = a.pos_sorted[slot];
          sm.xyz[0][e] = a.pos[j];
          sm.xyz[1][e] = a.pos[n + j];
          sm.xyz[2][e] = a.pos[2 * n + j];
        }
      }
      __syncthreads();
      // mixed precision with at least two ions per warp: a warp filters each
      // staged candidate against two home ions at once (one load, two
      // ballots); each ion keeps its own queue, batches and sums, so its
      // result is that of the one-ion loop below (three ions per warp were
      // slower: 1.38 against 1.25 ms at 512000 ions)
      const int per_warp = (gn + kW - 1) / kW;
      const bool two = a.mixed && per_warp >= 2;
      if (two) scan_ions_mixed<2>(a, sm.p, s_l, sm.j, sm.queue[warp], g0, gn, len, warp, kW, lane, sm.f);
      for (int gi = warp; gi < (two ? 0 : gn); gi += kW) {
        const int islot = g0 + gi;
        const int i = a.cell_ions[islot];
        const double x = a.pos[i], y = a.pos[n + i], z = a.pos[2 * n + i];
        const int t = a.type[i];
        float4 pi32, ril = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.mixed) {
          pi32 = a.rel_hi_sorted[islot];
          ril = a.rel_lo_sorted[islot];
        } else {
          pi32 = a.pos_sorted[islot];
        }
        const int self = a.mixed ? islot : i;
        int* q = sm.queue[warp];
        int qn = 0;
        PairSum ps;
        auto eval = [&](int e2) {
          if (a.mixed) {
            const float4 h = sm.p[e2], l = s_l[e2];
            const float dx = disp_df(pi32.x, ril.x, h.x, l.x, 0.f, 0.f);
            const float dy = disp_df(pi32.y, ril.y, h.y, l.y, 0.f, 0.f);
            const float dz = disp_df(pi32.z, ril.z, h.z, l.z, 0.f, 0.f);
            pair_f(a, t + (int)l.w, dx, dy, dz, ps);
          } else {
            pair_add(a, t, x, y, z, pi32, a.type[sm.j[e2]], sm.p[e2], sm.xyz[0][e2], sm.xyz[1][e2], sm.xyz[2][e2], ps);
          }
        };
        for (int e0 = 0; e0 < len; e0 += 32) {
          const int e = e0 + lane;
          bool pass = false;
          if (e < len && sm.j[e] != self) {
            if (a.mixed) {
              const float4 h = sm.p[e];
              const float dx = h.x - pi32.x, dy = h.y - pi32.y, dz = h.z - pi32.z;
              pass = dx * dx + dy * dy + dz * dz < a.rc2_filter;
            } else {
              pass = pair_filter(a, pi32, sm.p[e]);
            }
          }
          const unsigned m = __ballot_sync(0xffffffffu, pass);
          if (pass) q[qn + __popc(m & ((1u << lane) - 1u))] = e;
          qn += __popc(m);
          __syncwarp();
          if (qn >= 32) {
            eval(q[lane]);
            __syncwarp();
            if (lane < qn - 32) q[lane] = q[32 + lane];
            __syncwarp();
            qn -= 32;
          }
        }
        if (lane < qn) eval(q[lane]);
        __syncwarp();
        double fx, fy, fz, v;
        pair_total(a, ps, fx, fy, fz, v);
        if (lane == 0) {
          sm.f[gi][4] += fx;
          sm.f[gi][5] += fy;
          sm.f[gi][6] += fz;
          sm.f[gi][7] += v;
        }
      }
    }
    __syncthreads();
    if (kPairsOnly) {
      for (int e = threadIdx.x; e < gn * 4; e += blockDim.x)
        a.pair_out[(size_t)a.cell_ions[g0 + (e >> 2)] * 4 + (e & 3)] = sm.f[e >> 2][4 + (e & 3)];
      __syncthreads();
      continue;
    }
    for (int gi = warp; gi < gn; gi += kW) {
      double gx, gy, gz, vd;
      gather_el(a, a.cell_ions[g0 + gi], lane, gx, gy, gz, vd);
      if (lane == 0) {
        sm.f[gi][0] = gx;
        sm.f[gi][1] = gy;
        sm.f[gi][2] = gz;
        sm.f[gi][3] = vd;
      }
    }
    __syncthreads();
    // finish the group's ions, one per thread
    if (threadIdx.x < gn) {
      const double* r = sm.f[threadIdx.x];
      finish_ion(a, a.cell_ions[g0 + threadIdx.x], r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7], acc);
    }
    __syncthreads();
  }
}

// S8 in FP64 with every pair evaluated once (Newton's third law), and S7 of
// the cell's ions (to a.gath; S9 then runs one thread per ion), for boxes
// with a cell list of reach 1: block b takes cell b. Its candidates are the
// ions of the cell itself (a pair counted once: the candidate's slot after
// the home ion's) and of the 13 cells of the upper half of its neighbourhood
// (offsets (dz, dy, dx) after (0, 0, 0) in lexicographic order; with at
// least 3 cells per edge the 27 neighbour cells are distinct, so no cell
// pair is visited twice). Each surviving pair's force goes to both ions:
// the home ion's share is summed over the warp in a fixed order, the
// partner's share into a 64-bit fixed-point accumulator of the staged
// candidate with shared-memory integer atomics (the home ion's share is the
// same rounded integer with the opposite sign); both then reach the per-ion
// sums a.pair_fix ([n][4]: force x, y, z and pair energy, each pair's
// energy given to both ions as the one-ion loop does) with 64-bit integer
// atomics. Integer sums are exact, so the result does not depend on the
// order the blocks run in. Fixed point: 2^-40 eV/A (9.1e-13) per unit, the
// conversions done on the integer pipe (fix40), range +-8.4e6 eV/A; a pair
// closer than 0.5 A (forces approaching that range) marks the step
// non-finite. Staged candidates carry the periodic image of their cell
// relative to the home cell (cells are at least r_cut wide, so for every
// pair within r_cut that image is the minimum image, and any other pair is
// at least r_cut apart in every image): no per-pair image arithmetic.

// round(v * 2^40) as a 64-bit integer from v's bits, integer operations only
// (the FP64 pipe's conversions are slow); |v| < 2^23, rounding half away
// from zero, |v| < 2^-41 gives 0.
__device__ __forceinline__ long long fix40(double v) { return round_scaled(v, 40); }
constexpr int kHalfChunk = 384;
constexpr int kHalfNbr = 14;                        // the cell itself and 13 neighbours
template <int kW>
struct HalfSmem {
  float4 p[kHalfChunk];                            // FP32 positions (filter)
  __align__(16) double xyz[3][kHalfChunk];         // FP64 positions
  int j[kHalfChunk];                               // ion
  int slot[kHalfChunk];                            // cell-list slot
  unsigned long long acc[4][kHalfChunk];           // partners' shares, fixed point (component-major:
                                                   // a warp's atomics on 32 candidates hit distinct banks)
  int lo[kHalfNbr], cum[kHalfNbr + 1];
  unsigned long long f[kCellGroup][4];             // home ions' shares, fixed point
  int queue[kW][64];
  int bad;
};

// kGather: also S7 of the home ions (the single-kernel form); without it the
// pairs alone (the form that runs beside the solve, whose potential S7 needs).
template <int kW, bool kGather = true>
__device__ __forceinline__ void pairs_half_cell(const ForceArgs& a, int c, HalfSmem<kW>& sm) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int n = a.n, nc = a.nc;
  const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
  if (threadIdx.x < kHalfNbr) {
    // entry 0: the cell itself; then the 13 offsets after (0, 0, 0)
    const int t = threadIdx.x == 0 ? 13 : (threadIdx.x - 1) + 14;
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int cc = (cx + dx + nc) % nc + nc * ((cy + dy + nc) % nc + nc * ((cz + dz + nc) % nc));
    sm.lo[threadIdx.x] = a.cell_start[cc];
    sm.cum[threadIdx.x + 1] = a.cell_start[cc + 1] - a.cell_start[cc];
  }
  if (threadIdx.x == 0) sm.bad = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.cum[0] = 0;
    for (int t = 0; t < kHalfNbr; ++t) sm.cum[t + 1] += sm.cum[t];
  }
  __syncthreads();
  const int total = sm.cum[kHalfNbr];
  const int self_end = sm.cum[1];                    // candidates [0, self_end) are the cell's own ions
  const int c0 = a.cell_start[c], cn = a.cell_start[c + 1] - c0;
  bool bad = false;
  for (int g0 = c0; g0 < c0 + cn; g0 += kCellGroup) {
    const int gn = min(kCellGroup, c0 + cn - g0);
    for (int e = threadIdx.x; e < gn * 4; e += blockDim.x) sm.f[e >> 2][e & 3] = 0ull;
    for (int ch0 = 0; ch0 < total; ch0 += kHalfChunk) {
      const int len = min(kHalfChunk, total - ch0);
      __syncthreads();
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int tt = ch0 + e;
        int k = 0;
        while (k + 1 < kHalfNbr && sm.cum[k + 1] <= tt) ++k;
        const int slot = sm.lo[k] + (tt - sm.cum[k]);
        const int j = a.cell_ions[slot];
        // the image of neighbour cell k next to the home cell
        const int t = k == 0 ? 13 : (k - 1) + 14;
        const int ox = cx + t % 3 - 1, oy = cy + (t / 3) % 3 - 1, oz = cz + t / 9 - 1;
        const double shx = ox < 0 ? -a.L : (ox >= nc ? a.L : 0.0);
        const double shy = oy < 0 ? -a.L : (oy >= nc ? a.L : 0.0);
        const double shz = oz < 0 ? -a.L : (oz >= nc ? a.L : 0.0);
        const float fx = ox < 0 ? -a.Lf : (ox >= nc ? a.Lf : 0.f);
        const float fy = oy < 0 ? -a.Lf : (oy >= nc ? a.Lf : 0.f);
        const float fz = oz < 0 ? -a.Lf : (oz >= nc ? a.Lf : 0.f);
        const float4 pj = a.pos_sorted[slot];
        sm.j[e] = j;
        sm.slot[e] = tt < self_end ? slot : 0x7fffffff;
        sm.p[e] = make_float4(pj.x + fx, pj.y + fy, pj.z + fz, pj.w);
        sm.xyz[0][e] = a.pos[j] + shx;
        sm.xyz[1][e] = a.pos[n + j] + shy;
        sm.xyz[2][e] = a.pos[2 * n + j] + shz;
        sm.acc[0][e] = sm.acc[1][e] = sm.acc[2][e] = sm.acc[3][e] = 0ull;
      }
      __syncthreads();
      // The warp's home ions share one queue of passing candidates: a batch of
      // 32 may hold the last pairs of one ion (the "previous" one, its
      // entries first in the queue) and the first of the next, so the FP64
      // arithmetic runs on full warps (the FP64 pipe issues a warp
      // instruction at the same cost however many lanes are active).
      int* q = sm.queue[warp];
      int qn = 0;           // queued entries
      int qc = 0;           // of which the first qc belong to the previous ion
      int pgi = -1, pion = 0, pti = 0;
      long long px = 0, py = 0, pz = 0, pv = 0;   // the previous ion's per-lane sums, 2^-40 units
      auto flush_prev = [&]() {
        const long long tx = warp_isum(px), ty = warp_isum(py), tz = warp_isum(pz), tv = warp_isum(pv);
        if (lane == 0) {
          sm.f[pgi][0] += (unsigned long long)tx;
          sm.f[pgi][1] += (unsigned long long)ty;
          sm.f[pgi][2] += (unsigned long long)tz;
          sm.f[pgi][3] += (unsigned long long)tv;
        }
        px = py = pz = pv = 0;
      };
      double x = 0, y = 0, z = 0;   // the current home ion
      int ti = 0;
      long long sfx = 0, sfy = 0, sfz = 0, sv = 0;   // its per-lane sums, 2^-40 units
      // pair (home, candidate e2); prv: the home ion is the previous one
      auto eval = [&](int e2, bool prv) {
        const double hx = prv ? a.pos[pion] : x, hy = prv ? a.pos[n + pion] : y, hz = prv ? a.pos[2 * n + pion] : z;
        const double ddx = sm.xyz[0][e2] - hx, ddy = sm.xyz[1][e2] - hy, ddz = sm.xyz[2][e2] - hz;
        const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        // (r2 >= 0: the integer order of the bit patterns is the numeric one)
        if (__double_as_longlong(r2) >= __double_as_longlong(a.rc2)) return;
        double fr, V;
        tf_pair(a, (prv ? pti : ti) + a.type[sm.j[e2]], r2, fr, V);
        // force on the partner +fr d, on the home ion -fr d: the same 2^-40
        // integers with opposite signs (the pair's momentum balance is exact)
        const long long qx = fix40(fr * ddx), qy = fix40(fr * ddy), qz = fix40(fr * ddz), qv = fix40(V);
        if (prv) {
          px -= qx;
          py -= qy;
          pz -= qz;
          pv += qv;
        } else {
          sfx -= qx;
          sfy -= qy;
          sfz -= qz;
          sv += qv;
        }
        atomicAdd(&sm.acc[0][e2], (unsigned long long)qx);
        atomicAdd(&sm.acc[1][e2], (unsigned long long)qy);
        atomicAdd(&sm.acc[2][e2], (unsigned long long)qz);
        atomicAdd(&sm.acc[3][e2], (unsigned long long)qv);
      };
      for (int gi = warp; gi < gn; gi += kW) {
        const int islot = g0 + gi;
        const int i = a.cell_ions[islot];
        x = a.pos[i];
        y = a.pos[n + i];
        z = a.pos[2 * n + i];
        ti = a.type[i];
        const float4 pi32 = a.pos_sorted[islot];
        sfx = sfy = sfz = sv = 0;
        for (int e0 = 0; e0 < len; e0 += 32) {
          const int e = e0 + lane;
          bool pass = false;
          // own-cell partners only after the home ion (every pair once); the
          // other cells' candidates carry slot INT_MAX
          if (e < len && sm.slot[e] > islot) {
            const float4 pj = sm.p[e];
            const float dx = pj.x - pi32.x, dy = pj.y - pi32.y, dz = pj.z - pi32.z;
            const float r2f = dx * dx + dy * dy + dz * dz;
            pass = r2f < a.rc2_filter;
            bad = bad || r2f < 0.25f;
          }
          const unsigned m = __ballot_sync(0xffffffffu, pass);
          if (pass) q[qn + __popc(m & ((1u << lane) - 1u))] = e;
          qn += __popc(m);
          __syncwarp();
          if (qn >= 32) {
            eval(q[lane], lane < qc);
            __syncwarp();
            if (qc > 0) {   // the previous ion's last entries are done
              flush_prev();
              qc = 0;
            }
            if (lane < qn - 32) q[lane] = q[32 + lane];
            __syncwarp();
            qn -= 32;
          }
        }
        if (qc > 0) {
          // the previous ion is still queued (this one passed too few
          // candidates to fill a batch): finish both now
          if (lane < qn) eval(q[lane], lane < qc);
          __syncwarp();
          flush_prev();
          qc = 0;
          qn = 0;
          px = sfx;
          py = sfy;
          pz = sfz;
          pv = sv;
          pgi = gi;
          flush_prev();
        } else {
          // this ion's remaining entries wait for the next ion's (none left:
          // its sums are complete)
          qc = qn;
          pgi = gi;
          pion = i;
          pti = ti;
          px = sfx;
          py = sfy;
          pz = sfz;
          pv = sv;
          if (qc == 0) flush_prev();
        }
      }
      if (qn > 0) {
        if (lane < qn) eval(q[lane], true);
        __syncwarp();
      }
      if (pgi >= 0) flush_prev();
      __syncthreads();
      // the partners' shares of this chunk to the per-ion sums
      for (int e = threadIdx.x; e < len * 4; e += blockDim.x) {
        const unsigned long long v = sm.acc[e & 3][e >> 2];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(a.pair_fix) + (size_t)sm.j[e >> 2] * 4 + (e & 3), v);
      }
    }
    // S7 for the home ions (their potential neighbourhood is the cell's)
    if (kGather)
      for (int gi = warp; gi < gn; gi += kW) {
        const int i = a.cell_ions[g0 + gi];
        double gx, gy, gz, vd;
        gather_el(a, i, lane, gx, gy, gz, vd);
        if (lane == 0) {
          a.gath[(size_t)i * 4] = gx;
          a.gath[(size_t)i * 4 + 1] = gy;
          a.gath[(size_t)i * 4 + 2] = gz;
          a.gath[(size_t)i * 4 + 3] = vd;
        }
      }
    __syncthreads();
    for (int e = threadIdx.x; e < gn * 4; e += blockDim.x)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.pair_fix) + (size_t)a.cell_ions[g0 + (e >> 2)] * 4 + (e & 3),
                sm.f[e >> 2][e & 3]);
  }
  if (bad) atomicOr(&sm.bad, 1);
  __syncthreads();
  if (threadIdx.x == 0 && sm.bad) atomicCAS(&a.rec->status, MAZE_OK, MAZE_ERR_NONFINITE);
}

// S7 alone for the ions of cell c (to a.gath), one warp per ion.
template <int kW>
__device__ __forceinline__ void gather_cell(const ForceArgs& a, int c) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int c0 = a.cell_start[c], cn = a.cell_start[c + 1] - c0;
  for (int gi = warp; gi < cn; gi += kW) {
    const int i = a.cell_ions[c0 + gi];
    double gx, gy, gz, vd;
    gather_el(a, i, lane, gx, gy, gz, vd);
    if (lane == 0) {
      a.gath[(size_t)i * 4] = gx;
      a.gath[(size_t)i * 4 + 1] = gy;
      a.gath[(size_t)i * 4 + 2] = gz;
      a.gath[(size_t)i * 4 + 3] = vd;
    }
  }
}

// The mixed-precision form of pairs_half_cell (boxes above 64^3, which run
// one at a time): candidates staged as cell-relative hi + lo floats with the
// neighbour cell's offset folded in by TwoSum, displacements as exact FP32
// sums, the pair arithmetic in FP32; the same once-per-pair bookkeeping with
// 2^-40 fixed-point sums, and the FP32 gather of the cell's ions.
// kDF: the FP64 boxes' form, the same staging with the displacement kept as
// a double-float pair (the hi parts' difference exact by TwoSum, the lo
// parts' difference added), r^2 from exact squares, the pair by tf_pair_df
// and the 2^-40 integers from both halves of each product; the gather in
// FP64. Every quantity reaches ~1e-13 relative (the cell-relative hi + lo
// coordinates hold a position to ~2^-44 A), the FP64 force bar is 1e-10.
template <int kW>
struct HalfSmemF {
  float4 h[kHalfChunk];                            // hi parts (offset folded), type in l.w
  float4 l[kHalfChunk];
  int j[kHalfChunk];
  int slot[kHalfChunk];
  unsigned long long acc[4][kHalfChunk];   // component-major
  int lo[kHalfNbr], cum[kHalfNbr + 1];
  unsigned long long f[kCellGroup][4];
  int queue[kW][64];
  int bad;
};

template <int kW, bool kGather = true, bool kDF = false>
__device__ __forceinline__ void pairs_half_cell_mixed(const ForceArgs& a, int c, HalfSmemF<kW>& sm) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nc = a.nc;
  const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
  if (threadIdx.x < kHalfNbr) {
    const int t = threadIdx.x == 0 ? 13 : (threadIdx.x - 1) + 14;
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int cc = (cx + dx + nc) % nc + nc * ((cy + dy + nc) % nc + nc * ((cz + dz + nc) % nc));
    sm.lo[threadIdx.x] = a.cell_start[cc];
    sm.cum[threadIdx.x + 1] = a.cell_start[cc + 1] - a.cell_start[cc];
  }
  if (threadIdx.x == 0) sm.bad = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.cum[0] = 0;
    for (int t = 0; t < kHalfNbr; ++t) sm.cum[t + 1] += sm.cum[t];
  }
  __syncthreads();
  const int total = sm.cum[kHalfNbr];
  const int self_end = sm.cum[1];
  const int c0 = a.cell_start[c], cn = a.cell_start[c + 1] - c0;
  bool bad = false;
  for (int g0 = c0; g0 < c0 + cn; g0 += kCellGroup) {
    const int gn = min(kCellGroup, c0 + cn - g0);
    for (int e = threadIdx.x; e < gn * 4; e += blockDim.x) sm.f[e >> 2][e & 3] = 0ull;
    for (int ch0 = 0; ch0 < total; ch0 += kHalfChunk) {
      const int len = min(kHalfChunk, total - ch0);
      __syncthreads();
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int tt = ch0 + e;
        int k = 0;
        while (k + 1 < kHalfNbr && sm.cum[k + 1] <= tt) ++k;
        const int slot = sm.lo[k] + (tt - sm.cum[k]);
        const int t = k == 0 ? 13 : (k - 1) + 14;
        const float ox = (float)(t % 3 - 1), oy = (float)((t / 3) % 3 - 1), oz = (float)(t / 9 - 1);
        const float4 hh = a.rel_hi_sorted[slot], ll = a.rel_lo_sorted[slot];
        // (rel + offset * cell_len) as hi + lo: TwoSum with the offset's hi part
        const float sx = __fadd_rn(hh.x, ox * a.cell_len_h), sy = __fadd_rn(hh.y, oy * a.cell_len_h),
                    sz = __fadd_rn(hh.z, oz * a.cell_len_h);
        const float bx = __fsub_rn(sx, hh.x), by = __fsub_rn(sy, hh.y), bz = __fsub_rn(sz, hh.z);
        const float ex = __fadd_rn(__fsub_rn(hh.x, __fsub_rn(sx, bx)), __fsub_rn(ox * a.cell_len_h, bx));
        const float ey = __fadd_rn(__fsub_rn(hh.y, __fsub_rn(sy, by)), __fsub_rn(oy * a.cell_len_h, by));
        const float ez = __fadd_rn(__fsub_rn(hh.z, __fsub_rn(sz, bz)), __fsub_rn(oz * a.cell_len_h, bz));
        sm.h[e] = make_float4(sx, sy, sz, hh.w);
        sm.l[e] = make_float4(__fadd_rn(ex, __fadd_rn(ll.x, ox * a.cell_len_l)),
                              __fadd_rn(ey, __fadd_rn(ll.y, oy * a.cell_len_l)),
                              __fadd_rn(ez, __fadd_rn(ll.z, oz * a.cell_len_l)), ll.w);
        sm.j[e] = a.cell_ions[slot];
        sm.slot[e] = tt < self_end ? slot : 0x7fffffff;
        sm.acc[0][e] = sm.acc[1][e] = sm.acc[2][e] = sm.acc[3][e] = 0ull;
      }
      __syncthreads();
      // one queue of passing candidates for the warp's home ions, as in the
      // FP64 kernel: batches of 32 on full warps, a batch's first entries
      // possibly the previous ion's
      int* q = sm.queue[warp];
      int qn = 0, qc = 0;
      int pgi = -1, pslot = 0;
      long long px = 0, py = 0, pz = 0, pv = 0;   // the previous ion's per-lane sums, 2^-40 units
      auto flush_prev = [&]() {
        const long long tx = warp_isum(px), ty = warp_isum(py), tz = warp_isum(pz), tv = warp_isum(pv);
        if (lane == 0) {
          sm.f[pgi][0] += (unsigned long long)tx;
          sm.f[pgi][1] += (unsigned long long)ty;
          sm.f[pgi][2] += (unsigned long long)tz;
          sm.f[pgi][3] += (unsigned long long)tv;
        }
        px = py = pz = pv = 0;
      };
      int islot = 0;
      long long sfx = 0, sfy = 0, sfz = 0, sv = 0;   // the current ion's per-lane sums, 2^-40 units
      auto eval = [&](int e2, bool prv) {
        const int hs = prv ? pslot : islot;
        const float4 ph = a.rel_hi_sorted[hs], pl = a.rel_lo_sorted[hs];
        const int ti = (int)pl.w;
        const float4 h = sm.h[e2], l = sm.l[e2];
        const int kind = ti + (int)l.w;
        long long qx, qy, qz, qv;
        if constexpr (kDF) {
          const dfl sx = df_two_sum(h.x, -ph.x), sy = df_two_sum(h.y, -ph.y), sz = df_two_sum(h.z, -ph.z);
          // (Fast2Sum: the lo parts' difference is below 2^-18 A, so it can
          // exceed the hi difference only for a component of that size,
          // whose rounding then stays below 2^-42 A)
          const dfl dx = df_fast_sum(sx.h, __fadd_rn(sx.l, __fsub_rn(l.x, pl.x)));
          const dfl dy = df_fast_sum(sy.h, __fadd_rn(sy.l, __fsub_rn(l.y, pl.y)));
          const dfl dz = df_fast_sum(sz.h, __fadd_rn(sz.l, __fsub_rn(l.z, pl.z)));
          const dfl px = df_two_prod(dx.h, dx.h), py = df_two_prod(dy.h, dy.h), pz = df_two_prod(dz.h, dz.h);
          const dfl s1 = df_two_sum(px.h, py.h);
          const dfl s2 = df_two_sum(s1.h, pz.h);
          float lo = __fadd_rn(s1.l, s2.l);
          lo = __fadd_rn(lo, __fmaf_rn(__fadd_rn(dx.h, dx.h), dx.l, px.l));
          lo = __fadd_rn(lo, __fmaf_rn(__fadd_rn(dy.h, dy.h), dy.l, py.l));
          lo = __fadd_rn(lo, __fmaf_rn(__fadd_rn(dz.h, dz.h), dz.l, pz.l));
          const dfl r2 = df_fast_sum(s2.h, lo);
          if (!df_less(r2, f2df(a.pdf.rc2))) return;
          dfl fr, V;
          tf_pair_df(a, kind, r2, fr, V);
          const dfl fx = df_mul(fr, dx), fy = df_mul(fr, dy), fz = df_mul(fr, dz);
          qx = df_fix40(fx);
          qy = df_fix40(fy);
          qz = df_fix40(fz);
          qv = df_fix40(V);
        } else {
          const float dx = disp_df(ph.x, pl.x, h.x, l.x, 0.f, 0.f);
          const float dy = disp_df(ph.y, pl.y, h.y, l.y, 0.f, 0.f);
          const float dz = disp_df(ph.z, pl.z, h.z, l.z, 0.f, 0.f);
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 >= a.rc2f) return;
          const float ir = rsqrtf(r2);
          const float r = r2 * ir;
          const float ir2 = ir * ir;
          const float ir6 = ir2 * ir2 * ir2;
          const float ir8 = ir6 * ir2;
          const float exv = a.Af[kind] * expf(a.Bf * (a.sf[kind] - r));
          const float V = exv - a.Cf[kind] * ir6 - a.Df[kind] * ir8 - a.Vcf[kind];
          const float fr = a.Bf * exv * ir - 6.f * a.Cf[kind] * ir8 - 8.f * a.Df[kind] * ir8 * ir2;
          qx = round_scaled_f(fr * dx, 40);
          qy = round_scaled_f(fr * dy, 40);
          qz = round_scaled_f(fr * dz, 40);
          qv = round_scaled_f(V, 40);
        }
        // the partner +f, the home ion -f: the same 2^-40 integers
        if (prv) {
          px -= qx;
          py -= qy;
          pz -= qz;
          pv += qv;
        } else {
          sfx -= qx;
          sfy -= qy;
          sfz -= qz;
          sv += qv;
        }
        atomicAdd(&sm.acc[0][e2], (unsigned long long)qx);
        atomicAdd(&sm.acc[1][e2], (unsigned long long)qy);
        atomicAdd(&sm.acc[2][e2], (unsigned long long)qz);
        atomicAdd(&sm.acc[3][e2], (unsigned long long)qv);
      };
      for (int gi = warp; gi < gn; gi += kW) {
        islot = g0 + gi;
        const float4 ph = a.rel_hi_sorted[islot];
        sfx = sfy = sfz = sv = 0;
        for (int e0 = 0; e0 < len; e0 += 32) {
          const int e = e0 + lane;
          bool pass = false;
          if (e < len && sm.slot[e] > islot) {
            const float4 h = sm.h[e];
            const float dx = h.x - ph.x, dy = h.y - ph.y, dz = h.z - ph.z;
            const float r2f = dx * dx + dy * dy + dz * dz;
            pass = r2f < a.rc2_filter;
            bad = bad || r2f < 0.25f;
          }
          const unsigned m = __ballot_sync(0xffffffffu, pass);
          if (pass) q[qn + __popc(m & ((1u << lane) - 1u))] = e;
          qn += __popc(m);
          __syncwarp();
          if (qn >= 32) {
            eval(q[lane], lane < qc);
            __syncwarp();
            if (qc > 0) {
              flush_prev();
              qc = 0;
            }
            if (lane < qn - 32) q[lane] = q[32 + lane];
            __syncwarp();
            qn -= 32;
          }
        }
        if (qc > 0) {
          // the previous ion is still queued: finish both now
          if (lane < qn) eval(q[lane], lane < qc);
          __syncwarp();
          flush_prev();
          qc = 0;
          qn = 0;
          px = sfx;
          py = sfy;
          pz = sfz;
          pv = sv;
          pgi = gi;
          flush_prev();
        } else {
          qc = qn;
          pgi = gi;
          pslot = islot;
          px = sfx;
          py = sfy;
          pz = sfz;
          pv = sv;
          if (qc == 0) flush_prev();
        }
      }
      if (qn > 0) {
        if (lane < qn) eval(q[lane], true);
        __syncwarp();
      }
      if (pgi >= 0) flush_prev();
      __syncthreads();
      for (int e = threadIdx.x; e < len * 4; e += blockDim.x) {
        const unsigned long long v = sm.acc[e & 3][e >> 2];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(a.pair_fix) + (size_t)sm.j[e >> 2] * 4 + (e & 3), v);
      }
    }
    if (kGather)
      for (int gi = warp; gi < gn; gi += kW) {
        const int i = a.cell_ions[g0 + gi];
        double gx, gy, gz, vd;
        gather_el(a, i, lane, gx, gy, gz, vd);
        if (lane == 0) {
          a.gath[(size_t)i * 4] = gx;
          a.gath[(size_t)i * 4 + 1] = gy;
          a.gath[(size_t)i * 4 + 2] = gz;
          a.gath[(size_t)i * 4 + 3] = vd;
        }
      }
    __syncthreads();
    for (int e = threadIdx.x; e < gn * 4; e += blockDim.x)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.pair_fix) + (size_t)a.cell_ions[g0 + (e >> 2)] * 4 + (e & 3),
                sm.f[e >> 2][e & 3]);
  }
  if (bad) atomicOr(&sm.bad, 1);
  __syncthreads();
  if (threadIdx.x == 0 && sm.bad) atomicCAS(&a.rec->status, MAZE_OK, MAZE_ERR_NONFINITE);
}

}  // namespace maze
