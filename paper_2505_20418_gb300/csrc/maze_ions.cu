// Ion-side kernels of the MaZe step:
//   k_ion_update  S1 half kick + drift (velocity Verlet) and S3 charge spreading
//   k_cell_*      S2 cell list (counting sort, deterministic order within a cell)
//   k_forces      S7 gather of Eq. F_nostra, S8 Tosi-Fumi pairs, S9 half kick,
//                 energies and momentum (deterministic block + last-block sums)
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

// B-spline weights of one axis for an ion at grid coordinate u (Sec. II.A).
// The support starts at node floor(u) - (P/2 - 1); t = u - floor(u).
// P = 2: linear B-spline (1 - t, t).
// P = 4: cubic B-spline ((1-t)^3, 3t^3 - 6t^2 + 4, -3t^3 + 3t^2 + 3t + 1, t^3) / 6.
// Split u into the first support node and the fractional offset t.
__device__ __forceinline__ int axis_split(double u, int P, int N, double& t) {
  const double fl = floor(u);
  t = u - fl;
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

__device__ __forceinline__ int wrap_idx(int a, int N) { return a >= N ? a - N : a; }

__device__ __forceinline__ double wrap_pos(double x, double L, double inv_L) {
  x -= L * floor(x * inv_L);
  if (x < 0.0) x += L;
  if (x >= L) x -= L;
  return x;
}

// S1: one thread per ion for the Verlet half kick and drift, the FP32 copy,
// the cell count and the B-spline weights of the new position (stored: the
// spread and the gather of the same step reuse them).
__global__ void __launch_bounds__(kIonThreads) k_move(IonArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // the first kernel of a step decides, once, whether the step runs at all
  const bool skip = a.rec->status != MAZE_OK;
  if (i == 0) *a.gate = skip ? 1 : 0;
  if (skip) return;
  const int N = a.N, P = a.P;
  if (i < a.n) {
    double x = a.pos[i], y = a.pos[a.n + i], z = a.pos[2 * a.n + i];
    const int t = a.type[i];
    if (a.do_move) {
      const double kick = t ? a.kick1 : a.kick0;
      double vx = a.vel[i] + kick * a.force[i];
      double vy = a.vel[a.n + i] + kick * a.force[a.n + i];
      double vz = a.vel[2 * a.n + i] + kick * a.force[2 * a.n + i];
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
    const double Q = t ? a.charge1 : a.charge0;
    a.pos32[i] = make_float4((float)x, (float)y, (float)z, (float)Q);
    if (a.nc >= 3) {
      const double cs = a.cell_scale;
      int cx = min((int)(x * cs), a.nc - 1), cy = min((int)(y * cs), a.nc - 1), cz = min((int)(z * cs), a.nc - 1);
      const int c = cx + a.nc * (cy + a.nc * cz);
      a.cell_of[i] = c;
      atomicAdd(&a.cell_count[c], 1);
    }
    double tx, ty, tz;
    const int fx = axis_split(x * a.inv_h, P, N, tx);
    const int fy = axis_split(y * a.inv_h, P, N, ty);
    const int fz = axis_split(z * a.inv_h, P, N, tz);
    if (a.wbuf32) {
      // mixed precision: FP32 weights from the exact fractional offsets
      float w[12];
      bspline_weights<float>((float)tx, P, w);
      bspline_weights<float>((float)ty, P, w + 4);
      bspline_weights<float>((float)tz, P, w + 8);
      float4* gw = reinterpret_cast<float4*>(a.wbuf32 + (size_t)i * 12);
      gw[0] = make_float4(w[0], w[1], w[2], w[3]);
      gw[1] = make_float4(w[4], w[5], w[6], w[7]);
      gw[2] = make_float4(w[8], w[9], w[10], w[11]);
    } else {
      double w[12];
      bspline_weights<double>(tx, P, w);
      bspline_weights<double>(ty, P, w + 4);
      bspline_weights<double>(tz, P, w + 8);
      double* gw = a.wbuf + (size_t)i * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) gw[k] = w[k];
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
__global__ void __launch_bounds__(kSpreadThreads) k_spread(IonArgs a) {
  if (*a.gate) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (kSpreadThreads / 32) + (threadIdx.x >> 5);
  if (i >= a.n) return;
  const int N = a.N, P = a.P, P3 = P * P * P;
  const int4 b = a.wbase[i];
  const double Q = a.type[i] ? a.charge1 : a.charge0;
  long long v[2] = {0, 0};
  int idx[2] = {-1, -1};
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int sidx = lane + 32 * u;
    if (sidx >= P3) continue;
    const int ia = sidx % P, ib = (sidx / P) % P, ic = sidx / (P * P);
    if (a.wbuf32) {
      // mixed precision: FP32 products
      const float* w = a.wbuf32 + (size_t)i * 12;
      v[u] = __float2ll_rn((float)Q * w[8 + ic] * w[4 + ib] * w[ia] * (float)kQScale);
    } else {
      const double* w = a.wbuf + (size_t)i * 12;
      v[u] = __double2ll_rn(Q * w[8 + ic] * w[4 + ib] * w[ia] * kQScale);
    }
    const int ix = wrap_idx(b.x + ia, N), iy = wrap_idx(b.y + ib, N), iz = wrap_idx(b.z + ic, N);
    idx[u] = (int)(((size_t)iz * N + iy) * N + ix);
  }
  const long long total = warp_isum(v[0] + v[1]);
  if (lane == 0) v[0] += __double2ll_rn(Q * kQScale) - total;
#pragma unroll
  for (int u = 0; u < 2; ++u)
    if (idx[u] >= 0) atomicAdd(&a.qfix[idx[u]], (unsigned long long)v[u]);
}

__global__ void k_q_to_double(const unsigned long long* qfix, double* q, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (double)(long long)qfix[i] * kQInv;
}

cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t s) {
  k_move<<<(a.n + kIonThreads - 1) / kIonThreads, kIonThreads, 0, s>>>(a);
  if (a.qfix) {
    const int per = kSpreadThreads / 32;
    k_spread<<<(a.n + per - 1) / per, kSpreadThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_q_to_double(const unsigned long long* qfix, double* q, int n, cudaStream_t s) {
  k_q_to_double<<<(n + 255) / 256, 256, 0, s>>>(qfix, q, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S2: cell list. One block scans the counts (and clears them for the next
// step), ions claim slots, then each cell sorts its slots by ion index so the
// pair sums run in a fixed order.

__global__ void k_cell_scan(CellArgs a) {
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
}

__global__ void k_cell_fill(CellArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int slot = atomicAdd(&a.cursor[a.cell_of[i]], 1);
  a.cell_ions[slot] = i;
}

// One warp per cell: each slot's rank among the cell's (distinct) ion indices
// gives its sorted position. Cells larger than the shared buffer fall back to
// an insertion sort by lane 0.
constexpr int kSortWarps = 4;
constexpr int kSortCap = 256;
__global__ void __launch_bounds__(kSortWarps * 32) k_cell_sort(CellArgs a) {
  __shared__ int s_ids[kSortWarps][kSortCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * kSortWarps + warp;
  if (c >= a.ncell) return;
  const int lo = a.cell_start[c], hi = a.cell_start[c + 1], m = hi - lo;
  if (m <= 1) return;
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
    return;
  }
  int* ids = s_ids[warp];
  for (int u = lane; u < m; u += 32) ids[u] = a.cell_ions[lo + u];
  __syncwarp();
  for (int u = lane; u < m; u += 32) {
    const int v = ids[u];
    int rank = 0;
    for (int k = 0; k < m; ++k) rank += ids[k] < v;
    a.cell_ions[lo + rank] = v;
  }
}

cudaError_t launch_cells(const CellArgs& a, cudaStream_t s) {
  k_cell_scan<<<1, 1024, 0, s>>>(a);
  k_cell_fill<<<(a.n + 255) / 256, 256, 0, s>>>(a);
  k_cell_sort<<<(a.ncell + kSortWarps - 1) / kSortWarps, kSortWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S7-S9: one warp per ion.

__device__ __forceinline__ void tf_pair(const ForceArgs& a, int kind, double r2, double& fr, double& V) {
  // V = A exp(B (s - r)) - C r^-6 - D r^-8 - V(r_c);  fr = -(dV/dr) / r.
  // 1/r by Newton-Raphson for the reciprocal square root, y <- y (3 - r2 y^2)/2,
  // from an FP32 seed (two steps: ~2^-22 -> 2^-44 -> FP64 rounding), so no FP64
  // square root or division is needed.
  double ir = (double)rsqrtf((float)r2);
  ir = ir * (1.5 - 0.5 * r2 * ir * ir);
  ir = ir * (1.5 - 0.5 * r2 * ir * ir);
  const double r = r2 * ir;
  const double ir2 = ir * ir;
  const double ir6 = ir2 * ir2 * ir2;
  const double ir8 = ir6 * ir2;
  const double ex = a.A[kind] * exp(a.B * (a.s[kind] - r));
  V = ex - a.C[kind] * ir6 - a.D[kind] * ir8 - a.Vc[kind];
  fr = a.B * ex * ir - 6.0 * a.C[kind] * ir8 - 8.0 * a.D[kind] * ir8 * ir2;
}

__global__ void __launch_bounds__(kForceThreads) k_forces(ForceArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * (kForceThreads / 32) + warp;
  // a step whose solve hit max_iter still completes (forces, energies, step
  // count); any other error stops the step
  const int st0 = a.rec->status;
  const bool live = i < a.n && *a.gate == 0 && (st0 == MAZE_OK || st0 == MAZE_ERR_NOT_CONVERGED);
  // per-ion contributions to the block sums:
  // 0 KE, 1 V_TF (pairs counted twice), 2 1/2 phi.q, 3 dV_work, 4-6 momentum
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  __shared__ int s_queue[kForceThreads / 32][64];
  if (live) {
    const int n = a.n, N = a.N, P = a.P;
    const double x = a.pos[i], y = a.pos[n + i], z = a.pos[2 * n + i];
    const int t = a.type[i];
    const double Q = t ? a.charge1 : a.charge0;
    // --- S7: Eq. F_nostra, F = -k_e Q sum_n W (phi_{n+e} - phi_{n-e}) / 2h,
    // with the weights k_ion_update stored for this position
    const int4 first = a.wbase[i];
    const int P3 = P * P * P;
    double gx = 0, gy = 0, gz = 0, vd = 0;
    const size_t NN = (size_t)N * N;
    if (a.mixed) {
      // mixed precision: FP32 weights, differences of the double-float
      // potential in FP32, FP32 sums
      const float* w = a.wbuf32 + (size_t)i * 12;
      const float2* f = reinterpret_cast<const float2*>(a.phi);
      float sx = 0.f, sy = 0.f, sz = 0.f, s0 = 0.f;
      for (int sidx = lane; sidx < P3; sidx += 32) {
        const int ia = sidx % P, ib = (sidx / P) % P, ic = sidx / (P * P);
        const int ix = wrap_idx(first.x + ia, N), iy = wrap_idx(first.y + ib, N), iz = wrap_idx(first.z + ic, N);
        const float wt = w[ia] * w[4 + ib] * w[8 + ic];
        const size_t row = iz * NN + (size_t)iy * N;
        const float2 xp = f[row + (ix == N - 1 ? 0 : ix + 1)], xm = f[row + (ix == 0 ? N - 1 : ix - 1)];
        const float2 yp = f[iz * NN + (size_t)(iy == N - 1 ? 0 : iy + 1) * N + ix];
        const float2 ym = f[iz * NN + (size_t)(iy == 0 ? N - 1 : iy - 1) * N + ix];
        const float2 zp = f[(size_t)(iz == N - 1 ? 0 : iz + 1) * NN + (size_t)iy * N + ix];
        const float2 zm = f[(size_t)(iz == 0 ? N - 1 : iz - 1) * NN + (size_t)iy * N + ix];
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
      for (int sidx = lane; sidx < P3; sidx += 32) {
        const int ia = sidx % P, ib = (sidx / P) % P, ic = sidx / (P * P);
        const int ix = wrap_idx(first.x + ia, N), iy = wrap_idx(first.y + ib, N), iz = wrap_idx(first.z + ic, N);
        const double wt = w[ia] * w[4 + ib] * w[8 + ic];
        const size_t row = iz * NN + (size_t)iy * N;
        const size_t ixp = row + (ix == N - 1 ? 0 : ix + 1), ixm = row + (ix == 0 ? N - 1 : ix - 1);
        const size_t iyp = iz * NN + (size_t)(iy == N - 1 ? 0 : iy + 1) * N + ix;
        const size_t iym = iz * NN + (size_t)(iy == 0 ? N - 1 : iy - 1) * N + ix;
        const size_t izp = (size_t)(iz == N - 1 ? 0 : iz + 1) * NN + (size_t)iy * N + ix;
        const size_t izm = (size_t)(iz == 0 ? N - 1 : iz - 1) * NN + (size_t)iy * N + ix;
        double px, py, pz, p0;
        if (a.phi_df) {
          // double-float potential: differences of the (hi, lo) pairs in FP32
          const float2* f = reinterpret_cast<const float2*>(a.phi);
          const float2 xp = f[ixp], xm = f[ixm], yp = f[iyp], ym = f[iym], zp = f[izp], zm = f[izm], c0 = f[row + ix];
          px = (double)((xp.x - xm.x) + (xp.y - xm.y));
          py = (double)((yp.x - ym.x) + (yp.y - ym.y));
          pz = (double)((zp.x - zm.x) + (zp.y - zm.y));
          p0 = (double)c0.x + (double)c0.y;
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
      gx = warp_sum(gx);
      gy = warp_sum(gy);
      gz = warp_sum(gz);
      vd = warp_sum(vd);
    }
    const double fe = -MAZE_KE_EV_ANGSTROM * Q * a.inv_2h;
    const double Fex = fe * gx, Fey = fe * gy, Fez = fe * gz;
    // --- S8: Tosi-Fumi pairs, minimum image, r < r_c. Candidates pass an
    // FP32 pre-filter with a safety margin; survivors are queued per warp and
    // evaluated 32 at a time in FP64 (exact cutoff test), so the FP64 pipe
    // sees full warps instead of the ~10 % of lanes that pass the filter.
    const float4 pi32 = a.pos32[i];
    const float Lf = a.Lf;
    int* q = s_queue[warp];
    int qn = 0;
    double ftx = 0, fty = 0, ftz = 0, vtf = 0;
    float ftxf = 0.f, ftyf = 0.f, ftzf = 0.f, vtff = 0.f;
    auto pair = [&](int j) {
      const float4 pj = a.pos32[j];
      if (a.mixed) {
        // mixed precision: displacement in FP64 (exact minimum image), pair
        // energy and force in FP32
        const float iL = a.inv_Lf;
        const float sx = rintf((pj.x - pi32.x) * iL), sy = rintf((pj.y - pi32.y) * iL), sz = rintf((pj.z - pi32.z) * iL);
        const float dx = (float)((a.pos[j] - x) - (double)sx * a.L);
        const float dy = (float)((a.pos[n + j] - y) - (double)sy * a.L);
        const float dz = (float)((a.pos[2 * n + j] - z) - (double)sz * a.L);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= a.rc2f) return;
        const int kind = t + a.type[j];
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        const float ir2 = ir * ir;
        const float ir6 = ir2 * ir2 * ir2;
        const float ir8 = ir6 * ir2;
        const float ex = a.Af[kind] * expf(a.Bf * (a.sf[kind] - r));
        const float V = ex - a.Cf[kind] * ir6 - a.Df[kind] * ir8 - a.Vcf[kind];
        const float fr = a.Bf * ex * ir - 6.f * a.Cf[kind] * ir8 - 8.f * a.Df[kind] * ir8 * ir2;
        ftxf -= fr * dx;
        ftyf -= fr * dy;
        ftzf -= fr * dz;
        vtff += V;
        return;
      }
      const float iL = a.inv_Lf;
      const float sx = rintf((pj.x - pi32.x) * iL), sy = rintf((pj.y - pi32.y) * iL), sz = rintf((pj.z - pi32.z) * iL);
      const double ddx = (a.pos[j] - x) - (double)sx * a.L;
      const double ddy = (a.pos[n + j] - y) - (double)sy * a.L;
      const double ddz = (a.pos[2 * n + j] - z) - (double)sz * a.L;
      const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
      if (r2 >= a.rc2) return;
      double fr, V;
      tf_pair(a, t + a.type[j], r2, fr, V);
      ftx -= fr * ddx;
      fty -= fr * ddy;
      ftz -= fr * ddz;
      vtf += V;
    };
    auto offer = [&](int j, bool valid) {
      bool pass = false;
      if (valid && j != i) {
        const float4 pj = a.pos32[j];
        float dx = pj.x - pi32.x, dy = pj.y - pi32.y, dz = pj.z - pi32.z;
        dx -= rintf(dx * a.inv_Lf) * Lf;
        dy -= rintf(dy * a.inv_Lf) * Lf;
        dz -= rintf(dz * a.inv_Lf) * Lf;
        pass = dx * dx + dy * dy + dz * dz < a.rc2_filter;
      }
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) q[qn + __popc(m & ((1u << lane) - 1u))] = j;
      qn += __popc(m);
      __syncwarp();
      if (qn >= 32) {
        pair(q[lane]);
        __syncwarp();
        if (lane < qn - 32) q[lane] = q[32 + lane];
        __syncwarp();
        qn -= 32;
      }
    };
    if (a.nc >= 3) {
      const int nc = a.nc;
      const int c = a.cell_of[i];
      const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
      for (int dz = -1; dz <= 1; ++dz) {
        const int zz = (cz + dz + nc) % nc;
        for (int dy = -1; dy <= 1; ++dy) {
          const int yy = (cy + dy + nc) % nc;
          for (int dx = -1; dx <= 1; ++dx) {
            const int xx = (cx + dx + nc) % nc;
            const int cc = xx + nc * (yy + nc * zz);
            const int lo = a.cell_start[cc], hi = a.cell_start[cc + 1];
            for (int u0 = lo; u0 < hi; u0 += 32) {
              const int u = u0 + lane;
              offer(u < hi ? a.cell_ions[u] : -1, u < hi);
            }
          }
        }
      }
    } else {
      for (int j0 = 0; j0 < n; j0 += 32) offer(j0 + lane, j0 + lane < n);
    }
    if (lane < qn) pair(q[lane]);
    if (a.mixed) {
      for (int o = 16; o > 0; o >>= 1) {
        ftxf += __shfl_xor_sync(0xffffffffu, ftxf, o);
        ftyf += __shfl_xor_sync(0xffffffffu, ftyf, o);
        ftzf += __shfl_xor_sync(0xffffffffu, ftzf, o);
        vtff += __shfl_xor_sync(0xffffffffu, vtff, o);
      }
      ftx = ftxf;
      fty = ftyf;
      ftz = ftzf;
      vtf = vtff;
    } else {
      ftx = warp_sum(ftx);
      fty = warp_sum(fty);
      ftz = warp_sum(ftz);
      vtf = warp_sum(vtf);
    }
    if (lane == 0) {
      const double Fx = Fex + ftx, Fy = Fey + fty, Fz = Fez + ftz;
      double vx = a.vel[i], vy = a.vel[n + i], vz = a.vel[2 * n + i];
      const double m = t ? a.mass1 : a.mass0;
      if (a.do_kick) {
        // Eq. E_nostra, trapezoid rule: dV_work = -1/2 (F_el^k + F_el^{k+1}) . dt v_half
        const double ox = a.force_el[i], oy = a.force_el[n + i], oz = a.force_el[2 * n + i];
        acc[3] = -0.5 * a.dt * ((ox + Fex) * vx + (oy + Fey) * vy + (oz + Fez) * vz);
        const double kick = t ? a.kick1 : a.kick0;
        vx += kick * Fx;
        vy += kick * Fy;
        vz += kick * Fz;
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
      acc[0] = a.ke_coef * m * (vx * vx + vy * vy + vz * vz);
      acc[1] = 0.5 * vtf;
      acc[2] = 0.5 * MAZE_KE_EV_ANGSTROM * Q * vd;
      acc[4] = m * vx;
      acc[5] = m * vy;
      acc[6] = m * vz;
    }
  }
  // deterministic block sum: lane 0 of each warp holds its ion's values
  __shared__ double s_acc[kForceThreads / 32][7];
  if (lane == 0)
    for (int k = 0; k < 7; ++k) s_acc[warp][k] = acc[k];
  __syncthreads();
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    double b[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int wv = 0; wv < kForceThreads / 32; ++wv)
      for (int k = 0; k < 7; ++k) b[k] += s_acc[wv][k];
    for (int k = 0; k < 7; ++k) a.part[blockIdx.x * 8 + k] = b[k];
    __threadfence();
    const unsigned tk = atomicAdd(a.ticket, 1u);
    s_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  // last block: sum the block partials in index order and publish the record
  __threadfence();
  if (threadIdx.x < 32) {
    double tot[7];
    for (int k = 0; k < 7; ++k) {
      double v = 0;
      for (int bb = threadIdx.x; bb < (int)gridDim.x; bb += 32) v += a.part[bb * 8 + k];
      tot[k] = warp_sum(v);
    }
    if (threadIdx.x == 0) {
      maze_stats* r = a.rec;
      *a.ticket = 0;
      if (*a.gate == 0 && (r->status == MAZE_OK || r->status == MAZE_ERR_NOT_CONVERGED)) {
        r->ke = tot[0];
        r->v_tf = tot[1];
        r->v_disc = tot[2];
        r->v_work += tot[3];
        r->e_tot = tot[0] + tot[1] + r->v_work;
        r->momentum[0] = tot[4];
        r->momentum[1] = tot[5];
        r->momentum[2] = tot[6];
        if (a.count_step) r->step += 1;
        if (!isfinite(r->e_tot)) r->status = MAZE_ERR_NONFINITE;
      }
    }
  }
}

int force_blocks(int n_ions) { return (n_ions + kForceThreads / 32 - 1) / (kForceThreads / 32); }

cudaError_t launch_forces(const ForceArgs& a, int blocks, cudaStream_t s) {
  k_forces<<<blocks, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace maze
