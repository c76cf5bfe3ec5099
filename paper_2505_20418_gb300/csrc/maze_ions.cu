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
__device__ __forceinline__ int axis_weights(double u, int P, int N, double* w) {
  const double fl = floor(u);
  const double t = u - fl;
  int first = (int)fl - (P / 2 - 1);
  if (P == 2) {
    w[0] = 1.0 - t;
    w[1] = t;
  } else {
    const double t2 = t * t, t3 = t2 * t;
    const double s = 1.0 - t;
    w[0] = s * s * s * (1.0 / 6.0);
    w[1] = (3.0 * t3 - 6.0 * t2 + 4.0) * (1.0 / 6.0);
    w[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) * (1.0 / 6.0);
    w[3] = t3 * (1.0 / 6.0);
  }
  if (first < 0) first += N;
  if (first >= N) first -= N;
  return first;
}

__device__ __forceinline__ int wrap_idx(int a, int N) { return a >= N ? a - N : a; }

__device__ __forceinline__ double wrap_pos(double x, double L) {
  x -= L * floor(x / L);
  if (x >= L) x -= L;
  return x;
}

__global__ void k_ion_update(IonArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // the first kernel of a step decides, once, whether the step runs at all
  const bool skip = a.rec->status != MAZE_OK;
  if (i == 0) *a.gate = skip ? 1 : 0;
  if (i >= a.n || skip) return;
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
    x = wrap_pos(x + a.dt * vx, a.L);
    y = wrap_pos(y + a.dt * vy, a.L);
    z = wrap_pos(z + a.dt * vz, a.L);
    a.pos[i] = x;
    a.pos[a.n + i] = y;
    a.pos[2 * a.n + i] = z;
  }
  const double Q = t ? a.charge1 : a.charge0;
  a.pos32[i] = make_float4((float)x, (float)y, (float)z, (float)Q);
  if (a.nc >= 3) {
    const double cs = a.nc / a.L;
    int cx = min((int)(x * cs), a.nc - 1), cy = min((int)(y * cs), a.nc - 1), cz = min((int)(z * cs), a.nc - 1);
    const int c = cx + a.nc * (cy + a.nc * cz);
    a.cell_of[i] = c;
    atomicAdd(&a.cell_count[c], 1);
  }
  if (!a.qfix) return;
  // S3: q_n += Q W(r - r_n) over the P^3 support, fixed-point atomics
  double wx[4], wy[4], wz[4];
  const int N = a.N, P = a.P;
  const int fx = axis_weights(x / a.h, P, N, wx);
  const int fy = axis_weights(y / a.h, P, N, wy);
  const int fz = axis_weights(z / a.h, P, N, wz);
  for (int c = 0; c < P; ++c) {
    const int iz = wrap_idx(fz + c, N);
    const double qz = Q * wz[c];
    for (int b = 0; b < P; ++b) {
      const int iy = wrap_idx(fy + b, N);
      const double qzy = qz * wy[b];
      const size_t row = ((size_t)iz * N + iy) * N;
      for (int aa = 0; aa < P; ++aa) {
        const int ix = wrap_idx(fx + aa, N);
        const long long v = __double2ll_rn(qzy * wx[aa] * kQScale);
        atomicAdd(&a.qfix[row + ix], (unsigned long long)v);
      }
    }
  }
}

__global__ void k_q_to_double(const unsigned long long* qfix, double* q, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (double)(long long)qfix[i] * kQInv;
}

cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t s) {
  const int th = 128;
  k_ion_update<<<(a.n + th - 1) / th, th, 0, s>>>(a);
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

__global__ void k_cell_sort(CellArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ncell) return;
  const int lo = a.cell_start[c], hi = a.cell_start[c + 1];
  for (int u = lo + 1; u < hi; ++u) {
    const int v = a.cell_ions[u];
    int w = u - 1;
    while (w >= lo && a.cell_ions[w] > v) {
      a.cell_ions[w + 1] = a.cell_ions[w];
      --w;
    }
    a.cell_ions[w + 1] = v;
  }
}

cudaError_t launch_cells(const CellArgs& a, cudaStream_t s) {
  k_cell_scan<<<1, 1024, 0, s>>>(a);
  k_cell_fill<<<(a.n + 255) / 256, 256, 0, s>>>(a);
  k_cell_sort<<<(a.ncell + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S7-S9: one warp per ion.

__device__ __forceinline__ void tf_pair(const ForceArgs& a, int kind, double r2, double& fr, double& V) {
  // V = A exp(B (s - r)) - C r^-6 - D r^-8 - V(r_c);  fr = -(dV/dr) / r
  const double r = sqrt(r2);
  const double ir2 = 1.0 / r2;
  const double ir6 = ir2 * ir2 * ir2;
  const double ir8 = ir6 * ir2;
  const double ex = a.A[kind] * exp(a.B * (a.s[kind] - r));
  V = ex - a.C[kind] * ir6 - a.D[kind] * ir8 - a.Vc[kind];
  fr = (a.B * ex) / r - 6.0 * a.C[kind] * ir8 - 8.0 * a.D[kind] * ir8 * ir2;
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
  if (live) {
    const int n = a.n, N = a.N, P = a.P;
    const double x = a.pos[i], y = a.pos[n + i], z = a.pos[2 * n + i];
    const int t = a.type[i];
    const double Q = t ? a.charge1 : a.charge0;
    // --- S7: Eq. F_nostra, F = -k_e Q sum_n W (phi_{n+e} - phi_{n-e}) / 2h
    double w[3][4];
    int first[3];
    first[0] = axis_weights(x / a.h, P, N, w[0]);
    first[1] = axis_weights(y / a.h, P, N, w[1]);
    first[2] = axis_weights(z / a.h, P, N, w[2]);
    const int P3 = P * P * P;
    double gx = 0, gy = 0, gz = 0, vd = 0;
    const size_t NN = (size_t)N * N;
    for (int sidx = lane; sidx < P3; sidx += 32) {
      const int ia = sidx % P, ib = (sidx / P) % P, ic = sidx / (P * P);
      const int ix = wrap_idx(first[0] + ia, N), iy = wrap_idx(first[1] + ib, N), iz = wrap_idx(first[2] + ic, N);
      const double wt = w[0][ia] * w[1][ib] * w[2][ic];
      const size_t row = iz * NN + (size_t)iy * N;
      const double* ph = a.phi;
      const double px = ph[row + (ix == N - 1 ? 0 : ix + 1)] - ph[row + (ix == 0 ? N - 1 : ix - 1)];
      const double py = ph[iz * NN + (size_t)(iy == N - 1 ? 0 : iy + 1) * N + ix] -
                        ph[iz * NN + (size_t)(iy == 0 ? N - 1 : iy - 1) * N + ix];
      const double pz = ph[(size_t)(iz == N - 1 ? 0 : iz + 1) * NN + (size_t)iy * N + ix] -
                        ph[(size_t)(iz == 0 ? N - 1 : iz - 1) * NN + (size_t)iy * N + ix];
      gx += wt * px;
      gy += wt * py;
      gz += wt * pz;
      vd += wt * ph[row + ix];
    }
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    gz = warp_sum(gz);
    vd = warp_sum(vd);
    const double fe = -MAZE_KE_EV_ANGSTROM * Q / (2.0 * a.h);
    const double Fex = fe * gx, Fey = fe * gy, Fez = fe * gz;
    // --- S8: Tosi-Fumi pairs, minimum image, r < r_c. FP32 pre-filter with a
    // margin, exact FP64 test and arithmetic for the survivors.
    const float4 pi32 = a.pos32[i];
    const float Lf = a.Lf;
    double ftx = 0, fty = 0, ftz = 0, vtf = 0;
    auto visit = [&](int j) {
      if (j == i) return;
      const float4 pj = a.pos32[j];
      float dx = pj.x - pi32.x, dy = pj.y - pi32.y, dz = pj.z - pi32.z;
      const float sx = rintf(dx / Lf), sy = rintf(dy / Lf), sz = rintf(dz / Lf);
      dx -= sx * Lf;
      dy -= sy * Lf;
      dz -= sz * Lf;
      if (dx * dx + dy * dy + dz * dz >= a.rc2_filter) return;
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
            for (int u = lo + lane; u < hi; u += 32) visit(a.cell_ions[u]);
          }
        }
      }
    } else {
      for (int j = lane; j < n; j += 32) visit(j);
    }
    ftx = warp_sum(ftx);
    fty = warp_sum(fty);
    ftz = warp_sum(ftz);
    vtf = warp_sum(vtf);
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
