// Mixed-precision S4-S6 (precision MAZE_MIXED), multigrid solver: the device
// body, shared by the single-box launch forms and the batched step kernel.
//
// The outer SHAKE iteration keeps FP64-level accuracy without FP64
// instructions (GB300 runs FP64 at 1/64 of the FP32 rate): phi^k, phi^{k-1},
// phi_p, y and sigma_p are stored as double-float pairs (hi + lo, two FP32
// values, ~48-bit significand) and combined with error-free transformations
// (Knuth's TwoSum, Dekker's FastTwoSum, and the FMA-based TwoProduct). Each
// outer iteration
//   r = sigma_p - M y                         (double-float; max|r| is the
//                                              paper's residual, Eq. res_poisson_maze)
//   e = V-cycle(M e = r) from e = 0           (FP32: smoothing, residual,
//                                              full weighting, prolongation)
//   y = y + e                                 (double-float)
// is, by linearity, the same V-cycle the FP64 solver applies to (y, sigma_p),
// so iteration counts match the FP64 path. S4 and S6 (Eqs. SHAKE,
// SHAKEPhiFinal) run in double-float. Grid reductions are exact integer sums
// (FP64-grade), as in the FP64 kernels.
//
// Two launch forms share one body: a single thread-block cluster (small
// boxes; hardware cluster barriers and DSMEM reductions) and a cooperative
// grid (any box; grid barriers and flag-carrying reductions).
#pragma once
#include <math.h>

#include "maze_internal.cuh"

namespace maze {

namespace {

// ---- double-float arithmetic ------------------------------------------------
struct df {
  float h, l;
};

__device__ __forceinline__ df df_from(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 df_to(df a) { return make_float2(a.h, a.l); }

// Knuth TwoSum of the high parts, low parts added, FastTwoSum renormalise.
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b) {
  const float s = __fadd_rn(a.h, b);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  e = __fadd_rn(e, a.l);
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

// a * b for double-float b (TwoProduct with FMA for the high parts).
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// a * 2 (exact per part).
__device__ __forceinline__ df df_twice(df a) { return {a.h * 2.f, a.l * 2.f}; }

// a * c for a float c (TwoProduct of the high part, low part added).
__device__ __forceinline__ df df_mul_f(df a, float c) {
  const float p = __fmul_rn(a.h, c);
  float e = __fmaf_rn(a.h, c, -p);
  e = __fmaf_rn(a.l, c, e);
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// Fixed-point grid charge (2^-50 e units) as a double-float.
__device__ __forceinline__ df df_from_fix(long long x) {
  const float h = (float)x;  // rounds to 24 bits
  const long long rest = x - (long long)h;
  return {h * (float)kQInv, (float)rest * (float)kQInv};
}

// ---- sync domains ------------------------------------------------------------
struct GridSync {
  LLRec* recs;
  unsigned* bar;
  maze_stats* rec;
  unsigned epoch = 0, bar_epoch = 0;
  __device__ int rank() const { return blockIdx.x; }
  __device__ int size() const { return gridDim.x; }
  __device__ bool barrier() { return grid_barrier(bar, bar_epoch, rec); }
  template <int K>
  __device__ bool reduce(const double (&v)[K], const bool (&is_max)[K], double (&out)[K]) {
    return grid_reduce<K>(v, is_max, recs, ++epoch, rec, out);
  }
};

// One cluster: barrier.cluster for synchronisation; reductions combine the
// CTAs' exact block partials read from each CTA's shared memory over DSMEM.
struct ClusterSync {
  int parity = 0;
  __device__ int rank() const {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
  }
  __device__ int size() const {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return (int)r;
  }
  __device__ bool barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  }
  template <int K>
  __device__ bool reduce(const double (&v)[K], const bool (&is_max)[K], double (&out)[K]) {
    static_assert(K <= 8, "at most 8 values per reduction");
    __shared__ long long s_part[2][8][2];   // [parity][k] {S or max bits, E}
    __shared__ long long s_w[32][8];
    __shared__ int s_e[32][8];
    __shared__ double s_out[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (is_max[k]) {
        const unsigned long long m = warp_umax64((unsigned long long)__double_as_longlong(fabs(v[k])));
        if (lane == 0) s_w[warp][k] = (long long)m;
      } else {
        const int e = (int)__reduce_max_sync(0xffffffffu, (unsigned)dbl_exp(v[k]));
        if (lane == 0) s_e[warp][k] = e;
      }
    }
    __syncthreads();
    int Eb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (is_max[k]) continue;
      int E = 0;
      for (int u = 0; u < nw; ++u) E = max(E, s_e[u][k]);
      Eb[k] = E;
      const long long S = warp_isum(dbl_to_fix(v[k], E));
      if (lane == 0) s_w[warp][k] = S;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (is_max[k]) {
          unsigned long long m = 0;
          for (int u = 0; u < nw; ++u) m = max(m, (unsigned long long)s_w[u][k]);
          s_part[parity][k][0] = (long long)m;
          s_part[parity][k][1] = 0;
        } else {
          long long S = 0;
          for (int u = 0; u < nw; ++u) S += s_w[u][k];
          s_part[parity][k][0] = S;
          s_part[parity][k][1] = Eb[k];
        }
      }
    }
    barrier();
    if (warp == 0) {
      const int nc = size();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        long long a = 0, e = 0;
        if (lane < nc) {
          const unsigned loc0 = (unsigned)__cvta_generic_to_shared(&s_part[parity][k][0]);
          unsigned r0, r1;
          asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r0) : "r"(loc0), "r"((unsigned)lane));
          asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r1) : "r"(loc0 + 8u), "r"((unsigned)lane));
          asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(a) : "r"(r0) : "memory");
          asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(e) : "r"(r1) : "memory");
        }
        double tot;
        if (is_max[k]) {
          tot = __longlong_as_double((long long)warp_umax64((unsigned long long)a));
        } else {
          // re-align the CTAs' exact partials to the largest exponent
          const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
          const double part = fix_to_dbl(a, (int)e);
          tot = fix_to_dbl(warp_isum(dbl_to_fix(part, E + 11)), E + 11);
        }
        if (lane == 0) s_out[k] = tot;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = s_out[k];
    parity ^= 1;
    __syncthreads();
    return true;
  }
};

// ---- grid helpers --------------------------------------------------------------
// Point of colour c (0 red, 1 black) with half-index h on an N^3 grid, N
// even; lg = log2(N) when N is a power of two (shifts), else -1.
__device__ __forceinline__ int colour_point(int h, int N, int lg, int c, int& i, int& j, int& k) {
  int row, t;
  if (lg > 0) {
    row = h >> (lg - 1);
    t = h & ((N >> 1) - 1);
    k = row >> lg;
    j = row & (N - 1);
  } else {
    const int half = N >> 1;
    row = h / half;
    t = h - row * half;
    k = row / N;
    j = row - k * N;
  }
  i = 2 * t + ((j + k + c) & 1);
  return i + N * (j + N * k);
}

__device__ __forceinline__ void split3(int m, int N, int lg, int& i, int& j, int& k) {
  if (lg > 0) {
    i = m & (N - 1);
    j = (m >> lg) & (N - 1);
    k = m >> (2 * lg);
  } else {
    k = m / (N * N);
    j = (m / N) % N;
    i = m % N;
  }
}

__device__ __forceinline__ int wrapi(int a, int N) { return a < 0 ? a + N : (a >= N ? a - N : a); }

template <typename T>
__device__ __forceinline__ void nbr_idx(int i, int j, int k, int N, int (&q)[6]) {
  const int NN = N * N, n = i + N * j + NN * k;
  q[0] = i == 0 ? n + N - 1 : n - 1;
  q[1] = i == N - 1 ? n - N + 1 : n + 1;
  q[2] = j == 0 ? n + NN - N : n - N;
  q[3] = j == N - 1 ? n - NN + N : n + N;
  q[4] = k == 0 ? n + NN * (N - 1) : n - NN;
  q[5] = k == N - 1 ? n - NN * (N - 1) : n + NN;
}

__device__ __forceinline__ float fsum6(const float* x, const int (&q)[6]) {
  return ((x[q[0]] + x[q[1]]) + (x[q[2]] + x[q[3]])) + (x[q[4]] + x[q[5]]);
}

__device__ __forceinline__ df dsum6(const float2* x, const int (&q)[6]) {
  const df a = df_add(df_from(x[q[0]]), df_from(x[q[1]]));
  const df b = df_add(df_from(x[q[2]]), df_from(x[q[3]]));
  const df c = df_add(df_from(x[q[4]]), df_from(x[q[5]]));
  return df_add(df_add(a, b), c);
}

// One red-black half-sweep of colour c on a level: x = (sum of the six
// neighbours - b) / 6 at every point of that colour (from_zero: the level's
// guess is zero, so x = -b/6). A thread takes up to four points per round and
// issues all of their loads before any store (the loads read the other
// colour, the stores write this one, so batching is exact).
__device__ __forceinline__ void half_sweep(float* x, const float* __restrict__ b, int N, int lg, int c,
                                           bool from_zero, int tid, int stride) {
  const int hcount = N * N * N / 2;
  for (int h0 = tid; h0 < hcount; h0 += 4 * stride) {
    int mm[4];
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int h = h0 + u * stride;
      mm[u] = -1;
      v[u] = 0.f;
      if (h < hcount) {
        int i, j, k;
        mm[u] = colour_point(h, N, lg, c, i, j, k);
        if (from_zero) {
          v[u] = -b[mm[u]] * (1.f / 6.f);
        } else {
          int q[6];
          nbr_idx<float>(i, j, k, N, q);
          v[u] = (fsum6(x, q) - b[mm[u]]) * (1.f / 6.f);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (mm[u] >= 0) x[mm[u]] = v[u];
  }
}

// The body shared by both launch forms. ``S`` is the sync domain; the
// participating blocks stride over the points with tid/stride.
template <class S>
__device__ void mixed_body(const MixedArgs& a, S& sync) {
  const int n = a.n, N0 = a.N;
  const int tid = sync.rank() * blockDim.x + threadIdx.x;
  const int stride = sync.size() * blockDim.x;
  const df c_sig = {a.c_sig_h, a.c_sig_l};
  const df c_phi = {a.c_phi_h, a.c_phi_l};
  const bool mmax[2] = {true, true};
  const bool msum[4] = {false, false, false, false};

  // ---- S4: phi_p = 2 phi^k - phi^{k-1}, sigma_p = (h/4pi) M phi_p + q
  for (int m = tid; m < n; m += stride) {
    int i, j, k;
    split3(m, N0, a.lg[0], i, j, k);
    int q[6];
    nbr_idx<float>(i, j, k, N0, q);
    const long long qi = (long long)a.qfix[m];
    a.qfix[m] = 0ull;
    if (a.q_out) a.q_out[m] = (double)qi * kQInv;
    df php = {0.f, 0.f}, Mphp = {0.f, 0.f};
    if (a.zero_phi) {
    } else if (a.static_guess) {
      php = df_from(a.phi_k[m]);
      Mphp = df_sub(dsum6(a.phi_k, q), df_mul_f(php, 6.f));
    } else {
      php = df_sub(df_twice(df_from(a.phi_k[m])), df_from(a.phi_km1[m]));
      const df nk = dsum6(a.phi_k, q), nm = dsum6(a.phi_km1, q);
      const df s6 = df_sub(df_twice(nk), nm);
      Mphp = df_sub(s6, df_mul_f(php, 6.f));
    }
    a.phi_out[m] = df_to(php);
    a.sigma[m] = df_to(df_add(df_mul(Mphp, c_sig), df_from_fix(qi)));
  }
  if (!sync.barrier()) return;

  int it = 0;
  double res = 0.0, ymax_all = 0.0;
  while (true) {
    // ---- outer residual r = sigma - M y (double-float), its max, r -> FP32
    {
      float rmax = 0.f, ymax = 0.f;
      for (int m0 = tid; m0 < n; m0 += 2 * stride) {
        float rf[2];
        int mm[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int m = m0 + u * stride;
          mm[u] = m < n ? m : -1;
          rf[u] = 0.f;
          if (m < n) {
            int i, j, k;
            split3(m, N0, a.lg[0], i, j, k);
            int q[6];
            nbr_idx<float>(i, j, k, N0, q);
            const df ym = df_from(a.y[m]);
            ymax = fmaxf(ymax, fabsf(ym.h));
            const df My = df_sub(dsum6(a.y, q), df_mul_f(ym, 6.f));
            const df r = df_sub(df_from(a.sigma[m]), My);
            rf[u] = r.h + r.l;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (mm[u] >= 0) {
            a.r0[mm[u]] = rf[u];
            rmax = fmaxf(rmax, fabsf(rf[u]));
          }
      }
      const double v[2] = {(double)rmax, (double)ymax};
      double t[2];
      if (!sync.reduce(v, mmax, t)) return;
      res = t[0];
      ymax_all = t[1];
    }
    if (!isfinite(res) || res < a.tol || it >= a.max_iter) break;
    // ---- FP32 V-cycle on M e = r from e = 0
    for (int l = 0; l < a.L - 1; ++l) {
      const int N = a.Nl[l], NN = N * N, hcount = N * NN / 2, lg = a.lg[l];
      float* x = l == 0 ? a.e0 : a.lx + a.off[l];
      const float* __restrict__ b = l == 0 ? a.r0 : a.lb + a.off[l];
      for (int s = 0; s < a.nu1; ++s) {
        for (int c = 0; c < 2; ++c) {
          half_sweep(x, b, N, lg, c, s == 0 && c == 0, tid, stride);
          if (!sync.barrier()) return;
        }
      }
      float* __restrict__ rl = a.lr + a.off[l];
      const float* __restrict__ xr = x;
      for (int m = tid; m < N * NN; m += stride) {
        int i, j, k;
        split3(m, N, lg, i, j, k);
        int q[6];
        nbr_idx<float>(i, j, k, N, q);
        rl[m] = b[m] - (fsum6(xr, q) - 6.f * xr[m]);
      }
      if (!sync.barrier()) return;
      // coarse rhs = 4 * 27-point full weighting of the residual
      const int Nc = a.Nl[l + 1], NNc = Nc * Nc;
      float* bc = a.lb + a.off[l + 1];
      for (int m = tid; m < Nc * NNc; m += stride) {
        const int K = m / NNc, J = (m - K * NNc) / Nc, I = m - K * NNc - J * Nc;
        float acc = 0.f;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
          const int z = wrapi(2 * K + dz, N);
          const float wz = dz == 0 ? 0.5f : 0.25f;
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrapi(2 * J + dy, N);
            const float wzy = wz * (dy == 0 ? 0.5f : 0.25f);
            const float* row = rl + (size_t)z * NN + (size_t)yy * N;
            acc += wzy * (0.25f * row[wrapi(2 * I - 1, N)] + 0.5f * row[2 * I] + 0.25f * row[wrapi(2 * I + 1, N)]);
          }
        }
        bc[m] = 4.f * acc;
      }
      if (!sync.barrier()) return;
    }
    {
      // coarsest: exact zero-mean solve by the pseudo-inverse kernel. Every
      // block stages the coarse rhs and the kernel (at most 7^3 values each)
      // in shared memory; one warp per output point splits the sum.
      __shared__ float s_cb[343], s_cg[343];
      const int Nc = a.Nl[a.L - 1], NNc = Nc * Nc, nc3 = Nc * NNc;
      const float* bc = a.lb + a.off[a.L - 1];
      float* xc = a.lx + a.off[a.L - 1];
      for (int q = threadIdx.x; q < nc3; q += blockDim.x) {
        s_cb[q] = bc[q];
        s_cg[q] = a.gkerf[q];
      }
      __syncthreads();
      const int lane = threadIdx.x & 31;
      const int wid = tid >> 5, nwarps = stride >> 5;
      for (int p = wid; p < nc3; p += nwarps) {
        const int pk = p / NNc, pj = (p - pk * NNc) / Nc, pi = p - pk * NNc - pj * Nc;
        float acc = 0.f;
        for (int q = lane; q < nc3; q += 32) {
          const int qk = q / NNc, qj = (q - qk * NNc) / Nc, qi = q - qk * NNc - qj * Nc;
          acc += s_cg[wrapi(pi - qi, Nc) + Nc * (wrapi(pj - qj, Nc) + Nc * wrapi(pk - qk, Nc))] * s_cb[q];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) xc[p] = acc;
      }
      if (!sync.barrier()) return;
    }
    for (int l = a.L - 2; l >= 0; --l) {
      const int N = a.Nl[l], NN = N * N, hcount = N * NN / 2, lg = a.lg[l];
      const int Nc = a.Nl[l + 1], NNc = Nc * Nc;
      float* x = l == 0 ? a.e0 : a.lx + a.off[l];
      const float* __restrict__ b = l == 0 ? a.r0 : a.lb + a.off[l];
      const float* __restrict__ xc = a.lx + a.off[l + 1];
      for (int h = tid; h < hcount; h += stride) {
        int i, j, k;
        const int m = colour_point(h, N, lg, 1, i, j, k);
        const int i0 = i >> 1, i1 = (i & 1) ? wrapi(i0 + 1, Nc) : i0;
        const int j0 = j >> 1, j1 = (j & 1) ? wrapi(j0 + 1, Nc) : j0;
        const int k0 = k >> 1, k1 = (k & 1) ? wrapi(k0 + 1, Nc) : k0;
        const float* c0 = xc + (size_t)k0 * NNc;
        const float* c1 = xc + (size_t)k1 * NNc;
        x[m] += 0.125f * (((c0[j0 * Nc + i0] + c0[j0 * Nc + i1]) + (c0[j1 * Nc + i0] + c0[j1 * Nc + i1])) +
                          ((c1[j0 * Nc + i0] + c1[j0 * Nc + i1]) + (c1[j1 * Nc + i0] + c1[j1 * Nc + i1])));
      }
      if (!sync.barrier()) return;
      for (int s = 0; s < a.nu2; ++s) {
        for (int c = 0; c < 2; ++c) {
          half_sweep(x, b, N, lg, c, false, tid, stride);
          if (!sync.barrier()) return;
        }
      }
    }
    // ---- y += e (double-float)
    for (int m = tid; m < n; m += stride) a.y[m] = df_to(df_add_f(df_from(a.y[m]), a.e0[m]));
    ++it;
    if (!sync.barrier()) return;
  }
  // ---- S6: mean of y, exact and independent of how the points are split
  // over blocks: every point's hi and lo parts are rounded to one fixed-point
  // grid set by max|y| over the box (2^-41 of it), the integers are summed
  // modulo 2^64 (the true sum fits), and the sum crosses the domain as four
  // 16-bit chunk sums, small integers that the reduction adds exactly.
  {
    const int E = dbl_exp(ymax_all) + 11;
    unsigned long long u = 0;
    if (ymax_all > 0.0)
      for (int m = tid; m < n; m += stride) {
        const float2 yv = a.y[m];
        u += (unsigned long long)(dbl_to_fix((double)yv.x, E) + dbl_to_fix((double)yv.y, E));
      }
    const double v[4] = {(double)(u & 0xffffu), (double)((u >> 16) & 0xffffu), (double)((u >> 32) & 0xffffu),
                         (double)(u >> 48)};
    double t[4];
    if (!sync.reduce(v, msum, t)) return;
    const unsigned long long tot = (unsigned long long)(long long)t[0] + ((unsigned long long)(long long)t[1] << 16) +
                                   ((unsigned long long)(long long)t[2] << 32) +
                                   ((unsigned long long)(long long)t[3] << 48);
    const double ybar = ymax_all > 0.0 ? fix_to_dbl((long long)tot, E) * a.inv_n : 0.0;
    const float ybh = (float)ybar;
    const df yb = {ybh, (float)(ybar - (double)ybh)};
    for (int m = tid; m < n; m += stride) {
      const df yv = df_sub(df_from(a.y[m]), yb);
      a.y[m] = df_to(yv);
      a.phi_out[m] = df_to(df_sub(df_from(a.phi_out[m]), df_mul(yv, c_phi)));
    }
  }
  if (tid == 0) {
    maze_stats* r = a.rec;
    r->iters = it;
    r->resid = res * a.res_scale;
    r->total_iters += it;
    if (!isfinite(res)) r->status = MAZE_ERR_NONFINITE;
    else if (!(res < a.tol)) r->status = MAZE_ERR_NOT_CONVERGED;
  }
  // no block leaves while another may still read its shared memory (DSMEM)
  sync.barrier();
}

}  // namespace

}  // namespace maze
