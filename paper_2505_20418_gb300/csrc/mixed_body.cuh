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
  __device__ bool reduce_u64(unsigned long long v, unsigned long long& out) {
    return grid_reduce_u64(v, recs, ++epoch, rec, out);
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
  // sum of one unsigned 64-bit value per thread over the cluster, modulo
  // 2^64 (exact integer total in every thread)
  __device__ bool reduce_u64(unsigned long long v, unsigned long long& out) {
    __shared__ unsigned long long s_p[2];   // [parity]: this CTA's partial
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned long long w = (unsigned long long)warp_isum((long long)v);
    if (lane == 0) s_w[warp] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long S = 0;
      for (int u = 0; u < nw; ++u) S += s_w[u];
      s_p[parity] = S;
    }
    barrier();
    if (warp == 0) {
      long long a = 0;
      if (lane < size()) {
        const unsigned loc = (unsigned)__cvta_generic_to_shared(&s_p[parity]);
        unsigned r;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(loc), "r"((unsigned)lane));
        asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(a) : "r"(r) : "memory");
      }
      const long long t = warp_isum(a);
      if (lane == 0) s_t = (unsigned long long)t;
    }
    __syncthreads();
    out = s_t;
    parity ^= 1;
    __syncthreads();
    return true;
  }
};

// ---- grid helpers --------------------------------------------------------------
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

__device__ __forceinline__ df dsum6(const float2* x, const int (&q)[6]) {
  const df a = df_add(df_from(x[q[0]]), df_from(x[q[1]]));
  const df b = df_add(df_from(x[q[2]]), df_from(x[q[3]]));
  const df c = df_add(df_from(x[q[4]]), df_from(x[q[5]]));
  return df_add(df_add(a, b), c);
}

// ---- storage of the FP32 V-cycle ----------------------------------------------
// Level l's correction x, right-hand side b and red-point residual r are held
// as z-slabs: a "part" q of Q owns planes [q P_l, min((q+1) P_l, N_l)) with
// P_l = ceil(N_l / Q) and stores x, b (P_l N_l^2 values each) and, above the
// coarsest level, r (P_l N_l^2 / 2) of every level at the same offsets.
// The smoothed levels keep x and b in red-black order: the red points (i + j
// + k even) of the part first, then the black ones, each colour plane by
// plane and row by row, point (i, j) of a row at half-row index t = i / 2.
// A half-sweep then reads whole lines of the other colour and writes whole
// lines of its own (the natural order would move every line twice); a
// point's x-neighbours sit at t or t -+ 1 of the other colour, its y- and
// z-neighbours at the same t. r holds the red points in the same order. The
// coarsest level (solved exactly, never swept) stays in natural order.
// Two forms share every phase:
//  * cluster-resident: a part per CTA of the cluster, in its dynamic shared
//    memory; planes owned by another CTA are read over DSMEM (generic
//    addresses from mapa). Threads stride over their own CTA's points.
//  * global: one part (Q = 1) in a global scratch buffer; the threads of the
//    whole sync domain stride over all points.
// Every point is computed by the same arithmetic in both forms and in either
// order, so results do not depend on the form or on how many CTAs take part.
struct RLevel {
  int N, NN, P, lg;
  int z0, z1;        // planes of this part
  unsigned off;      // float offset of x in a part; b at off + P NN, r at off + 2 P NN
  unsigned Pinv;     // ceil(2^32 / P) for P > 1: z / P = umulhi(z, Pinv) for z < 2^16
  unsigned mH, mN, mNN;  // ceil(2^32 / d) for d = N/2, N, N^2 when N <= 64 (else 0: divide)
  int split;         // x and b in red-black order (every level but the coarsest)
};

// x / d by a multiply-high with m = ceil(2^32 / d): exact while x d < 2^32
// (every index of a grid of at most 64^3 points against d <= 4096); m = 0
// falls back to the division.
__device__ __forceinline__ int fdiv(int x, int d, unsigned m) {
  return m ? (int)__umulhi((unsigned)x, m) : x / d;
}

// Plane (local), in-plane offset, row and column of the natural-order index
// m of a level: shifts when N is a power of two, else the multiply-high
// division (or the division itself above 64^3).
__device__ __forceinline__ void point_kji(const RLevel& v, int m, int& kl, int& rem, int& j, int& i) {
  if (v.lg > 0) {
    kl = m >> (2 * v.lg);
    rem = m & (v.NN - 1);
    j = rem >> v.lg;
    i = rem & (v.N - 1);
  } else {
    kl = fdiv(m, v.NN, v.mNN);
    rem = m - kl * v.NN;
    j = fdiv(rem, v.N, v.mN);
    i = rem - j * v.N;
  }
}

struct Slabs {
  float* sm;         // this part's storage
  unsigned me, Q;    // part index and count
  int L;
  int tail;          // first level held whole by part 0 (the tail of the V-cycle)
  bool dsmem;
  RLevel lv[kMaxLevels];
  // pointer to plane z (0 <= z < N_l) of array arr (0 x, 1 b) of level v (a
  // register copy of lv[l]); one part (the global form) needs no lookup
  __device__ __forceinline__ float* plane(const RLevel& v, int arr, int z) const {
    if (Q == 1) return sm + v.off + (unsigned)(arr * v.P * v.NN) + (unsigned)(z * v.NN);
    const unsigned q = v.P == 1 ? (unsigned)z : __umulhi((unsigned)z, v.Pinv);
    float* p = sm + v.off + (unsigned)(arr * v.P * v.NN) + (unsigned)((z - (int)q * v.P) * v.NN);
    if (q == me) return p;
    float* r;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(p), "r"(q));
    return r;
  }
  __device__ __forceinline__ float* plane(int l, int arr, int z) const { return plane(lv[l], arr, z); }
  // pointer to the colour-c half of plane z of array arr of a red-black
  // ordered level v (N_l^2 / 2 values, row j at j N_l / 2)
  __device__ __forceinline__ float* cplane(const RLevel& v, int arr, int c, int z) const {
    const unsigned HH = (unsigned)(v.NN >> 1);
    if (Q == 1) return sm + v.off + (unsigned)(arr * v.P * v.NN) + (unsigned)(c * v.P) * HH + (unsigned)z * HH;
    const unsigned q = v.P == 1 ? (unsigned)z : __umulhi((unsigned)z, v.Pinv);
    float* p = sm + v.off + (unsigned)(arr * v.P * v.NN) + (unsigned)(c * v.P) * HH + (unsigned)(z - (int)q * v.P) * HH;
    if (q == me) return p;
    float* r;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(p), "r"(q));
    return r;
  }
  // pointer to the red-point residuals of plane z of level v (N_l^2 / 2 values)
  __device__ __forceinline__ float* rplane(const RLevel& v, int z) const {
    if (Q == 1) return sm + v.off + (unsigned)(2 * v.P * v.NN) + (unsigned)(z * (v.NN / 2));
    const unsigned q = v.P == 1 ? (unsigned)z : __umulhi((unsigned)z, v.Pinv);
    float* p = sm + v.off + (unsigned)(2 * v.P * v.NN) + (unsigned)((z - (int)q * v.P) * (v.NN / 2));
    if (q == me) return p;
    float* r;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(p), "r"(q));
    return r;
  }
};

// The tail of the V-cycle: the coarse levels run by one CTA (part 0) with
// block barriers instead of cluster or grid barriers. In a cluster, the
// levels of at most 8^3 points (a 16^3 half-sweep already costs one SM
// ~0.8 us, as much as a cluster barrier phase; an 8^3 one ~0.2 us); in the
// global form (one part, grid barriers of ~2 us), those of at most 16^3.
// The global form keeps every level whole in its one part either way. A
// box's tail_n overrides the size (the batch autotuner chooses it).
__host__ __device__ __forceinline__ int tail_level(const MixedArgs& a, int Q) {
  const int tn = a.tail_n > 0 ? a.tail_n : (Q == 1 ? 16 : 8);
  for (int l = 0; l < a.L; ++l)
    if (a.Nl[l] <= tn) return l;
  return a.L - 1;
}

// Planes per part of level l for Q parts (tail levels: all planes in part 0).
__host__ __device__ __forceinline__ int slab_planes(const MixedArgs& a, int l, int Q) {
  return l >= tail_level(a, Q) ? a.Nl[l] : (a.Nl[l] + Q - 1) / Q;
}

// Floats of one part for Q parts.
__host__ __device__ __forceinline__ size_t slab_floats(const MixedArgs& a, int Q) {
  size_t tot = 0;
  for (int l = 0; l < a.L; ++l) {
    const size_t N = (size_t)a.Nl[l], P = (size_t)slab_planes(a, l, Q);
    tot += 2 * P * N * N + (l < a.L - 1 ? P * (N * N / 2) : 0);
  }
  return tot;
}

__host__ __device__ __forceinline__ size_t resident_bytes(const MixedArgs& a, int C) {
  return slab_floats(a, C) * sizeof(float);
}

// ceil(2^32 / d) for d >= 2 in 32-bit arithmetic: (2^32 - 1) / d + 1.
__device__ __forceinline__ unsigned ceil_recip32(unsigned d) { return 0xffffffffu / d + 1u; }

// The level descriptors of the slab storage, built by the block's first L
// threads (one level each; offsets then by a prefix sum in thread 0), then a
// block barrier.
__device__ __forceinline__ void slabs_setup(Slabs& R, const MixedArgs& a, float* sm, unsigned me, unsigned Q,
                                            bool dsmem) {
  __shared__ unsigned s_size[kMaxLevels];
  const int l = threadIdx.x;
  if (l < a.L) {
    RLevel& v = R.lv[l];
    v.N = a.Nl[l];
    v.NN = v.N * v.N;
    v.P = slab_planes(a, l, (int)Q);
    v.lg = a.lg[l];
    v.z0 = min(v.N, (int)me * v.P);
    v.z1 = min(v.N, ((int)me + 1) * v.P);
    // (P = 1 would need 2^32, which does not fit: owner() treats it apart)
    v.Pinv = v.P > 1 ? ceil_recip32((unsigned)v.P) : 0u;
    auto magic = [&](int d) -> unsigned { return (v.N <= 64 && d > 1) ? ceil_recip32((unsigned)d) : 0u; };
    v.mH = magic(v.N / 2);
    v.mN = magic(v.N);
    v.mNN = magic(v.NN);
    v.split = l < a.L - 1 ? 1 : 0;
    s_size[l] = 2u * (unsigned)(v.P * v.NN) + (l < a.L - 1 ? (unsigned)(v.P * (v.NN / 2)) : 0u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R.sm = sm;
    R.me = me;
    R.Q = Q;
    R.L = a.L;
    R.tail = tail_level(a, (int)Q);
    R.dsmem = dsmem;
    unsigned off = 0;
    for (int k = 0; k < a.L; ++k) {
      R.lv[k].off = off;
      off += s_size[k];
    }
  }
}

// Own point h of colour c (0 red = i+j+k even, 1 black) of a red-black
// ordered level v: local plane kl, row j, half-row index t (h is also the
// point's index within its colour); returns the column parity p, i = 2t + p.
__device__ __forceinline__ int colour_point(const RLevel& v, int h, int c, int& t, int& j, int& kl) {
  const int half = v.N >> 1;
  int row;
  if (v.lg > 0) {
    row = h >> (v.lg - 1);
    t = h & (half - 1);
    kl = row >> v.lg;
    j = row & (v.N - 1);
  } else {
    row = fdiv(h, half, v.mH);
    t = h - row * half;
    kl = fdiv(row, v.N, v.mN);
    j = row - kl * v.N;
  }
  return (j + v.z0 + kl + c) & 1;
}

// Sum of the six neighbours (all of the other colour, array xo of the part,
// boundary planes xlo / xhi) of the own point (t, j, kl) with parity p, in the
// fixed order ((x- + x+) + (y- + y+)) + (z- + z+).
// (F: transform of each loaded neighbour value; the identity for a sweep)
struct Ident {
  __device__ float operator()(float v) const { return v; }
};
template <class F = Ident>
__device__ __forceinline__ float colour_nbr_sum(const float* xo, const float* xlo, const float* xhi, int N, int own,
                                                int t, int j, int kl, int p, F f = F()) {
  const int H = N >> 1, HH = H * N;
  const int rowb = kl * HH + j * H;
  const float sx = f(xo[rowb + (p ? t : (t == 0 ? H - 1 : t - 1))]) + f(xo[rowb + (p ? (t == H - 1 ? 0 : t + 1) : t)]);
  const float sy =
      f(xo[kl * HH + (j == 0 ? N - 1 : j - 1) * H + t]) + f(xo[kl * HH + (j == N - 1 ? 0 : j + 1) * H + t]);
  const float zm = f(kl > 0 ? xo[rowb - HH + t] : xlo[j * H + t]);
  const float zp = f(kl < own - 1 ? xo[rowb + HH + t] : xhi[j * H + t]);
  return (sx + sy) + (zm + zp);
}

// 16-byte loads and stores of four consecutive values.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Four consecutive own points (half-row indices t .. t+3 of one row, t a
// multiple of 4, parity p): the six-neighbour sums in the order of
// colour_nbr_sum. Their y- and z-neighbours are the other colour's values at
// the same t (four loads of 16 bytes), their x-neighbours the other colour's
// t .. t+3 of the row and one more value at t-1 (p = 0) or t+4 (p = 1).
template <class F = Ident>
__device__ __forceinline__ float4 colour_nbr_sum4(const float* xo, const float* xlo, const float* xhi, int N, int own,
                                                  int t, int j, int kl, int p, F f = F()) {
  const int H = N >> 1, HH = H * N;
  const int rowb = kl * HH + j * H;
  auto f4 = [&](float4 v) { return make_float4(f(v.x), f(v.y), f(v.z), f(v.w)); };
  const float4 xr = f4(ld4(xo + rowb + t));
  const float xe = f(p ? xo[rowb + (t + 4 == H ? 0 : t + 4)] : xo[rowb + (t == 0 ? H - 1 : t - 1)]);
  const float4 ym = f4(ld4(xo + kl * HH + (j == 0 ? N - 1 : j - 1) * H + t));
  const float4 yp = f4(ld4(xo + kl * HH + (j == N - 1 ? 0 : j + 1) * H + t));
  const float4 zm = f4(ld4((kl > 0 ? xo + rowb - HH : xlo + j * H) + t));
  const float4 zp = f4(ld4((kl < own - 1 ? xo + rowb + HH : xhi + j * H) + t));
  const float4 xmn = p ? xr : make_float4(xe, xr.x, xr.y, xr.z);
  const float4 xpl = p ? make_float4(xr.y, xr.z, xr.w, xe) : xr;
  float4 s;
  s.x = ((xmn.x + xpl.x) + (ym.x + yp.x)) + (zm.x + zp.x);
  s.y = ((xmn.y + xpl.y) + (ym.y + yp.y)) + (zm.y + zp.y);
  s.z = ((xmn.z + xpl.z) + (ym.z + yp.z)) + (zm.z + zp.z);
  s.w = ((xmn.w + xpl.w) + (ym.w + yp.w)) + (zm.w + zp.w);
  return s;
}

// Levels whose rows hold a multiple of 4 values of each colour (N a multiple
// of 8) take the four-point forms; their storage offsets are then multiples
// of 16 bytes.
__device__ __forceinline__ bool quad_level(const RLevel& v) { return (v.N & 7) == 0; }

// One red-black half-sweep of colour c: x = (sum of the six neighbours - b) / 6
// at the part's points of that colour. A thread issues the loads of its
// points before their stores (the loads read the other colour, the stores
// write this one).
__device__ __forceinline__ void res_half_sweep(const Slabs& R, int l, int c, int t0, int ts) {
  const RLevel v = R.lv[l];
  const int own = v.z1 - v.z0;
  if (own <= 0) return;
  const int PH = v.P * (v.NN >> 1);
  float* xc = R.sm + v.off + c * PH;
  const float* xo = R.sm + v.off + (1 - c) * PH;
  const float* bc = R.sm + v.off + v.P * v.NN + c * PH;
  const int N = v.N;
  const int hcount = own * (v.NN >> 1);
  const float* xlo = R.cplane(v, 0, 1 - c, (v.z0 - 1 + N) % N);
  const float* xhi = R.cplane(v, 0, 1 - c, v.z1 % N);
  if (quad_level(v)) {
    for (int g = t0; g < (hcount >> 2); g += ts) {
      const int h = g << 2;
      const float4 b = ld4(bc + h);
      int t, j, kl;
      const int p = colour_point(v, h, c, t, j, kl);
      const float4 s = colour_nbr_sum4(xo, xlo, xhi, N, own, t, j, kl, p);
      st4(xc + h, make_float4((s.x - b.x) * (1.f / 6.f), (s.y - b.y) * (1.f / 6.f), (s.z - b.z) * (1.f / 6.f),
                              (s.w - b.w) * (1.f / 6.f)));
    }
    return;
  }
  for (int h0 = t0; h0 < hcount; h0 += 2 * ts) {
    float val[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int h = h0 + u * ts;
      val[u] = 0.f;
      if (h < hcount) {
        int t, j, kl;
        const int p = colour_point(v, h, c, t, j, kl);
        val[u] = (colour_nbr_sum(xo, xlo, xhi, N, own, t, j, kl, p) - bc[h]) * (1.f / 6.f);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (h0 + u * ts < hcount) xc[h0 + u * ts] = val[u];
  }
}

// The first sweep from the zero guess in one phase: the red half-sweep sets
// x = -b/6 at the red points, and the black half-sweep that follows reads
// those values, so its red neighbours are formed from b directly (the same
// products as the red half-sweep computes, hence the same values).
// (__fmul_rn: the product is rounded on its own, never contracted into the
// sum that follows, exactly as the stored red values are.)
struct NegSixth {
  __device__ float operator()(float v) const { return __fmul_rn(-v, 1.f / 6.f); }
};
__device__ __forceinline__ void res_first_sweep(const Slabs& R, int l, int t0, int ts) {
  const RLevel v = R.lv[l];
  const int own = v.z1 - v.z0;
  if (own <= 0) return;
  const int PH = v.P * (v.NN >> 1);
  float* xr = R.sm + v.off;
  float* xb = xr + PH;
  const float* br = R.sm + v.off + v.P * v.NN;
  const float* bb = br + PH;
  const int N = v.N;
  const int hcount = own * (v.NN >> 1);
  const float* blo = R.cplane(v, 1, 0, (v.z0 - 1 + N) % N);
  const float* bhi = R.cplane(v, 1, 0, v.z1 % N);
  const NegSixth f;
  if (quad_level(v)) {
    for (int g = t0; g < (hcount >> 2); g += ts) {
      const int h = g << 2;
      const float4 r = ld4(br + h);
      st4(xr + h, make_float4(f(r.x), f(r.y), f(r.z), f(r.w)));
      int t, j, kl;
      const int p = colour_point(v, h, 1, t, j, kl);
      const float4 s = colour_nbr_sum4(br, blo, bhi, N, own, t, j, kl, p, f);
      const float4 b = ld4(bb + h);
      st4(xb + h, make_float4((s.x - b.x) * (1.f / 6.f), (s.y - b.y) * (1.f / 6.f), (s.z - b.z) * (1.f / 6.f),
                              (s.w - b.w) * (1.f / 6.f)));
    }
    return;
  }
  for (int h = t0; h < hcount; h += ts) {
    xr[h] = f(br[h]);
    int t, j, kl;
    const int p = colour_point(v, h, 1, t, j, kl);
    xb[h] = (colour_nbr_sum(br, blo, bhi, N, own, t, j, kl, p, f) - bb[h]) * (1.f / 6.f);
  }
}

// Residual r = b - M x of level l at the part's red points (after the black
// half-sweep the residual at the black points is zero).
__device__ __forceinline__ void res_residual(const Slabs& R, int l, int t0, int ts) {
  const RLevel v = R.lv[l];
  const int own = v.z1 - v.z0;
  if (own <= 0) return;
  const int PH = v.P * (v.NN >> 1);
  const float* xr = R.sm + v.off;
  const float* xb = xr + PH;
  const float* br = R.sm + v.off + v.P * v.NN;
  float* r = R.sm + v.off + 2 * v.P * v.NN;
  const int N = v.N;
  const int hcount = own * (v.NN >> 1);
  const float* xlo = R.cplane(v, 0, 1, (v.z0 - 1 + N) % N);
  const float* xhi = R.cplane(v, 0, 1, v.z1 % N);
  if (quad_level(v)) {
    for (int g = t0; g < (hcount >> 2); g += ts) {
      const int h = g << 2;
      int t, j, kl;
      const int p = colour_point(v, h, 0, t, j, kl);
      const float4 s6 = colour_nbr_sum4(xb, xlo, xhi, N, own, t, j, kl, p);
      const float4 b = ld4(br + h), x = ld4(xr + h);
      st4(r + h, make_float4(b.x - (s6.x - 6.f * x.x), b.y - (s6.y - 6.f * x.y), b.z - (s6.z - 6.f * x.z),
                             b.w - (s6.w - 6.f * x.w)));
    }
    return;
  }
  for (int h = t0; h < hcount; h += ts) {
    int t, j, kl;
    const int p = colour_point(v, h, 0, t, j, kl);
    const float s6 = colour_nbr_sum(xb, xlo, xhi, N, own, t, j, kl, p);
    r[h] = br[h] - (s6 - 6.f * xr[h]);
  }
}

// Coarse rhs of level l+1 = 4 x 27-point full weighting of the fine residual
// (4 because M is h^2-scaled): with the residual zero at the black fine
// points only the centre (weight 1/8) and the 12 edge neighbours (1/32),
// all red, count. Coarse plane K is computed by the part that owns fine
// plane 2K and stored into the part that owns K (another CTA's shared
// memory when they differ), red-black ordered unless level l+1 is the
// coarsest.
__device__ __forceinline__ void res_restrict(const Slabs& R, int l, int t0, int ts) {
  const RLevel f = R.lv[l];
  const RLevel cv = R.lv[l + 1];
  const int K0 = (f.z0 + 1) / 2, own = (f.z1 + 1) / 2 - K0;
  if (own <= 0) return;
  const int N = f.N, H = N / 2, Nc = cv.N, NNc = cv.NN;
  const int count = own * NNc;
  if (quad_level(f) && cv.split) {
    // four coarse columns I .. I+3 (I a multiple of 4) of one coarse row: the
    // red fine residuals they read lie at half-row indices I-1 .. I+3 of
    // nine fine rows (16-byte loads plus one value at I-1 where needed);
    // the even columns go to colour (J + K) & 1, the odd ones to the other
    // (8-byte stores).
    const int Hc = Nc >> 1;
    for (int g = t0; g < (count >> 2); g += ts) {
      const int m = g << 2;
      int kl, rem, J, I;
      point_kji(cv, m, kl, rem, J, I);
      const int K = K0 + kl;
      const int j0 = 2 * J, jm = j0 == 0 ? N - 1 : j0 - 1, jp = j0 + 1 == N ? 0 : j0 + 1;
      const int Im = I == 0 ? H - 1 : I - 1;
      const float* rz = R.rplane(f, 2 * K);
      const float* rl = R.rplane(f, (2 * K - 1 + N) % N);
      const float* rh = R.rplane(f, (2 * K + 1) % N);
      // per fine row: the values at I .. I+3 and (where read) at I-1
      const float4 a_jm = ld4(rz + jm * H + I), a_j0 = ld4(rz + j0 * H + I), a_jp = ld4(rz + jp * H + I);
      const float e_jm = rz[jm * H + Im], e_jp = rz[jp * H + Im];
      const float4 l_j0 = ld4(rl + j0 * H + I), l_jm = ld4(rl + jm * H + I), l_jp = ld4(rl + jp * H + I);
      const float4 h_j0 = ld4(rh + j0 * H + I), h_jm = ld4(rh + jm * H + I), h_jp = ld4(rh + jp * H + I);
      const float el_j0 = rl[j0 * H + Im], eh_j0 = rh[j0 * H + Im];
      auto col = [](float4 v, float e, int u) -> float { return u == 0 ? e : (u == 1 ? v.x : (u == 2 ? v.y : v.z)); };
      auto at = [](float4 v, int u) -> float { return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w)); };
      float o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // fine columns im = 2(I+u)-1 -> half index I+u-1, ip = 2(I+u)+1 and
        // i0 = 2(I+u) -> I+u
        const float edges = ((col(a_jm, e_jm, u) + at(a_jm, u)) + (col(a_jp, e_jp, u) + at(a_jp, u))) +
                            ((col(l_j0, el_j0, u) + at(l_j0, u)) + (col(h_j0, eh_j0, u) + at(h_j0, u))) +
                            ((at(l_jm, u) + at(l_jp, u)) + (at(h_jm, u) + at(h_jp, u)));
        o[u] = 4.f * (0.125f * at(a_j0, u) + 0.03125f * edges);
      }
      const int ce = (I + J + K) & 1, th = rem >> 1;   // = J Hc + I / 2
      *reinterpret_cast<float2*>(R.cplane(cv, 1, ce, K) + th) = make_float2(o[0], o[2]);
      *reinterpret_cast<float2*>(R.cplane(cv, 1, 1 - ce, K) + th) = make_float2(o[1], o[3]);
      (void)Hc;
    }
    return;
  }
  for (int m = t0; m < count; m += ts) {
    int kl, rem, J, I;
    point_kji(cv, m, kl, rem, J, I);
    const int K = K0 + kl;
    const float* rp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) rp[d] = R.rplane(f, (2 * K - 1 + d + N) % N);
    // red-point residual at fine (i, j) of plane 2K + dz
    auto res = [&](int i, int j, int dz) -> float { return rp[dz + 1][j * H + (i >> 1)]; };
    const int i0 = 2 * I, j0 = 2 * J;
    const int im = i0 == 0 ? N - 1 : i0 - 1, ip = i0 + 1 == N ? 0 : i0 + 1;
    const int jm = j0 == 0 ? N - 1 : j0 - 1, jp = j0 + 1 == N ? 0 : j0 + 1;
    const float edges = ((res(im, jm, 0) + res(ip, jm, 0)) + (res(im, jp, 0) + res(ip, jp, 0))) +
                        ((res(im, j0, -1) + res(ip, j0, -1)) + (res(im, j0, 1) + res(ip, j0, 1))) +
                        ((res(i0, jm, -1) + res(i0, jp, -1)) + (res(i0, jm, 1) + res(i0, jp, 1)));
    const float val = 4.f * (0.125f * res(i0, j0, 0) + 0.03125f * edges);
    if (cv.split)
      R.cplane(cv, 1, (I + J + K) & 1, K)[J * (Nc >> 1) + (I >> 1)] = val;
    else
      R.plane(cv, 1, K)[J * Nc + I] = val;
  }
}

// Trilinear prolongation of level l+1's correction onto level l's black
// points (the next red half-sweep overwrites the red ones).
__device__ __forceinline__ void res_prolong(const Slabs& R, int l, int t0, int ts) {
  const RLevel f = R.lv[l];
  const RLevel cv = R.lv[l + 1];
  const int own = f.z1 - f.z0;
  if (own <= 0) return;
  float* xb = R.sm + f.off + f.P * (f.NN >> 1);
  const int Nc = cv.N, Hc = Nc >> 1, hcount = own * (f.NN >> 1);
  if (quad_level(f) && cv.split) {
    // four black points t .. t+3 of a fine row (t a multiple of 4, parity p):
    // point u reads coarse columns I0 = t + u and I1 = t + u + p of the
    // coarse rows J in {j0, j1} and planes K in {k0, k1}. Of the coarse
    // columns t .. t+4 of one (J, K), the even ones lie in colour (J + K) & 1
    // at half-row indices t/2 .. t/2 + 2 and the odd ones in the other
    // colour at t/2, t/2 + 1 (8-byte loads; t + 4 wraps to column 0).
    for (int g = t0; g < (hcount >> 2); g += ts) {
      const int h = g << 2;
      int t, j, kl;
      const int p = colour_point(f, h, 1, t, j, kl);
      const int k = f.z0 + kl;
      const int j0 = j >> 1, j1 = (j & 1) ? (j0 + 1 == Nc ? 0 : j0 + 1) : j0;
      const int k0 = k >> 1, k1 = (k & 1) ? (k0 + 1 == Nc ? 0 : k0 + 1) : k0;
      const int th = t >> 1, te = t + 4 == Nc ? 0 : th + 2;
      float V[4][5];   // [(J, K) = (j0,k0), (j1,k0), (j0,k1), (j1,k1)][column t .. t+4]
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int J = (q & 1) ? j1 : j0, K = (q & 2) ? k1 : k0;
        const int ce = (J + K) & 1;
        const float* pe = R.cplane(cv, 0, ce, K) + J * Hc;
        const float* po = R.cplane(cv, 0, 1 - ce, K) + J * Hc;
        const float2 ev = *reinterpret_cast<const float2*>(pe + th);
        const float2 od = *reinterpret_cast<const float2*>(po + th);
        V[q][0] = ev.x;
        V[q][1] = od.x;
        V[q][2] = ev.y;
        V[q][3] = od.y;
        V[q][4] = p ? pe[te] : 0.f;
      }
      float4 x = ld4(xb + h);
      float o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // column I1 is t + u + p (a select: no runtime index into V)
        const float b0 = p ? V[0][u + 1] : V[0][u], b1 = p ? V[1][u + 1] : V[1][u];
        const float b2 = p ? V[2][u + 1] : V[2][u], b3 = p ? V[3][u + 1] : V[3][u];
        o[u] = 0.125f * (((V[0][u] + b0) + (V[1][u] + b1)) + ((V[2][u] + b2) + (V[3][u] + b3)));
      }
      x.x += o[0];
      x.y += o[1];
      x.z += o[2];
      x.w += o[3];
      st4(xb + h, x);
    }
    return;
  }
  for (int h = t0; h < hcount; h += ts) {
    int t, j, kl;
    const int p = colour_point(f, h, 1, t, j, kl);
    const int i = 2 * t + p;
    const int k = f.z0 + kl;
    const int i0 = i >> 1, i1 = (i & 1) ? (i0 + 1 == Nc ? 0 : i0 + 1) : i0;
    const int j0 = j >> 1, j1 = (j & 1) ? (j0 + 1 == Nc ? 0 : j0 + 1) : j0;
    const int k0 = k >> 1, k1 = (k & 1) ? (k0 + 1 == Nc ? 0 : k0 + 1) : k0;
    float c8[8];
    if (cv.split) {
      // coarse point (I, J, K) lies in colour (I + J + K) & 1 at J Hc + I / 2
      const float* c0r = R.cplane(cv, 0, 0, k0);
      const float* c0b = R.cplane(cv, 0, 1, k0);
      const float* c1r = R.cplane(cv, 0, 0, k1);
      const float* c1b = R.cplane(cv, 0, 1, k1);
      auto at = [&](int I, int J, int K, const float* pr, const float* pb) -> float {
        return (((I + J + K) & 1) ? pb : pr)[J * Hc + (I >> 1)];
      };
      c8[0] = at(i0, j0, k0, c0r, c0b);
      c8[1] = at(i1, j0, k0, c0r, c0b);
      c8[2] = at(i0, j1, k0, c0r, c0b);
      c8[3] = at(i1, j1, k0, c0r, c0b);
      c8[4] = at(i0, j0, k1, c1r, c1b);
      c8[5] = at(i1, j0, k1, c1r, c1b);
      c8[6] = at(i0, j1, k1, c1r, c1b);
      c8[7] = at(i1, j1, k1, c1r, c1b);
    } else {
      const float* c0 = R.plane(cv, 0, k0);
      const float* c1 = R.plane(cv, 0, k1);
      c8[0] = c0[j0 * Nc + i0];
      c8[1] = c0[j0 * Nc + i1];
      c8[2] = c0[j1 * Nc + i0];
      c8[3] = c0[j1 * Nc + i1];
      c8[4] = c1[j0 * Nc + i0];
      c8[5] = c1[j0 * Nc + i1];
      c8[6] = c1[j1 * Nc + i0];
      c8[7] = c1[j1 * Nc + i1];
    }
    xb[h] += 0.125f * (((c8[0] + c8[1]) + (c8[2] + c8[3])) + ((c8[4] + c8[5]) + (c8[6] + c8[7])));
  }
}

// Coarsest level (at most 8^3 points, solved by one CTA): the exact
// zero-mean solve. M is circulant, so the discrete Fourier transform
// diagonalises it: x = F^-1 (F b / lambda) with lambda(k) = 2 (cos kx + cos
// ky + cos kz) - 6 and the k = 0 mode dropped. The three forward and three
// inverse passes are direct N_c-point transforms along one axis each, one
// point per thread (s_re / s_im in shared memory, the pass's outputs kept in
// registers across a barrier); s_il holds 1/(N_c^3 lambda), s_tc / s_ts the
// cosines and sines of 2 pi t / N_c, s_co the packed coordinates. Needs
// blockDim.x >= N_c^3 (512 threads).
__device__ __noinline__ void res_coarsest(const Slabs& R, const float* s_il, const float* s_tc, const float* s_ts,
                                          const int* s_co, float* s_re, float* s_im, maze_stats* rec) {
  const int l = R.L - 1;
  const RLevel& v = R.lv[l];
  const int Nc = v.N, NNc = v.NN, nc3 = Nc * NNc;
  // (the host admits coarsest levels of at most 8^3 points and launches 512
  // or more threads; anything else is an error, never an overrun)
  if (Nc > 8 || nc3 > (int)blockDim.x) {
    if (threadIdx.x == 0) atomicCAS(&rec->status, MAZE_OK, MAZE_ERR_INVALID);
    return;
  }
  const int p = threadIdx.x;
  int pi = 0, pj = 0, pk = 0;
  if (p < nc3) {
    const int c = s_co[p];
    pi = c & 255;
    pj = (c >> 8) & 255;
    pk = c >> 16;
    s_re[p] = R.plane(l, 1, pk)[pj * Nc + pi];
    s_im[p] = 0.f;
  }
  __syncthreads();
  for (int pass = 0; pass < 6; ++pass) {
    const int ax = pass % 3;
    const float sg = pass < 3 ? -1.f : 1.f;   // forward e^{-i..}, inverse e^{+i..}
    float re = 0.f, im = 0.f;
    if (p < nc3) {
      const int idx = ax == 0 ? pi : (ax == 1 ? pj : pk);
      const int stride = ax == 0 ? 1 : (ax == 1 ? Nc : NNc);
      const int base = p - idx * stride;
      int t = 0;   // idx * m mod N_c
      for (int m = 0; m < Nc; ++m) {
        const float ar = s_re[base + m * stride], ai = s_im[base + m * stride];
        const float c = s_tc[t], sn = sg * s_ts[t];
        re += ar * c - ai * sn;
        im += ar * sn + ai * c;
        t += idx;
        if (t >= Nc) t -= Nc;
      }
      if (pass == 2) {
        re *= s_il[p];
        im *= s_il[p];
      }
    }
    __syncthreads();
    if (p < nc3) {
      s_re[p] = re;
      s_im[p] = im;
    }
    __syncthreads();
  }
  if (p < nc3) R.plane(l, 0, pk)[pj * Nc + pi] = s_re[p];
}

// Level-0 pointers of the outer passes. The arrays are distinct (the three
// potentials rotate through separate buffers, y and y2 are separate, the
// V-cycle storage is its own region), so the passes take them as restrict
// parameters: each point's loads may then issue together, ahead of the
// previous point's stores.
//
// S4 fused with the first outer residual r = sigma_p - M y at the part's
// level-0 points: phi_p and sigma_p written, r into the V-cycle's level-0
// right-hand side b0 (red-black order), max|r| and max|y| returned.
// A point pair (i0, i0 + 1) of a row and the neighbours of both: x- of the
// first, x+ of the second, and the pairs of the rows j -+ 1 and planes
// k -+ 1 (16-byte loads; m even).
struct Pair6 {
  float2 a, b, xm, xp, jmA, jmB, jpA, jpB, kmA, kmB, kpA, kpB;
};
__device__ __forceinline__ Pair6 load_pair6(const float2* __restrict__ x, int m, int xm, int xp, int jm, int jp,
                                            int km, int kp) {
  auto ld = [&](int at, float2& u, float2& w) {
    const float4 v = *reinterpret_cast<const float4*>(x + at);
    u = make_float2(v.x, v.y);
    w = make_float2(v.z, v.w);
  };
  Pair6 P;
  ld(m, P.a, P.b);
  P.xm = x[xm];
  P.xp = x[xp];
  ld(jm, P.jmA, P.jmB);
  ld(jp, P.jpA, P.jpB);
  ld(km, P.kmA, P.kmB);
  ld(kp, P.kpA, P.kpB);
  return P;
}
// Six double-float values summed by Sum2 (Ogita, Rump and Oishi, SIAM J.
// Sci. Comput. 26, 2005): the high parts by an error-free TwoSum chain whose
// errors collect with the low parts in c, then one renormalisation; the
// accuracy of a double-float sum at ~40 % of its operations.
__device__ __forceinline__ df sum6_df(float2 x0, float2 x1, float2 x2, float2 x3, float2 x4, float2 x5) {
  const float2 x[6] = {x0, x1, x2, x3, x4, x5};
  float sh = x[0].x, c = 0.f;
#pragma unroll
  for (int u = 1; u < 6; ++u) {
    const float s2 = __fadd_rn(sh, x[u].x);
    const float bb = __fsub_rn(s2, sh);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(sh, __fsub_rn(s2, bb)), __fsub_rn(x[u].x, bb)));
    sh = s2;
  }
  c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fadd_rn(x[0].y, x[1].y), __fadd_rn(x[2].y, x[3].y)), __fadd_rn(x[4].y, x[5].y)));
  const float h = __fadd_rn(sh, c);
  return {h, __fsub_rn(c, __fsub_rn(h, sh))};
}
// the six-neighbour sums of the pair (x-, x+, y-, y+, z-, z+)
__device__ __forceinline__ df pair_sumA(const Pair6& P) { return sum6_df(P.xm, P.b, P.jmA, P.jpA, P.kmA, P.kpA); }
__device__ __forceinline__ df pair_sumB(const Pair6& P) { return sum6_df(P.a, P.xp, P.jmB, P.jpB, P.kmB, P.kpB); }

// S4 for one point from its potentials' centre values and neighbour sums:
// phi_p = 2 phi_k - phi_{k-1} (or phi_k, or 0) and M phi_p.
__device__ __forceinline__ void s4_php(bool zero_phi, bool static_guess, float2 pk, float2 pm, df nk, df nm, df& php,
                                       df& Mphp) {
  php = {0.f, 0.f};
  Mphp = {0.f, 0.f};
  if (zero_phi) {
  } else if (static_guess) {
    php = df_from(pk);
    Mphp = df_sub(nk, df_mul_f(php, 6.f));
  } else {
    php = df_sub(df_twice(df_from(pk)), df_from(pm));
    const df s6 = df_sub(df_twice(nk), nm);
    Mphp = df_sub(s6, df_mul_f(php, 6.f));
  }
}

// S4 fused with the first outer residual r = sigma_p - M y at the part's
// level-0 points: phi_p and sigma_p written, r into the V-cycle's level-0
// right-hand side b0 (red-black order), max|r| and max|y| returned. A thread
// takes two x-adjacent points at a time (16-byte loads and stores).
__device__ __forceinline__ void s4_pass(const RLevel& v0, int t0, int ts, df c_sig, bool zero_phi, bool static_guess,
                                        unsigned long long* __restrict__ qfix, double* __restrict__ q_out,
                                        const float2* __restrict__ phk, const float2* __restrict__ phm,
                                        float2* __restrict__ phout, float2* __restrict__ sig,
                                        const float2* __restrict__ y, float* __restrict__ b0, float& rmax_o,
                                        float& ymax_o) {
  const int N0 = v0.N, NN0 = v0.NN, cnt0 = (v0.z1 - v0.z0) * NN0, H0 = N0 >> 1, HH0 = NN0 >> 1;
  const int PH0 = v0.P * HH0;
  float rmax = 0.f, ymax = 0.f;
  for (int g = t0; g < (cnt0 >> 1); g += ts) {
    const int ml = g << 1;
    int kl, rem, j, i0;
    point_kji(v0, ml, kl, rem, j, i0);
    const int k = v0.z0 + kl;
    const int m = k * NN0 + rem;
    const int xm = i0 == 0 ? m + N0 - 1 : m - 1, xp = i0 + 2 == N0 ? m + 2 - N0 : m + 2;
    const int jm = j == 0 ? m + NN0 - N0 : m - N0, jp = j == N0 - 1 ? m - NN0 + N0 : m + N0;
    const int km = k == 0 ? m + NN0 * (N0 - 1) : m - NN0, kp = k == N0 - 1 ? m - NN0 * (N0 - 1) : m + NN0;
    const ulonglong2 qq = *reinterpret_cast<const ulonglong2*>(qfix + m);
    const long long qA = (long long)qq.x, qB = (long long)qq.y;
    df phA, phB, MA, MB;
    if (zero_phi) {
      s4_php(true, false, {}, {}, {}, {}, phA, MA);
      s4_php(true, false, {}, {}, {}, {}, phB, MB);
    } else {
      const Pair6 K6 = load_pair6(phk, m, xm, xp, jm, jp, km, kp);
      const df nkA = pair_sumA(K6), nkB = pair_sumB(K6);
      if (static_guess) {
        s4_php(false, true, K6.a, {}, nkA, {}, phA, MA);
        s4_php(false, true, K6.b, {}, nkB, {}, phB, MB);
      } else {
        const Pair6 M6 = load_pair6(phm, m, xm, xp, jm, jp, km, kp);
        s4_php(false, false, K6.a, M6.a, nkA, pair_sumA(M6), phA, MA);
        s4_php(false, false, K6.b, M6.b, nkB, pair_sumB(M6), phB, MB);
      }
    }
    const df sgA = df_add(df_mul(MA, c_sig), df_from_fix(qA)), sgB = df_add(df_mul(MB, c_sig), df_from_fix(qB));
    const Pair6 Y6 = load_pair6(y, m, xm, xp, jm, jp, km, kp);
    const df yA = df_from(Y6.a), yB = df_from(Y6.b);
    const df rA = df_sub(sgA, df_sub(pair_sumA(Y6), df_mul_f(yA, 6.f)));
    const df rB = df_sub(sgB, df_sub(pair_sumB(Y6), df_mul_f(yB, 6.f)));
    const float rfA = rA.h + rA.l, rfB = rB.h + rB.l;
    *reinterpret_cast<ulonglong2*>(qfix + m) = make_ulonglong2(0ull, 0ull);
    if (q_out) *reinterpret_cast<double2*>(q_out + m) = make_double2((double)qA * kQInv, (double)qB * kQInv);
    *reinterpret_cast<float4*>(phout + m) = make_float4(phA.h, phA.l, phB.h, phB.l);
    *reinterpret_cast<float4*>(sig + m) = make_float4(sgA.h, sgA.l, sgB.h, sgB.l);
    const int c0 = (i0 + j + k) & 1, hb = kl * HH0 + j * H0 + (i0 >> 1);
    b0[c0 * PH0 + hb] = rfA;
    b0[(1 - c0) * PH0 + hb] = rfB;
    ymax = fmaxf(ymax, fmaxf(abs_nan_inf(yA.h), abs_nan_inf(yB.h)));
    rmax = fmaxf(rmax, fmaxf(abs_nan_inf(rfA), abs_nan_inf(rfB)));
  }
  rmax_o = rmax;
  ymax_o = ymax;
}

// One point of the update pass: y_next = y + e (returned in ynew) and the
// residual r = sigma_p - (sum of the six (y + e) neighbours - 6 y_next) as a
// float; yn / en are the neighbours' y and e in the order x-, x+, y-, y+,
// z-, z+.
__device__ __forceinline__ void upd_point(const float2 (&yn)[6], const float (&en)[6], float2 yo, float eo, float2 sg,
                                          float2& ynew, float& rf) {
  // the neighbour sum of y + e: the high parts summed error-free (TwoSum
  // chain, errors collected in c), the low parts and the corrections e added
  // into c, one renormalisation (Ogita, Rump and Oishi's Sum2, SIAM J. Sci.
  // Comput. 26, 2005): the accuracy of the double-float sum at ~40 % of its
  // operations
  float sh = yn[0].x, c = 0.f;
#pragma unroll
  for (int u = 1; u < 6; ++u) {
    const float s2 = __fadd_rn(sh, yn[u].x);
    const float bb = __fsub_rn(s2, sh);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(sh, __fsub_rn(s2, bb)), __fsub_rn(yn[u].x, bb)));
    sh = s2;
  }
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(yn[0].y, yn[1].y), __fadd_rn(yn[2].y, yn[3].y)),
                             __fadd_rn(yn[4].y, yn[5].y));
  const float es = __fadd_rn(__fadd_rn(__fadd_rn(en[0], en[1]), __fadd_rn(en[2], en[3])), __fadd_rn(en[4], en[5]));
  c = __fadd_rn(c, __fadd_rn(lo, es));
  const float snh = __fadd_rn(sh, c);
  const df sn = {snh, __fsub_rn(c, __fsub_rn(snh, sh))};
  const df ym = df_add_f(df_from(yo), eo);
  const df r = df_sub(df_from(sg), df_sub(sn, df_mul_f(ym, 6.f)));
  ynew = df_to(ym);
  rf = r.h + r.l;
}

// y_next = y + e and the next outer residual r = sigma_p - M y_next at the
// part's level-0 points (e0: this part's correction, red-black ordered;
// elo0/elo1, ehi0/ehi1: red / black halves of the neighbouring parts'
// boundary planes); r into b0 (red-black order), max|r| and max|y_next|
// returned. A thread takes two x-adjacent points at a time (one of each
// colour): 16-byte loads of y and sigma_p, each point's partner supplies one
// of its x-neighbours.
__device__ __forceinline__ void update_pass(const RLevel& v0, int t0, int ts, const float* __restrict__ e0,
                                            const float* elo0, const float* elo1, const float* ehi0,
                                            const float* ehi1, const float2* __restrict__ ycur,
                                            float2* __restrict__ ynext, const float2* __restrict__ sig,
                                            float* __restrict__ b0, float& rmax_o, float& ymax_o) {
  const int N0 = v0.N, NN0 = v0.NN, own0 = v0.z1 - v0.z0, cnt0 = own0 * NN0;
  const int H0 = N0 >> 1, HH0 = NN0 >> 1, PH0 = v0.P * HH0;
  auto ld2x2 = [](const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  };
  float rmax = 0.f, ymax = 0.f;
  for (int g = t0; g < (cnt0 >> 1); g += ts) {
    const int ml = g << 1;
    int kl, rem, j, i0;
    point_kji(v0, ml, kl, rem, j, i0);
    const int k = v0.z0 + kl;
    const int m = k * NN0 + rem;
    // the pair: A = (i0, j, k) of colour c0, B = (i0 + 1, j, k) of colour 1 - c0
    const int c0 = (i0 + j + k) & 1, t = i0 >> 1, rowb = kl * HH0 + j * H0;
    const float* EA = e0 + c0 * PH0;
    const float* EB = e0 + (1 - c0) * PH0;
    const int rjm = kl * HH0 + (j == 0 ? N0 - 1 : j - 1) * H0 + t, rjp = kl * HH0 + (j == N0 - 1 ? 0 : j + 1) * H0 + t;
    const float* lA = kl > 0 ? EB + rowb - HH0 : (c0 ? elo0 : elo1) + j * H0;
    const float* lB = kl > 0 ? EA + rowb - HH0 : (c0 ? elo1 : elo0) + j * H0;
    const float* hA = kl < own0 - 1 ? EB + rowb + HH0 : (c0 ? ehi0 : ehi1) + j * H0;
    const float* hB = kl < own0 - 1 ? EA + rowb + HH0 : (c0 ? ehi1 : ehi0) + j * H0;
    const float eA = EA[rowb + t], eB = EB[rowb + t];
    const float enA[6] = {EB[rowb + (i0 == 0 ? H0 - 1 : t - 1)], eB, EB[rjm], EB[rjp], lA[t], hA[t]};
    const float enB[6] = {eA, EA[rowb + (i0 + 2 == N0 ? 0 : t + 1)], EA[rjm], EA[rjp], lB[t], hB[t]};
    float2 yA, yB, ymA, ymB, ypA, ypB, zmA, zmB, zpA, zpB, sA, sB;
    ld2x2(ycur + m, yA, yB);
    ld2x2(ycur + (j == 0 ? m + NN0 - N0 : m - N0), ymA, ymB);
    ld2x2(ycur + (j == N0 - 1 ? m - NN0 + N0 : m + N0), ypA, ypB);
    ld2x2(ycur + (k == 0 ? m + NN0 * (N0 - 1) : m - NN0), zmA, zmB);
    ld2x2(ycur + (k == N0 - 1 ? m - NN0 * (N0 - 1) : m + NN0), zpA, zpB);
    ld2x2(sig + m, sA, sB);
    const float2 yxm = ycur[i0 == 0 ? m + N0 - 1 : m - 1];
    const float2 yxp = ycur[i0 + 2 == N0 ? m + 2 - N0 : m + 2];
    const float2 ynA[6] = {yxm, yB, ymA, ypA, zmA, zpA};
    const float2 ynB[6] = {yA, yxp, ymB, ypB, zmB, zpB};
    float2 nA, nB;
    float rA, rB;
    upd_point(ynA, enA, yA, eA, sA, nA, rA);
    upd_point(ynB, enB, yB, eB, sB, nB, rB);
    *reinterpret_cast<float4*>(ynext + m) = make_float4(nA.x, nA.y, nB.x, nB.y);
    b0[c0 * PH0 + rowb + t] = rA;
    b0[(1 - c0) * PH0 + rowb + t] = rB;
    ymax = fmaxf(ymax, fmaxf(abs_nan_inf(nA.x), abs_nan_inf(nB.x)));
    rmax = fmaxf(rmax, fmaxf(abs_nan_inf(rA), abs_nan_inf(rB)));
  }
  rmax_o = rmax;
  ymax_o = ymax;
}

// update_pass on four-point levels: a thread takes four x-adjacent points
// P0 .. P3 (i0 a multiple of 4; P0, P2 of colour c0 at half-row indices t,
// t+1, P1, P3 of the other colour at the same indices), each with the
// arithmetic and neighbour order of update_pass (same results): 16-byte
// loads of y, sigma_p and the neighbour rows, 8-byte loads of e, 8-byte
// stores of r.
__device__ __forceinline__ void update_pass4(const RLevel& v0, int t0, int ts, const float* __restrict__ e0,
                                             const float* elo0, const float* elo1, const float* ehi0,
                                             const float* ehi1, const float2* __restrict__ ycur,
                                             float2* __restrict__ ynext, const float2* __restrict__ sig,
                                             float* __restrict__ b0, float& rmax_o, float& ymax_o) {
  const int N0 = v0.N, NN0 = v0.NN, own0 = v0.z1 - v0.z0, cnt0 = own0 * NN0;
  const int H0 = N0 >> 1, HH0 = NN0 >> 1, PH0 = v0.P * HH0;
  auto ld2x2 = [](const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  };
  auto ldf2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
  float rmax = 0.f, ymax = 0.f;
  for (int g = t0; g < (cnt0 >> 2); g += ts) {
    const int ml = g << 2;
    int kl, rem, j, i0;
    point_kji(v0, ml, kl, rem, j, i0);
    const int k = v0.z0 + kl;
    const int m = k * NN0 + rem;
    const int c0 = (i0 + j + k) & 1, t = i0 >> 1, rowb = kl * HH0 + j * H0;
    const float* EA = e0 + c0 * PH0;
    const float* EB = e0 + (1 - c0) * PH0;
    const int rjm = kl * HH0 + (j == 0 ? N0 - 1 : j - 1) * H0 + t, rjp = kl * HH0 + (j == N0 - 1 ? 0 : j + 1) * H0 + t;
    const float* lA = kl > 0 ? EB + rowb - HH0 : (c0 ? elo0 : elo1) + j * H0;
    const float* lB = kl > 0 ? EA + rowb - HH0 : (c0 ? elo1 : elo0) + j * H0;
    const float* hA = kl < own0 - 1 ? EB + rowb + HH0 : (c0 ? ehi0 : ehi1) + j * H0;
    const float* hB = kl < own0 - 1 ? EA + rowb + HH0 : (c0 ? ehi1 : ehi0) + j * H0;
    const float2 eA = ldf2(EA + rowb + t), eB = ldf2(EB + rowb + t);
    const float eBm = EB[rowb + (t == 0 ? H0 - 1 : t - 1)], eAp = EA[rowb + (t + 2 == H0 ? 0 : t + 2)];
    const float2 eBjm = ldf2(EB + rjm), eBjp = ldf2(EB + rjp), eAjm = ldf2(EA + rjm), eAjp = ldf2(EA + rjp);
    const float2 lA2 = ldf2(lA + t), lB2 = ldf2(lB + t), hA2 = ldf2(hA + t), hB2 = ldf2(hB + t);
    float2 y0, y1, y2, y3, ym0, ym1, ym2, ym3, yp0, yp1, yp2, yp3, zm0, zm1, zm2, zm3, zp0, zp1, zp2, zp3, s0, s1, s2, s3;
    const int mjm = j == 0 ? m + NN0 - N0 : m - N0, mjp = j == N0 - 1 ? m - NN0 + N0 : m + N0;
    const int mkm = k == 0 ? m + NN0 * (N0 - 1) : m - NN0, mkp = k == N0 - 1 ? m - NN0 * (N0 - 1) : m + NN0;
    ld2x2(ycur + m, y0, y1);
    ld2x2(ycur + m + 2, y2, y3);
    ld2x2(ycur + mjm, ym0, ym1);
    ld2x2(ycur + mjm + 2, ym2, ym3);
    ld2x2(ycur + mjp, yp0, yp1);
    ld2x2(ycur + mjp + 2, yp2, yp3);
    ld2x2(ycur + mkm, zm0, zm1);
    ld2x2(ycur + mkm + 2, zm2, zm3);
    ld2x2(ycur + mkp, zp0, zp1);
    ld2x2(ycur + mkp + 2, zp2, zp3);
    ld2x2(sig + m, s0, s1);
    ld2x2(sig + m + 2, s2, s3);
    const float2 yxm = ycur[i0 == 0 ? m + N0 - 1 : m - 1];
    const float2 yxp = ycur[i0 + 4 == N0 ? m + 4 - N0 : m + 4];
    float2 n0, n1, n2, n3;
    float r0, r1, r2, r3;
    {
      const float2 yn[6] = {yxm, y1, ym0, yp0, zm0, zp0};
      const float en[6] = {eBm, eB.x, eBjm.x, eBjp.x, lA2.x, hA2.x};
      upd_point(yn, en, y0, eA.x, s0, n0, r0);
    }
    {
      const float2 yn[6] = {y0, y2, ym1, yp1, zm1, zp1};
      const float en[6] = {eA.x, eA.y, eAjm.x, eAjp.x, lB2.x, hB2.x};
      upd_point(yn, en, y1, eB.x, s1, n1, r1);
    }
    {
      const float2 yn[6] = {y1, y3, ym2, yp2, zm2, zp2};
      const float en[6] = {eB.x, eB.y, eBjm.y, eBjp.y, lA2.y, hA2.y};
      upd_point(yn, en, y2, eA.y, s2, n2, r2);
    }
    {
      const float2 yn[6] = {y2, yxp, ym3, yp3, zm3, zp3};
      const float en[6] = {eA.y, eAp, eAjm.y, eAjp.y, lB2.y, hB2.y};
      upd_point(yn, en, y3, eB.y, s3, n3, r3);
    }
    *reinterpret_cast<float4*>(ynext + m) = make_float4(n0.x, n0.y, n1.x, n1.y);
    *reinterpret_cast<float4*>(ynext + m + 2) = make_float4(n2.x, n2.y, n3.x, n3.y);
    *reinterpret_cast<float2*>(b0 + c0 * PH0 + rowb + t) = make_float2(r0, r2);
    *reinterpret_cast<float2*>(b0 + (1 - c0) * PH0 + rowb + t) = make_float2(r1, r3);
    ymax = fmaxf(ymax, fmaxf(fmaxf(abs_nan_inf(n0.x), abs_nan_inf(n1.x)), fmaxf(abs_nan_inf(n2.x), abs_nan_inf(n3.x))));
    rmax = fmaxf(rmax, fmaxf(fmaxf(abs_nan_inf(r0), abs_nan_inf(r1)), fmaxf(abs_nan_inf(r2), abs_nan_inf(r3))));
  }
  rmax_o = rmax;
  ymax_o = ymax;
}

// The solve (S4-S6) shared by every launch form. ``S`` is the sync domain;
// ``dsm`` is the CTA's dynamic shared memory for the cluster-resident form,
// or nullptr for the global form (a.scratch). The outer SHAKE iteration
// runs on double-float y (double-buffered: y_next = y + e is formed inside
// the next residual pass), the V-cycle on the FP32 slabs.
template <class S>
__device__ void mixed_body(const MixedArgs& a, S& sync, float* dsm) {
  __shared__ Slabs R;
  const unsigned me = (unsigned)sync.rank(), C = (unsigned)sync.size();
  const int tid = (int)me * blockDim.x + threadIdx.x;
  const int stride = (int)C * blockDim.x;
  // the coarsest level's pseudo-inverse kernel, staged once per solve
  __shared__ float s_cg[512];   // 1/(N_c^3 lambda) of the coarsest level
  __shared__ int s_co[512];
  __shared__ float s_re[512], s_im[512];
  __shared__ float s_tc[8], s_ts[8];
  if (dsm)
    slabs_setup(R, a, dsm, me, C, true);
  else
    slabs_setup(R, a, a.scratch, 0, 1, false);
  {
    const int Nc = a.Nl[a.L - 1];
    // (at most 8^3 values: larger coarsest levels are rejected below)
    if (threadIdx.x < Nc && Nc <= 8) {
      s_tc[threadIdx.x] = a.gkerf[Nc * Nc * Nc + threadIdx.x];
      s_ts[threadIdx.x] = a.gkerf[Nc * Nc * Nc + Nc + threadIdx.x];
    }
    for (int q = threadIdx.x; q < min(Nc * Nc * Nc, 512); q += blockDim.x) {
      s_cg[q] = a.gkerf[q];
      const int qk = q / (Nc * Nc), qj = (q - qk * Nc * Nc) / Nc;
      s_co[q] = (q - qk * Nc * Nc - qj * Nc) | (qj << 8) | (qk << 16);
    }
  }
  __syncthreads();
  // the storage must hold the layout (uniform decision: every CTA computes
  // the same sizes); a mismatch is an error, never an out-of-bounds access
  unsigned dyn_bytes;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
  if (dsm ? resident_bytes(a, (int)C) > (size_t)dyn_bytes : slab_floats(a, 1) > a.scratch_floats) {
    if (tid == 0) a.rec->status = MAZE_ERR_INVALID;
    sync.barrier();
    return;
  }
  // this thread's first point and stride within its part
  const int t0 = dsm ? (int)threadIdx.x : tid, ts = dsm ? (int)blockDim.x : stride;
  const df c_sig = {a.c_sig_h, a.c_sig_l};
  const df c_phi = {a.c_phi_h, a.c_phi_l};
  const bool mmax[2] = {true, true};
  const RLevel v0 = R.lv[0];
  const int N0 = v0.N, NN0 = v0.NN, own0 = v0.z1 - v0.z0, cnt0 = own0 * NN0;
  float* e0 = R.sm + v0.off;
  float* r0 = e0 + v0.P * NN0;
  float2* ycur = a.y;
  float2* ynext = a.y2;
  int it = 0;
  double res = 0.0, ymax_all = 0.0;
  // ---- S4 fused with the first outer residual r = sigma_p - M y
  {
    float rmax, ymax;
    s4_pass(v0, t0, ts, c_sig, a.zero_phi, a.static_guess, a.qfix, a.q_out, a.phi_k, a.phi_km1, a.phi_out, a.sigma,
            ycur, r0, rmax, ymax);
    const double vv[2] = {(double)rmax, (double)ymax};
    double t[2];
    if (!sync.reduce(vv, mmax, t)) return;
    res = t[0];
    ymax_all = t[1];
  }
  while (isfinite(res) && isfinite(ymax_all) && !(res < a.tol) && it < a.max_iter) {
    // ---- FP32 V-cycle on M e = r from e = 0: the levels above the tail
    // across the sync domain, the tail in one CTA
    const int lt = R.tail;
    for (int l = 0; l < lt; ++l) {
      res_first_sweep(R, l, t0, ts);
      if (!sync.barrier()) return;
      for (int s = 1; s < a.nu1; ++s)
        for (int c = 0; c < 2; ++c) {
          res_half_sweep(R, l, c, t0, ts);
          if (!sync.barrier()) return;
        }
      res_residual(R, l, t0, ts);
      if (!sync.barrier()) return;
      res_restrict(R, l, t0, ts);
      if (!sync.barrier()) return;
    }
    if (lt == a.L - 1) {
      // the coarsest level alone below the domain's levels: its exact solve
      // in the first CTA
      if (sync.rank() == 0) res_coarsest(R, s_cg, s_tc, s_ts, s_co, s_re, s_im, a.rec);
      if (!sync.barrier()) return;
    } else if (sync.rank() == 0) {
      const int u0 = threadIdx.x, us = blockDim.x;
      for (int l = lt; l < a.L - 1; ++l) {
        res_first_sweep(R, l, u0, us);
        __syncthreads();
        for (int s = 1; s < a.nu1; ++s)
          for (int c = 0; c < 2; ++c) {
            res_half_sweep(R, l, c, u0, us);
            __syncthreads();
          }
        res_residual(R, l, u0, us);
        __syncthreads();
        res_restrict(R, l, u0, us);
        __syncthreads();
      }
      res_coarsest(R, s_cg, s_tc, s_ts, s_co, s_re, s_im, a.rec);
      __syncthreads();
      for (int l = a.L - 2; l >= lt; --l) {
        res_prolong(R, l, u0, us);
        __syncthreads();
        for (int s = 0; s < a.nu2; ++s)
          for (int c = 0; c < 2; ++c) {
            res_half_sweep(R, l, c, u0, us);
            __syncthreads();
          }
      }
    }
    if (lt > 0 && lt < a.L - 1 && !sync.barrier()) return;
    for (int l = lt - 1; l >= 0; --l) {
      res_prolong(R, l, t0, ts);
      if (!sync.barrier()) return;
      for (int s = 0; s < a.nu2; ++s)
        for (int c = 0; c < 2; ++c) {
          res_half_sweep(R, l, c, t0, ts);
          if (!sync.barrier()) return;
        }
    }
    if (lt == 0 && !sync.barrier()) return;
    // ---- y_next = y + e and the next outer residual r = sigma_p - M y_next
    {
      const int zlo = (v0.z0 - 1 + N0) % N0, zhi = v0.z1 % N0;
      float rmax, ymax;
      if (quad_level(v0))
        update_pass4(v0, t0, ts, e0, R.cplane(v0, 0, 0, zlo), R.cplane(v0, 0, 1, zlo), R.cplane(v0, 0, 0, zhi),
                     R.cplane(v0, 0, 1, zhi), ycur, ynext, a.sigma, r0, rmax, ymax);
      else
        update_pass(v0, t0, ts, e0, R.cplane(v0, 0, 0, zlo), R.cplane(v0, 0, 1, zlo), R.cplane(v0, 0, 0, zhi),
                    R.cplane(v0, 0, 1, zhi), ycur, ynext, a.sigma, r0, rmax, ymax);
      ++it;
      float2* t2 = ycur;
      ycur = ynext;
      ynext = t2;
      const double vv[2] = {(double)rmax, (double)ymax};
      double t[2];
      if (!sync.reduce(vv, mmax, t)) return;
      res = t[0];
      ymax_all = t[1];
    }
  }
  // ---- S6: mean of y, exact and independent of how the points are split:
  // every point's hi and lo parts are rounded to one fixed-point grid set by
  // max|y| over the box (2^-41 of it) and the integers are summed modulo
  // 2^64 across the domain (the true sum fits). Then the correction
  // phi = phi_p - (4pi/h)(y - mean y) and y -> a.y.
  {
    const int E = dbl_exp(ymax_all) + 11;
    unsigned long long u = 0;
    if (ymax_all > 0.0) {
      const float2* yc = ycur + v0.z0 * NN0;
      for (int ml = t0; ml < cnt0; ml += 4 * ts) {
        float2 yv[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) yv[w] = ml + w * ts < cnt0 ? yc[ml + w * ts] : make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          u += (unsigned long long)(dbl_to_fix((double)yv[w].x, E) + dbl_to_fix((double)yv[w].y, E));
      }
    }
    unsigned long long tot;
    if (!sync.reduce_u64(u, tot)) return;
    const double ybar = ymax_all > 0.0 ? fix_to_dbl((long long)tot, E) * a.inv_n : 0.0;
    const float ybh = (float)ybar;
    const df yb = {ybh, (float)(ybar - (double)ybh)};
    for (int ml = t0; ml < cnt0; ml += 2 * ts) {
      // both points' loads ahead of the stores (a.y may be ycur itself)
      const int m0 = v0.z0 * NN0 + ml, m1 = m0 + ts;
      const bool two = ml + ts < cnt0;
      const float2 y0 = ycur[m0], p0 = a.phi_out[m0];
      const float2 y1 = two ? ycur[m1] : make_float2(0.f, 0.f), p1 = two ? a.phi_out[m1] : make_float2(0.f, 0.f);
      const df yv0 = df_sub(df_from(y0), yb), yv1 = df_sub(df_from(y1), yb);
      a.y[m0] = df_to(yv0);
      a.phi_out[m0] = df_to(df_sub(df_from(p0), df_mul(yv0, c_phi)));
      if (two) {
        a.y[m1] = df_to(yv1);
        a.phi_out[m1] = df_to(df_sub(df_from(p1), df_mul(yv1, c_phi)));
      }
    }
  }
  if (tid == 0) {
    maze_stats* r = a.rec;
    r->iters = it;
    r->resid = res * a.res_scale;
    r->total_iters += it;
    if (!isfinite(res) || !isfinite(ymax_all)) r->status = MAZE_ERR_NONFINITE;
    else if (!(res < a.tol)) r->status = MAZE_ERR_NOT_CONVERGED;
  }
  // no block leaves (or reuses its shared memory) while another may still
  // read it
  sync.barrier();
}

}  // namespace

}  // namespace maze
