// Ion-side kernels of the single-box MaZe step (bodies in ion_body.cuh):
//   k_move, k_spread  S1 half kick + drift and S3 charge spreading
//   k_cell_*          S2 cell list (counting sort, deterministic order within a cell)
//   k_forces*         S7 gather of Eq. F_nostra, S8 Tosi-Fumi pairs, S9 half kick,
//                     energies and momentum (deterministic block + last-block sums)
#include "ion_body.cuh"

namespace maze {

// S1: one thread per ion. The first kernel of a step decides, once, whether
// the step runs at all.
__global__ void __launch_bounds__(kIonThreads) k_move(IonArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool skip = a.rec->status != MAZE_OK;
  if (i == 0) *a.gate = skip ? 1 : 0;
  if (skip) return;
  if (i < a.n) move_ion(a, i);
}

// S3: one warp per ion.
__global__ void __launch_bounds__(kSpreadThreads) k_spread(IonArgs a) {
  if (*a.gate) return;
  const int i = blockIdx.x * (kSpreadThreads / 32) + (threadIdx.x >> 5);
  if (i < a.n) spread_ion(a, i, threadIdx.x & 31);
}

__global__ void k_q_to_double(const unsigned long long* qfix, double* q, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = fix_to_dbl((long long)qfix[i], 1075 - 50);   // qfix 2^-50
}

cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t s, int part) {
  if (part != 2) k_move<<<(a.n + kIonThreads - 1) / kIonThreads, kIonThreads, 0, s>>>(a);
  if (a.qfix && part != 1) {
    const int per = kSpreadThreads / 32;
    k_spread<<<(a.n + per - 1) / per, kSpreadThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// The read-back of maze_step_io's exchange, by the SMs on pinned host
// memory (device addresses of the host allocations; no copy engine between
// the step's kernels and the host): the device's [3][n] positions and
// velocities (velocities after positions) -> [n][3] order into the arrays
// the exchange descriptor names, and the record's words. (The inputs are
// read by the step's S1 itself: IonArgs::io.)

__global__ void k_io_out(const double* __restrict__ soa, const IoDesc* __restrict__ io, int n,
                         const unsigned long long* __restrict__ rec, unsigned long long* __restrict__ rec_out,
                         int rec_words) {
  const int n3 = 3 * n;
  double* const po = io->pos_out;
  double* const vo = io->vel_out;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n3 + rec_words; e += gridDim.x * blockDim.x) {
    if (e < 2 * n3) {
      const int a = e >= n3 ? 1 : 0, r = e - a * n3, i = r / 3, d = r - 3 * i;
      (a ? vo : po)[r] = soa[a * n3 + d * n + i];
    } else {
      rec_out[e - 2 * n3] = rec[e - 2 * n3];
    }
  }
}

static int io_blocks(int items) { return std::max(1, std::min(1216, (items + 255) / 256)); }

cudaError_t launch_io_out(const double* soa, const IoDesc* io, int n, const void* rec, void* rec_out, size_t rec_bytes,
                          cudaStream_t s) {
  const int words = (int)(rec_bytes / 8);
  k_io_out<<<io_blocks(6 * n + words), 256, 0, s>>>(soa, io, n, static_cast<const unsigned long long*>(rec),
                                                    static_cast<unsigned long long*>(rec_out), words);
  return cudaGetLastError();
}

cudaError_t launch_q_to_double(const unsigned long long* qfix, double* q, int n, cudaStream_t s) {
  k_q_to_double<<<(n + 255) / 256, 256, 0, s>>>(qfix, q, n);
  return cudaGetLastError();
}

// S2: one block scans, one thread per ion claims a slot, one warp per cell sorts.
__global__ void k_cell_scan(CellArgs a) { cell_scan_block(a); }

// The same scan with the counts staged in shared memory (boxes whose counts
// fit): coalesced loads and stores instead of each thread walking its own
// run of cells in global memory; each thread then scans a contiguous run of
// the staged counts, and one block scan joins the runs.
__global__ void __launch_bounds__(1024) k_cell_scan_smem(CellArgs a) {
  extern __shared__ int s_cnt[];             // [ncell]
  __shared__ int s_part[1024];
  const int T = blockDim.x, nc = a.ncell;
  for (int c = threadIdx.x; c < nc; c += T) {
    s_cnt[c] = a.cell_count[c];
    a.cell_count[c] = 0;                     // cleared for the next step
  }
  __syncthreads();
  const int chunk = (nc + T - 1) / T;
  const int lo = min(threadIdx.x * chunk, nc), hi = min(lo + chunk, nc);
  int sum = 0;
  for (int c = lo; c < hi; ++c) sum += s_cnt[c];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {          // Hillis-Steele inclusive scan of the runs' sums
    const int v = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s_part[threadIdx.x] - sum;
  for (int c = lo; c < hi; ++c) {            // exclusive prefix sums, in place
    const int v = s_cnt[c];
    s_cnt[c] = run;
    run += v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += T) {
    const int v = s_cnt[c];
    a.cell_start[c] = v;
    a.cursor[c] = v;
  }
  if (threadIdx.x == T - 1) a.cell_start[nc] = s_part[T - 1];
}

__global__ void k_cell_fill(CellArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) cell_fill_ion(a, i);
}

constexpr int kSortWarps = 4;
__global__ void __launch_bounds__(kSortWarps * 32) k_cell_sort(CellArgs a) {
  __shared__ int s_ids[kSortWarps][kSortCap];
  const int warp = threadIdx.x >> 5;
  const int c = blockIdx.x * kSortWarps + warp;
  if (c < a.ncell) cell_sort_one(a, c, threadIdx.x & 31, s_ids[warp]);
}

cudaError_t launch_cells(const CellArgs& a, cudaStream_t s) {
  int dev = 0, smem_max = 0;                 // opt-in shared memory per block of this device
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    smem_max = 0;
  }
  const int need = a.ncell * (int)sizeof(int);
  if (need + 8192 <= smem_max) {             // (the static 4 KB of partial sums beside it)
    cudaError_t e = cudaFuncSetAttribute(k_cell_scan_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e != cudaSuccess) return e;
    k_cell_scan_smem<<<1, 1024, need, s>>>(a);
  } else {
    k_cell_scan<<<1, 1024, 0, s>>>(a);
  }
  k_cell_fill<<<(a.n + 255) / 256, 256, 0, s>>>(a);
  k_cell_sort<<<(a.ncell + kSortWarps - 1) / kSortWarps, kSortWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

// Exact sum (integer fixed point at the largest exponent + 16, see
// grid_reduce) of the seven values of partials [first, first + count) of
// part (8 doubles per partial), by all threads of the block; every thread
// gets the seven totals, each rounded once to a double.
__device__ __forceinline__ void combine_partials(const double* part, int first, int count, double (&tot)[7]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ int c_e[32][8];
  __shared__ long long c_s[32][8];
  __shared__ int c_E[8];
  __shared__ double c_tot[8];
  int e[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int bb = threadIdx.x; bb < count; bb += blockDim.x)
#pragma unroll
    for (int k = 0; k < 7; ++k) e[k] = max(e[k], dbl_exp(__ldcg(&part[(first + bb) * 8 + k])));
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int m = (int)__reduce_max_sync(0xffffffffu, (unsigned)e[k]);
    if (lane == 0) c_e[warp][k] = m;
  }
  __syncthreads();
  if (warp == 0 && lane < 7) {
    int m = 0;
    for (int u = 0; u < nw; ++u) m = max(m, c_e[u][lane]);
    c_E[lane] = m + 16;   // up to 2^25 partials
  }
  __syncthreads();
  long long x[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int bb = threadIdx.x; bb < count; bb += blockDim.x)
#pragma unroll
    for (int k = 0; k < 7; ++k) x[k] += dbl_to_fix(__ldcg(&part[(first + bb) * 8 + k]), c_E[k]);
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const long long S = warp_isum(x[k]);
    if (lane == 0) c_s[warp][k] = S;
  }
  __syncthreads();
  if (warp == 0 && lane < 7) {
    long long S = 0;
    for (int u = 0; u < nw; ++u) S += c_s[u][lane];
    c_tot[lane] = fix_to_dbl(S, c_E[lane]);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 7; ++k) tot[k] = c_tot[k];
  __syncthreads();
}

// Deterministic energy sums: every thread holds the terms of the ions it
// finished; the block sums them exactly (integer fixed point, see
// grid_reduce) and rounds the block's sums once; the last block to finish
// combines all block partials the same way and publishes the step record.
// Large grids (more than 2 kEnergyGroup blocks) combine in two
// levels: the last block of each group of kEnergyGroup blocks combines its
// group into a group partial, the last group combines the groups, so that no
// single block sweeps every partial. ticket[0] counts groups (or blocks),
// ticket[1 + g] the blocks of group g; all reset by their last user.
__device__ __forceinline__ void energy_reduce(const ForceArgs& a, const double (&acc)[7]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ int s_e[32][8];
  __shared__ long long s_s[32][8];
  __shared__ int s_E[8];
  __shared__ int s_last;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int e = (int)__reduce_max_sync(0xffffffffu, (unsigned)dbl_exp(acc[k]));
    if (lane == 0) s_e[warp][k] = e;
  }
  __syncthreads();
  if (warp == 0 && lane < 7) {
    int m = 0;
    for (int u = 0; u < nw; ++u) m = max(m, s_e[u][lane]);
    s_E[lane] = m + 4;   // headroom for the sum over warps
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const long long S = warp_isum(dbl_to_fix(acc[k], s_E[k]));
    if (lane == 0) s_s[warp][k] = S;
  }
  __syncthreads();
  const int G = gridDim.x;
  const bool two_level = G > 2 * kEnergyGroup;
  const int ngroups = (G + kEnergyGroup - 1) / kEnergyGroup;
  const int g = blockIdx.x / kEnergyGroup;
  if (warp == 0) {
    if (lane < 7) {
      long long S = 0;
      for (int u = 0; u < nw; ++u) S += s_s[u][lane];
      a.part[blockIdx.x * 8 + lane] = fix_to_dbl(S, s_E[lane]);
      __threadfence();
    }
    __syncwarp();
    if (lane == 0) {
      if (two_level) {
        const int gsize = min(kEnergyGroup, G - g * kEnergyGroup);
        s_last = atomicAdd(&a.ticket[1 + g], 1u) == (unsigned)(gsize - 1) ? 1 : 0;
      } else {
        s_last = atomicAdd(a.ticket, 1u) == (unsigned)(G - 1) ? 2 : 0;
      }
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot[7];
  if (s_last == 1) {
    // the group's last block: its group partial, then the group ticket
    const int gsize = min(kEnergyGroup, G - g * kEnergyGroup);
    combine_partials(a.part, g * kEnergyGroup, gsize, tot);
    if (threadIdx.x == 0) {
      a.ticket[1 + g] = 0;
      for (int k = 0; k < 7; ++k) a.part[(G + g) * 8 + k] = tot[k];
      __threadfence();
      s_last = atomicAdd(a.ticket, 1u) == (unsigned)(ngroups - 1) ? 2 : 0;
    }
    __syncthreads();
    if (s_last != 2) return;
    __threadfence();
    combine_partials(a.part, G, ngroups, tot);
  } else {
    combine_partials(a.part, 0, G, tot);
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

// One warp per ion (small boxes: the pair work spread over every SM). The
// warps leave their sums in shared memory and the block finishes its ions
// one per thread (FP64 work on full lanes).
__global__ void __launch_bounds__(kForceThreads) k_forces(ForceArgs a) {
  constexpr int kW = kForceThreads / 32;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kW + warp;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  __shared__ int s_queue[kW][64];
  __shared__ double s_r[kW][8];
  const bool live = forces_live(a);
  if (i < a.n && live) {
    double r[8];
    forces_ion_warp(a, i, lane, s_queue[warp], r);
    if (lane == 0)
      for (int k = 0; k < 8; ++k) s_r[warp][k] = r[k];
  }
  __syncthreads();
  if (live && threadIdx.x < kW) {
    const int ii = blockIdx.x * kW + threadIdx.x;
    if (ii < a.n) {
      const double* r = s_r[threadIdx.x];
      finish_ion(a, ii, r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7], acc);
    }
  }
  energy_reduce(a, acc);
}

// One block per (cell, slice): small boxes split each cell's ions over
// several blocks so that the grid fills the GPU.
__global__ void __launch_bounds__(kForceThreads) k_forces_cells(ForceArgs a) {
  __shared__ CellSmem<kForceThreads / 32> sm;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (forces_live(a)) {
    const int c = blockIdx.x / a.cell_split, s = blockIdx.x - c * a.cell_split;
    forces_cell_slice<kForceThreads / 32>(a, c, s, a.cell_split, sm, acc);
  }
  energy_reduce(a, acc);
}

// S8 alone, one block per (cell, slice): the pair sums of every ion to
// a.pair_out (run beside the solve, which it does not depend on).
__global__ void __launch_bounds__(kForceThreads) k_pairs_cells(ForceArgs a) {
  __shared__ CellSmem<kForceThreads / 32> sm;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (forces_live(a)) {
    const int c = blockIdx.x / a.cell_split, s = blockIdx.x - c * a.cell_split;
    forces_cell_slice<kForceThreads / 32, true>(a, c, s, a.cell_split, sm, acc);
  }
}

// S7 + S9 after the solve: one warp gathers each ion's electrostatic force,
// its pair sums come from a.pair_out, and the block finishes its ions one
// per thread (the per-ion arithmetic of k_forces_cells).
__global__ void __launch_bounds__(kForceThreads) k_gather_finish(ForceArgs a) {
  constexpr int kW = kForceThreads / 32;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kW + warp;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  __shared__ double s_r[kW][8];
  const bool live = forces_live(a);
  if (i < a.n && live) {
    double gx, gy, gz, vd;
    gather_el(a, i, lane, gx, gy, gz, vd);
    if (lane == 0) {
      s_r[warp][0] = gx;
      s_r[warp][1] = gy;
      s_r[warp][2] = gz;
      s_r[warp][3] = vd;
    }
    if (lane < 4) s_r[warp][4 + lane] = a.pair_out[(size_t)i * 4 + lane];
  }
  __syncthreads();
  if (live && threadIdx.x < kW) {
    const int ii = blockIdx.x * kW + threadIdx.x;
    if (ii < a.n) {
      const double* r = s_r[threadIdx.x];
      finish_ion(a, ii, r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7], acc);
    }
  }
  energy_reduce(a, acc);
}

// S8 with each pair once (Newton's third law), FP64, one block per cell.
__global__ void __launch_bounds__(kForceThreads) k_pairs_half(ForceArgs a) {
  __shared__ HalfSmem<kForceThreads / 32> sm;
  if (forces_live(a)) pairs_half_cell<kForceThreads / 32>(a, blockIdx.x, sm);
}

// The mixed-precision form (FP32 pair arithmetic on hi + lo positions).
__global__ void __launch_bounds__(kForceThreads) k_pairs_half_mixed(ForceArgs a) {
  __shared__ HalfSmemF<kForceThreads / 32> sm;
  if (forces_live(a)) pairs_half_cell_mixed<kForceThreads / 32>(a, blockIdx.x, sm);
}

// The FP64 boxes' form with the pair arithmetic in double-float on the FP32
// pipe (the gather in FP64).
__global__ void __launch_bounds__(kForceThreads) k_pairs_half_df(ForceArgs a) {
  __shared__ HalfSmemF<kForceThreads / 32> sm;
  if (forces_live(a)) pairs_half_cell_mixed<kForceThreads / 32, true, true>(a, blockIdx.x, sm);
}

// S8 alone (no gather), persistent: gridDim.x blocks take the cells in turn
// (FP64, or the FP32 pair arithmetic of mixed precision).
// The block's shared memory is padded (dynamic size set by the launcher) so
// that no more of these blocks share an SM than the launcher intends: the
// form that runs beside the solve.
__global__ void __launch_bounds__(kForceThreads) k_pairs_only(ForceArgs a) {
  extern __shared__ __align__(16) unsigned char pairs_smem[];
  HalfSmem<kForceThreads / 32>& sm = *reinterpret_cast<HalfSmem<kForceThreads / 32>*>(pairs_smem);
  if (!forces_live(a)) return;
  const int ncell = a.nc * a.nc * a.nc;
  for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
    pairs_half_cell<kForceThreads / 32, false>(a, c, sm);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kForceThreads) k_pairs_only_mixed(ForceArgs a) {
  extern __shared__ __align__(16) unsigned char pairs_smem[];
  HalfSmemF<kForceThreads / 32>& sm = *reinterpret_cast<HalfSmemF<kForceThreads / 32>*>(pairs_smem);
  if (!forces_live(a)) return;
  const int ncell = a.nc * a.nc * a.nc;
  for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
    pairs_half_cell_mixed<kForceThreads / 32, false>(a, c, sm);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kForceThreads) k_pairs_only_df(ForceArgs a) {
  extern __shared__ __align__(16) unsigned char pairs_smem[];
  HalfSmemF<kForceThreads / 32>& sm = *reinterpret_cast<HalfSmemF<kForceThreads / 32>*>(pairs_smem);
  if (!forces_live(a)) return;
  const int ncell = a.nc * a.nc * a.nc;
  for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
    pairs_half_cell_mixed<kForceThreads / 32, false, true>(a, c, sm);
    __syncthreads();
  }
}

// S7 alone, one block per cell (after the solve, beside which k_pairs_only ran).
__global__ void __launch_bounds__(kForceThreads) k_gather_cells(ForceArgs a) {
  if (forces_live(a)) gather_cell<kForceThreads / 32>(a, blockIdx.x);
}

cudaError_t launch_pairs_only(const ForceArgs& a, int blocks, int smem_bytes, cudaStream_t s) {
  const int need = (a.mixed || a.pair_df) ? (int)sizeof(HalfSmemF<kForceThreads / 32>)
                                          : (int)sizeof(HalfSmem<kForceThreads / 32>);
  if (smem_bytes < need) smem_bytes = need;
  if (a.pair_df) {
    cudaError_t e = cudaFuncSetAttribute(k_pairs_only_df, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    k_pairs_only_df<<<blocks, kForceThreads, smem_bytes, s>>>(a);
  } else if (a.mixed) {
    cudaError_t e = cudaFuncSetAttribute(k_pairs_only_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    k_pairs_only_mixed<<<blocks, kForceThreads, smem_bytes, s>>>(a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_pairs_only, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    k_pairs_only<<<blocks, kForceThreads, smem_bytes, s>>>(a);
  }
  return cudaGetLastError();
}

int pairs_only_regs(bool mixed, bool df) {
  cudaFuncAttributes fa;
  const void* k = df ? (const void*)k_pairs_only_df : mixed ? (const void*)k_pairs_only_mixed : (const void*)k_pairs_only;
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 255;
  return fa.numRegs;
}

cudaError_t launch_gather_cells(const ForceArgs& a, cudaStream_t s) {
  k_gather_cells<<<a.nc * a.nc * a.nc, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pairs_half(const ForceArgs& a, cudaStream_t s) {
  if (a.mixed)
    k_pairs_half_mixed<<<a.nc * a.nc * a.nc, kForceThreads, 0, s>>>(a);
  else if (a.pair_df)
    k_pairs_half_df<<<a.nc * a.nc * a.nc, kForceThreads, 0, s>>>(a);
  else
    k_pairs_half<<<a.nc * a.nc * a.nc, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// S9 after k_pairs_half, one thread per ion: the gather sums (a.gath) and
// the fixed-point pair sums (a.pair_fix, cleared for the next step).
__global__ void __launch_bounds__(kForceThreads) k_finish_fix(ForceArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (i < a.n) {
    long long* pf = a.pair_fix + (size_t)i * 4;
    if (forces_live(a)) {
      const double* g = a.gath + (size_t)i * 4;
      // 2^-40 units to doubles on the integer pipe
      finish_ion(a, i, g[0], g[1], g[2], g[3], fix_to_dbl(pf[0], 1075 - 40), fix_to_dbl(pf[1], 1075 - 40),
                 fix_to_dbl(pf[2], 1075 - 40), fix_to_dbl(pf[3], 1075 - 40), acc);
    }
    pf[0] = pf[1] = pf[2] = pf[3] = 0;   // never carried over to the next step
  }
  energy_reduce(a, acc);
}

cudaError_t launch_finish_fix(const ForceArgs& a, cudaStream_t s) {
  k_finish_fix<<<(a.n + kForceThreads - 1) / kForceThreads, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pairs(const ForceArgs& a, cudaStream_t s) {
  k_pairs_cells<<<a.nc * a.nc * a.nc * a.cell_split, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather_finish(const ForceArgs& a, int blocks, cudaStream_t s) {
  k_gather_finish<<<blocks, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

int force_blocks(int n_ions) { return (n_ions + kForceThreads / 32 - 1) / (kForceThreads / 32); }

cudaError_t launch_forces(const ForceArgs& a, int blocks, cudaStream_t s) {
  if (a.by_cell)
    k_forces_cells<<<a.nc * a.nc * a.nc * a.cell_split, kForceThreads, 0, s>>>(a);
  else
    k_forces<<<blocks, kForceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace maze
