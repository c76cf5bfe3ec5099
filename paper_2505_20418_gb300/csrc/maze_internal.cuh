// Internal declarations shared by the CUDA translation units of libmaze.
// Device-side helpers: bounded grid barrier, deterministic block and grid
// reductions, periodic neighbour indexing, fixed-point charge accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/maze.h"

namespace maze {

// Grid charges are accumulated as 64-bit fixed point with 50 fractional bits:
// integer atomics make the spread order-independent (bit-reproducible), the
// resolution 2^-50 e is below FP64 rounding of O(1) values, and the range
// +-8192 e per grid point is far above any physical charge on one node.
constexpr double kQScale = 1125899906842624.0;         // 2^50
constexpr double kQInv = 1.0 / 1125899906842624.0;

// Spin limit of every device-side wait (about a second of polling).
constexpr unsigned kSpinLimit = 1u << 22;
// Largest cooperative grid the flag-carrying reduction supports.
constexpr int kMaxReduceBlocks = 256;

constexpr int kSolveThreads = 256;
constexpr int kForceThreads = 256;   // 8 ions (one warp each) per block
constexpr int kEnergyGroup = 128;    // force blocks per group of the two-level energy combine
constexpr int kIonThreads = 128;
constexpr int kSpreadThreads = 256;  // 8 ions (one warp each) per block

struct LLRec;  // flag-carrying reduction record (defined below)

// ---------------------------------------------------------------------------
// Kernel argument blocks (plain device pointers).

// O part of the OVRVO Langevin integrator: v <- a v + sd[type] xi over a half
// step, xi from Philox-4x32-10 with counter (ion, step, stage, 0).
struct LangevinArgs {
  int on;
  double a;              // exp(-gamma dt / 2)
  double sd0, sd1;       // sqrt((1 - a^2) k_B T / m) per species, Angstrom/fs
  unsigned key0, key1;   // generator key (seed)
};

// maze_step_io's exchange buffers as device addresses of pinned host memory:
// the caller's own arrays when they are pinned, else the context's stage.
struct IoDesc {
  const double* pos_in;   // [n][3]
  const double* vel_in;   // [n][3]
  double* pos_out;        // [n][3]
  double* vel_out;        // [n][3]
};

struct IonArgs {
  int n;                 // ions
  double L, h;           // box edge, grid spacing
  double inv_L, inv_h;   // 1/L, 1/h
  double cell_scale;     // nc / L
  int N, P;              // grid edge, assignment order
  double* pos;           // [3][n] SoA
  double* vel;           // [3][n]
  const double* force;   // [3][n] total force of the previous step
  const int* type;       // [n]
  float4* pos32;         // [n] FP32 copy (x, y, z, charge) for the pair pre-filter
  unsigned long long* qfix;  // [N^3] fixed-point charge grid (accumulated)
  int* cell_of;          // [n]
  int* cell_count;       // [nc^3] (accumulated) or nullptr
  int nc;                // cells per edge (0 = no cell list)
  double charge0, charge1;
  double kick0, kick1;   // dt/2 * acc_unit / m per species
  double dt;
  int do_move;           // 1: half kick + drift before spreading
  maze_stats* rec;
  int* gate;             // set to 1 when the step starts after an error
  double* wbuf;          // [n][3][4] B-spline weights of the new positions
  float* wbuf32;         // [n][3][4] FP32 weights (mixed precision) or nullptr
  float4* rel_hi;        // [n] (x, y, z, Q): position relative to the own cell's
  float4* rel_lo;        //     corner as hi + lo floats (mixed precision) or nullptr
  double cell_len;       // L / nc (L when there is no cell list)
  int4* wbase;           // [n] first support node per axis
  double* wdbuf;         // [n][3][4] weight derivatives dW/dt (Eq. F_Benoit, FP64) or nullptr
  float* wdbuf32;        // the same in FP32 (mixed precision) or nullptr
  LangevinArgs ou;       // OVRVO O steps (off when ou.on == 0)
  const IoDesc* io;      // maze_step_io's exchange (device memory): this step's positions and
                         // velocities in the caller's [n][3] order, read instead of pos / vel
                         // (positions wrapped as maze_set wraps them), or nullptr
};

struct CellArgs {
  int n, ncell;
  const int* cell_of;
  int* cell_count;       // read and cleared by the scan
  int* cell_start;       // [ncell + 1]
  int* cursor;           // [ncell]
  int* cell_ions;        // [n]
  const float4* pos32;   // [n] FP32 positions by ion
  float4* pos_sorted;    // [n] FP32 positions by cell slot (written by the sort)
  const float4* rel_hi;  // [n] cell-relative hi/lo positions (mixed) or nullptr
  const float4* rel_lo;
  float4* rel_hi_sorted; // [n] the same in cell-slot order
  float4* rel_lo_sorted;
  maze_stats* rec;
};

// Tosi-Fumi constants as (hi, lo) float pairs for the double-float pair
// arithmetic of FP64 boxes (each pair the double's value to ~2^-48).
struct PairDf {
  float2 B, rc2;
  float2 Ec[3], C[3], D[3], Vc[3], C6[3], D8[3];
};

struct ForceArgs {
  int n;
  double L, h;
  double inv_2h;         // 1 / (2h)
  int N, P;
  const double* pos;     // [3][n]
  double* vel;           // [3][n]
  double* force;         // [3][n] total force (out)
  double* force_el;      // [3][n] electrostatic force (in: previous, out: new)
  const float4* pos32;
  const int* type;
  const double* phi;     // [N^3] doubles, or double-float pairs when phi_df
  int phi_df;            // 1: phi holds (hi, lo) float pairs (mixed precision)
  const double* wbuf;    // [n][3][4] weights written by k_ion_update
  const float* wbuf32;   // [n][3][4] FP32 weights (mixed precision)
  const int4* wbase;     // [n]
  const double* wdbuf;   // [n][3][4] weight derivatives (force estimator of Eq. F_Benoit)
  const float* wdbuf32;
  int gradw;             // 1: F = -k_e Q sum_n grad W phi_n (Eq. F_Benoit), else Eq. F_nostra
  int mixed;             // 1: FP32 gather and pair arithmetic
  int by_cell;           // 1: one block per cell (k_forces_cells), else one warp per ion
  int cell_split;        // blocks per cell in k_forces_cells (each takes a slice of the cell's ions)
  const float4* rel_hi;  // [n] cell-relative hi/lo positions (mixed precision)
  const float4* rel_lo;
  const float4* rel_hi_sorted;  // [n] the same in cell-slot order
  const float4* rel_lo_sorted;
  float cell_len_h, cell_len_l;  // L / nc as hi + lo floats
  float L_h, L_l;                // L as hi + lo floats
  float Af[3], sf[3], Cf[3], Df[3], Vcf[3], Bf, rc2f;
  int nc;                // cells per edge; < 3 means all pairs
  int reach;             // neighbour cells within +-reach per axis (cells >= r_cut / reach)
  const int* cell_start;
  const int* cell_ions;
  const float4* pos_sorted;  // [n] FP32 positions in cell-slot order
  const int* cell_of;
  double charge0, charge1, mass0, mass1;
  double kick0, kick1;
  double dt;
  double ke_coef;        // 1 / (2 acc_unit): 1/2 m v^2 in eV
  // Tosi-Fumi table by pair kind (0,0) (0,1) (1,1)
  double A[3], s[3], C[3], D[3], Vc[3];
  double Ec[3];          // B s + ln A: the repulsion A exp(B (s - r)) = exp(Ec - B r)
  double C6[3], D8[3];   // 6 C, 8 D (the force's dispersion terms)
  const double* exp2tab; // [64] 2^(j/64), j = 0..63 (exp_tab)
  int pair_df;           // 1: FP64 box whose pair arithmetic runs in double-float on the FP32 pipe
  PairDf pdf;            // the Tosi-Fumi table for it
  const float2* exp2tab_f;  // [64] 2^(j/64) as (hi, lo) floats (df_exp)
  double B;
  double rc2;            // r_cut^2
  float rc2_filter;      // (r_cut + margin)^2 for the FP32 pre-filter
  float Lf, inv_Lf;
  int do_kick;           // 1: second half kick + V_work increment
  int count_step;        // 1: this completes an MD step
  LangevinArgs ou;       // second O step after the kick (when do_kick)
  double* part;          // [gridDim][8] block partials
  unsigned* ticket;      // last-block ticket (self-resetting)
  double* pair_out;      // [n][4] pair sums per ion (the split step: S8 apart from S7/S9) or nullptr
  long long* pair_fix;   // [n][4] pair sums per ion in 2^-40 fixed point (FP64, pairs once each), zero
                         // before the pair kernel, cleared by the kernel that reads them; or nullptr
  double* gath;          // [n][4] gather sums per ion (with pair_fix: written by the pair kernel)
  maze_stats* rec;
  const int* gate;       // 1: this step was skipped
};

struct SolveArgs {
  int N, n;
  const double* phi_k;
  const double* phi_km1;
  double* phi_out;       // phi_p, then phi^{k+1}
  unsigned long long* qfix;  // read and cleared
  double* q_out;         // optional copy of q (nullptr = skip)
  double* sigma;
  double* y;
  double* r;
  double* p;             // search direction, double-buffered with p1
  double* p1;
  double* Mp;
  LLRec* recs;           // [2][gridDim][4] reduction records, zero at launch
  unsigned* bar;         // grid barrier counter, zero at launch
  maze_stats* rec;
  double c_sig;          // h / 4pi
  double c_phi;          // 4pi / h
  double inv_n;          // 1 / N^3
  double tol;
  int max_iter;
  int zero_phi;          // step 0: phi^k = phi^{k-1} = 0
  int static_guess;      // 1: phi_p = phi^k (direct solve from the previous potential)
  double res_scale;      // reported residual = res_scale * max|M y - sigma_p|
  const int* gate;       // 1: this step was skipped
};

// Multigrid hierarchy (levels 0..L-1, level 0 is the SHAKE grid itself).
constexpr int kMaxLevels = 10;
struct MgArgs {
  int L;
  int Nl[kMaxLevels];
  int lg[kMaxLevels];      // log2(N_l) for powers of two, else -1
  size_t off[kMaxLevels];  // offsets of each level in x, b, r (level 0 at 0)
  double* x;               // corrections on levels >= 1 (level 0 uses y)
  double* b;               // right-hand sides, stored as -b/6, all levels (level 0: -sigma_p/6)
  double* r;               // residuals (at red points), all levels
                           // (MAZE_FP64_FIXMG: x, b, r hold int64 in units of
                           // 2^-F, b unscaled, level 0 of x is the correction e)
  const double* gker;      // [Nc^3] -6 times the pseudo-inverse kernel of the coarsest M
  int nu1, nu2;
};

// Threads per block of the cooperative multigrid kernels for a grid of n
// points: grids of 128^3 points and more run one 1024-thread block per SM
// (every SM carries the same work); smaller grids, whose phases give each
// thread only a few points, run blocks of 256 threads over more SMs.
constexpr int kMgThreads = 1024;
inline int mg_threads(int n) { return n >= (1 << 21) ? kMgThreads : 256; }

// Mixed-precision solve (double-float outer iteration, FP32 V-cycle).
constexpr int kMixedClusterThreads = 512;   // one cluster per box
constexpr int kMixedGridThreads = 1024;     // cooperative grid (large boxes)
// Dynamic shared memory a CTA may give the cluster-resident V-cycle.
constexpr int kResidentSmem = 200 * 1024;
struct MixedArgs {
  int N, n;
  const float2* phi_k;     // double-float grids (hi, lo)
  const float2* phi_km1;
  float2* phi_out;
  float2* sigma;
  float2* y;
  float2* y2;              // second y buffer of the cluster-resident form
  int resident;            // 1: V-cycle vectors in the cluster's shared memory
  unsigned long long* qfix;  // read and cleared
  double* q_out;           // optional copy of q
  float* scratch;          // global form of the V-cycle storage (slab layout of one part)
  size_t scratch_floats;   // its size; the kernels refuse a layout that does not fit
  const float* gkerf;      // [Nc^3] 1/(Nc^3 lambda(k)) of the coarsest M (0 at k = 0), then [Nc] cos and
                           // [Nc] sin of 2 pi t / Nc
  int L;
  int Nl[kMaxLevels];
  int lg[kMaxLevels];      // log2(N_l) for powers of two, else -1
  int nu1, nu2;
  int tail_n;              // levels of at most tail_n^3 points run in one CTA (0: 8 in a cluster, 16 in
                           // the global form); the arithmetic, hence every result, is the same either way
  float c_sig_h, c_sig_l;  // h/4pi as a double-float
  float c_phi_h, c_phi_l;  // 4pi/h as a double-float
  double tol;
  int max_iter;
  double inv_n;
  int zero_phi;
  int static_guess;        // 1: phi_p = phi^k (direct solve from the previous potential)
  int y_reset;             // 1: the solve starts from y = 0 (direct schemes; batch kernel clears y)
  double res_scale;        // reported residual = res_scale * max|M y - sigma_p|
  LLRec* recs;             // grid form only
  unsigned* bar;           // grid form only
  maze_stats* rec;
  const int* gate;
};

// Host-side launchers (defined in the .cu files).
// S1 and S3: part 0 both, 1 the move (S1) only, 2 the spread (S3) only.
cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t s, int part = 0);   // k_move, then k_spread if a.qfix
cudaError_t launch_q_to_double(const unsigned long long* qfix, double* q, int n, cudaStream_t s);
// maze_step_io's exchange (device-accessible pinned pointers): the device's
// [2][3][n] positions and velocities -> [2][n][3] host order, and the
// record (rec_bytes a multiple of 8)
cudaError_t launch_io_out(const double* soa, const IoDesc* io, int n, const void* rec, void* rec_out, size_t rec_bytes,
                          cudaStream_t s);
cudaError_t launch_cells(const CellArgs& a, cudaStream_t s);
cudaError_t launch_forces(const ForceArgs& a, int blocks, cudaStream_t s);
cudaError_t launch_pairs(const ForceArgs& a, cudaStream_t s);
// S8 once per pair and S7 (FP64, a.pair_fix, a.gath), one block per cell;
// then S9 one thread per ion.
cudaError_t launch_pairs_half(const ForceArgs& a, cudaStream_t s);
cudaError_t launch_pairs_only(const ForceArgs& a, int blocks, int smem_bytes, cudaStream_t s);
int pairs_only_regs(bool mixed, bool df);   // registers per thread of k_pairs_only(_mixed, _df)
void fill_pair_consts(const maze_config& g, ForceArgs& a);   // Tosi-Fumi table (host)
int mgfix_regs();                  // and of k_mgfix_solve
int mixed_grid_regs();             // and of k_mixed_grid
cudaError_t launch_gather_cells(const ForceArgs& a, cudaStream_t s);
cudaError_t launch_finish_fix(const ForceArgs& a, cudaStream_t s);
cudaError_t launch_cluster_front(const IonArgs& ia, const CellArgs& ca, const MixedArgs& ma, int cluster,
                                 cudaStream_t s);
cudaError_t launch_gather_finish(const ForceArgs& a, int blocks, cudaStream_t s);
int force_blocks(int n_ions);
cudaError_t launch_cg_solve(const SolveArgs& a, int blocks, cudaStream_t s);
int solve_blocks(int n_points);
// The 64 entries 2^(j/64) of exp_tab's table (host).
void exp2_table(double* out64);
cudaError_t launch_mg_solve(const SolveArgs& a, const MgArgs& g, int blocks, cudaStream_t s);
int mg_blocks(int n_points);
cudaError_t launch_mgfix_solve(const SolveArgs& a, const MgArgs& g, int blocks, int threads, cudaStream_t s);
int mgfix_blocks(int n_points);
// threads > 0: the cooperative grid form with that many threads per block
// (at least 512; fewer than kMixedGridThreads leave room beside it)
cudaError_t launch_mixed_solve(const MixedArgs& a, int cluster, int blocks, cudaStream_t s, int threads = 0);
int mixed_cluster_size();
int cluster_step_size();
// S1-S6 of one mixed-precision step of a box up to 64^3 in one cluster launch.
cudaError_t launch_cluster_step(const IonArgs& ia, const CellArgs& ca, const MixedArgs& ma, int cluster,
                                cudaStream_t s);
// Shared-memory bytes per CTA of the cluster-resident V-cycle for C CTAs.
size_t resident_bytes_host(const MixedArgs& a, int C);
int mixed_grid_blocks(int n_points);
// Sets the message returned by maze_last_error on the calling thread.
void set_last_error(const char* msg);

// ---------------------------------------------------------------------------
// Device helpers

#ifdef __CUDACC__

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch. ``epoch`` counts this block's
// barriers (thread 0 only); the counter grows monotonically and barrier e is
// complete when it reaches e * gridDim.x. A wait longer than kSpinLimit polls
// records MAZE_ERR_TIMEOUT and returns false in every thread of the block.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& epoch, maze_stats* rec) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    int ok = 1;
    unsigned spins = 0;
    while (ld_acquire_u32(bar) < target) {
      if (++spins > kSpinLimit) {
        ok = 0;
        atomicCAS(&rec->status, MAZE_OK, MAZE_ERR_TIMEOUT);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Flag-carrying grid reduction. Each block publishes its partials as 16-byte
// records {lo32, flag, hi32, flag}: each 8-byte half pairs half of the double
// with the epoch number, so a reader that sees both flags equal to the epoch
// holds the whole value (8-byte stores and loads are single-copy atomic).
// One round of publish + poll replaces a barrier followed by a second trip to
// read the partials. Records are double-buffered by epoch parity and must be
// zero when the kernel starts. Release: __syncthreads,
// then a gpu-scope release store of the record by the publishing thread;
// acquire: gpu-scope acquire loads of the records, then __syncthreads.
struct LLRec {
  unsigned lo, f0, hi, f1;
};

// Release store: the block's earlier global writes (ordered before this
// thread by __syncthreads) become visible no later than the record.
__device__ __forceinline__ void ll_store(LLRec* r, double v, unsigned epoch) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  asm volatile("st.release.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(r), "r"((unsigned)b), "r"(epoch),
               "r"((unsigned)(b >> 32)), "r"(epoch)
               : "memory");
}

// Acquire load: once the flags match, the publisher's earlier writes are
// visible to this thread (and, after __syncthreads, to its block).
__device__ __forceinline__ bool ll_load(const LLRec* r, unsigned epoch, double& v) {
  unsigned lo, f0, hi, f1;
  asm volatile("ld.acquire.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(lo), "=r"(f0), "=r"(hi), "=r"(f1) : "l"(r)
               : "memory");
  if (f0 != epoch || f1 != epoch) return false;
  v = __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
  return true;
}

// 1/d by Newton-Raphson on the mantissa: d = m 2^e with m in [1,2), an FP32
// seed for 1/m, then two steps y <- y (2 - m y) (the error squares at each
// step: ~2^-23 -> 2^-46 -> below FP64 rounding), and the exponent restored by
// integer arithmetic. A handful of FP64 operations instead of the long FP64
// division sequence; used for the scalar recurrences of the solvers. Zero,
// denormal, infinite and NaN inputs take the ordinary division.
__device__ __forceinline__ double recip_newton(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0 || e == 2047) return 1.0 / d;
  const double m = __longlong_as_double((b & (long long)0x800fffffffffffffULL) | (1023LL << 52));
  double y = (double)(1.0f / (float)m);
  y = y * (2.0 - m * y);
  y = y * (2.0 - m * y);
  const long long yb = __double_as_longlong(y) - ((long long)(e - 1023) << 52);
  return __longlong_as_double(yb);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// round(v * 2^S) as a 64-bit integer from v's bits, integer operations only
// (GB300's FP64-pipe conversions take several issue slots each): rounding
// half away from zero, 0 when |v 2^S| < 1/2; requires |v 2^S| < 2^62.
__device__ __forceinline__ long long round_scaled(double v, int S) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const int sh = 1075 - S - e;   // v 2^S = m 2^(e - 1075 + S)
  if (sh > 53) return 0;
  const long long m = (b & 0xfffffffffffffLL) | (1LL << 52);
  const long long x = sh > 0 ? (m + (1LL << (sh - 1))) >> sh : m << (-sh);
  return b < 0 ? -x : x;
}

// round(v * 2^S) for an FP32 v, integer operations only (as round_scaled).
__device__ __forceinline__ long long round_scaled_f(float v, int S) {
  const int b = __float_as_int(v);
  const int e = (b >> 23) & 0xff;
  const int sh = 150 - S - e;   // v 2^S = m 2^(e - 150 + S)
  if (sh > 24) return 0;
  const long long m = (long long)((b & 0x7fffff) | 0x800000);
  const long long x = sh > 0 ? (m + (1LL << (sh - 1))) >> sh : m << (-sh);
  return b < 0 ? -x : x;
}

// Max-norm accumulation on the integer pipe: |v| as its IEEE bit pattern. For
// non-negative doubles the integer order is the numeric order and every NaN
// sorts above +inf, so a NaN entry is never dropped (fmax would drop it).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}
// The accumulated maximum as a double, a NaN reported as +inf (non-finite
// either way, and +inf survives an fmax-based combine).
__device__ __forceinline__ double absmax_value(unsigned long long u) {
  return u > 0x7ff0000000000000ULL ? __longlong_as_double(0x7ff0000000000000LL) : __longlong_as_double((long long)u);
}
// FP32 form: |v|, a NaN mapped to +inf.
__device__ __forceinline__ float abs_nan_inf(float v) {
  const float a = fabsf(v);
  return a == a ? a : __int_as_float(0x7f800000);
}

// Periodic neighbours of flat index n = i + jN + kN^2.
struct Nbr {
  int xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nbr neighbours(int n, int N) {
  const int NN = N * N;
  int i, j, k;
  if ((N & (N - 1)) == 0) {   // powers of two: shifts, not divisions
    const int lg = __ffs(N) - 1;
    i = n & (N - 1);
    j = (n >> lg) & (N - 1);
    k = n >> (2 * lg);
  } else {
    k = n / NN;
    const int rem = n - k * NN;
    j = rem / N;
    i = rem - j * N;
  }
  Nbr b;
  b.xm = (i == 0) ? n + N - 1 : n - 1;
  b.xp = (i == N - 1) ? n - N + 1 : n + 1;
  b.ym = (j == 0) ? n + NN - N : n - N;
  b.yp = (j == N - 1) ? n - NN + N : n + N;
  b.zm = (k == 0) ? n + NN * (N - 1) : n - NN;
  b.zp = (k == N - 1) ? n - NN * (N - 1) : n + NN;
  return b;
}

// Point of colour c (0 red, 1 black; red = i + j + k even) with half-index h
// on an N^3 grid (N even): h = t + (N/2)(j + N k), i = 2t + ((j + k + c) & 1).
// lg = log2 N for powers of two (shift decode), else -1.
__device__ __forceinline__ void colour_point(int h, int N, int lg, int c, int& i, int& j, int& k) {
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
}

// Identity post step of grid_reduce.
struct NoPost {
  __device__ double operator()(const double*) const { return 0.0; }
};

// ---------------------------------------------------------------------------
// Exact sums of doubles on the integer pipe. GB300 issues FP64 at 1/64 of the
// FP32 rate and a dependent FP64 add costs ~150 cycles, so a shuffle tree of
// FP64 adds is slow. Instead every value is rounded to a 64-bit fixed-point
// grid aligned to the largest exponent in the group (the value's 53-bit
// significand shifted right by the exponent difference, round to nearest),
// and the integers are summed exactly: each int64 is cut into four 16-bit
// chunks and each chunk summed with __reduce_add_sync (32 lanes x 2^16 < 2^21),
// then recombined modulo 2^64. The total is exact for the rounded inputs, so
// the result is independent of summation order (bit-reproducible) and its
// error is at most half an ulp of the largest input per input.

__device__ __forceinline__ int dbl_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7ff); }

// v as an integer multiple of 2^(E - 1075); requires the exponent of v <= E.
__device__ __forceinline__ long long dbl_to_fix(double v, int E) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;  // zero and denormals (below 2^-1022) count as zero
  const long long m = (b & 0xfffffffffffffLL) | (1LL << 52);
  const int sh = E - e;
  long long x;
  if (sh <= 0) x = m;
  else if (sh >= 62) x = 0;
  else x = (m + (1LL << (sh - 1))) >> sh;
  return b < 0 ? -x : x;
}

// S * 2^(E - 1075) as a double, built with integer operations only:
// normalise |S| to a 53-bit significand (round half up) and set the exponent.
__device__ __forceinline__ double fix_to_dbl(long long S, int E) {
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? 0x8000000000000000ULL : 0ULL;
  const unsigned long long u = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  int sh = (64 - __clzll((long long)u)) - 53;
  unsigned long long m;
  if (sh > 0) {
    m = (u + (1ULL << (sh - 1))) >> sh;
    if (m >> 53) {
      m >>= 1;
      ++sh;
    }
  } else {
    m = u << (-sh);
  }
  const int ed = sh + E;
  if (ed <= 0) return 0.0;
  if (ed >= 2047) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ULL));
  return __longlong_as_double((long long)(sign | ((unsigned long long)ed << 52) | (m & 0xfffffffffffffULL)));
}

__device__ __forceinline__ long long warp_isum(long long x) {
  const unsigned long long u = (unsigned long long)x;
  const unsigned c0 = __reduce_add_sync(0xffffffffu, (unsigned)(u & 0xffffu));
  const unsigned c1 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 16) & 0xffffu));
  const unsigned c2 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 32) & 0xffffu));
  const unsigned c3 = __reduce_add_sync(0xffffffffu, (unsigned)(u >> 48));
  return (long long)((unsigned long long)c0 + ((unsigned long long)c1 << 16) + ((unsigned long long)c2 << 32) +
                     ((unsigned long long)c3 << 48));
}

// Max of non-negative doubles by integer max of their bit patterns (IEEE
// ordering of non-negative values equals integer ordering).
__device__ __forceinline__ unsigned long long warp_umax64(unsigned long long u) {
  const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(u >> 32));
  const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(u >> 32) == hi ? (unsigned)u : 0u);
  return ((unsigned long long)hi << 32) | lo;
}

// Exact warp sum of doubles (every lane gets the result as fixed point S, E).
__device__ __forceinline__ void warp_dsum_fix(double v, long long& S, int& E) {
  E = (int)__reduce_max_sync(0xffffffffu, (unsigned)dbl_exp(v));
  S = warp_isum(dbl_to_fix(v, E));
}

// The same, rounded once to a double (every lane gets it).
__device__ __forceinline__ double warp_dsum(double v) {
  long long S;
  int E;
  warp_dsum_fix(v, S, E);
  return fix_to_dbl(S, E);
}

// FP32 <-> FP64 conversions on the integer pipe. On GB300 a conversion that
// involves FP64 (F2F, I2F, F2I) occupies the FP64 pipe for many issue slots,
// so the FP64 hot loops build the other format's bits instead.

// v to FP32, rounding to nearest even (as the conversion instruction; FP32
// subnormal results included, overflow to infinity, NaN kept).
__device__ __forceinline__ float dbl_to_flt(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffULL;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int ef = e - 1023 + 127;
  int sh = 29;                                   // significand bits dropped
  unsigned long long sig = m, base = (unsigned long long)(ef > 0 ? ef : 0) << 23;
  if (ef <= 0) {                                 // FP32 subnormal (or zero)
    if (e == 0 || ef < -24) return __uint_as_float(sign);
    sig = m | (1ULL << 52);
    sh = 30 - ef;
  }
  unsigned long long r = base | (sig >> sh);
  const unsigned long long rem = sig & ((1ULL << sh) - 1), halfway = 1ULL << (sh - 1);
  if (rem > halfway || (rem == halfway && (r & 1))) ++r;   // a carry moves into the exponent
  if (r >= 0x7f800000ULL) r = 0x7f800000ULL;
  return __uint_as_float(sign | (unsigned)r);
}

// f to FP64 (exact).
__device__ __forceinline__ double flt_to_dbl(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const int e = (int)((b >> 23) & 0xff);
  const unsigned long long m = b & 0x7fffffu;
  if (e == 0xff) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ULL | (m << 29)));
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    const int p = 31 - __clz((int)m);            // value m 2^-149 = 1.f 2^(p - 149)
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(p - 149 + 1023) << 52) | ((m << (52 - p)) & 0xfffffffffffffULL)));
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | (m << 29)));
}

// floor(v) as an integer for finite v with |v| < 2^62.
__device__ __forceinline__ long long floor_ll(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const bool neg = b < 0;
  if (e < 0) return (neg && (b & 0x7fffffffffffffffLL)) ? -1 : 0;   // |v| < 1
  const long long m = (b & 0xfffffffffffffLL) | (1LL << 52);
  if (e >= 52) return neg ? -(m << (e - 52)) : (m << (e - 52));
  const long long ip = m >> (52 - e);
  const bool frac = (m & ((1LL << (52 - e)) - 1)) != 0;
  return neg ? -(ip + (frac ? 1 : 0)) : ip;
}

// exp(x) by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15, 1989):
// x = (64 m + j) ln2/64 + r with |r| <= ln2/128, so exp(x) = 2^m 2^(j/64) e^r;
// 2^(j/64) comes from a 64-entry table, e^r - 1 from its degree-5 Taylor
// polynomial (the remainder r^6/720 is below 2^-54 there), the 2^m scaling is
// an integer add to the exponent field. 10 FP64 operations and no conversion;
// |x| >= 512, infinities and NaN take exp(). Within 2 ulp of exp() (checked
// against it by maze_exp_probe).
__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ tab) {
  if (((__double_as_longlong(x) >> 52) & 0x7ff) >= 1023 + 9) return exp(x);
  const double kd = fma(x, 0x1.71547652b82fep+6, 0x1.8p52);   // 64/ln2, then round to an integer
  const int k = (int)(unsigned)__double_as_longlong(kd);       // (the low bits of 1.5 2^52 + k)
  const double kf = kd - 0x1.8p52;
  double r = fma(-kf, 0x1.62e42fefa39efp-7, x);                 // ln2/64 in two parts (Cody-Waite)
  r = fma(-kf, 0x1.abc9e3b39803fp-62, r);
  const double c4 = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  const double c3 = fma(r, c4, 1.0 / 6.0);
  const double c2 = fma(r, c3, 0.5);
  const double p = r * fma(r, c2, 1.0);                         // e^r - 1
  const double t = __ldg(tab + (k & 63));
  const double e = fma(t, p, t);
  return __longlong_as_double(__double_as_longlong(e) + ((long long)(k >> 6) << 52));
}

// S4 at grid point m with periodic neighbours b (Eq. SHAKE): the charge q
// (read from the fixed-point grid, which is cleared; converted on the integer
// pipe, exact for |q| < 8), phi_p = 2 phi^k -
// phi^{k-1} (phi^k for the direct scheme from the previous potential, 0 at
// step 0) and sigma_p = (h/4pi) M phi_p + q. phi_p goes to phi_out, sigma_p
// to sigma and is returned.
__device__ __forceinline__ double shake_rhs(const SolveArgs& a, int m, const Nbr& b) {
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
      Mphp = fma(-6.0, php, nk);
    } else {
      php = fma(2.0, pk[m], -pm[m]);
      const double nm = (pm[b.xm] + pm[b.xp]) + (pm[b.ym] + pm[b.yp]) + (pm[b.zm] + pm[b.zp]);
      Mphp = fma(-6.0, php, fma(2.0, nk, -nm));
    }
  }
  const double sg = fma(a.c_sig, Mphp, q);
  a.phi_out[m] = php;
  a.sigma[m] = sg;
  return sg;
}

// Grid-wide reduction of K <= 4 values (sum, or max of non-negative values
// where is_max[k]) over all blocks of a cooperative launch. ``v`` holds this
// thread's contributions; on return every thread of every block holds the
// identical totals in ``out``. Blocks publish their partials through the
// flag-carrying records (``recs`` is [2][gridDim][4], zero at launch;
// ``epoch`` counts rounds from 1). ``post`` runs once per block, in one lane,
// on the totals; its result comes back in ``extra``. A poll that exceeds
// kSpinLimit records MAZE_ERR_TIMEOUT and returns false.
template <int K, typename Post = NoPost>
__device__ __forceinline__ bool grid_reduce(const double (&v)[K], const bool (&is_max)[K], LLRec* recs, unsigned epoch,
                                            maze_stats* rec, double (&out)[K], Post post = Post(),
                                            double* extra = nullptr) {
  __shared__ long long s_s[32][4];
  __shared__ int s_e[32][4];
  __shared__ double s_out[5];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // block stage 1: warp exponent maxima (sums) or bit maxima (maxima)
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (is_max[k]) {
      const unsigned long long m = warp_umax64((unsigned long long)__double_as_longlong(fabs(v[k])));
      if (lane == 0) s_s[warp][k] = (long long)m;
    } else {
      const int e = (int)__reduce_max_sync(0xffffffffu, (unsigned)dbl_exp(v[k]));
      if (lane == 0) s_e[warp][k] = e;
    }
  }
  __syncthreads();
  // block stage 2: align every value to the block's largest exponent, sum exactly
  int Eb[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (is_max[k]) continue;
    int E = 0;
    for (int u = 0; u < nw; ++u) E = max(E, s_e[u][k]);
    Eb[k] = E;
    const long long S = warp_isum(dbl_to_fix(v[k], E));
    if (lane == 0) s_s[warp][k] = S;
  }
  __syncthreads();
  LLRec* buf = recs + (size_t)(epoch & 1u) * gridDim.x * 4;
  if (warp == 0) {
    // publish the block partials (as doubles; one rounding of the exact sum)
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        double w;
        if (is_max[k]) {
          unsigned long long m = 0;
          for (int u = 0; u < nw; ++u) m = max(m, (unsigned long long)s_s[u][k]);
          w = __longlong_as_double((long long)m);
        } else {
          long long S = 0;
          for (int u = 0; u < nw; ++u) S += s_s[u][k];
          w = fix_to_dbl(S, Eb[k]);
        }
        ll_store(&buf[blockIdx.x * 4 + k], w, epoch);
      }
    }
    // read every block's records; all of this lane's loads are in flight at once
    constexpr int kMaxPer = kMaxReduceBlocks / 32;
    double val[K][kMaxPer];
    unsigned pending = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < kMaxPer; ++j) {
        val[k][j] = 0.0;
        if (lane + 32 * j < (int)gridDim.x) pending |= 1u << (k * kMaxPer + j);
      }
    int ok = 1;
    unsigned spins = 0;
    while (pending) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int j = 0; j < kMaxPer; ++j) {
          const unsigned bit = 1u << (k * kMaxPer + j);
          if (pending & bit) {
            if (ll_load(&buf[(lane + 32 * j) * 4 + k], epoch, val[k][j])) pending &= ~bit;
          }
        }
      if (pending && ++spins > kSpinLimit) {
        ok = 0;
        break;
      }
    }
    // combine the block partials exactly (same integer algorithm)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double tot;
      if (is_max[k]) {
        unsigned long long m = 0;
#pragma unroll
        for (int j = 0; j < kMaxPer; ++j) m = max(m, (unsigned long long)__double_as_longlong(val[k][j]));
        tot = __longlong_as_double((long long)warp_umax64(m));
      } else {
        int e = 0;
#pragma unroll
        for (int j = 0; j < kMaxPer; ++j) e = max(e, dbl_exp(val[k][j]));
        const int E = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
        long long x = 0;
#pragma unroll
        for (int j = 0; j < kMaxPer; ++j) x += dbl_to_fix(val[k][j], E);
        tot = fix_to_dbl(warp_isum(x), E);
      }
      if (lane == 0) s_out[k] = tot;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
      if (!ok) atomicCAS(&rec->status, MAZE_OK, MAZE_ERR_TIMEOUT);
      s_ok = ok;
      s_out[4] = post(s_out);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = s_out[k];
  if (extra) *extra = s_out[4];
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

// Grid-wide sum of one unsigned 64-bit value per thread, modulo 2^64 (exact
// integer totals; same publication records and epochs as grid_reduce). Every
// thread of every block gets the total in ``out``.
__device__ __forceinline__ bool grid_reduce_u64(unsigned long long v, LLRec* recs, unsigned epoch, maze_stats* rec,
                                                unsigned long long& out) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_tot;
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long w = (unsigned long long)warp_isum((long long)v);
  if (lane == 0) s_w[warp] = w;
  __syncthreads();
  LLRec* buf = recs + (size_t)(epoch & 1u) * gridDim.x * 4;
  if (warp == 0) {
    if (lane == 0) {
      unsigned long long S = 0;
      for (int u = 0; u < nw; ++u) S += s_w[u];
      ll_store(&buf[blockIdx.x * 4], __longlong_as_double((long long)S), epoch);
    }
    constexpr int kMaxPer = kMaxReduceBlocks / 32;
    double val[kMaxPer];
    unsigned pending = 0;
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
      val[j] = 0.0;
      if (lane + 32 * j < (int)gridDim.x) pending |= 1u << j;
    }
    int ok = 1;
    unsigned spins = 0;
    while (pending) {
#pragma unroll
      for (int j = 0; j < kMaxPer; ++j)
        if ((pending >> j) & 1u)
          if (ll_load(&buf[(lane + 32 * j) * 4], epoch, val[j])) pending &= ~(1u << j);
      if (pending && ++spins > kSpinLimit) {
        ok = 0;
        break;
      }
    }
    unsigned long long x = 0;
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) x += (unsigned long long)__double_as_longlong(val[j]);
    const unsigned long long t = (unsigned long long)warp_isum((long long)x);
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
      if (!ok) atomicCAS(&rec->status, MAZE_OK, MAZE_ERR_TIMEOUT);
      s_ok = ok;
      s_tot = t;
    }
  }
  __syncthreads();
  out = s_tot;
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

#endif  // __CUDACC__

}  // namespace maze
