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

constexpr int kSolveThreads = 256;
constexpr int kForceThreads = 256;   // 8 ions (one warp each) per block

// ---------------------------------------------------------------------------
// Kernel argument blocks (plain device pointers).

struct IonArgs {
  int n;                 // ions
  double L, h;           // box edge, grid spacing
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
};

struct CellArgs {
  int n, ncell;
  const int* cell_of;
  int* cell_count;       // read and cleared by the scan
  int* cell_start;       // [ncell + 1]
  int* cursor;           // [ncell]
  int* cell_ions;        // [n]
  maze_stats* rec;
};

struct ForceArgs {
  int n;
  double L, h;
  int N, P;
  const double* pos;     // [3][n]
  double* vel;           // [3][n]
  double* force;         // [3][n] total force (out)
  double* force_el;      // [3][n] electrostatic force (in: previous, out: new)
  const float4* pos32;
  const int* type;
  const double* phi;     // [N^3]
  int nc;                // cells per edge; < 3 means all pairs
  const int* cell_start;
  const int* cell_ions;
  const int* cell_of;
  double charge0, charge1, mass0, mass1;
  double kick0, kick1;
  double dt;
  double ke_coef;        // 1 / (2 acc_unit): 1/2 m v^2 in eV
  // Tosi-Fumi table by pair kind (0,0) (0,1) (1,1)
  double A[3], s[3], C[3], D[3], Vc[3];
  double B;
  double rc2;            // r_cut^2
  float rc2_filter;      // (r_cut + margin)^2 for the FP32 pre-filter
  float Lf;
  int do_kick;           // 1: second half kick + V_work increment
  int count_step;        // 1: this completes an MD step
  double* part;          // [gridDim][8] block partials
  unsigned* ticket;      // last-block ticket (self-resetting)
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
  double* p;
  double* Mp;
  double* part;          // [2][gridDim][4] double-buffered block partials
  unsigned* bar;         // barrier counter, zero at launch
  maze_stats* rec;
  double c_sig;          // h / 4pi
  double c_phi;          // 4pi / h
  double tol;
  int max_iter;
  int zero_phi;          // step 0: phi^k = phi^{k-1} = 0
  const int* gate;       // 1: this step was skipped
};

// Host-side launchers (defined in the .cu files).
cudaError_t launch_ion_update(const IonArgs& a, cudaStream_t s);
cudaError_t launch_q_to_double(const unsigned long long* qfix, double* q, int n, cudaStream_t s);
cudaError_t launch_cells(const CellArgs& a, cudaStream_t s);
cudaError_t launch_forces(const ForceArgs& a, int blocks, cudaStream_t s);
int force_blocks(int n_ions);
cudaError_t launch_cg_solve(const SolveArgs& a, int blocks, cudaStream_t s);
int solve_blocks(int n_points);
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
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    unsigned spins = 0;
    while (ld_acquire_u32(bar) < target) {
      if (++spins > kSpinLimit) {
        ok = 0;
        atomicCAS(&rec->status, MAZE_OK, MAZE_ERR_TIMEOUT);
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
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

// Periodic neighbours of flat index n = i + jN + kN^2.
struct Nbr {
  int xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nbr neighbours(int n, int N) {
  const int NN = N * N;
  const int k = n / NN;
  const int rem = n - k * NN;
  const int j = rem / N;
  const int i = rem - j * N;
  Nbr b;
  b.xm = (i == 0) ? n + N - 1 : n - 1;
  b.xp = (i == N - 1) ? n - N + 1 : n + 1;
  b.ym = (j == 0) ? n + NN - N : n - N;
  b.yp = (j == N - 1) ? n - NN + N : n + N;
  b.zm = (k == 0) ? n + NN * (N - 1) : n - NN;
  b.zp = (k == N - 1) ? n - NN * (N - 1) : n + NN;
  return b;
}

#endif  // __CUDACC__

}  // namespace maze
