// C ABI of libmaze: context lifetime, configuration checks, the order of the
// kernels in one MaZe step, CUDA-graph replay of the step, host transfers and
// checkpoints. See include/maze.h for the contract of each entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <cmath>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <functional>
#include <condition_variable>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "maze_ctx.h"
#include "maze_trace.h"

using namespace maze;

namespace {
thread_local std::string g_err;
constexpr uint64_t kBlobMagic = 0x4d415a4530314250ull;  // "MAZE01BP"
}  // namespace

maze_status maze::fail(maze_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? MAZE_ERR_OOM : MAZE_ERR_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    }                                                                                         \
  } while (0)

void maze::set_last_error(const char* msg) { g_err = msg; }


namespace maze {

template <typename T>
maze_status dalloc(maze_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  if (c->arena) {
    v = c->arena->alloc(count * sizeof(T) + 16);
    if (!v) return fail(MAZE_ERR_OOM, "the batch's device memory arena is full");
  } else {
    cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MAZE_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
  }
  c->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return MAZE_OK;
}

void exp2_table(double* out64) {
  for (int j = 0; j < 64; ++j) out64[j] = exp2(j / 64.0);
}

// Whether the multigrid hierarchy halves level L - 1 of edge N once more:
// while the edge is even and above 8, and an 8^3 finest level once (so that
// every hierarchy has at least two levels). The coarsest level, of at most
// 8^3 points, is solved exactly.
bool mg_halves(int N, int L) { return N % 2 == 0 && (N > 8 || (N == 8 && L == 1)); }

maze_status validate(const maze_config* c) {
  if (!c) return fail(MAZE_ERR_INVALID, "config is NULL");
  if (c->n_ions < 2) return fail(MAZE_ERR_INVALID, "n_ions must be >= 2");
  if (c->grid_N < 8 || c->grid_N > 1024 || c->grid_N % 2)
    return fail(MAZE_ERR_INVALID, "grid_N must be even and in [8, 1024]");
  if (!(c->box_L > 0) || !isfinite(c->box_L)) return fail(MAZE_ERR_INVALID, "box_L must be > 0");
  if (!(c->r_cut > 0) || c->r_cut > 0.5 * c->box_L * (1 + 1e-12))
    return fail(MAZE_ERR_INVALID, "r_cut must be in (0, L/2]");
  if (!(c->dt > 0)) return fail(MAZE_ERR_INVALID, "dt must be > 0");
  if (!(c->tol > 0)) return fail(MAZE_ERR_INVALID, "tol must be > 0");
  if (c->max_iter < 1) return fail(MAZE_ERR_INVALID, "max_iter must be >= 1");
  if (c->solver != MAZE_SOLVER_CG && c->solver != MAZE_SOLVER_MG)
    return fail(MAZE_ERR_INVALID, "solver must be MAZE_SOLVER_CG or MAZE_SOLVER_MG");
  if (c->solver == MAZE_SOLVER_MG && (c->mg_pre < 1 || c->mg_post < 1 || c->mg_pre > 8 || c->mg_post > 8))
    return fail(MAZE_ERR_INVALID, "mg_pre and mg_post must be in [1, 8]");
  if (c->solver == MAZE_SOLVER_MG) {
    // the hierarchy halves the edge while it is even and above 8; its
    // coarsest level is solved exactly by a dense kernel of at most 8^3 points
    int Nc = c->grid_N;
    for (int L = 1; mg_halves(Nc, L); ++L) Nc /= 2;
    if (Nc > 8)
      return fail(MAZE_ERR_INVALID, "multigrid needs grid_N = m * 2^k with a coarsest edge m <= 8 (e.g. 32, 48, 56)");
  }
  if (c->order_P != 2 && c->order_P != 4) return fail(MAZE_ERR_INVALID, "order_P must be 2 or 4");
  for (int k = 0; k < 3; ++k)
    if (!(c->tf_A[k] >= 0) || !isfinite(c->tf_A[k]))
      return fail(MAZE_ERR_INVALID, "tf_A must be finite and >= 0 (a repulsive prefactor)");
  if (c->precision != MAZE_FP64 && c->precision != MAZE_MIXED && c->precision != MAZE_FP64_FIXMG)
    return fail(MAZE_ERR_INVALID, "precision must be MAZE_FP64, MAZE_MIXED or MAZE_FP64_FIXMG");
  if (c->precision == MAZE_FP64_FIXMG && c->solver != MAZE_SOLVER_MG)
    return fail(MAZE_ERR_INVALID, "precision MAZE_FP64_FIXMG runs the multigrid solver (MAZE_SOLVER_MG)");
  if (c->precision == MAZE_MIXED && c->solver != MAZE_SOLVER_MG)
    return fail(MAZE_ERR_INVALID, "precision MAZE_MIXED runs the multigrid solver (MAZE_SOLVER_MG)");
  if (c->scheme != MAZE_SCHEME_MAZE && c->scheme != MAZE_SCHEME_MG_STATIC && c->scheme != MAZE_SCHEME_MG_TIMEPROP)
    return fail(MAZE_ERR_INVALID, "scheme must be one of MAZE_SCHEME_*");
  if (c->force_estimator != MAZE_FORCE_CD && c->force_estimator != MAZE_FORCE_GRADW)
    return fail(MAZE_ERR_INVALID, "force_estimator must be MAZE_FORCE_CD or MAZE_FORCE_GRADW");
  if (!(c->langevin_gamma >= 0) || !isfinite(c->langevin_gamma))
    return fail(MAZE_ERR_INVALID, "langevin_gamma must be finite and >= 0");
  if (!(c->langevin_T >= 0) || !isfinite(c->langevin_T))
    return fail(MAZE_ERR_INVALID, "langevin_T must be finite and >= 0");
  if (!c->pos || !c->vel || !c->type) return fail(MAZE_ERR_INVALID, "pos, vel and type must be non-NULL");
  if (!(c->mass[0] > 0) || !(c->mass[1] > 0)) return fail(MAZE_ERR_INVALID, "masses must be > 0");
  double qsum = 0, qabs = 0;
  for (int i = 0; i < c->n_ions; ++i) {
    const int t = c->type[i];
    if (t != 0 && t != 1) return fail(MAZE_ERR_INVALID, "type must be 0 or 1");
    qsum += c->charge[t];
    qabs += fabs(c->charge[t]);
    for (int d = 0; d < 3; ++d)
      if (!isfinite(c->pos[3 * i + d]) || !isfinite(c->vel[3 * i + d]))
        return fail(MAZE_ERR_INVALID, "non-finite position or velocity");
  }
  if (fabs(qsum) > 1e-9 * qabs) return fail(MAZE_ERR_INVALID, "the system must be charge neutral");
  return MAZE_OK;
}

double wrap_host(double x, double L) {
  if (x >= 0.0 && x < L) return x;
  x -= L * floor(x / L);
  if (x < 0.0) x += L;   // (x / L rounded up to the next integer)
  if (x >= L) x = 0.0;   // (within rounding of L, i.e. of 0)
  return x;
}

// --- argument blocks for the current rotation ------------------------------

LangevinArgs langevin_args(maze_ctx* c) {
  LangevinArgs o = {};
  const maze_config& g = c->cfg;
  o.on = g.langevin_gamma > 0 ? 1 : 0;
  o.a = exp(-0.5 * g.langevin_gamma * g.dt);
  const double v2 = (1.0 - o.a * o.a) * MAZE_KB_EV_PER_K * g.langevin_T * MAZE_ACC_UNIT;
  o.sd0 = sqrt(v2 / g.mass[0]);
  o.sd1 = sqrt(v2 / g.mass[1]);
  o.key0 = (unsigned)(g.seed & 0xffffffffu);
  o.key1 = (unsigned)(g.seed >> 32);
  return o;
}

IonArgs ion_args(maze_ctx* c, int do_move, int do_spread) {
  IonArgs a;
  a.n = c->n;
  a.L = c->L;
  a.h = c->h;
  a.inv_L = 1.0 / c->L;
  a.inv_h = 1.0 / c->h;
  a.cell_scale = c->nc / c->L;
  a.N = c->N;
  a.P = c->P;
  a.pos = c->pos;
  a.vel = c->vel;
  a.force = c->force;
  a.type = c->type;
  a.pos32 = c->pos32;
  a.qfix = do_spread ? c->qfix : nullptr;
  a.cell_of = c->cell_of;
  a.cell_count = c->cell_count;
  a.nc = c->nc;
  a.charge0 = c->cfg.charge[0];
  a.charge1 = c->cfg.charge[1];
  a.kick0 = 0.5 * c->cfg.dt * MAZE_ACC_UNIT / c->cfg.mass[0];
  a.kick1 = 0.5 * c->cfg.dt * MAZE_ACC_UNIT / c->cfg.mass[1];
  a.dt = c->cfg.dt;
  a.do_move = do_move;
  a.rec = c->rec;
  a.gate = c->gate;
  a.wbuf = c->wbuf;
  a.wbuf32 = c->mixed ? c->wbuf32 : nullptr;
  a.wbase = c->wbase;
  a.io = (do_move && c->io_capture) ? c->io_desc : nullptr;
  a.rel_hi = (c->mixed || c->pair_df) ? c->rel_hi : nullptr;
  a.rel_lo = (c->mixed || c->pair_df) ? c->rel_lo : nullptr;
  a.cell_len = c->nc >= 3 ? c->L / c->nc : c->L;
  a.wdbuf = c->wdbuf;
  a.wdbuf32 = c->wdbuf32;
  a.ou = langevin_args(c);
  return a;
}

CellArgs cell_args(maze_ctx* c) {
  CellArgs a;
  a.n = c->n;
  a.ncell = c->ncell;
  a.cell_of = c->cell_of;
  a.cell_count = c->cell_count;
  a.cell_start = c->cell_start;
  a.cursor = c->cursor;
  a.cell_ions = c->cell_ions;
  a.pos32 = c->pos32;
  a.pos_sorted = c->pos_sorted;
  a.rel_hi = (c->mixed || c->pair_df) ? c->rel_hi : nullptr;
  a.rel_lo = c->rel_lo;
  a.rel_hi_sorted = c->rel_hi_s;
  a.rel_lo_sorted = c->rel_lo_s;
  a.rec = c->rec;
  return a;
}

// The Tosi-Fumi table of the pair kernels from the configuration, V(r) =
// A exp(B (s - r)) - C r^-6 - D r^-8 - V(r_cut) per pair kind, in FP64 and as
// (hi, lo) float pairs for the double-float form.
void fill_pair_consts(const maze_config& g, ForceArgs& a) {
  const double rc = g.r_cut;
  for (int k = 0; k < 3; ++k) {
    a.A[k] = g.tf_A[k];
    a.s[k] = g.tf_s[k];
    a.C[k] = g.tf_C[k];
    a.D[k] = g.tf_D[k];
    a.Vc[k] = g.tf_A[k] * exp(g.tf_B * (g.tf_s[k] - rc)) - g.tf_C[k] / pow(rc, 6) - g.tf_D[k] / pow(rc, 8);
    a.Ec[k] = g.tf_B * g.tf_s[k] + log(g.tf_A[k]);   // (A = 0: -inf, exp gives 0)
    a.C6[k] = 6.0 * g.tf_C[k];
    a.D8[k] = 8.0 * g.tf_D[k];
  }
  a.B = g.tf_B;
  a.rc2 = rc * rc;
  auto split = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  a.pdf.B = split(g.tf_B);
  a.pdf.rc2 = split(a.rc2);
  for (int k = 0; k < 3; ++k) {
    // (A = 0 makes Ec -inf: a large negative finite value gives the same 0)
    a.pdf.Ec[k] = split(std::isfinite(a.Ec[k]) ? a.Ec[k] : -1e4);
    a.pdf.C[k] = split(a.C[k]);
    a.pdf.D[k] = split(a.D[k]);
    a.pdf.Vc[k] = split(a.Vc[k]);
    a.pdf.C6[k] = split(a.C6[k]);
    a.pdf.D8[k] = split(a.D8[k]);
  }
}

ForceArgs force_args(maze_ctx* c, const double* phi, int do_kick, int count_step) {
  ForceArgs a;
  const maze_config& g = c->cfg;
  a.n = c->n;
  a.L = c->L;
  a.h = c->h;
  a.inv_2h = 0.5 / c->h;
  a.N = c->N;
  a.P = c->P;
  a.pos = c->pos;
  a.vel = c->vel;
  a.force = c->force;
  a.force_el = c->force_el;
  a.pos32 = c->pos32;
  a.type = c->type;
  a.phi = phi;
  a.phi_df = c->mixed ? 1 : 0;
  a.mixed = c->mixed ? 1 : 0;
  a.rel_hi = c->rel_hi;
  a.rel_lo = c->rel_lo;
  a.rel_hi_sorted = c->rel_hi_s;
  a.rel_lo_sorted = c->rel_lo_s;
  {
    const double cl = c->nc >= 3 ? c->L / c->nc : c->L;
    a.cell_len_h = (float)cl;
    a.cell_len_l = (float)(cl - (double)a.cell_len_h);
    a.L_h = (float)c->L;
    a.L_l = (float)(c->L - (double)a.L_h);
  }
  // one block per cell when the box has cells and either enough of them to
  // fill the GPU or FP32 pair arithmetic (mixed precision)
  a.by_cell = (c->nc >= 3 && (c->mixed || c->ncell >= 2 * c->num_sms)) ? 1 : 0;
  a.cell_split = c->cell_split;
  a.wbuf32 = c->wbuf32;
  a.wbuf = c->wbuf;
  a.wbase = c->wbase;
  a.wdbuf = c->wdbuf;
  a.wdbuf32 = c->wdbuf32;
  a.gradw = c->cfg.force_estimator == MAZE_FORCE_GRADW ? 1 : 0;
  a.nc = c->nc;
  a.reach = c->reach;
  a.cell_start = c->cell_start;
  a.cell_ions = c->cell_ions;
  a.pos_sorted = c->pos_sorted;
  a.cell_of = c->cell_of;
  a.charge0 = g.charge[0];
  a.charge1 = g.charge[1];
  a.mass0 = g.mass[0];
  a.mass1 = g.mass[1];
  a.kick0 = 0.5 * g.dt * MAZE_ACC_UNIT / g.mass[0];
  a.kick1 = 0.5 * g.dt * MAZE_ACC_UNIT / g.mass[1];
  a.dt = g.dt;
  a.ke_coef = 0.5 / MAZE_ACC_UNIT;
  const double rc = g.r_cut;
  fill_pair_consts(g, a);
  a.exp2tab = c->exp2tab;
  a.pair_df = c->pair_df ? 1 : 0;
  a.exp2tab_f = c->exp2tab_f;
  for (int k = 0; k < 3; ++k) {
    a.Af[k] = (float)a.A[k];
    a.sf[k] = (float)a.s[k];
    a.Cf[k] = (float)a.C[k];
    a.Df[k] = (float)a.D[k];
    a.Vcf[k] = (float)a.Vc[k];
  }
  a.Bf = (float)g.tf_B;
  a.rc2f = (float)(rc * rc);
  const double rcf = rc + 1e-3 + 1e-6 * c->L;
  a.rc2_filter = (float)(rcf * rcf);
  a.Lf = (float)c->L;
  a.inv_Lf = (float)(1.0 / c->L);
  a.do_kick = do_kick;
  a.count_step = count_step;
  a.ou = langevin_args(c);
  a.part = c->fpart;
  a.ticket = c->ticket;
  a.pair_out = c->pair_out;
  a.pair_fix = c->pair_fix;
  a.gath = c->gath;
  a.rec = c->rec;
  a.gate = c->gate;
  return a;
}

// The direct schemes solve M phi = -4pi q/h from phi_p; in correction form
// phi = phi_p - (4pi/h) y with M y = sigma(phi_p) from y = 0, and their
// residual max|M phi + (4pi/h) q| (Eq. res_poisson) is (4pi/h) max|M y - sigma|.
void set_scheme(maze_ctx* c, int zero_phi, int& static_guess, double& tol, double& res_scale) {
  const bool direct = !zero_phi && c->cfg.scheme != MAZE_SCHEME_MAZE;
  static_guess = (!zero_phi && c->cfg.scheme == MAZE_SCHEME_MG_STATIC) ? 1 : 0;
  res_scale = direct ? 4.0 * kPi / c->h : 1.0;
  tol = c->cfg.tol / res_scale;
}

SolveArgs solve_args(maze_ctx* c, int zero_phi, double* q_out) {
  SolveArgs a;
  a.N = c->N;
  a.n = (int)c->ng;
  a.phi_k = c->phi[c->ik];
  a.phi_km1 = c->phi[(c->ik + 1) % 3];
  a.phi_out = c->phi[(c->ik + 2) % 3];
  a.qfix = c->qfix;
  a.q_out = q_out;
  a.sigma = c->sigma;
  a.y = c->y;
  a.r = c->r;
  a.p = c->p;
  a.p1 = c->p1;
  a.Mp = c->Mp;
  a.recs = c->recs;
  a.bar = c->bar;
  a.rec = c->rec;
  a.c_sig = c->h / (4.0 * kPi);
  a.c_phi = 4.0 * kPi / c->h;
  a.inv_n = 1.0 / (double)c->ng;
  a.tol = c->cfg.tol;
  a.max_iter = zero_phi ? c->max_iter_init : c->cfg.max_iter;
  a.zero_phi = zero_phi;
  set_scheme(c, zero_phi, a.static_guess, a.tol, a.res_scale);
  a.gate = c->gate;
  return a;
}

// --- sequences ------------------------------------------------------------

MixedArgs mixed_args(maze_ctx* c, int zero_phi, double* q_out) {
  MixedArgs a = c->mx;
  a.phi_k = reinterpret_cast<const float2*>(c->phi[c->ik]);
  a.phi_km1 = reinterpret_cast<const float2*>(c->phi[(c->ik + 1) % 3]);
  a.phi_out = reinterpret_cast<float2*>(c->phi[(c->ik + 2) % 3]);
  a.sigma = reinterpret_cast<float2*>(c->sigma);
  a.y = reinterpret_cast<float2*>(c->y);
  a.y2 = reinterpret_cast<float2*>(c->y2);
  a.qfix = c->qfix;
  a.q_out = q_out;
  a.max_iter = zero_phi ? c->max_iter_init : c->cfg.max_iter;
  a.zero_phi = zero_phi;
  set_scheme(c, zero_phi, a.static_guess, a.tol, a.res_scale);
  a.y_reset = (!zero_phi && c->cfg.scheme != MAZE_SCHEME_MAZE) ? 1 : 0;
  a.recs = c->recs;
  a.bar = c->bar;
  a.rec = c->rec;
  a.gate = c->gate;
  return a;
}

maze_status enqueue_solve(maze_ctx* c, int zero_phi, double* q_out, bool narrow = false) {
  // (the one-cluster mixed solve synchronises and reduces in shared memory:
  // no grid counters or reduction records to clear)
  const bool cluster = c->mixed && c->mx_cluster > 0;
  if (!cluster) CK(cudaMemsetAsync(c->recs, 0, c->recs_bytes, c->stream));
  if (!zero_phi && c->cfg.scheme != MAZE_SCHEME_MAZE) CK(cudaMemsetAsync(c->y, 0, c->ng * 8, c->stream));
  if (c->mixed) {
    if (!cluster) CK(cudaMemsetAsync(c->bar, 0, sizeof(unsigned), c->stream));
    CK(launch_mixed_solve(mixed_args(c, zero_phi, q_out), c->mx_cluster, narrow ? c->ov_blocks : c->mx_blocks,
                          c->stream, narrow ? c->ov_threads : 0));
  } else if (c->cfg.solver == MAZE_SOLVER_MG) {
    CK(cudaMemsetAsync(c->bar, 0, sizeof(unsigned), c->stream));
    if (c->fixmg)
      CK(launch_mgfix_solve(solve_args(c, zero_phi, q_out), c->mg, narrow ? c->ov_blocks : c->sblocks,
                            narrow ? c->ov_threads : 0, c->stream));
    else CK(launch_mg_solve(solve_args(c, zero_phi, q_out), c->mg, c->sblocks, c->stream));
  } else {
    CK(launch_cg_solve(solve_args(c, zero_phi, q_out), c->sblocks, c->stream));
  }
  return MAZE_OK;
}

// Pseudo-inverse of the periodic h^2-scaled Laplacian on an Nc^3 grid as a
// convolution kernel: g(d) = (1/Nc^3) sum_{k != 0} cos(2 pi k.d / Nc) / lambda(k),
// lambda(k) = -6 + 2 cos(2 pi kx/Nc) + 2 cos(2 pi ky/Nc) + 2 cos(2 pi kz/Nc)
// (the plane waves diagonalise the circulant M). g * b is the zero-mean
// exact solution of M x = b - mean(b).
std::vector<double> coarse_kernel(int Nc) {
  const int n3 = Nc * Nc * Nc;
  std::vector<double> c(Nc), g(n3, 0.0);
  for (int t = 0; t < Nc; ++t) c[t] = cos(2.0 * kPi * t / Nc);
  for (int dz = 0; dz < Nc; ++dz)
    for (int dy = 0; dy < Nc; ++dy)
      for (int dx = 0; dx < Nc; ++dx) {
        double s = 0.0;
        for (int kz = 0; kz < Nc; ++kz)
          for (int ky = 0; ky < Nc; ++ky)
            for (int kx = 0; kx < Nc; ++kx) {
              if (!kx && !ky && !kz) continue;
              const double lam = -6.0 + 2.0 * (c[kx] + c[ky] + c[kz]);
              s += c[(kx * dx + ky * dy + kz * dz) % Nc] / lam;
            }
        g[dx + Nc * (dy + Nc * dz)] = s / n3;
      }
  return g;
}

// S7 + S8 (+ S9): one force kernel, or for FP64 boxes with pair_fix the
// once-per-pair kernel followed by the gather and finish.
maze_status enqueue_forces(maze_ctx* c, const ForceArgs& fa, cudaStream_t st) {
  if (c->pair_fix) {
    CK(launch_pairs_half(fa, st));
    CK(launch_finish_fix(fa, st));
  } else {
    CK(launch_forces(fa, c->fblocks, st));
  }
  return MAZE_OK;
}

maze_status enqueue_cells(maze_ctx* c) {
  if (c->nc >= 3) CK(launch_cells(cell_args(c), c->stream));
  return MAZE_OK;
}

// One MaZe step for the current rotation (does not rotate). With timing on,
// events bracket the four phases.
maze_status enqueue_step(maze_ctx* c, int timed) {
  if (c->mixed && c->fused_step) {
    // mixed precision up to 64^3: S1-S6 in one cluster launch, then the
    // forces; the move/spread and cell phases are timed as part of the solve
    if (timed) {
      CK(cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal));
      CK(cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal));
      CK(cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal));
    }
    CK(launch_cluster_step(ion_args(c, 1, 1), cell_args(c), mixed_args(c, 0, nullptr), c->mx_cluster, c->stream));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[3], c->stream, cudaEventRecordExternal));
    CK(launch_forces(force_args(c, c->phi[(c->ik + 2) % 3], 1, 1), c->fblocks, c->stream));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[4], c->stream, cudaEventRecordExternal));
    return MAZE_OK;
  }
  if (c->pair_out) {
    // mixed precision, one-cluster solve: S1-S3 in one cluster launch, then
    // S8 (pairs) on the side stream beside the solve (S4-S6, one cluster on
    // a few SMs), joined before S7/S9
    if (timed) {
      CK(cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal));
      CK(cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal));
    }
    CK(launch_cluster_front(ion_args(c, 1, 1), cell_args(c), mixed_args(c, 0, nullptr), c->mx_cluster, c->stream));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal));
    maze_status s;
    const ForceArgs fa = force_args(c, c->phi[(c->ik + 2) % 3], 1, 1);
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    CK(launch_pairs(fa, c->side_stream));
    CK(cudaEventRecord(c->ev_join, c->side_stream));
    s = enqueue_solve(c, 0, nullptr);
    if (timed && s == MAZE_OK) CK(cudaEventRecordWithFlags(c->ev[3], c->stream, cudaEventRecordExternal));
    // join the side stream before any return (a capture must not end forked)
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (s != MAZE_OK) return s;
    CK(launch_gather_finish(fa, c->fblocks, c->stream));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[4], c->stream, cudaEventRecordExternal));
    return MAZE_OK;
  }
  if (c->overlap) {
    // S8 needs only the positions and the cell list: after S1 and S2 it runs
    // on the side stream, sharing every SM with S3 and the solve (S4-S6),
    // whose V-cycle is bound by memory latency and integer work while the
    // pairs are bound by instruction issue; then S7 (needs phi^{k+1}) and S9.
    // (Timed phases: S1; S2 and S3; the solve S4-S6; S7-S9.) The cell list
    // on the side stream too (beside S3) made the step slower: the pairs
    // then started late and ended after the solve.
    if (timed) CK(cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal));
    const IonArgs ia = ion_args(c, 1, 1);
    CK(launch_ion_update(ia, c->stream, 1));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal));
    maze_status s = enqueue_cells(c);
    if (s != MAZE_OK) return s;
    const ForceArgs fa = force_args(c, c->phi[(c->ik + 2) % 3], 1, 1);
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    CK(launch_pairs_only(fa, c->ov_pair_blocks, c->ov_pair_smem, c->side_stream));
    CK(cudaEventRecord(c->ev_join, c->side_stream));
    CK(launch_ion_update(ia, c->stream, 2));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal));
    s = enqueue_solve(c, 0, nullptr, true);
    if (timed && s == MAZE_OK) CK(cudaEventRecordWithFlags(c->ev[3], c->stream, cudaEventRecordExternal));
    // join the side stream before any return (a capture must not end forked)
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (s != MAZE_OK) return s;
    CK(launch_gather_cells(fa, c->stream));
    CK(launch_finish_fix(fa, c->stream));
    if (timed) CK(cudaEventRecordWithFlags(c->ev[4], c->stream, cudaEventRecordExternal));
    return MAZE_OK;
  }
  if (timed) CK(cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal));
  CK(launch_ion_update(ion_args(c, 1, 1), c->stream));
  if (timed) CK(cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal));
  maze_status s = enqueue_cells(c);
  if (s != MAZE_OK) return s;
  if (timed) CK(cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal));
  s = enqueue_solve(c, 0, nullptr);
  if (s != MAZE_OK) return s;
  if (timed) CK(cudaEventRecordWithFlags(c->ev[3], c->stream, cudaEventRecordExternal));
  {
    const maze_status fs = enqueue_forces(c, force_args(c, c->phi[(c->ik + 2) % 3], 1, 1), c->stream);
    if (fs != MAZE_OK) return fs;
  }
  if (timed) CK(cudaEventRecordWithFlags(c->ev[4], c->stream, cudaEventRecordExternal));
  return MAZE_OK;
}

void rotate(maze_ctx* c, int steps) { c->ik = (c->ik + 2 * (steps % 3)) % 3; }

// Capture one step per rotation state (phi^k in phi[0], phi[1], phi[2]);
// on any capture failure fall back to direct launches.
maze_status build_graphs(maze_ctx* c, int timed) {
  c->graphs_tried[timed] = true;
  const int ik0 = c->ik;
  for (int g = 0; g < 3; ++g) {
    c->ik = g;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c->ik = ik0;
      return MAZE_OK;
    }
    maze_status s = enqueue_step(c, timed);
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (s != MAZE_OK || e != cudaSuccess || !graph) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      c->ik = ik0;
      return MAZE_OK;
    }
    e = cudaGraphInstantiate(&c->graph[timed][g], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->graph[timed][g] = nullptr;
      c->ik = ik0;
      return MAZE_OK;
    }
  }
  c->ik = ik0;
  c->graphs_ok[timed] = true;
  return MAZE_OK;
}

maze_status clear_status(maze_ctx* c) {
  c->rec_dirty = true;
  c->staged_fresh[0] = c->staged_fresh[1] = false;
  CK(cudaMemsetAsync(&c->rec->status, 0, sizeof(int32_t), c->stream));
  return MAZE_OK;
}

maze_status read_stats(maze_ctx* c) {
  CK(cudaMemcpyAsync(c->rec_host, c->rec, sizeof(maze_stats), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->rec_dirty = false;
  return MAZE_OK;
}

// The pinned staging buffer k of the per-ion host copies (3 n doubles), made
// on first use in pairs: stages 0 and 1 (uploads of the positions and
// velocities) are one block, 2 and 3 (their reads) another, each laid out as
// the device's positions followed by its velocities, so that both move in
// one copy.
maze_status stage_buffer(maze_ctx* c, int k) {
  if (c->stage[k]) return MAZE_OK;
  const int k0 = k & ~1;
  const size_t n3 = 3 * (size_t)c->n;
  double* b = nullptr;
  if (cudaMallocHost(&b, 2 * n3 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MAZE_ERR_OOM, "cudaMallocHost failed");
  }
  c->stage[k0] = b;
  c->stage[k0 + 1] = b + n3;
  if (k0 == 0)
    for (int q = 0; q < 2; ++q) CK(cudaEventCreateWithFlags(&c->stage_ev[q], cudaEventDisableTiming));
  return MAZE_OK;
}

maze_status status_message(maze_ctx* c) {
  const int s = c->rec_host->status;
  if (s == MAZE_OK) return MAZE_OK;
  char buf[160];
  if (s == MAZE_ERR_NOT_CONVERGED)
    snprintf(buf, sizeof buf, "constraint solve not converged: residual %.3e after %d iterations",
             c->rec_host->resid, c->rec_host->iters);
  else if (s == MAZE_ERR_TIMEOUT)
    snprintf(buf, sizeof buf, "a device-side wait timed out; the context must be destroyed");
  else if (s == MAZE_ERR_NONFINITE)
    snprintf(buf, sizeof buf, "non-finite residual or energy");
  else
    snprintf(buf, sizeof buf, "device status %d", s);
  return fail((maze_status)s, buf);
}

void free_ctx(maze_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int t = 0; t < 2; ++t)
    for (int g = 0; g < 3; ++g)
      if (c->graph[t][g]) cudaGraphExecDestroy(c->graph[t][g]);
  for (int g = 0; g < 3; ++g)
    if (c->io_graph[g]) cudaGraphExecDestroy(c->io_graph[g]);
  if (c->io_stage) cudaFreeHost(c->io_stage);
  if (c->io_desc_host) cudaFreeHost(c->io_desc_host);
  if (c->io_desc) cudaFree(c->io_desc);
  for (int k = 0; k < 5; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  for (void* p : c->allocs) {
    if (c->arena) c->arena->release(p);
    else cudaFree(p);
  }
  if (c->rec_host) cudaFreeHost(c->rec_host);
  for (int k = 0; k < 4; ++k)
    if (c->stage[k] && !(k & 1)) cudaFreeHost(c->stage[k]);   // (odd stages live in the even ones' blocks)
  for (int k = 0; k < 2; ++k)
    if (c->stage_ev[k]) cudaEventDestroy(c->stage_ev[k]);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// Host threads for the exchange's copies: created once per process and
// kept (a thread started and joined per call costs more than a share of the
// copies on the GPU machine's Arm cores), woken per job; the caller runs task 0,
// the workers the rest. Jobs from several host threads run one at a time.
class HostPool {
 public:
  explicit HostPool(int workers) {
    for (int w = 0; w < workers; ++w) std::thread([this] { loop(); }).detach();
  }
  void run(int tasks, const std::function<void(int)>& job) {
    std::lock_guard<std::mutex> one(run_mutex_);
    {
      std::lock_guard<std::mutex> g(m_);
      job_ = &job;
      tasks_ = tasks;
      next_.store(1);
      left_.store(tasks - 1);
      ++gen_;
    }
    cv_.notify_all();
    job(0);
    work();
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [&] { return left_.load() == 0; });
  }

 private:
  void loop() {
    unsigned seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
      }
      work();
    }
  }
  void work() {
    for (int t; (t = next_.fetch_add(1)) < tasks_;) {
      (*job_)(t);
      if (left_.fetch_sub(1) == 1) {
        std::lock_guard<std::mutex> g(m_);
        done_.notify_all();
      }
    }
  }
  std::mutex run_mutex_, m_;
  std::condition_variable cv_, done_;
  unsigned gen_ = 0;
  int tasks_ = 0;
  std::atomic<int> next_{0}, left_{0};
  const std::function<void(int)>* job_ = nullptr;
};

HostPool& host_pool() {
  static HostPool* pool = new HostPool(15);   // never destroyed: its threads wait until the process ends
  return *pool;
}

// fn(lo, hi) over [0, n) in chunks on host threads for large n (the per-ion
// host loops of big boxes), else in the calling thread.
template <class F>
void host_ranges(int n, F fn) {
  constexpr int kMinPerThread = 16384;
  const unsigned hw = std::thread::hardware_concurrency();
  const int T = std::min(std::min(16, hw > 1 ? (int)hw / 2 : 1), n / kMinPerThread);
  if (T <= 1) {
    fn(0, n);
    return;
  }
  const int chunk = (n + T - 1) / T;
  const std::function<void(int)> job = [&](int t) { fn(std::min(n, t * chunk), std::min(n, (t + 1) * chunk)); };
  host_pool().run(T, job);
}

bool ion_finite(const maze_ctx* c, const double* in) {
  std::atomic<bool> bad{false};
  host_ranges(c->n, [&](int lo, int hi) {
    bool b = false;
    for (size_t i = 3 * (size_t)lo; i < 3 * (size_t)hi; ++i) b |= !isfinite(in[i]);
    if (b) bad.store(true, std::memory_order_relaxed);
  });
  return !bad.load();
}

// [n][3] host order -> [3][n] (positions wrapped into [0, L) when wrap).
void to_soa(const double* in, double* out, int n, bool wrap, double L) {
  host_ranges(n, [=](int lo, int hi) {
    double* o0 = out;
    double* o1 = out + n;
    double* o2 = out + 2 * (size_t)n;
    for (int i = lo; i < hi; ++i) {
      const double* p = in + 3 * (size_t)i;
      o0[i] = wrap ? wrap_host(p[0], L) : p[0];
      o1[i] = wrap ? wrap_host(p[1], L) : p[1];
      o2[i] = wrap ? wrap_host(p[2], L) : p[2];
    }
  });
}

// [3][n] -> [n][3] host order.
void to_aos(const double* in, double* out, int n) {
  host_ranges(n, [=](int lo, int hi) {
    const double* i0 = in;
    const double* i1 = in + n;
    const double* i2 = in + 2 * (size_t)n;
    for (int i = lo; i < hi; ++i) {
      double* p = out + 3 * (size_t)i;
      p[0] = i0[i];
      p[1] = i1[i];
      p[2] = i2[i];
    }
  });
}

// Upload of the positions (in[0], wrapped into [0, L)) and / or velocities
// (in[1]) from host memory in [n][3] order, checked finite by the caller.
// The values go through pinned stages of the context, so the upload is
// asynchronous on the stream: the caller's buffers are read only here. Both
// together move in one copy (the device keeps the velocities right after
// the positions, the stages likewise).
maze_status upload_ions(maze_ctx* c, const double* const (&in)[2]) {
  const int n = c->n;
  const size_t n3 = 3 * (size_t)n;
  if (c->arena) {   // a batch box: a temporary and a synchronous copy
    std::vector<double> tmp(n3);
    for (int k = 0; k < 2; ++k) {
      if (!in[k]) continue;
      c->staged_fresh[k] = false;
      to_soa(in[k], tmp.data(), n, k == 0, c->L);
      CK(cudaMemcpyAsync(k == 0 ? c->pos : c->vel, tmp.data(), n3 * 8, cudaMemcpyHostToDevice, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    return MAZE_OK;
  }
  maze_status st = stage_buffer(c, 0);
  if (st != MAZE_OK) return st;
  for (int k = 0; k < 2; ++k) {
    if (!in[k]) continue;
    c->staged_fresh[k] = false;
    CK(cudaEventSynchronize(c->stage_ev[k]));   // the stage's previous upload has been read
    to_soa(in[k], c->stage[k], n, k == 0, c->L);
  }
  if (in[0] && in[1]) {
    CK(cudaMemcpyAsync(c->pos, c->stage[0], 2 * n3 * 8, cudaMemcpyHostToDevice, c->stream));
  } else {
    const int k = in[0] ? 0 : 1;
    CK(cudaMemcpyAsync(k == 0 ? c->pos : c->vel, c->stage[k], n3 * 8, cudaMemcpyHostToDevice, c->stream));
  }
  for (int k = 0; k < 2; ++k)
    if (in[k]) CK(cudaEventRecord(c->stage_ev[k], c->stream));
  return MAZE_OK;
}

}  // namespace maze

extern "C" {

const char* maze_last_error(void) { return g_err.c_str(); }

const char* maze_version(void) { return "maze-gb300 0.1"; }

}  // extern "C"

namespace maze {

// Checks, layout and device buffers of a context (no uploads, no kernels).
// With a counting arena nothing is allocated and no stream is created.
maze_status ctx_setup(const maze_config* cfg, Arena* arena, maze_ctx** out) {
  *out = nullptr;
  maze_status s = validate(cfg);
  if (s != MAZE_OK) return s;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3)
    return fail(MAZE_ERR_CUDA, "libmaze is built for sm_103a (GB300); this device is sm_" +
                                   std::to_string(prop.major) + std::to_string(prop.minor));
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(MAZE_ERR_CUDA, "device does not support cooperative launch");

  maze_ctx* c = new maze_ctx();
  c->arena = arena;
  c->cfg = *cfg;
  c->cfg.pos = c->cfg.vel = nullptr;
  c->cfg.type = nullptr;
  c->n = cfg->n_ions;
  c->N = cfg->grid_N;
  c->P = cfg->order_P;
  c->ng = (size_t)c->N * c->N * c->N;
  c->L = cfg->box_L;
  c->h = cfg->box_L / cfg->grid_N;
  if (cfg->cuda_stream) {
    c->stream = (cudaStream_t)cfg->cuda_stream;
  } else if (!(arena && arena->counting())) {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(MAZE_ERR_CUDA, "cudaStreamCreate failed");
    }
    c->own_stream = true;
  }
  const int n = c->n;
  const size_t ng = c->ng;
  // cell list: cells of at least r_cut with a 3^3 neighbourhood (the force
  // kernels also take cells of r_cut / 2 with a 5^3 neighbourhood, reach 2,
  // but with ~3 ions per cell the per-cell staging costs more than the fewer
  // candidates save: measured 5x slower on the 512000-ion box)
  c->reach = 1;
  c->nc = (int)floor(c->L / cfg->r_cut);
  if (c->nc < 3) c->nc = 0;
  c->ncell = c->nc * c->nc * c->nc;
  c->fixmg = cfg->precision == MAZE_FP64_FIXMG;
  c->sblocks = cfg->solver != MAZE_SOLVER_MG ? solve_blocks((int)ng)
               : c->fixmg                    ? mgfix_blocks((int)ng)
                                             : mg_blocks((int)ng);
  c->fblocks = force_blocks(n);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) c->num_sms = 1;
  if (c->ncell > 0) {
    // few cells (small boxes): split each cell's ions over several blocks of
    // the by-cell force kernel, about one ion per warp, up to two blocks per SM
    const int per_warp = (n + c->ncell - 1) / c->ncell;
    const int by_ions = (per_warp + kForceThreads / 32 - 1) / (kForceThreads / 32);
    const int by_sms = (2 * c->num_sms + c->ncell - 1) / c->ncell;
    c->cell_split = std::max(1, std::min(by_ions, by_sms));
  }
#define AL(p, cnt)                          \
  do {                                      \
    maze_status s_ = dalloc(c, &(p), (cnt)); \
    if (s_ != MAZE_OK) {                    \
      free_ctx(c);                          \
      return s_;                            \
    }                                       \
  } while (0)
  AL(c->pos, 6 * (size_t)n);   // the velocities right after the positions (one copy moves both)
  c->vel = c->pos + 3 * (size_t)n;
  AL(c->force, 3 * (size_t)n);
  AL(c->force_el, 3 * (size_t)n);
  AL(c->type, (size_t)n);
  AL(c->pos32, (size_t)n);
  // each precision allocates only the buffers its kernels touch
  const bool mixed = cfg->precision == MAZE_MIXED;
  const bool gradw = cfg->force_estimator == MAZE_FORCE_GRADW;
  if (mixed) {
    AL(c->wbuf32, 12 * (size_t)n);
    if (gradw) AL(c->wdbuf32, 12 * (size_t)n);
    AL(c->rel_hi, (size_t)n);
    AL(c->rel_lo, (size_t)n);
  } else {
    AL(c->wbuf, 12 * (size_t)n);
    if (gradw) AL(c->wdbuf, 12 * (size_t)n);
  }
  AL(c->wbase, (size_t)n);
  AL(c->exp2tab, 64);
  AL(c->qfix, ng);
  AL(c->qd, ng);
  for (int g = 0; g < 3; ++g) AL(c->phi[g], ng);
  AL(c->sigma, ng);
  AL(c->y, ng);
  if (cfg->solver == MAZE_SOLVER_CG) {
    AL(c->r, ng);
    AL(c->p, ng);
    AL(c->p1, ng);
    AL(c->Mp, ng);
  }
  c->recs_bytes = 2 * (size_t)c->sblocks * 4 * 16;
  AL(c->recs, 2 * (size_t)c->sblocks * 4);
  AL(c->bar, 4);
  std::vector<double>& gk = c->gk;
  if (cfg->solver == MAZE_SOLVER_MG) {
    // hierarchy: halve while the edge is even and above 8 (an 8^3 box: once)
    MgArgs& g = c->mg;
    g.L = 0;
    size_t tot = 0;
    for (int N = c->N;; N /= 2) {
      g.Nl[g.L] = N;
      g.lg[g.L] = -1;
      for (int b = 1; b < 16; ++b)
        if ((1 << b) == N) g.lg[g.L] = b;
      g.off[g.L] = tot;
      tot += (size_t)N * N * N;
      ++g.L;
      if (!mg_halves(N, g.L) || g.L == kMaxLevels) break;
    }
    g.nu1 = cfg->mg_pre;
    g.nu2 = cfg->mg_post;
    if (!mixed) {
      AL(c->mg_x, tot);
      AL(c->mg_b, tot);
      AL(c->mg_r, tot);
    }
    const int Nc = g.Nl[g.L - 1];
    gk = coarse_kernel(Nc);
    if (!mixed) {
      // the FP64 V-cycle keeps its right-hand sides as -b/6: fold the -6
      // into the coarsest solve's kernel
      for (double& v : gk) v *= -6.0;
      AL(c->mg_g, gk.size());
    }
    g.x = c->mg_x;
    g.b = c->mg_b;
    g.r = c->mg_r;
    g.gker = c->mg_g;
  }
  if (cfg->precision == MAZE_MIXED) {
    c->mixed = true;
    MixedArgs& m = c->mx;
    m.N = c->N;
    m.n = (int)ng;
    m.L = c->mg.L;
    for (int l = 0; l < m.L; ++l) {
      m.Nl[l] = c->mg.Nl[l];
      m.lg[l] = -1;
      for (int b = 1; b < 16; ++b)
        if ((1 << b) == m.Nl[l]) m.lg[l] = b;
    }
    m.nu1 = cfg->mg_pre;
    m.nu2 = cfg->mg_post;
    // the global form of the V-cycle storage: one part holding every level,
    // sized by the same layout function the kernels use
    const size_t tot = resident_bytes_host(m, 1) / sizeof(float);
    m.scratch_floats = tot;
    AL(c->y2, ng);
    AL(c->mx_scratch, tot);
    // the coarsest level's spectral solve: 1/(N_c^3 lambda(k)), then cos
    // and sin of 2 pi t / N_c
    AL(c->mx_g, gk.size() + 2 * (size_t)c->mg.Nl[c->mg.L - 1]);
    m.scratch = c->mx_scratch;
    m.gkerf = c->mx_g;
    const double cs = c->h / (4.0 * kPi), cp = 4.0 * kPi / c->h;
    m.c_sig_h = (float)cs;
    m.c_sig_l = (float)(cs - (double)m.c_sig_h);
    m.c_phi_h = (float)cp;
    m.c_phi_l = (float)(cp - (double)m.c_phi_h);
    m.tol = cfg->tol;
    m.inv_n = 1.0 / (double)ng;
    // one cluster for boxes up to 64^3 (cluster barriers), a cooperative
    // grid above
    if (c->N <= 64) {
      // the step's cluster launch and the step-0 solve use the same size
      const int cs = cluster_step_size();
      c->mx_cluster = cs > 0 ? std::min(cs, mixed_cluster_size()) : mixed_cluster_size();
      // standalone boxes with a cell list take the split step (S8 beside the
      // solve); the others S1-S6 in one cluster launch
      c->split_step = cs > 0 && cs >= c->mx_cluster && !arena && c->nc >= 3;
      c->fused_step = cs > 0 && cs >= c->mx_cluster && !c->split_step;
      m.resident = resident_bytes_host(m, c->mx_cluster) <= (size_t)kResidentSmem ? 1 : 0;
    } else {
      c->mx_blocks = mixed_grid_blocks((int)ng);
      if (c->mx_blocks > c->sblocks) c->mx_blocks = c->sblocks;
    }
  }
  AL(c->cell_of, (size_t)n);
  if (c->nc >= 3) {
    AL(c->cell_count, (size_t)c->ncell);
    AL(c->cell_start, (size_t)c->ncell + 1);
    AL(c->cursor, (size_t)c->ncell);
    AL(c->cell_ions, (size_t)n);
    AL(c->pos_sorted, (size_t)n);
    if (mixed) {
      AL(c->rel_hi_s, (size_t)n);
      AL(c->rel_lo_s, (size_t)n);
    }
  }
  {
    // block partials, then group partials; a ticket per group after the
    // global one (the force kernel's two-level energy combine)
    const size_t G = (size_t)std::max(c->fblocks, c->ncell * c->cell_split);
    const size_t ngroups = (G + kEnergyGroup - 1) / kEnergyGroup;
    AL(c->fpart, (G + ngroups) * 8);
    AL(c->ticket, ngroups + 4);
    c->ticket_count = ngroups + 4;
  }
  // boxes whose forces run one block per cell, FP64 or mixed above 64^3
  // (mixed boxes up to 64^3 take the split step, and only those run in
  // batches): the pairs once each (Newton's third law) in their own kernel
  // with the gather, then the finish
  if (c->nc >= 3 && c->reach == 1 && c->ncell >= 2 * c->num_sms && !arena && !c->split_step &&
      (!c->mixed || c->N > 64)) {
    AL(c->pair_fix, 4 * (size_t)n);
    AL(c->gath, 4 * (size_t)n);
    // FP64 boxes: the pair arithmetic in double-float on the FP32 pipe, from
    // cell-relative hi + lo positions (MAZE_PAIRS_FP64=1: in FP64 arithmetic)
    const char* pf = getenv("MAZE_PAIRS_FP64");
    if (!c->mixed && !(pf && pf[0] == '1')) {
      c->pair_df = true;
      AL(c->rel_hi, (size_t)n);
      AL(c->rel_lo, (size_t)n);
      AL(c->rel_hi_s, (size_t)n);
      AL(c->rel_lo_s, (size_t)n);
      AL(c->exp2tab_f, 64);
    }
    // the split of each SM: P pair blocks of kForceThreads and one solve
    // block of T threads, T the largest whose registers fit beside them. The
    // register file is split over the SM's 4 sub-partitions, warps are
    // dealt to them in turn, and a warp takes 32 x (registers per thread,
    // rounded up to 8): so per sub-partition ceil(pair warps / 4) pair warps
    // and T / 128 solve warps must fit in a quarter of the file.
    // MAZE_OVERLAP: "0" off, "TxP" (T 0: the largest that fits)
    const char* ov = getenv("MAZE_OVERLAP");
    int ot = 0, op = 1;
    if (ov && sscanf(ov, "%dx%d", &ot, &op) != 2) ot = -1;
    int regs_sm = 0;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const int rp = (pairs_only_regs(c->mixed, c->pair_df) + 7) / 8 * 8;
    const int rs = ((c->mixed ? mixed_grid_regs() : mgfix_regs()) + 7) / 8 * 8;
    const int pair_warps = op * kForceThreads / 32;
    const int per_part = regs_sm / 4 - (pair_warps + 3) / 4 * 32 * rp;
    int tmax = per_part > 0 ? per_part / (32 * rs) * 4 * 32 : 0;
    if (tmax > kMgThreads) tmax = kMgThreads;
    if (ot == 0 || ot > tmax) ot = tmax;
    // (the integer V-cycle on grids of 128^3 and more; the mixed solve in its
    // cooperative grid form, which needs at least 512 threads per block)
    const bool form = (c->fixmg && mg_threads((int)ng) == kMgThreads) ||
                      (c->mixed && c->mx_cluster == 0 && c->N >= 128 && ot >= 512);
    if (form && ot >= 256 && ot % 32 == 0 && op >= 1 && op <= 3) {
      int smem_sm = 0;
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      c->overlap = true;
      c->ov_threads = ot;
      c->ov_blocks = c->num_sms;               // one solve block per SM
      c->ov_pair_blocks = op * c->num_sms;
      c->ov_pair_smem = smem_sm / (op + 1) + 1024;   // no more than op pair blocks fit on an SM
      if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return fail(MAZE_ERR_CUDA, "cudaStreamCreate / cudaEventCreate failed");
      }
    }
  }
  if (c->split_step) {
    AL(c->pair_out, 4 * (size_t)n);
    if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      free_ctx(c);
      return fail(MAZE_ERR_CUDA, "cudaStreamCreate / cudaEventCreate failed");
    }
  }
  AL(c->rec, 1);
  AL(c->gate, 1);
#undef AL
  *out = c;
  return MAZE_OK;
}

// Full creation: setup, pinned stats buffer, upload, step 0 (spread, solve
// from zero, phi^{-1} = phi^0, y = 0, forces F^0 and energies).
maze_status ctx_create(const maze_config* cfg, Arena* arena, maze_ctx** out, bool defer_status) {
  if (!out) return fail(MAZE_ERR_INVALID, "out is NULL");
  maze_ctx* c = nullptr;
  maze_status s = ctx_setup(cfg, arena, &c);
  if (s != MAZE_OK) return s;
  const int n = c->n;
  const size_t ng = c->ng;
  const std::vector<double>& gk = c->gk;
  std::vector<float> gkf;
  if (c->mixed) {
    // M e^{i k.p} = lambda(k) e^{i k.p}, lambda = 2 (cos kx + cos ky + cos kz) - 6
    // (k in units of 2 pi / N_c): the zero-mean inverse multiplies the
    // transform by 1 / lambda (0 at k = 0); the 1 / N_c^3 of the inverse
    // transform is folded in
    const int Nc = c->mg.Nl[c->mg.L - 1], nc3 = Nc * Nc * Nc;
    gkf.assign((size_t)nc3 + 2 * Nc, 0.f);
    std::vector<double> cs(Nc);
    for (int t = 0; t < Nc; ++t) cs[t] = cos(2.0 * kPi * t / Nc);
    for (int kz = 0; kz < Nc; ++kz)
      for (int ky = 0; ky < Nc; ++ky)
        for (int kx = 0; kx < Nc; ++kx) {
          if (!kx && !ky && !kz) continue;
          const double lam = 2.0 * (cs[kx] + cs[ky] + cs[kz]) - 6.0;
          gkf[kx + Nc * (ky + Nc * kz)] = (float)(1.0 / (lam * nc3));
        }
    for (int t = 0; t < Nc; ++t) {
      gkf[nc3 + t] = (float)cs[t];
      gkf[nc3 + Nc + t] = (float)sin(2.0 * kPi * t / Nc);
    }
  }
  if (cudaMallocHost(&c->rec_host, sizeof(maze_stats)) != cudaSuccess) {
    free_ctx(c);
    return fail(MAZE_ERR_OOM, "cudaMallocHost failed");
  }
  // upload (AoS host -> SoA device)
  std::vector<double> tmp(3 * (size_t)n);
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < n; ++i) tmp[(size_t)d * n + i] = wrap_host(cfg->pos[3 * i + d], c->L);
  cudaStream_t st = c->stream;
#define CKC(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      free_ctx(c);                                                         \
      return fail(MAZE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                      \
  } while (0)
  CKC(cudaMemcpyAsync(c->pos, tmp.data(), tmp.size() * 8, cudaMemcpyHostToDevice, st));
  CKC(cudaStreamSynchronize(st));
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < n; ++i) tmp[(size_t)d * n + i] = cfg->vel[3 * i + d];
  CKC(cudaMemcpyAsync(c->vel, tmp.data(), tmp.size() * 8, cudaMemcpyHostToDevice, st));
  CKC(cudaMemcpyAsync(c->type, cfg->type, (size_t)n * 4, cudaMemcpyHostToDevice, st));
  if (!gk.empty() && c->mg_g) CKC(cudaMemcpyAsync(c->mg_g, gk.data(), gk.size() * 8, cudaMemcpyHostToDevice, st));
  std::vector<double> e2(64);
  exp2_table(e2.data());
  CKC(cudaMemcpyAsync(c->exp2tab, e2.data(), 64 * 8, cudaMemcpyHostToDevice, st));
  std::vector<float2> e2f(64);
  for (int j = 0; j < 64; ++j) e2f[j] = make_float2((float)e2[j], (float)(e2[j] - (double)(float)e2[j]));
  if (c->exp2tab_f) CKC(cudaMemcpyAsync(c->exp2tab_f, e2f.data(), 64 * sizeof(float2), cudaMemcpyHostToDevice, st));
  if (!gkf.empty()) CKC(cudaMemcpyAsync(c->mx_g, gkf.data(), gkf.size() * 4, cudaMemcpyHostToDevice, st));
  CKC(cudaMemsetAsync(c->force, 0, 3 * (size_t)n * 8, st));
  CKC(cudaMemsetAsync(c->force_el, 0, 3 * (size_t)n * 8, st));
  if (c->pair_fix) CKC(cudaMemsetAsync(c->pair_fix, 0, 4 * (size_t)n * 8, st));
  CKC(cudaMemsetAsync(c->qfix, 0, ng * 8, st));
  CKC(cudaMemsetAsync(c->y, 0, ng * 8, st));
  CKC(cudaMemsetAsync(c->phi[0], 0, ng * 8, st));
  CKC(cudaMemsetAsync(c->phi[1], 0, ng * 8, st));
  CKC(cudaMemsetAsync(c->phi[2], 0, ng * 8, st));
  CKC(cudaMemsetAsync(c->rec, 0, sizeof(maze_stats), st));
  CKC(cudaMemsetAsync(c->ticket, 0, c->ticket_count * sizeof(unsigned), st));
  CKC(cudaMemsetAsync(c->gate, 0, 4, st));
  if (c->nc >= 3) CKC(cudaMemsetAsync(c->cell_count, 0, (size_t)c->ncell * 4, st));
  CKC(cudaStreamSynchronize(st));
#undef CKC
  // step 0: spread, solve M y = q from zero, phi^0 = -(4pi/h)(y - mean y),
  // phi^{-1} = phi^0, y = 0, forces F^0 and energies
  c->ik = 1;  // solve writes phi[(ik+2)%3] = phi[0]
  s = MAZE_OK;
  auto run = [&]() -> maze_status {
    CK(launch_ion_update(ion_args(c, 0, 1), st));
    maze_status r = enqueue_cells(c);
    if (r != MAZE_OK) return r;
    r = enqueue_solve(c, 1, c->qd);
    if (r != MAZE_OK) return r;
    c->ik = 0;
    CK(cudaMemcpyAsync(c->phi[1], c->phi[0], ng * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(c->y, 0, ng * 8, st));
    r = enqueue_forces(c, force_args(c, c->phi[0], 0, 0), st);
    if (r != MAZE_OK) return r;
    if (defer_status) return MAZE_OK;
    r = read_stats(c);
    if (r != MAZE_OK) return r;
    return status_message(c);
  };
  s = run();
  if (s != MAZE_OK) {
    std::string keep = g_err;
    free_ctx(c);
    g_err = keep;
    return s;
  }
  *out = c;
  return MAZE_OK;
}

maze_status ctx_bytes(const maze_config* cfg, size_t* bytes) {
  if (!bytes) return fail(MAZE_ERR_INVALID, "bytes is NULL");
  Arena counter(nullptr, (size_t)1 << 62);
  maze_ctx* c = nullptr;
  maze_status s = ctx_setup(cfg, &counter, &c);
  if (s != MAZE_OK) return s;
  *bytes = counter.used();
  free_ctx(c);
  return MAZE_OK;
}

// The exchange graphs of maze_step_io (one per rotation): the step's status
// cleared, positions and velocities uploaded from their pinned stages, one
// step, positions, velocities and the record read back into pinned memory:
// the operations maze_set, maze_step and maze_get issue, in their order, on
// the same stream. On any capture failure the calls keep their separate form.
maze_status build_io_graphs(maze_ctx* c) {
  c->io_tried = true;
  const size_t n6 = 6 * (size_t)c->n;
  if (cudaMallocHost(&c->io_stage, 2 * n6 * sizeof(double)) != cudaSuccess) {
    c->io_stage = nullptr;
    cudaGetLastError();
    return MAZE_OK;   // (no exchange stage: the separate form)
  }
  static_assert(sizeof(maze_stats) % 8 == 0, "the record moves as 8-byte words");
  void *st = nullptr, *rec_out = nullptr;
  if (cudaHostGetDevicePointer(&st, c->io_stage, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(&rec_out, c->rec_host, 0) != cudaSuccess) {
    cudaGetLastError();
    return MAZE_OK;   // (no device addresses: the separate form)
  }
  c->io_stage_dev = static_cast<const double*>(st);
  if (cudaMallocHost(&c->io_desc_host, sizeof(IoDesc)) != cudaSuccess ||
      cudaMalloc(&c->io_desc, sizeof(IoDesc)) != cudaSuccess) {
    cudaGetLastError();
    return MAZE_OK;
  }
  // read by the captured step's S1, and only there: cleared on every way out
  c->io_capture = true;
  struct Clear {
    maze_ctx* c;
    ~Clear() { c->io_capture = false; }
  } clear{c};
  const int ik0 = c->ik;
  for (int g = 0; g < 3; ++g) {
    c->ik = g;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c->ik = ik0;
      return MAZE_OK;
    }
    // the pinned stages and record are read and written by the SMs
    // directly (device addresses of the host allocations)
    // (this exchange's buffer addresses, written by the host before each launch)
    bool ok = cudaMemcpyAsync(c->io_desc, c->io_desc_host, sizeof(IoDesc), cudaMemcpyHostToDevice, c->stream) ==
              cudaSuccess;
    ok = ok && cudaMemsetAsync(&c->rec->status, 0, sizeof(int32_t), c->stream) == cudaSuccess;
    ok = ok && enqueue_step(c, 0) == MAZE_OK;
    ok = ok && launch_io_out(c->pos, c->io_desc, c->n, c->rec, rec_out, sizeof(maze_stats), c->stream) ==
                   cudaSuccess;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (!ok || e != cudaSuccess || !graph ||
        cudaGraphInstantiate(&c->io_graph[g], graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      for (int q = 0; q < 3; ++q)
        if (c->io_graph[q]) {
          cudaGraphExecDestroy(c->io_graph[q]);
          c->io_graph[q] = nullptr;
        }
      c->ik = ik0;
      return MAZE_OK;
    }
    cudaGraphDestroy(graph);
  }
  c->ik = ik0;
  c->io_ok = true;
  return MAZE_OK;
}

// maze_step_io of one step with every input and output, through the
// exchange graph.
maze_status step_io_graph(maze_ctx* c, const double* pos_in, const double* vel_in, double* pos_out,
                          double* vel_out, maze_stats* stats_out) {
  if (c->rec_dirty) {   // (the step count before the step, as maze_step keeps it)
    maze_status s = read_stats(c);
    if (s != MAZE_OK) return s;
  }
  const int64_t before = c->rec_host->step;
  const int ik0 = c->ik;
  // Pinned caller arrays are read and written by the device directly (their
  // device addresses go to the graph through the descriptor); other arrays
  // pass through the context's pinned stage. Either way the inputs are
  // checked on the host first (a non-finite value: nothing runs), and S1
  // wraps the positions into [0, L) as maze_set does.
  const size_t n3 = 3 * (size_t)c->n;
  double* in = c->io_stage;
  const double* out = c->io_stage + 2 * n3;
  auto pinned = [](const void* p) -> void* {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
  };
  const void* dpi = pinned(pos_in);
  const void* dvi = pinned(vel_in);
  void* dpo = pinned(pos_out);
  void* dvo = pinned(vel_out);
  const bool direct_in = dpi && dvi, direct_out = dpo && dvo;
  std::atomic<bool> bad{false};
  if (direct_in) {
    host_ranges(c->n, [&](int lo, int hi) {
      bool b = false;
      for (size_t e = 3 * (size_t)lo; e < 3 * (size_t)hi; ++e) b |= !isfinite(pos_in[e]) || !isfinite(vel_in[e]);
      if (b) bad.store(true, std::memory_order_relaxed);
    });
  } else {
    const double L = c->L;
    host_ranges(c->n, [&, in, L](int lo, int hi) {
      bool b = false;
      for (size_t e = 3 * (size_t)lo; e < 3 * (size_t)hi; ++e) {
        const double x = pos_in[e], v = vel_in[e];
        b |= !isfinite(x) || !isfinite(v);
        in[e] = wrap_host(x, L);
        in[n3 + e] = v;
      }
      if (b) bad.store(true, std::memory_order_relaxed);
    });
  }
  if (bad.load()) return fail(MAZE_ERR_INVALID, "non-finite input");   // (nothing uploaded or run)
  IoDesc& d = *c->io_desc_host;
  d.pos_in = direct_in ? static_cast<const double*>(dpi) : c->io_stage_dev;
  d.vel_in = direct_in ? static_cast<const double*>(dvi) : c->io_stage_dev + n3;
  d.pos_out = direct_out ? static_cast<double*>(dpo) : const_cast<double*>(c->io_stage_dev) + 2 * n3;
  d.vel_out = direct_out ? static_cast<double*>(dvo) : const_cast<double*>(c->io_stage_dev) + 3 * n3;
  c->rec_dirty = true;
  c->staged_fresh[0] = c->staged_fresh[1] = false;
  c->want_ion[0] = c->want_ion[1] = false;
  CK(cudaGraphLaunch(c->io_graph[c->ik], c->stream));
  rotate(c, 1);
  CK(cudaStreamSynchronize(c->stream));
  c->rec_dirty = false;
  if (c->rec_host->status != MAZE_OK) {
    // the step was skipped on the device: the rotation stays where it was
    const int64_t done = c->rec_host->step - before;
    c->ik = (int)((ik0 + 2 * (done % 3)) % 3);
  }
  if (!direct_out)
    host_ranges(c->n, [=](int lo, int hi) {
      memcpy(pos_out + 3 * (size_t)lo, out + 3 * (size_t)lo, 3 * (size_t)(hi - lo) * sizeof(double));
      memcpy(vel_out + 3 * (size_t)lo, out + n3 + 3 * (size_t)lo, 3 * (size_t)(hi - lo) * sizeof(double));
    });
  if (stats_out) *stats_out = *c->rec_host;
  return status_message(c);
}

}  // namespace maze

extern "C" {

maze_status maze_create(const maze_config* cfg, maze_ctx** out) {
  maze::TraceRange tr("maze_create");
  return ctx_create(cfg, nullptr, out);
}


void maze_destroy(maze_ctx* ctx) { free_ctx(ctx); }

maze_status maze_spread(maze_ctx* c) {
  maze::TraceRange tr("maze_spread");
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  maze_status s = clear_status(c);
  if (s != MAZE_OK) return s;
  CK(cudaMemsetAsync(c->qfix, 0, c->ng * 8, c->stream));
  CK(launch_ion_update(ion_args(c, 0, 1), c->stream));
  s = enqueue_cells(c);
  if (s != MAZE_OK) return s;
  CK(launch_q_to_double(c->qfix, c->qd, (int)c->ng, c->stream));
  return MAZE_OK;
}

maze_status maze_solve(maze_ctx* c, int32_t* iters, double* resid) {
  maze::TraceRange tr("maze_solve");
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  maze_status s = clear_status(c);
  if (s != MAZE_OK) return s;
  s = enqueue_solve(c, 0, c->qd);
  if (s != MAZE_OK) return s;
  rotate(c, 1);
  s = read_stats(c);
  if (s != MAZE_OK) return s;
  if (iters) *iters = c->rec_host->iters;
  if (resid) *resid = c->rec_host->resid;
  return status_message(c);
}

maze_status maze_gather(maze_ctx* c) {
  maze::TraceRange tr("maze_gather");
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  maze_status s = clear_status(c);
  if (s != MAZE_OK) return s;
  CK(launch_ion_update(ion_args(c, 0, 0), c->stream));
  s = enqueue_cells(c);
  if (s != MAZE_OK) return s;
  s = enqueue_forces(c, force_args(c, c->phi[c->ik], 0, 0), c->stream);
  if (s != MAZE_OK) return s;
  s = read_stats(c);
  if (s != MAZE_OK) return s;
  return status_message(c);
}

maze_status maze_step_async(maze_ctx* c, int32_t nsteps) {
  maze::TraceRange tr("maze_step_async");
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  if (nsteps < 0) return fail(MAZE_ERR_INVALID, "nsteps must be >= 0");
  c->rec_dirty = true;
  c->staged_fresh[0] = c->staged_fresh[1] = false;
  const int t = c->timing;
  if (!c->graphs_tried[t]) {
    maze_status s = build_graphs(c, t);
    if (s != MAZE_OK) return s;
  }
  for (int k = 0; k < nsteps; ++k) {
    if (c->graphs_ok[t]) {
      CK(cudaGraphLaunch(c->graph[t][c->ik], c->stream));
    } else {
      maze_status s = enqueue_step(c, t);
      if (s != MAZE_OK) return s;
    }
    rotate(c, 1);
  }
  return MAZE_OK;
}

maze_status maze_step(maze_ctx* c, int32_t nsteps) {
  maze::TraceRange tr("maze_step");
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  maze_status s = MAZE_OK;
  if (c->rec_dirty) {   // (the record a synchronising call left is current)
    s = read_stats(c);
    if (s != MAZE_OK) return s;
  }
  const int64_t before = c->rec_host->step;
  s = clear_status(c);
  if (s != MAZE_OK) return s;
  const int ik0 = c->ik;
  s = maze_step_async(c, nsteps);
  if (s != MAZE_OK) return s;
  // positions and velocities were read back after the previous step: queue
  // their copies now, so that the record read below waits for all at once
  bool queued[2] = {false, false};
  if (!c->arena && (c->want_ion[0] || c->want_ion[1]) && stage_buffer(c, 2) == MAZE_OK) {
    const size_t n3 = 3 * (size_t)c->n;
    if (c->want_ion[0] && c->want_ion[1]) {
      CK(cudaMemcpyAsync(c->stage[2], c->pos, 2 * n3 * 8, cudaMemcpyDeviceToHost, c->stream));
    } else {
      const int k = c->want_ion[0] ? 0 : 1;
      CK(cudaMemcpyAsync(c->stage[2 + k], k == 0 ? c->pos : c->vel, n3 * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    for (int k = 0; k < 2; ++k) {
      queued[k] = c->want_ion[k];
      c->want_ion[k] = false;
    }
  }
  s = read_stats(c);
  if (s != MAZE_OK) return s;
  c->staged_fresh[0] = queued[0];
  c->staged_fresh[1] = queued[1];
  if (s != MAZE_OK) return s;
  if (c->rec_host->status != MAZE_OK) {
    // later steps were skipped on the device: put the rotation where the
    // last completed step left it
    const int64_t done = c->rec_host->step - before;
    c->ik = (int)((ik0 + 2 * (done % 3)) % 3);
  }
  return status_message(c);
}

maze_status maze_set_timing(maze_ctx* c, int32_t on) {
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  if (on && !c->ev[0])
    for (int k = 0; k < 5; ++k) CK(cudaEventCreate(&c->ev[k]));
  c->timing = on ? 1 : 0;
  return MAZE_OK;
}

maze_status maze_get_timing(maze_ctx* c, double* out) {
  if (!c || !out) return fail(MAZE_ERR_INVALID, "NULL argument");
  if (!c->timing) return fail(MAZE_ERR_INVALID, "timing is off (maze_set_timing)");
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 4; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
    out[k] = ms;
  }
  return MAZE_OK;
}

maze_status maze_get_stats(maze_ctx* c, maze_stats* out) {
  if (!c || !out) return fail(MAZE_ERR_INVALID, "NULL argument");
  // a standalone context's record changes only through the calls that mark
  // it dirty, so a current copy is returned as is; a batch box's record is
  // written by the batch's launches and always read
  if (c->arena || c->rec_dirty) {
    maze_status s = read_stats(c);
    if (s != MAZE_OK) return s;
  }
  *out = *c->rec_host;
  return MAZE_OK;
}

maze_status maze_get(maze_ctx* c, int32_t what, double* out) {
  if (!c || !out) return fail(MAZE_ERR_INVALID, "NULL argument");
  const double* src = nullptr;
  bool ion = false;
  switch (what) {
    case MAZE_POS: src = c->pos; ion = true; break;
    case MAZE_VEL: src = c->vel; ion = true; break;
    case MAZE_FORCE: src = c->force; ion = true; break;
    case MAZE_FORCE_EL: src = c->force_el; ion = true; break;
    case MAZE_PHI: src = c->phi[c->ik]; break;
    case MAZE_PHI_PREV: src = c->phi[(c->ik + 1) % 3]; break;
    case MAZE_Y: src = c->y; break;
    case MAZE_CHARGE: src = c->qd; break;
    case MAZE_SIGMA: src = c->sigma; break;
    default: return fail(MAZE_ERR_INVALID, "unknown quantity");
  }
  if (ion) {
    // a standalone context reads through its pinned stage; a batch box (its
    // buffers in the batch's arena) through a temporary, so that admitting
    // and retiring boxes allocates no pinned memory
    const int n = c->n;
    std::vector<double> tmpv;
    double* tmp = nullptr;
    const int kk = what == MAZE_POS ? 0 : (what == MAZE_VEL ? 1 : -1);
    if (c->arena) {
      tmpv.resize(3 * (size_t)n);
      tmp = tmpv.data();
    } else {
      const int sk = kk == 0 ? 2 : 3;
      maze_status st = stage_buffer(c, sk);
      if (st != MAZE_OK) return st;
      tmp = c->stage[sk];
      if (kk >= 0)
        c->want_ion[kk] = true;
      else
        c->staged_fresh[1] = false;   // the forces go through the velocities' stage
    }
    if (kk >= 0 && !c->arena && c->staged_fresh[kk]) {
      // copied by the last maze_step together with its record read
    } else {
      CK(cudaMemcpyAsync(tmp, src, 3 * (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    to_aos(tmp, out, n);
  } else {
    CK(cudaMemcpyAsync(out, src, c->ng * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->mixed && what != MAZE_CHARGE) {
      // double-float pairs (hi, lo) -> hi + lo
      for (size_t i = 0; i < c->ng; ++i) {
        float2 v;
        memcpy(&v, &out[i], 8);
        out[i] = (double)v.x + (double)v.y;
      }
    }
  }
  return MAZE_OK;
}

maze_status maze_set(maze_ctx* c, int32_t what, const double* in) {
  if (!c || !in) return fail(MAZE_ERR_INVALID, "NULL argument");
  double* dst = nullptr;
  bool ion = false;
  switch (what) {
    case MAZE_POS: dst = c->pos; ion = true; break;
    case MAZE_VEL: dst = c->vel; ion = true; break;
    case MAZE_PHI: dst = c->phi[c->ik]; break;
    case MAZE_PHI_PREV: dst = c->phi[(c->ik + 1) % 3]; break;
    case MAZE_Y: dst = c->y; break;
    default: return fail(MAZE_ERR_INVALID, "quantity cannot be set");
  }
  if (ion) {
    if (!ion_finite(c, in)) return fail(MAZE_ERR_INVALID, "non-finite input");
    const double* const ins[2] = {what == MAZE_POS ? in : nullptr, what == MAZE_VEL ? in : nullptr};
    return upload_ions(c, ins);
  } else if (c->mixed) {
    // double -> double-float pair (hi = nearest float, lo = remainder)
    std::vector<float2> tmp(c->ng);
    for (size_t i = 0; i < c->ng; ++i) {
      const float hi = (float)in[i];
      tmp[i] = make_float2(hi, (float)(in[i] - (double)hi));
    }
    CK(cudaMemcpyAsync(dst, tmp.data(), c->ng * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    CK(cudaMemcpyAsync(dst, in, c->ng * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return MAZE_OK;
}

maze_status maze_step_io(maze_ctx* c, const double* pos_in, const double* vel_in, int32_t nsteps, double* pos_out,
                         double* vel_out, maze_stats* stats_out) {
  maze::TraceRange tr("maze_step_io");
  if (!c) return fail(MAZE_ERR_INVALID, "ctx is NULL");
  if (nsteps < 0) return fail(MAZE_ERR_INVALID, "nsteps must be >= 0");
  maze_status s;
  // the full exchange of one step: one graph launch and one synchronisation
  // (its staging pass checks the inputs before anything runs)
  if (!c->arena && nsteps == 1 && pos_in && vel_in && pos_out && vel_out && !c->timing) {
    if (!c->io_tried) {
      s = build_io_graphs(c);
      if (s != MAZE_OK) return s;
    }
    if (c->io_ok) return step_io_graph(c, pos_in, vel_in, pos_out, vel_out, stats_out);
  }
  // both inputs are checked before anything is uploaded or run
  if ((pos_in && !ion_finite(c, pos_in)) || (vel_in && !ion_finite(c, vel_in)))
    return fail(MAZE_ERR_INVALID, "non-finite input");
  if (pos_in || vel_in) {
    const double* const ins[2] = {pos_in, vel_in};
    if ((s = upload_ions(c, ins)) != MAZE_OK) return s;
  }
  // maze_step queues the copies of the wanted quantities together with its
  // record read (one synchronisation)
  if (!c->arena) {
    c->want_ion[0] = pos_out != nullptr;
    c->want_ion[1] = vel_out != nullptr;
  }
  s = maze_step(c, nsteps);
  if (c->rec_dirty) return s;   // the step did not reach its record read: no outputs
  double* outs[2] = {pos_out, vel_out};
  for (int k = 0; k < 2; ++k) {
    if (!outs[k]) continue;
    if (!c->arena && c->staged_fresh[k]) {
      to_aos(c->stage[2 + k], outs[k], c->n);
    } else {
      const maze_status g = maze_get(c, k == 0 ? MAZE_POS : MAZE_VEL, outs[k]);
      if (g != MAZE_OK) return g;
    }
  }
  if (stats_out) *stats_out = *c->rec_host;
  if (s != MAZE_OK) return status_message(c);   // (the step's message again, after maze_get)
  return MAZE_OK;
}

// Blob layout: header (magic, n, N, step, total_iters) + V_work, then
// pos, vel, force, force_el ([3][n] each), phi^k, phi^{k-1}, y ([N^3] each).
maze_status maze_get_state(maze_ctx* c, void* blob, size_t* nbytes) {
  if (!c || !nbytes) return fail(MAZE_ERR_INVALID, "NULL argument");
  const size_t ion = 3 * (size_t)c->n * 8, grid = c->ng * 8;
  const size_t need = 6 * 8 + 4 * ion + 3 * grid;
  if (!blob) {
    *nbytes = need;
    return MAZE_OK;
  }
  if (*nbytes < need) return fail(MAZE_ERR_INVALID, "blob too small");
  maze_status s = read_stats(c);
  if (s != MAZE_OK) return s;
  char* b = static_cast<char*>(blob);
  uint64_t hdr[5] = {kBlobMagic, (uint64_t)c->n, (uint64_t)c->N, (uint64_t)c->rec_host->step,
                     (uint64_t)c->rec_host->total_iters};
  memcpy(b, hdr, sizeof hdr);
  memcpy(b + 40, &c->rec_host->v_work, 8);
  char* q = b + 48;
  const double* ions[4] = {c->pos, c->vel, c->force, c->force_el};
  for (int k = 0; k < 4; ++k, q += ion) CK(cudaMemcpyAsync(q, ions[k], ion, cudaMemcpyDeviceToHost, c->stream));
  const double* grids[3] = {c->phi[c->ik], c->phi[(c->ik + 1) % 3], c->y};
  for (int k = 0; k < 3; ++k, q += grid) CK(cudaMemcpyAsync(q, grids[k], grid, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *nbytes = need;
  return MAZE_OK;
}

maze_status maze_set_state(maze_ctx* c, const void* blob, size_t nbytes) {
  if (!c || !blob) return fail(MAZE_ERR_INVALID, "NULL argument");
  const size_t ion = 3 * (size_t)c->n * 8, grid = c->ng * 8;
  const size_t need = 6 * 8 + 4 * ion + 3 * grid;
  if (nbytes != need) return fail(MAZE_ERR_INVALID, "blob size does not match this context");
  const char* b = static_cast<const char*>(blob);
  uint64_t hdr[5];
  memcpy(hdr, b, sizeof hdr);
  if (hdr[0] != kBlobMagic || hdr[1] != (uint64_t)c->n || hdr[2] != (uint64_t)c->N)
    return fail(MAZE_ERR_INVALID, "blob does not belong to a context of this shape");
  double vw;
  memcpy(&vw, b + 40, 8);
  c->ik = 0;
  const char* q = b + 48;
  double* ions[4] = {c->pos, c->vel, c->force, c->force_el};
  for (int k = 0; k < 4; ++k, q += ion) CK(cudaMemcpyAsync(ions[k], q, ion, cudaMemcpyHostToDevice, c->stream));
  double* grids[3] = {c->phi[0], c->phi[1], c->y};
  for (int k = 0; k < 3; ++k, q += grid) CK(cudaMemcpyAsync(grids[k], q, grid, cudaMemcpyHostToDevice, c->stream));
  maze_status s = read_stats(c);
  if (s != MAZE_OK) return s;
  maze_stats st = *c->rec_host;
  st.step = (int64_t)hdr[3];
  st.total_iters = (int64_t)hdr[4];
  st.v_work = vw;
  st.status = MAZE_OK;
  *c->rec_host = st;
  c->rec_dirty = true;
  c->staged_fresh[0] = c->staged_fresh[1] = false;
  CK(cudaMemcpyAsync(c->rec, c->rec_host, sizeof(maze_stats), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return MAZE_OK;
}

}  // extern "C"
