// Host-side state of one MaZe simulation (a context) and the internal host
// functions that the single-box entry points (maze_api.cu) and the batched
// engine (maze_batch.cu) share. Not part of the public C ABI.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "maze_internal.cuh"

namespace maze {

constexpr double kPi = 3.14159265358979323846;

// First-fit sub-allocator over one device allocation (256-byte aligned
// blocks, neighbouring free blocks merged on release). A counting arena
// (base == nullptr) hands out fake addresses and only measures.
class Arena {
 public:
  Arena(char* base, size_t capacity);
  void* alloc(size_t bytes);          // nullptr when no free block is large enough
  void release(void* p);
  size_t used() const { return used_bytes_; }
  size_t capacity() const { return cap_; }
  size_t largest_free() const;
  size_t high_water() const;          // end of the highest block in use
  bool counting() const { return counting_; }
  char* base() const { return base_; }

 private:
  char* base_;
  size_t cap_;
  bool counting_;
  size_t used_bytes_ = 0;
  std::map<size_t, size_t> free_;     // offset -> size
  std::map<size_t, size_t> taken_;    // offset -> size
};

}  // namespace maze

struct maze_ctx {
  maze_config cfg;
  int n = 0, N = 0, P = 4;
  size_t ng = 0;
  double L = 0, h = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // ions, SoA [3][n]
  double *pos = nullptr, *vel = nullptr, *force = nullptr, *force_el = nullptr;
  int* type = nullptr;
  float4* pos32 = nullptr;
  double* wbuf = nullptr;   // [n][3][4] B-spline weights of the current positions
  float* wbuf32 = nullptr;  // FP32 weights (mixed precision)
  double* wdbuf = nullptr;  // weight derivatives (force estimator of Eq. F_Benoit)
  float* wdbuf32 = nullptr;
  int4* wbase = nullptr;
  // grid
  unsigned long long* qfix = nullptr;
  double* qd = nullptr;
  double* phi[3] = {nullptr, nullptr, nullptr};
  int ik = 0;  // phi^k is phi[ik], phi^{k-1} phi[(ik+1)%3], scratch phi[(ik+2)%3]
  double *sigma = nullptr, *y = nullptr, *r = nullptr, *p = nullptr, *p1 = nullptr, *Mp = nullptr;
  double* y2 = nullptr;   // second y buffer (mixed precision, cluster-resident solve)
  maze::LLRec* recs = nullptr;
  size_t recs_bytes = 0;
  unsigned* bar = nullptr;
  // multigrid
  maze::MgArgs mg = {};
  double *mg_x = nullptr, *mg_b = nullptr, *mg_r = nullptr, *mg_g = nullptr;
  double* exp2tab = nullptr;   // [64] 2^(j/64), the pair forces' exponential
  float2* exp2tab_f = nullptr;  // [64] the same as (hi, lo) floats (double-float pairs)
  bool pair_df = false;         // FP64 once-per-pair kernel with double-float pair arithmetic
  // mixed precision: phi, y, sigma hold double-float pairs (float2, 8 B)
  bool mixed = false;
  bool fixmg = false;     // MAZE_FP64_FIXMG: the integer defect-correction V-cycle
  maze::MixedArgs mx = {};
  int mx_cluster = 0, mx_blocks = 0;
  bool fused_step = false;   // S1-S6 in one cluster launch (k_cluster_step)
  bool split_step = false;   // S8 beside the one-cluster solve (k_pairs_cells, k_gather_finish)
  float *mx_scratch = nullptr, *mx_g = nullptr;
  int sblocks = 0;
  // cells
  int nc = 0, ncell = 0, cell_split = 1, reach = 1;
  int *cell_of = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cursor = nullptr, *cell_ions = nullptr;
  float4* pos_sorted = nullptr;
  float4 *rel_hi = nullptr, *rel_lo = nullptr, *rel_hi_s = nullptr, *rel_lo_s = nullptr;
  // force reductions
  double* fpart = nullptr;
  unsigned* ticket = nullptr;
  size_t ticket_count = 0;
  int fblocks = 0;
  int num_sms = 0;
  maze_stats* rec = nullptr;       // device
  int* gate = nullptr;             // device: current step skipped
  maze_stats* rec_host = nullptr;  // pinned
  bool rec_dirty = true;           // device record may differ from rec_host
  // the split single-box step (mixed, one cluster): S8 on side_stream beside
  // the solve, joined before S7/S9
  double* pair_out = nullptr;
  long long* pair_fix = nullptr;   // FP64 large boxes: per-ion pair sums of the once-per-pair kernel
  double* gath = nullptr;          // ... and their gather sums
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // FP64 state with the integer V-cycle on a box with once-per-pair forces:
  // the pairs (k_pairs_only, ov_pair_blocks blocks padded to ov_pair_smem
  // bytes of shared memory) run on side_stream beside the solve (ov_blocks x
  // ov_threads), then S7 and S9; MAZE_OVERLAP=0 turns it off
  bool overlap = false;
  int ov_threads = 0, ov_blocks = 0, ov_pair_blocks = 0, ov_pair_smem = 0;
  // pinned staging of the per-ion host copies (standalone contexts, made on
  // first use): [0] maze_set of positions, [1] of velocities, [2] maze_get of
  // positions, [3] of velocities (and of the forces); an uploaded stage is
  // reused only after its copy's event
  double* stage[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  // positions / velocities read back after the last step: maze_step then
  // queues their copies with its record read (staged_fresh: the stage holds
  // the device values, nothing has been issued since)
  bool want_ion[2] = {false, false};
  bool staged_fresh[2] = {false, false};
  cudaGraphExec_t graph[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  bool graphs_tried[2] = {false, false}, graphs_ok[2] = {false, false};
  // one host exchange of maze_step_io (status clear, upload of positions and
  // velocities, one step, their read-back and the record's) per rotation
  cudaGraphExec_t io_graph[3] = {nullptr, nullptr, nullptr};
  bool io_tried = false, io_ok = false;
  double* io_stage = nullptr;   // pinned [2][2][n][3]: positions, velocities in; then out
  const double* io_stage_dev = nullptr;   // its device address
  maze::IoDesc* io_desc_host = nullptr;   // pinned: this exchange's buffers (device addresses)
  maze::IoDesc* io_desc = nullptr;        // device copy, filled by the graph's first node
  bool io_capture = false;                // S1 reads the exchange's inputs (while the graphs are captured)
  int timing = 0;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int max_iter_init = 20000;
  std::vector<void*> allocs;
  maze::Arena* arena = nullptr;   // device buffers come from this arena (batched boxes), else cudaMalloc
  std::vector<double> gk;         // coarsest-level kernel (host copy for the upload)
};


namespace maze {

maze_status fail(maze_status s, const std::string& msg);
maze_status validate(const maze_config* c);
IonArgs ion_args(maze_ctx* c, int do_move, int do_spread);
CellArgs cell_args(maze_ctx* c);
ForceArgs force_args(maze_ctx* c, const double* phi, int do_kick, int count_step);
MixedArgs mixed_args(maze_ctx* c, int zero_phi, double* q_out);
maze_status read_stats(maze_ctx* c);
maze_status status_message(maze_ctx* c);
void free_ctx(maze_ctx* c);
// Validates cfg, allocates every buffer (from ``arena`` when given), uploads
// the state and runs step 0 on ``stream`` (the config's stream when null).
// Builds a context and runs step 0. With defer_status the call returns once
// step 0 is queued on the context's stream, without waiting for it: a failure
// of step 0 then shows only in the device record (the batch's admission).
maze_status ctx_create(const maze_config* cfg, Arena* arena, maze_ctx** out, bool defer_status = false);
// Device bytes a context of this configuration takes from an arena.
maze_status ctx_bytes(const maze_config* cfg, size_t* bytes);

}  // namespace maze
