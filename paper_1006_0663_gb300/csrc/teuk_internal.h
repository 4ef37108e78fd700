// Internal state of a teuk handle, shared by the C ABI layer and the per-precision units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/teuk.h"

struct teuk_s {
  // problem (Sec. 3.A-3.B)
  double M = 1, a = 0;
  int s = 0, m = 0;
  teuk_grid grid{};
  int W = 1;            // words per real
  int rows_per_block = 0;  // step-kernel launch shape: rows of theta per block (0: default)
  int threads_theta = 0;   // threads along theta per row (0: n_theta rounded up to 32, <= 256)
  int kernel_variant = 0;  // register budget of the step kernels: 0 (<= 255), 1 (<= 128), 2 (rows:
                           // <= 102 in blocks of <= 128 threads; warp segments: <= 85)
  double* u2 = nullptr;    // second state buffer of kernel family 4 (boundary rows zero)
  int iteration_launches() const { return kernel_family == 4 && engine == 0 ? 1 : 2; }
  bool in_u2 = false;      // family 4 left the latest iteration in u2 (settled back by teuk_capi.cu)
  int kernel_family = 0;   // 0: rows per block (half_kernel/full_kernel), 1: one warp per 32 columns,
                           // 2: balanced (every resident block the same number of points),
                           // 3: persistent (persist_kernel: outer steps per cooperative launch),
                           // 4: fused iteration (fused_kernel: one launch per iteration, u <-> u2)
  int persist_steps = 1;   // family 3: outer steps per launch
  int* pflags = nullptr;   // family 3: neighbour counters and abort word of the launch
  int pflags_cap = 0;
  int bal_key = -1;        // (variant, threads) the balanced grid sizes below were computed for
  int bal_grid[2] = {0, 0};  // blocks of the balanced half / full kernels (resident capacity)
  int n_r = 0, n_th = 0, pitch = 0, parity = 1, radius = 5, k = 1;  // n_r: rows held (local)
  int row0 = 0;            // global index of local row 0 (r* slab: own_lo - 1 or 0)
  int own_lo = 0, own_hi = -1;  // global rows a slab advances; -1: the whole grid (no slab)
  bool is_slab() const { return own_hi >= 0; }
  double dt_outer = 0;  // leading word of the outer step
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // device buffers
  double* u = nullptr;       // [4][W][n_r][pitch]
  double* uh = nullptr;      // [4][W][n_r-1][pitch]   half-step scratch
  double* cn_raw = nullptr;  // [8][W][n_r][pitch]
  double* ch_raw = nullptr;  // [8][W][n_r-1][pitch]
  double* cn = nullptr;      // folded node tables
  double* ch = nullptr;      // folded half tables
  double* wts = nullptr;     // [2*radius+1][W][n_th]
  double* sin_th = nullptr;  // [W][n_th]
  double* lfac = nullptr;    // [2][W][n_th]: the theta operator's factors A2 and A1 cot(theta_j)
  double* cos_th = nullptr;  // [W][n_th]
  double* x_node = nullptr;  // [W][n_r]
  double* x_half = nullptr;  // [W][n_r-1]
  double* rs_node = nullptr; // [W][n_r]
  double* prof = nullptr;    // [W][n_th]
  unsigned int* status = nullptr;
  // CUDA graph of one outer step (k iterations), replayed by teuk_step
  bool use_graphs = true;
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_record = false;   // whether the captured step records an observer sample
  long long* d_ring_counter = nullptr;  // samples recorded so far (device copy)
  // observer ring
  int i_obs = -1;
  int64_t ring_cap = 0;
  double* ring = nullptr;    // [cap][2][W][n_th]
  int64_t n_recorded = 0;
  // per-kernel event timing (kind 0 = half step, 1 = full step)
  bool timing = false;
  struct EvPair { int kind; cudaEvent_t a, b; };
  std::vector<EvPair> pending;
  std::vector<EvPair> graph_events;  // timing events captured in the outer-step graph
  bool graph_events_fresh = false;   // a replay has recorded them since they were last read
  bool capturing = false;            // the outer-step graph is being captured
  bool time_this = true;             // whether the launches being issued are timed
  std::vector<cudaEvent_t> free_events;
  double ms[2] = {0, 0};
  int64_t n_timed[2] = {0, 0};
  // counters
  int64_t substeps_done = 0;
  int64_t launches = 0;
  // target-precision scalars kept as words
  double h4_w[4] = {0, 0, 0, 0}, h2_w[4] = {0, 0, 0, 0}, ln2_w[4] = {0, 0, 0, 0};
  double dr_d = 0, rsmin_d = 0;
  double dt_w[4] = {0, 0, 0, 0}, dr_w[4] = {0, 0, 0, 0};  // outer dt and dr* as words
  double ko_sigma = 0;                 // r* dissipation strength (0: off, the paper's scheme)
  double ko_eps_w[4] = {0, 0, 0, 0};   // sigma dt / (16 dr*) as words
  double ko_theta = 0;                 // theta dissipation strength (0: off, the paper's scheme)
  double* eps_th = nullptr;            // [W][n_r]: ko_theta c_th(i) dt / (4096 dtheta) per row
  double* u_ko = nullptr;              // output of the dissipation step (state layout)
  int filter_lcut = 0;                 // theta filter: removes multipoles l >= filter_lcut (0: off)
  int filter_period = 1;               // ... at every filter_period-th outer step
  long long* d_filter_ctr = nullptr;   // [2] device: outer steps begun, blocks finished
  double* filt = nullptr;              // its tables [2][n_ell][W][n_th] (analysis, synthesis)
  int filter_n_ell() const { return filter_lcut - std::max(std::abs(s), std::abs(m)); }
  // an operator runs once at the start of every outer step (dissipation or theta filter)
  bool dissipating() const { return ko_sigma > 0 || ko_theta > 0 || filter_lcut > 0; }
  // kernels those operators launch per outer step
  int outer_op_launches() const { return (ko_sigma > 0 || ko_theta > 0 ? 1 : 0) + (filter_lcut > 0 ? 1 : 0); }
  int engine = 0;                      // double-double arithmetic: 0 FP64 error-free transforms,
                                       // 1 integer engine (ix.cuh)
  uint4* ix_m = nullptr;               // integer-engine tables: node coefficients, half-node
  int* ix_e = nullptr;                 // coefficients, stencil weights (mantissas, exponent-sign)
  long long ix_stage_key = -1;         // launch shape the staging choice below was made for
  int ix_stage = 0;                    // integer-engine kernels copy their table rows to shared memory
  int test_stall_block = -1;           // test hook: block that arms its copy barrier without copies
  int wait_log2 = 20;                  // the engine kernels' copy wait gives up after 2^wait_log2 tries
  std::string last_error;
};

namespace teuk {
// per-precision entry points (teuk_prec.cu compiled with TEUK_WORDS = 1, 2, 4)
int setup_w1(teuk_s* h);
int setup_w2(teuk_s* h);
int setup_w4(teuk_s* h);
int pulse_w1(teuk_s* h, double center, double width, double ar, double ai, int ell);
int pulse_w2(teuk_s* h, double center, double width, double ar, double ai, int ell);
int pulse_w4(teuk_s* h, double center, double width, double ar, double ai, int ell);
int advance_counter(teuk_s* h);
int substep_w1(teuk_s* h, bool record, int64_t slot);
int substep_w2(teuk_s* h, bool record, int64_t slot);
int substep_w4(teuk_s* h, bool record, int64_t slot);
int substep_buffers_w1(teuk_s* h, const double* u_in, double* u_out, double* scratch);
int substep_buffers_w2(teuk_s* h, const double* u_in, double* u_out, double* scratch);
int substep_buffers_w4(teuk_s* h, const double* u_in, double* u_out, double* scratch);
int prepare_w1(teuk_s* h);
int prepare_w2(teuk_s* h);
int prepare_w4(teuk_s* h);
int persist_w1(teuk_s* h, int64_t n_outer, long long ring_base);
int persist_w2(teuk_s* h, int64_t n_outer, long long ring_base);
int persist_w4(teuk_s* h, int64_t n_outer, long long ring_base);
// Integer-engine kernels (double-double and quad-double; teuk_ixk.cu): the engine's tables,
// the step's kernel pair of register-budget variant 0..2, and the batched executor.
struct StepArgs;
struct BatchArgs;
struct IxArgs;
int ix_tables_w2(teuk_s* h);
int ix_tables_w4(teuk_s* h);
int ix_launch_pair_w2(teuk_s* h, const StepArgs& sa, dim3 blk, int variant);
int ix_launch_pair_w4(teuk_s* h, const StepArgs& sa, dim3 blk, int variant);
// (shared memory of `rows` engine rows of gstride columns without the staged tables)
size_t ix_row_smem_w2(int rows, int gstride);
size_t ix_row_smem_w4(int rows, int gstride);
cudaError_t batch_ix_occupancy_w2(int* per_sm, size_t smem);
cudaError_t batch_ix_occupancy_w4(int* per_sm, size_t smem);
cudaError_t batch_ix_launch_w2(const BatchArgs& args, const IxArgs* d_ix, int grid, size_t smem, cudaStream_t st);
cudaError_t batch_ix_launch_w4(const BatchArgs& args, const IxArgs* d_ix, int grid, size_t smem, cudaStream_t st);
int engine_w1(teuk_s* h, int engine);
int engine_w2(teuk_s* h, int engine);
int engine_w4(teuk_s* h, int engine);
int dissipation_w1(teuk_s* h, double sigma);
int dissipation_w2(teuk_s* h, double sigma);
int dissipation_w4(teuk_s* h, double sigma);
int dissipate_w1(teuk_s* h);
int dissipate_w2(teuk_s* h);
int dissipate_w4(teuk_s* h);
int filter_tables_w1(teuk_s* h, int l_cut);
int filter_tables_w2(teuk_s* h, int l_cut);
int filter_tables_w4(teuk_s* h, int l_cut);
// normalised sY_lm(theta_j) as quad-double words [n_ell][4][n_th] (times 2 pi w_j if weighted)
std::vector<double> harmonics_w4(int s, int m, int n_th, int ell_min, int ell_max, bool weighted);
int theta_dissipation_w1(teuk_s* h, double sigma, double* max_rate);
int theta_dissipation_w2(teuk_s* h, double sigma, double* max_rate);
int theta_dissipation_w4(teuk_s* h, double sigma, double* max_rate);
int project_w1(teuk_s* h, int ell_min, int ell_max, double* out, int64_t n, int64_t first);
int project_w2(teuk_s* h, int ell_min, int ell_max, double* out, int64_t n, int64_t first);
int project_w4(teuk_s* h, int ell_min, int ell_max, double* out, int64_t n, int64_t first);
int mw_eval_w1(int op, int device, const double* a, const double* b, double* out, int64_t n);
int mw_eval_w2(int op, int device, const double* a, const double* b, double* out, int64_t n);
int mw_eval_w4(int op, int device, const double* a, const double* b, double* out, int64_t n);

// Event pair around one launch when timing is on (records nothing otherwise).
cudaEvent_t take_event(teuk_s* h);
void time_begin(teuk_s* h, cudaEvent_t* a);
void time_end(teuk_s* h, int kind, cudaEvent_t a);

// Block shape of the row-family and balanced step kernels for the handle's launch shape:
// threads along theta (a multiple of 32 up to 256, or the row width) x rows per block. The
// register budget 2 allows at most 128 threads per block.
// Block of kernel family 4 (fused iteration): tx threads along theta x (R + 1) rows, R full-step
// rows per block, tx (R + 1) <= 256.
inline void fused_shape(const teuk_s* h, int& tx, int& R) {
  tx = ((h->n_th + 31) / 32) * 32;
  if (tx > 128) tx = 128;
  if (h->threads_theta > 0 && h->threads_theta < tx) tx = h->threads_theta;
  R = h->rows_per_block > 0 ? h->rows_per_block : 1;
  while (R > 1 && tx * (R + 1) > 256) --R;
}
inline size_t fused_smem(const teuk_s* h, int R) {
  return ((size_t)4 * h->W * (R + 1) * h->pitch + (size_t)(R + 1) * 2 * h->W * (h->n_th + 2 * h->radius)) *
         sizeof(double);
}

inline void row_block_shape(const teuk_s* h, int& tx, int& ty) {
  const int cap = h->kernel_variant == 2 ? 128 : 256;
  tx = ((h->n_th + 31) / 32) * 32;
  if (tx > cap) tx = cap;
  if (h->threads_theta > 0 && h->threads_theta < tx) tx = h->threads_theta;
  if (h->kernel_family == 2) {  // balanced kernels: one row of threads per block
    ty = 1;
    return;
  }
  ty = h->rows_per_block > 0 ? h->rows_per_block : (tx >= 128 ? 1 : 128 / tx);
  while (ty > 1 && tx * ty > cap) ty /= 2;
}

// Launches a step kernel with programmatic stream serialization: its blocks may be scheduled
// while the previous kernel of the stream runs; the kernel itself waits for that kernel's
// completion before reading what it wrote (step_dependency in teuk_kernels.cuh). On the legacy
// default stream it is an ordinary launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  const bool legacy = st == nullptr || st == (cudaStream_t)0x1;
  cfg.attrs = legacy ? nullptr : &attr;
  cfg.numAttrs = legacy ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

inline int cuda_fail(teuk_s* h, cudaError_t e, const char* what) {
  if (h) h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TEUK_ERR_OOM : TEUK_ERR_CUDA;
}
}  // namespace teuk

#define TEUK_CUDA(h, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return teuk::cuda_fail(h, e_, #call); \
  } while (0)
