// C ABI of the teuk library (include/teuk.h): argument checking, device memory, the
// per-outer-step launch sequence and host <-> device transfers.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "teuk_internal.h"

namespace {

int dispatch_setup(teuk_s* h) {
  switch (h->W) {
    case 1: return teuk::setup_w1(h);
    case 2: return teuk::setup_w2(h);
    default: return teuk::setup_w4(h);
  }
}
int dispatch_substep(teuk_s* h, bool record, int64_t slot) {
  switch (h->W) {
    case 1: return teuk::substep_w1(h, record, slot);
    case 2: return teuk::substep_w2(h, record, slot);
    default: return teuk::substep_w4(h, record, slot);
  }
}

int dispatch_persist(teuk_s* h, int64_t n_outer, long long ring_base) {
  switch (h->W) {
    case 1: return teuk::persist_w1(h, n_outer, ring_base);
    case 2: return teuk::persist_w2(h, n_outer, ring_base);
    default: return teuk::persist_w4(h, n_outer, ring_base);
  }
}

// Outer steps through the persistent kernel: one cooperative launch per persist_steps steps.
int step_persistent(teuk_s* h, int64_t n) {
  int64_t done = 0;
  while (done < n) {
    const int64_t chunk = std::min<int64_t>(h->persist_steps, n - done);
    const int rc = dispatch_persist(h, chunk, h->ring ? h->n_recorded : 0);
    if (rc != TEUK_OK) return rc;
    h->substeps_done += chunk * h->k;
    if (h->ring) h->n_recorded += chunk;
    done += chunk;
  }
  return TEUK_OK;
}

int dispatch_dissipate(teuk_s* h) {
  switch (h->W) {
    case 1: return teuk::dissipate_w1(h);
    case 2: return teuk::dissipate_w2(h);
    default: return teuk::dissipate_w4(h);
  }
}

// Kernel family 4 writes every other iteration into the second state buffer; this copies such
// a result back (queued on the stream), so that h->u holds the state again.
int settle_state(teuk_s* h) {
  if (!h->in_u2) return TEUK_OK;
  h->in_u2 = false;
  TEUK_CUDA(h, cudaMemcpyAsync(h->u, h->u2, (size_t)4 * h->W * h->n_r * h->pitch * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->stream));
  return TEUK_OK;
}

// The second state buffer of kernel family 4, zeroed once (its r* boundary rows stay zero).
int ensure_u2(teuk_s* h) {
  if (h->u2) return TEUK_OK;
  const size_t bytes = (size_t)4 * h->W * h->n_r * h->pitch * sizeof(double);
  TEUK_CUDA(h, cudaMalloc(&h->u2, bytes));
  TEUK_CUDA(h, cudaMemsetAsync(h->u2, 0, bytes, h->stream));
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

// One Lax-Wendroff iteration, preceded by the r* dissipation step when it is enabled and an
// outer step begins (the iteration count is a multiple of k); the state is in h->u after it.
int iterate(teuk_s* h, bool record, int64_t slot) {
  if (h->dissipating() && h->substeps_done % h->k == 0) {
    int rc = dispatch_dissipate(h);
    if (rc) return rc;
  }
  int rc = dispatch_substep(h, record, slot);
  if (rc == TEUK_OK) rc = settle_state(h);
  if (rc) return rc;
  ++h->substeps_done;
  return TEUK_OK;
}

// The theta filter's outer-step count restarts from the state's iteration count: the index of
// the next outer step to begin (the current one's when the count is a multiple of k).
int sync_filter_counter(teuk_s* h) {
  if (!h->d_filter_ctr) return TEUK_OK;
  const long long v[2] = {(long long)((h->substeps_done + h->k - 1) / h->k), 0};
  TEUK_CUDA(h, cudaMemcpyAsync(h->d_filter_ctr, v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

int invalid(teuk_s* h, const char* msg) {
  if (h) h->last_error = msg;
  return TEUK_ERR_INVALID_ARG;
}

void drop_graph(teuk_s* h);

void free_all(teuk_s* h) {
  double** bufs[] = {&h->u, &h->uh, &h->cn_raw, &h->ch_raw, &h->cn, &h->ch, &h->wts, &h->lfac, &h->sin_th,
                     &h->cos_th, &h->x_node, &h->x_half, &h->rs_node, &h->prof, &h->ring, &h->u_ko,
                     &h->eps_th, &h->filt};
  for (double** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  if (h->ix_m) cudaFree(h->ix_m);
  if (h->ix_e) cudaFree(h->ix_e);
  h->ix_m = nullptr;
  h->ix_e = nullptr;
  if (h->status) cudaFree(h->status);
  h->status = nullptr;
  if (h->d_filter_ctr) cudaFree(h->d_filter_ctr);
  h->d_filter_ctr = nullptr;
  if (h->u2) cudaFree(h->u2);
  h->u2 = nullptr;
  h->in_u2 = false;
  if (h->pflags) cudaFree(h->pflags);
  h->pflags = nullptr;
  h->pflags_cap = 0;
  if (h->d_ring_counter) cudaFree(h->d_ring_counter);
  h->d_ring_counter = nullptr;
  drop_graph(h);
}

// Copies a [C][W][rows][n_th] host array to / from the pitched device layout.
int copy_planes(teuk_s* h, double* dev, const double* host_in, double* host_out, int comps, int rows) {
  const size_t planes = (size_t)comps * h->W;
  const size_t dpitch = (size_t)h->pitch * sizeof(double), hpitch = (size_t)h->n_th * sizeof(double);
  const size_t height = planes * rows;
  if (dpitch == hpitch) {  // rows without padding: one contiguous copy
    if (host_in) {
      TEUK_CUDA(h, cudaMemcpyAsync(dev, host_in, hpitch * height, cudaMemcpyHostToDevice, h->stream));
    } else {
      TEUK_CUDA(h, cudaMemcpyAsync(host_out, dev, hpitch * height, cudaMemcpyDeviceToHost, h->stream));
    }
    TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
    return TEUK_OK;
  }
  if (host_in) {
    TEUK_CUDA(h, cudaMemcpy2DAsync(dev, dpitch, host_in, hpitch, hpitch, height, cudaMemcpyHostToDevice,
                                   h->stream));
  } else {
    TEUK_CUDA(h, cudaMemcpy2DAsync(host_out, hpitch, dev, dpitch, hpitch, height, cudaMemcpyDeviceToHost,
                                   h->stream));
  }
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

// Local row of the node nearest rstar_obs (ties toward the lower index, computed in FP64), or
// -1 if a slab does not own that node.
int observer_row(const teuk_s* h, double rstar_obs) {
  const double q = (rstar_obs - h->rsmin_d) / h->dr_d;
  int i = (int)std::ceil(q - 0.5);
  if (i < 0) i = 0;
  if (i > h->grid.n_r - 1) i = h->grid.n_r - 1;
  if (h->is_slab() && (i < h->own_lo || i > h->own_hi)) return -1;
  return i - h->row0;
}

__global__ void fp64_peak_kernel(double* out, double a, double b, int iters) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int it = 0; it < iters; ++it) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// One more sample in the observer ring (launched after the last iteration of a captured
// outer step; the kernels read the slot from this counter).
__global__ void advance_counter_kernel(long long* counter) { *counter += 1; }

// Reads the timing events of the last replay of the outer-step graph into the totals.
void read_graph_timing(teuk_s* h) {
  if (!h->graph_events_fresh) return;
  cudaStreamSynchronize(h->stream);
  for (auto& p : h->graph_events) {
    float t = 0;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      h->ms[p.kind] += t;
      h->n_timed[p.kind] += 1;
    } else {
      cudaGetLastError();  // a pair without a time is skipped; keep the error from later checks
    }
  }
  h->graph_events_fresh = false;
}

void drop_graph(teuk_s* h) {
  read_graph_timing(h);
  for (auto& p : h->graph_events) {
    h->free_events.push_back(p.a);
    h->free_events.push_back(p.b);
  }
  h->graph_events.clear();
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
}

// With timing on, the captured graph records an event pair around the two kernels of the
// last iteration of the outer step (event record nodes: a node per kernel would cost about
// what separate launches cost); the library reads the last replay's pairs when the timings
// are drained.
bool graphs_possible(const teuk_s* h) {
  const cudaStream_t legacy = (cudaStream_t)0x1;
  return h->use_graphs && h->stream != nullptr && h->stream != legacy &&
         (!h->dissipating() || h->substeps_done % h->k == 0);
}

// Captures one outer step: k iterations, the last one recording the observer row at slot
// *d_ring_counter % cap, then the counter increment.
int build_graph(teuk_s* h, bool record) {
  drop_graph(h);
  int prc;
  switch (h->W) {  // host-side set-up of the launch shape stays outside the capture
    case 1: prc = teuk::prepare_w1(h); break;
    case 2: prc = teuk::prepare_w2(h); break;
    default: prc = teuk::prepare_w4(h); break;
  }
  if (prc != TEUK_OK) return prc;
  const int64_t launches = h->launches;
  cudaGraph_t graph = nullptr;
  if (h->timing) {  // events for the capture come from the pool, made before it starts
    for (size_t n = h->free_events.size(); n < (size_t)(4 * h->k + 2); ++n) {
      cudaEvent_t ev = nullptr;
      TEUK_CUDA(h, cudaEventCreate(&ev));
      h->free_events.push_back(ev);
    }
  }
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return teuk::cuda_fail(h, e, "cudaStreamBeginCapture");
  h->capturing = true;
  int rc = h->dissipating() ? dispatch_dissipate(h) : TEUK_OK;
  for (int q = 0; q < h->k && rc == TEUK_OK; ++q) {
    h->time_this = q == h->k - 1;  // the graph times the last iteration of the outer step only
    rc = dispatch_substep(h, record && q == h->k - 1, -1);
  }
  if (rc == TEUK_OK) rc = settle_state(h);  // odd k with fused iterations: one copy per outer step
  h->in_u2 = false;
  h->time_this = true;
  if (rc == TEUK_OK && record) advance_counter_kernel<<<1, 1, 0, h->stream>>>(h->d_ring_counter);
  e = cudaStreamEndCapture(h->stream, &graph);
  h->capturing = false;
  h->launches = launches;
  if (rc != TEUK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return teuk::cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->graph_exec = nullptr;
    return teuk::cuda_fail(h, e, "cudaGraphInstantiate");
  }
  h->graph_record = record;
  return TEUK_OK;
}

void drain_timing(teuk_s* h) {
  read_graph_timing(h);
  if (h->pending.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto& p : h->pending) {
    float t = 0;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      h->ms[p.kind] += t;
      h->n_timed[p.kind] += 1;
    } else {
      cudaGetLastError();  // a pair without a time is skipped; keep the error from later checks
    }
    h->free_events.push_back(p.a);
    h->free_events.push_back(p.b);
  }
  h->pending.clear();
}

}  // namespace

namespace teuk {
cudaEvent_t take_event(teuk_s* h) {
  if (!h->free_events.empty()) {
    cudaEvent_t e = h->free_events.back();
    h->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// While the outer-step graph is captured, events are recorded as external event record
// nodes (recorded when the graph runs), not as capture-internal dependencies.
static void record_event(teuk_s* h, cudaEvent_t e) {
  if (h->capturing) cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
  else cudaEventRecord(e, h->stream);
}
void time_begin(teuk_s* h, cudaEvent_t* a) {
  if (!h->timing || !h->time_this) return;
  *a = take_event(h);
  record_event(h, *a);
}
void time_end(teuk_s* h, int kind, cudaEvent_t a) {
  if (!h->timing || !a) return;
  cudaEvent_t b = take_event(h);
  record_event(h, b);
  if (h->capturing) {  // recorded by every replay of the graph
    h->graph_events.push_back(teuk_s::EvPair{kind, a, b});
    return;
  }
  h->pending.push_back(teuk_s::EvPair{kind, a, b});
  if (h->pending.size() > 4096) drain_timing(h);
}
}  // namespace teuk

namespace {
int create_impl(teuk_t* out, double M, double a, int s, int m, const teuk_grid* grid, teuk_precision precision,
                void* cuda_stream, int own_lo, int own_hi);
}

extern "C" {

const char* teuk_strerror(int code) {
  switch (code) {
    case TEUK_OK: return "ok";
    case TEUK_ERR_INVALID_ARG: return "invalid argument";
    case TEUK_ERR_CUDA: return "CUDA runtime error";
    case TEUK_ERR_OOM: return "out of memory";
    case TEUK_ERR_NONFINITE: return "non-finite value in the evolution";
    case TEUK_ERR_STATE_MISMATCH: return "state does not match the handle";
    case TEUK_ERR_NO_DEVICE: return "no CUDA device";
    case TEUK_ERR_TIMEOUT: return "a wait inside a step kernel reached its limit";
    default: return "unknown error";
  }
}

const char* teuk_last_error(teuk_t h) { return h ? h->last_error.c_str() : ""; }

int teuk_create(teuk_t* out, double M, double a, int s, int m, const teuk_grid* grid,
                teuk_precision precision, void* cuda_stream) {
  return create_impl(out, M, a, s, m, grid, precision, cuda_stream, 0, -1);
}

int teuk_create_slab(teuk_t* out, double M, double a, int s, int m, const teuk_grid* grid,
                     teuk_precision precision, void* cuda_stream, int own_lo, int own_hi) {
  if (!grid || own_lo < 0 || own_hi < own_lo || own_hi > grid->n_r - 1) return TEUK_ERR_INVALID_ARG;
  const int lo = own_lo > 0 ? own_lo - 1 : 0, hi = own_hi < grid->n_r - 1 ? own_hi + 1 : own_hi;
  if (hi - lo + 1 < 3) return TEUK_ERR_INVALID_ARG;  // the kernels need three rows
  return create_impl(out, M, a, s, m, grid, precision, cuda_stream, own_lo, own_hi);
}

}  // extern "C"

namespace {
int create_impl(teuk_t* out, double M, double a, int s, int m, const teuk_grid* grid, teuk_precision precision,
                void* cuda_stream, int own_lo, int own_hi) {
  if (!out || !grid) return TEUK_ERR_INVALID_ARG;
  *out = nullptr;
  const int W = (int)precision;
  if (W != 1 && W != 2 && W != 4) return TEUK_ERR_INVALID_ARG;
  if (!(M > 0) || !(std::fabs(a) < M) || !std::isfinite(M) || !std::isfinite(a)) return TEUK_ERR_INVALID_ARG;
  if (s < -2 || s > 2) return TEUK_ERR_INVALID_ARG;
  const teuk_grid& g = *grid;
  if (g.n_r < 3 || g.n_theta < 6 || g.n_theta > 1024 || g.substeps < 1 || g.reserved != 0)
    return TEUK_ERR_INVALID_ARG;
  if (!(g.rstar_max > g.rstar_min) || !std::isfinite(g.rstar_min) || !std::isfinite(g.rstar_max))
    return TEUK_ERR_INVALID_ARG;
  if (g.dt < 0 || !std::isfinite(g.dt)) return TEUK_ERR_INVALID_ARG;
  const int order = g.theta_order == 0 ? 10 : g.theta_order;
  if (order != 10 && order != 2) return TEUK_ERR_INVALID_ARG;
  if (g.parity != 0 && g.parity != 1 && g.parity != -1 && g.parity != 2) return TEUK_ERR_INVALID_ARG;
  if (!(g.ko_sigma >= 0) || !(g.ko_theta >= 0) || g.ko_sigma > 4.0 || g.ko_theta > 4.0) return TEUK_ERR_INVALID_ARG;
  if (g.theta_filter < 0 || g.theta_filter_period < 0) return TEUK_ERR_INVALID_ARG;
  // slabs: no dissipation and no filter
  if (own_hi >= 0 && (g.ko_sigma > 0 || g.ko_theta > 0 || g.theta_filter > 0)) return TEUK_ERR_INVALID_ARG;
  if ((int64_t)g.n_r * g.n_theta > (int64_t)1 << 31) return TEUK_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TEUK_ERR_NO_DEVICE;

  teuk_s* h = new (std::nothrow) teuk_s;
  if (!h) return TEUK_ERR_OOM;
  h->M = M;
  h->a = a;
  h->s = s;
  h->m = m;
  h->grid = g;
  h->W = W;
  h->n_r = g.n_r;
  if (own_hi >= 0) {  // an r* slab: the owned rows and one halo row on each side inside the grid
    h->own_lo = own_lo;
    h->own_hi = own_hi;
    h->row0 = own_lo > 0 ? own_lo - 1 : 0;
    h->n_r = (own_hi < g.n_r - 1 ? own_hi + 1 : own_hi) - h->row0 + 1;
  }
  h->n_th = g.n_theta;
  h->pitch = ((g.n_theta + 15) / 16) * 16;
  h->parity = g.parity == 0 ? (((m + s) % 2 == 0) ? 1 : -1)
              : g.parity == 2 ? ((std::abs(m) % 2 == 0) ? 1 : -1) : g.parity;
  h->radius = order == 10 ? 5 : 1;
  h->k = g.substeps;
  cudaGetDevice(&h->device);
  int rc = TEUK_OK;
  auto fail = [&](int code) {
    free_all(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return code;
  };
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(TEUK_ERR_CUDA);
    h->own_stream = true;
  }
  const size_t P = h->pitch, nr = h->n_r, nh = h->n_r - 1;
  struct Alloc { double** p; size_t n; } allocs[] = {
      {&h->u, 4 * W * nr * P},      {&h->uh, 4 * W * nh * P},     {&h->cn_raw, 8 * W * nr * P},
      {&h->ch_raw, 8 * W * nh * P}, {&h->cn, 8 * W * nr * P},     {&h->ch, 8 * W * nh * P},
      {&h->wts, (size_t)(2 * h->radius + 1) * W * h->n_th},     {&h->sin_th, (size_t)W * h->n_th},
      {&h->lfac, (size_t)2 * W * h->n_th},
      {&h->cos_th, (size_t)W * h->n_th}, {&h->x_node, W * nr},  {&h->x_half, W * nh},
      {&h->rs_node, W * nr},        {&h->prof, (size_t)W * h->n_th}};
  for (auto& al : allocs) {
    if (cudaMalloc(al.p, al.n * sizeof(double)) != cudaSuccess) return fail(TEUK_ERR_OOM);
    if (cudaMemsetAsync(*al.p, 0, al.n * sizeof(double), h->stream) != cudaSuccess) return fail(TEUK_ERR_CUDA);
  }
  if (cudaMalloc(&h->status, sizeof(unsigned int)) != cudaSuccess) return fail(TEUK_ERR_OOM);
  cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->stream);
  if (cudaMalloc(&h->d_ring_counter, sizeof(long long)) != cudaSuccess) return fail(TEUK_ERR_OOM);
  cudaMemsetAsync(h->d_ring_counter, 0, sizeof(long long), h->stream);
  rc = dispatch_setup(h);
  if (rc != TEUK_OK) return fail(rc);
  if (g.ko_sigma > 0 && (rc = teuk_set_dissipation(h, g.ko_sigma)) != TEUK_OK) return fail(rc);
  if (g.ko_theta > 0 && (rc = teuk_set_theta_dissipation(h, g.ko_theta)) != TEUK_OK) return fail(rc);
  if (g.theta_filter > 0 && (rc = teuk_set_theta_filter(h, g.theta_filter, g.theta_filter_period)) != TEUK_OK)
    return fail(rc);
  *out = h;
  return TEUK_OK;
}
}  // namespace

extern "C" {

int teuk_destroy(teuk_t h) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  drain_timing(h);
  for (cudaEvent_t e : h->free_events) cudaEventDestroy(e);
  h->free_events.clear();
  free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return TEUK_OK;
}

// One state row [4][W][n_theta] between local row `row` and a buffer (device or host memory).
static int copy_row(teuk_s* h, int row, double* dst, const double* src) {
  const size_t plane = (size_t)h->n_r * h->pitch * sizeof(double), line = (size_t)h->n_th * sizeof(double);
  double* r = h->u + (size_t)row * h->pitch;
  if (dst) {
    TEUK_CUDA(h, cudaMemcpy2DAsync(dst, line, r, plane, line, (size_t)4 * h->W, cudaMemcpyDefault, h->stream));
  } else {
    TEUK_CUDA(h, cudaMemcpy2DAsync(r, plane, src, line, line, (size_t)4 * h->W, cudaMemcpyDefault, h->stream));
  }
  return TEUK_OK;
}

int teuk_get_halo_rows(teuk_t h, double* lo_out, double* hi_out) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (!h->is_slab()) return invalid(h, "halo rows: not a slab");
  int rc = TEUK_OK;
  if (lo_out) rc = copy_row(h, h->own_lo - h->row0, lo_out, nullptr);
  if (rc == TEUK_OK && hi_out) rc = copy_row(h, h->own_hi - h->row0, hi_out, nullptr);
  return rc;
}

int teuk_set_halo_rows(teuk_t h, const double* lo_in, const double* hi_in) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (!h->is_slab()) return invalid(h, "halo rows: not a slab");
  if ((lo_in && h->own_lo == 0) || (hi_in && h->own_hi == h->grid.n_r - 1))
    return invalid(h, "halo rows: no halo beyond an r* boundary row");
  int rc = TEUK_OK;
  if (lo_in) rc = copy_row(h, 0, nullptr, lo_in);
  if (rc == TEUK_OK && hi_in) rc = copy_row(h, h->n_r - 1, nullptr, hi_in);
  return rc;
}

int teuk_slab_rows(teuk_t h, int* row0, int* own_lo, int* own_hi) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (row0) *row0 = h->row0;
  if (own_lo) *own_lo = h->is_slab() ? h->own_lo : 0;
  if (own_hi) *own_hi = h->is_slab() ? h->own_hi : h->n_r - 1;
  return TEUK_OK;
}

int teuk_info(teuk_t h, int* words, int* n_r, int* n_theta, int* substeps, double* dt_outer) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (words) *words = h->W;
  if (n_r) *n_r = h->n_r;
  if (n_theta) *n_theta = h->n_th;
  if (substeps) *substeps = h->k;
  if (dt_outer) *dt_outer = h->dt_outer;
  return TEUK_OK;
}

int64_t teuk_kernel_launches(teuk_t h) { return h ? h->launches : -1; }

int teuk_set_initial(teuk_t h, const double* phi_pi) {
  if (!h || !phi_pi) return invalid(h, "null argument");
  int rc = copy_planes(h, h->u, phi_pi, nullptr, 4, h->n_r);
  if (rc) return rc;
  // Phi = Pi = 0 on the r* boundary rows (Sec. 3.B); a slab's halo rows are data
  const size_t ws = (size_t)h->n_r * h->pitch;
  const bool first = h->row0 == 0, last = h->row0 + h->n_r - 1 == h->grid.n_r - 1;
  for (int p = 0; p < 4 * h->W; ++p) {
    if (first) TEUK_CUDA(h, cudaMemsetAsync(h->u + p * ws, 0, h->pitch * sizeof(double), h->stream));
    if (last)
      TEUK_CUDA(h, cudaMemsetAsync(h->u + p * ws + (size_t)(h->n_r - 1) * h->pitch, 0, h->pitch * sizeof(double),
                                   h->stream));
  }
  h->substeps_done = 0;
  h->n_recorded = 0;
  h->in_u2 = false;
  TEUK_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->stream));
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return sync_filter_counter(h);
}

int teuk_set_initial_pulse(teuk_t h, double center, double width, double amp_re, double amp_im, int ell) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (ell < std::abs(h->m) || ell < std::abs(h->s) || ell > 40 || !(width > 0) || !std::isfinite(center))
    return invalid(h, "pulse: need max(|m|, |s|) <= ell <= 40, width > 0");
  int rc;
  switch (h->W) {
    case 1: rc = teuk::pulse_w1(h, center, width, amp_re, amp_im, ell); break;
    case 2: rc = teuk::pulse_w2(h, center, width, amp_re, amp_im, ell); break;
    default: rc = teuk::pulse_w4(h, center, width, amp_re, amp_im, ell); break;
  }
  h->substeps_done = 0;
  h->n_recorded = 0;
  h->in_u2 = false;
  if (rc == TEUK_OK) TEUK_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->stream));
  if (rc == TEUK_OK) rc = sync_filter_counter(h);
  return rc;
}

int teuk_substep(teuk_t h, int64_t n) {
  if (!h || n < 0) return TEUK_ERR_INVALID_ARG;
  if (h->is_slab() && n > 1)
    return invalid(h, "slab: one iteration per call (the halo rows are exchanged between iterations)");
  for (int64_t t = 0; t < n; ++t) {
    int rc = iterate(h, false, 0);
    if (rc) return rc;
  }
  return TEUK_OK;
}

int teuk_substep_host_state(teuk_t h, double* host_planes, int64_t n) {
  if (!h || !host_planes || n < 0) return TEUK_ERR_INVALID_ARG;
  const size_t dpitch = (size_t)h->pitch * sizeof(double), hpitch = (size_t)h->n_th * sizeof(double);
  const size_t height = (size_t)4 * h->W * h->n_r;
  for (int64_t t = 0; t < n; ++t) {
    TEUK_CUDA(h, cudaMemcpy2DAsync(h->u, dpitch, host_planes, hpitch, hpitch, height, cudaMemcpyHostToDevice,
                                   h->stream));
    int rc = iterate(h, false, 0);
    if (rc) return rc;
    TEUK_CUDA(h, cudaMemcpy2DAsync(host_planes, hpitch, h->u, dpitch, hpitch, height, cudaMemcpyDeviceToHost,
                                   h->stream));
    // the host loop owns the state between iterations
    TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return TEUK_OK;
}

int teuk_use_graphs(teuk_t h, int enable) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  h->use_graphs = enable != 0;
  if (!h->use_graphs) drop_graph(h);
  return TEUK_OK;
}

int teuk_set_engine(teuk_t h, int engine) {
  if (!h || engine < 0 || engine > 1) return TEUK_ERR_INVALID_ARG;
  if (engine == 1 && h->W == 1) return invalid(h, "the integer engine is for double-double and quad-double handles");
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  if (engine == 1) h->kernel_family = 0;
  switch (h->W) {
    case 1: return teuk::engine_w1(h, engine);
    case 2: return teuk::engine_w2(h, engine);
    default: return teuk::engine_w4(h, engine);
  }
}

int teuk_engine(teuk_t h) { return h ? h->engine : TEUK_ERR_INVALID_ARG; }

int teuk_test_stall_copies(teuk_t h, int block, int wait_log2) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (h->engine != 1 && h->kernel_family != 3)
    return invalid(h, "stall test: the bounded waits are the integer engine's and the persistent launches'");
  if (block < -1 || wait_log2 < 10 || wait_log2 > 20)
    return invalid(h, "stall test: block >= -1, 10 <= wait_log2 <= 20");
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  h->test_stall_block = block;
  h->wait_log2 = block < 0 ? 20 : wait_log2;
  return TEUK_OK;
}

int teuk_set_dissipation(teuk_t h, double sigma) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (!(sigma >= 0) || !std::isfinite(sigma) || sigma > 4.0)
    return invalid(h, "dissipation: need 0 <= sigma <= 4");
  if (h->is_slab() && sigma > 0) return invalid(h, "dissipation: not on a slab (it reads two rows beyond the halo)");
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (sigma > 0 && !h->u_ko)
    TEUK_CUDA(h, cudaMalloc(&h->u_ko, (size_t)4 * h->W * h->n_r * h->pitch * sizeof(double)));
  h->ko_sigma = sigma;
  drop_graph(h);
  switch (h->W) {
    case 1: return teuk::dissipation_w1(h, sigma);
    case 2: return teuk::dissipation_w2(h, sigma);
    default: return teuk::dissipation_w4(h, sigma);
  }
}

int teuk_set_theta_dissipation(teuk_t h, double sigma) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (!(sigma >= 0) || !std::isfinite(sigma) || sigma > 4.0)
    return invalid(h, "theta dissipation: need 0 <= sigma <= 4");
  if (h->is_slab() && sigma > 0) return invalid(h, "theta dissipation: not on a slab");
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  if (sigma == 0) {
    h->ko_theta = 0;
    return TEUK_OK;
  }
  if (!h->u_ko) TEUK_CUDA(h, cudaMalloc(&h->u_ko, (size_t)4 * h->W * h->n_r * h->pitch * sizeof(double)));
  if (!h->eps_th) TEUK_CUDA(h, cudaMalloc(&h->eps_th, (size_t)h->W * h->n_r * sizeof(double)));
  auto table = [&](double sg, double* rate) {
    switch (h->W) {
      case 1: return teuk::theta_dissipation_w1(h, sg, rate);
      case 2: return teuk::theta_dissipation_w2(h, sg, rate);
      default: return teuk::theta_dissipation_w4(h, sg, rate);
    }
  };
  double rate = 0;
  int rc = table(sigma, &rate);
  if (rc != TEUK_OK) return rc;
  if (rate > 2.0) {  // refused: the table of the sigma in use is restored
    double old_rate = 0;
    if (h->ko_theta > 0 && (rc = table(h->ko_theta, &old_rate)) != TEUK_OK) return rc;
    return invalid(h, "theta dissipation: sigma c_th dt / dtheta must not exceed 2 (the step would "
                      "amplify the grid-scale theta mode)");
  }
  h->ko_theta = sigma;
  return TEUK_OK;
}

double teuk_theta_dissipation(teuk_t h) { return h ? h->ko_theta : -1.0; }

int teuk_set_theta_filter(teuk_t h, int l_cut, int period) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  const int l_low = std::max(std::abs(h->s), std::abs(h->m));
  if (l_cut != 0 && (l_cut <= l_low || l_cut > 41 || 2 * (l_cut - 1) >= h->n_th))
    return invalid(h, "theta filter: need l_cut = 0 or max(|s|, |m|) < l_cut <= 41 with 2 (l_cut - 1) < n_theta");
  if (period < 0 || period > 1024) return invalid(h, "theta filter: need 0 <= period <= 1024 (0 = 1)");
  if (h->is_slab() && l_cut > 0) return invalid(h, "theta filter: not on a slab");
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  if (l_cut == 0) {
    h->filter_lcut = 0;
    return TEUK_OK;
  }
  int rc;
  switch (h->W) {
    case 1: rc = teuk::filter_tables_w1(h, l_cut); break;
    case 2: rc = teuk::filter_tables_w2(h, l_cut); break;
    default: rc = teuk::filter_tables_w4(h, l_cut); break;
  }
  if (rc != TEUK_OK) {
    h->filter_lcut = 0;  // the tables of the previous cut are gone
    return rc;
  }
  if (!h->d_filter_ctr) TEUK_CUDA(h, cudaMalloc(&h->d_filter_ctr, 2 * sizeof(long long)));
  h->filter_lcut = l_cut;
  h->filter_period = period > 0 ? period : 1;
  return sync_filter_counter(h);
}

int teuk_theta_filter_period(teuk_t h) { return h ? h->filter_period : -1; }

int teuk_theta_filter(teuk_t h) { return h ? h->filter_lcut : -1; }

int teuk_step(teuk_t h, int64_t n) {
  if (!h || n < 0) return TEUK_ERR_INVALID_ARG;
  if (h->is_slab()) return invalid(h, "slab: advance with teuk_substep(h, 1) and a halo exchange per iteration");
  if (n > 0 && h->kernel_family == 3 && h->engine == 0 && !h->dissipating() && h->substeps_done % h->k == 0)
    return step_persistent(h, n);
  if (n > 0 && graphs_possible(h)) {
    const bool record = h->ring != nullptr;
    if (!h->graph_exec || h->graph_record != record) {
      int rc = build_graph(h, record);
      if (rc != TEUK_OK) return rc;
    }
    if (record) {
      const long long recorded = h->n_recorded;
      TEUK_CUDA(h, cudaMemcpyAsync(h->d_ring_counter, &recorded, sizeof(recorded), cudaMemcpyHostToDevice,
                                   h->stream));
    }
    for (int64_t t = 0; t < n; ++t) TEUK_CUDA(h, cudaGraphLaunch(h->graph_exec, h->stream));
    if (!h->graph_events.empty()) h->graph_events_fresh = true;
    h->substeps_done += n * h->k;
    h->launches += n * (h->iteration_launches() * h->k + h->outer_op_launches());
    if (record) h->n_recorded += n;
    return TEUK_OK;
  }
  for (int64_t t = 0; t < n; ++t) {
    for (int q = 0; q < h->k; ++q) {
      const bool last = q == h->k - 1;
      const bool record = last && h->ring != nullptr;
      const int64_t slot = record ? h->n_recorded % h->ring_cap : 0;
      int rc = iterate(h, record, slot);
      if (rc) return rc;
    }
    if (h->ring) ++h->n_recorded;
  }
  return TEUK_OK;
}

int teuk_sync(teuk_t h) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  unsigned int st = 0;
  TEUK_CUDA(h, cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st & 1u) {
    h->last_error = "non-finite value produced by the Lax-Wendroff step";
    return TEUK_ERR_NONFINITE;
  }
  if (st & 2u) {
    h->last_error = "a copy into shared memory did not complete within its wait limit";
    return TEUK_ERR_TIMEOUT;
  }
  return TEUK_OK;
}

int teuk_observe(teuk_t h, double rstar_obs, double* out_phi, double* rstar_used) {
  if (!h || !out_phi || !std::isfinite(rstar_obs)) return TEUK_ERR_INVALID_ARG;
  const int i = observer_row(h, rstar_obs);
  if (i < 0) {
    h->last_error = "observer: the node is not one of this slab's rows";
    return TEUK_ERR_STATE_MISMATCH;
  }
  const size_t ws = (size_t)h->n_r * h->pitch;
  for (int p = 0; p < 2 * h->W; ++p)
    TEUK_CUDA(h, cudaMemcpyAsync(out_phi + (size_t)p * h->n_th, h->u + p * ws + (size_t)i * h->pitch,
                                 h->n_th * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (rstar_used) *rstar_used = h->rsmin_d + (i + h->row0) * h->dr_d;
  return TEUK_OK;
}

int teuk_set_observer(teuk_t h, double rstar_obs, int64_t capacity) {
  if (!h || capacity < 1 || !std::isfinite(rstar_obs)) return TEUK_ERR_INVALID_ARG;
  if (observer_row(h, rstar_obs) < 0) {
    h->last_error = "observer: the node is not one of this slab's rows";
    return TEUK_ERR_STATE_MISMATCH;
  }
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->ring) cudaFree(h->ring);
  h->ring = nullptr;
  const size_t n = (size_t)capacity * 2 * h->W * h->n_th;
  TEUK_CUDA(h, cudaMalloc(&h->ring, n * sizeof(double)));
  TEUK_CUDA(h, cudaMemsetAsync(h->ring, 0, n * sizeof(double), h->stream));
  h->ring_cap = capacity;
  h->i_obs = observer_row(h, rstar_obs);
  h->n_recorded = 0;
  drop_graph(h);
  return TEUK_OK;
}

int teuk_read_waveform(teuk_t h, double* out, int64_t* n_samples) {
  if (!h || !n_samples) return TEUK_ERR_INVALID_ARG;
  if (!h->ring) return TEUK_ERR_STATE_MISMATCH;
  const int64_t n = h->n_recorded < h->ring_cap ? h->n_recorded : h->ring_cap;
  *n_samples = n;
  if (!out || n == 0) return TEUK_OK;
  const size_t per = (size_t)2 * h->W * h->n_th;
  const int64_t first = h->n_recorded - n;  // oldest sample kept
  for (int64_t t = 0; t < n; ++t) {
    const int64_t slot = (first + t) % h->ring_cap;
    TEUK_CUDA(h, cudaMemcpyAsync(out + t * per, h->ring + slot * per, per * sizeof(double),
                                 cudaMemcpyDeviceToHost, h->stream));
  }
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

int teuk_read_multipoles(teuk_t h, int ell_min, int ell_max, double* out, int64_t* n_samples) {
  if (!h || !n_samples) return TEUK_ERR_INVALID_ARG;
  const int lo = std::max(std::abs(h->m), std::abs(h->s));
  if (ell_min < lo || ell_max < ell_min || ell_max > 40 || ell_max >= h->n_th)
    return invalid(h, "multipoles: need max(|m|, |s|) <= ell_min <= ell_max <= min(40, n_theta - 1)");
  if (!h->ring) return TEUK_ERR_STATE_MISMATCH;
  const int64_t n = h->n_recorded < h->ring_cap ? h->n_recorded : h->ring_cap;
  *n_samples = n;
  if (!out || n == 0) return TEUK_OK;
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  const int64_t first = h->n_recorded - n;  // oldest sample kept
  switch (h->W) {
    case 1: return teuk::project_w1(h, ell_min, ell_max, out, n, first);
    case 2: return teuk::project_w2(h, ell_min, ell_max, out, n, first);
    default: return teuk::project_w4(h, ell_min, ell_max, out, n, first);
  }
}

int teuk_get_state(teuk_t h, double* planes, int64_t* substeps_done) {
  if (!h || !planes) return TEUK_ERR_INVALID_ARG;
  int rc = copy_planes(h, h->u, nullptr, planes, 4, h->n_r);
  if (substeps_done) *substeps_done = h->substeps_done;
  return rc;
}

int teuk_set_state(teuk_t h, const double* planes, int64_t substeps_done) {
  if (!h || !planes || substeps_done < 0) return TEUK_ERR_INVALID_ARG;
  int rc = copy_planes(h, h->u, planes, nullptr, 4, h->n_r);
  if (rc) return rc;
  h->substeps_done = substeps_done;
  h->in_u2 = false;
  TEUK_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned int), h->stream));
  return sync_filter_counter(h);
}

int teuk_get_state_device(teuk_t h, double* dev_planes) {
  if (!h || !dev_planes) return TEUK_ERR_INVALID_ARG;
  const size_t dpitch = (size_t)h->pitch * sizeof(double), hpitch = (size_t)h->n_th * sizeof(double);
  TEUK_CUDA(h, cudaMemcpy2DAsync(dev_planes, hpitch, h->u, dpitch, hpitch, (size_t)4 * h->W * h->n_r,
                                 cudaMemcpyDeviceToDevice, h->stream));
  return TEUK_OK;
}

int teuk_get_coeffs(teuk_t h, int which, double* out) {
  if (!h || !out || (which != 0 && which != 1)) return TEUK_ERR_INVALID_ARG;
  return copy_planes(h, which ? h->ch_raw : h->cn_raw, nullptr, out, 8, which ? h->n_r - 1 : h->n_r);
}

int teuk_get_tortoise(teuk_t h, int which, double* x_out) {
  if (!h || !x_out || (which != 0 && which != 1)) return TEUK_ERR_INVALID_ARG;
  const size_t rows = which ? h->n_r - 1 : h->n_r;
  TEUK_CUDA(h, cudaMemcpyAsync(x_out, which ? h->x_half : h->x_node, rows * h->W * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

// Whether ty rows of the integer engine's kernels fit the shared memory of one block.
bool ix_shape_fits(const teuk_s* h, int ty) {
  if (h->W == 1) return true;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const int gs = h->n_th + 2 * h->radius;
  const size_t b = h->W == 2 ? teuk::ix_row_smem_w2(ty, gs) : teuk::ix_row_smem_w4(ty, gs);
  return b <= (size_t)optin;
}

// Whether the fused block with R full-step rows fits the shared memory a block can have.
bool fused_smem_fits(const teuk_s* h, int R) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return teuk::fused_smem(h, R) <= (size_t)optin;
}

int teuk_tune(teuk_t h, int* rows_per_block) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  const size_t n = (size_t)4 * h->W * h->n_r * h->pitch;
  double* saved = nullptr;
  unsigned int status = 0;
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  TEUK_CUDA(h, cudaMemcpy(&status, h->status, sizeof(status), cudaMemcpyDeviceToHost));
  TEUK_CUDA(h, cudaMalloc(&saved, n * sizeof(double)));
  cudaMemcpyAsync(saved, h->u, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  const bool timing = h->timing;
  h->timing = false;
  const int64_t launches = h->launches;
  const int tx_full = std::min(256, ((h->n_th + 31) / 32) * 32);
  int best = 0, best_tx = 0;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = TEUK_OK;
  // candidates: threads along theta (32 .. the row width, powers of two times 32, or the
  // row width itself) x rows per block, at most 256 threads
  int best_v = 0, best_f = 0;
  struct Cand { float ms; int f, v, tx, ty; };
  std::vector<Cand> cands;
  auto trial = [&](int f, int v, int tx, int ty) {
    if (h->engine == 1 && !ix_shape_fits(h, ty)) return;  // rows too wide for one block
    h->kernel_family = f;
    h->kernel_variant = v;
    h->threads_theta = tx;
    h->rows_per_block = ty;
    if ((rc = dispatch_substep(h, false, 0)) != TEUK_OK) return;  // warm-up
    cudaEventRecord(e0, h->stream);
    for (int t = 0; t < 4 && rc == TEUK_OK; ++t) rc = dispatch_substep(h, false, 0);
    cudaEventRecord(e1, h->stream);
    if (rc == TEUK_OK) rc = settle_state(h);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rc == TEUK_OK) cands.push_back(Cand{ms, f, v, tx, ty});
    if (rc == TEUK_OK && ms < best_ms) {
      best_ms = ms;
      best = ty;
      best_tx = tx;
      best_v = v;
      best_f = f;
    }
  };
  for (int v = 0; v < 3 && rc == TEUK_OK; ++v) {
    // rows-per-block kernels: threads along theta x rows per block, at most 256 threads
    // (128 with register budget 2)
    const int cap = v == 2 ? 128 : 256;
    const int tx_top = std::min(tx_full, cap);
    for (int tx = 32; tx <= tx_top && rc == TEUK_OK; tx = (tx * 2 > tx_top && tx < tx_top) ? tx_top : tx * 2) {
      for (int ty = 1; ty <= 8 && tx * ty <= cap && rc == TEUK_OK; ty *= 2) trial(0, v, tx, ty);
      if (tx == tx_top) break;
    }
    if (h->engine == 1) continue;  // the integer engine has the rows-per-block kernels only
    // one warp per (row, 32 columns)
    if (rc == TEUK_OK) trial(1, v, 0, 0);
    // balanced: the same number of points for every resident block
    for (int tx = 32; tx <= tx_top && rc == TEUK_OK; tx = (tx * 2 > tx_top && tx < tx_top) ? tx_top : tx * 2) {
      trial(2, v, tx, 1);
      if (tx == tx_top) break;
    }
  }
  // fused iterations (one launch each) for grids of up to 2^20 points, threads along theta x
  // (R + 1) rows, R = 1, 3, 7 full-step rows per block
  if (rc == TEUK_OK && h->engine == 0 && !h->is_slab() && (int64_t)h->n_r * h->n_th <= ((int64_t)1 << 20) &&
      (rc = ensure_u2(h)) == TEUK_OK) {
    const int tx_top = std::min(tx_full, 128);
    for (int tx = 32; tx <= tx_top && rc == TEUK_OK; tx = (tx * 2 > tx_top && tx < tx_top) ? tx_top : tx * 2) {
      for (int R = 1; R <= 7 && tx * (R + 1) <= 256 && rc == TEUK_OK; R = 2 * R + 1)
        if (fused_smem_fits(h, R)) trial(4, 0, tx, R);
      if (tx == tx_top) break;
    }
  }
  int best_p = 1;
  double* ring = h->ring;  // the observer ring is left alone by the steps below
  h->ring = nullptr;
  auto time_steps = [&](int outer, auto&& run) -> float {
    if ((rc = run(1)) != TEUK_OK) return 1e30f;  // warm-up (and graph build)
    cudaEventRecord(e0, h->stream);
    rc = run(outer);
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return rc == TEUK_OK ? ms : 1e30f;
  };
  auto regular = [&](int outer) -> int {
    if (graphs_possible(h)) {
      if (!h->graph_exec) {
        const int r = build_graph(h, false);
        if (r != TEUK_OK) return r;
      }
      for (int t = 0; t < outer; ++t) TEUK_CUDA(h, cudaGraphLaunch(h->graph_exec, h->stream));
      return TEUK_OK;
    }
    for (int t = 0; t < outer * h->k; ++t) {
      const int r = dispatch_substep(h, false, 0);
      if (r != TEUK_OK) return r;
    }
    return settle_state(h);
  };
  // Small problems run as replayed graphs, where launch costs differ from direct launches: the
  // four fastest shapes of the two-kernel families above and the two fastest fused ones are
  // timed again as teuk_step runs them, over four outer steps, when an outer step is short
  // (timed by direct launches, the fused shapes' single launch per iteration ranks them above
  // two-kernel shapes that replay faster).
  const bool rerank = rc == TEUK_OK && graphs_possible(h) && best_ms / 4 * h->k < 5.0f;
  if (rc == TEUK_OK && graphs_possible(h) && !rerank && best_f == 4) {
    // not re-timed as graphs: keep the fastest two-kernel shape rather than a fused one ranked
    // first by its launch count
    float two_ms = 1e30f;
    for (const Cand& c : cands)
      if (c.f != 4 && c.ms < two_ms) {
        two_ms = c.ms;
        best_f = c.f;
        best_v = c.v;
        best_tx = c.tx;
        best = c.ty;
      }
  }
  if (rerank) {
    std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    std::vector<Cand> pick;
    int n_two = 0, n_fused = 0;
    for (const Cand& c : cands) {
      if (c.f == 4 ? n_fused++ < 2 : n_two++ < 4) pick.push_back(c);
    }
    cands.swap(pick);
    float graph_best = 1e30f;
    for (size_t c = 0; c < cands.size() && rc == TEUK_OK; ++c) {
      h->kernel_family = cands[c].f;
      h->kernel_variant = cands[c].v;
      h->threads_theta = cands[c].tx;
      h->rows_per_block = cands[c].ty;
      drop_graph(h);
      const float ms = time_steps(4, regular);
      if (rc == TEUK_OK && ms < graph_best) {
        graph_best = ms;
        best_f = cands[c].f;
        best_v = cands[c].v;
        best_tx = cands[c].tx;
        best = cands[c].ty;
      }
    }
    drop_graph(h);
  }
  if (rc == TEUK_OK && h->engine == 0 && !h->dissipating() && h->substeps_done % h->k == 0) {
    // Persistent launches against the best shape above, both as teuk_step runs them (the
    // regular kernels as a replayed graph where possible), over the same outer steps.
    h->kernel_family = best_f;
    h->kernel_variant = best_v;
    h->threads_theta = best_tx;
    h->rows_per_block = best;
    const float reg_ms = time_steps(2, regular);
    drop_graph(h);
    float pers_ms = 1e30f;
    int pers_r = 0;
    for (int R = 1; R <= 8 && rc == TEUK_OK; R *= 2) {
      h->kernel_family = 3;
      h->rows_per_block = R;
      h->threads_theta = 0;
      const float ms = time_steps(2, [&](int outer) { return dispatch_persist(h, outer, 0); });
      if (rc == TEUK_ERR_INVALID_ARG) {  // the blocks of this shape cannot all be resident
        rc = TEUK_OK;
        continue;
      }
      if (ms < pers_ms) {
        pers_ms = ms;
        pers_r = R;
      }
    }
    if (rc == TEUK_OK && pers_r > 0 && pers_ms < reg_ms) {
      // outer steps per launch: one launch per step against one launch for eight
      h->rows_per_block = pers_r;
      const float one = time_steps(8, [&](int outer) {
        for (int t = 0; t < outer; ++t) {
          const int r = dispatch_persist(h, 1, 0);
          if (r != TEUK_OK) return r;
        }
        return (int)TEUK_OK;
      });
      const float eight = time_steps(8, [&](int outer) { return dispatch_persist(h, outer, 0); });
      best_f = 3;
      best = pers_r;
      best_tx = 0;
      best_v = 0;
      best_p = eight < one ? 8 : 1;
    }
  }
  h->ring = ring;
  cudaMemcpyAsync(h->u, saved, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->status, &status, sizeof(status), cudaMemcpyHostToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  cudaFree(saved);
  if (rc == TEUK_OK) rc = sync_filter_counter(h);
  h->persist_steps = best_p;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->timing = timing;
  h->launches = launches;
  h->rows_per_block = best;
  h->threads_theta = best_tx;
  h->kernel_variant = best_v;
  h->kernel_family = best_f;
  drop_graph(h);
  if (rows_per_block) *rows_per_block = best;
  return rc;
}

int teuk_set_persistent(teuk_t h, int threads_theta, int rows_per_block, int steps_per_launch) {
  if (!h || rows_per_block < 1 || rows_per_block > 8 || steps_per_launch < 1 || steps_per_launch > 4096)
    return invalid(h, "persistent: 1 <= rows_per_block <= 8, 1 <= steps_per_launch <= 4096");
  if (threads_theta != 0 && (threads_theta < 32 || threads_theta % 32 != 0 || threads_theta * rows_per_block > 256))
    return invalid(h, "persistent: threads_theta 0 or a multiple of 32 with threads_theta * rows <= 256");
  if (h->engine == 1) return invalid(h, "persistent: not on the integer engine");
  h->kernel_family = 3;
  h->kernel_variant = 0;
  h->threads_theta = threads_theta;
  h->rows_per_block = rows_per_block;
  h->persist_steps = steps_per_launch;
  drop_graph(h);
  return TEUK_OK;
}

int teuk_launch_shape(teuk_t h, int* threads_theta, int* rows_per_block, int* variant) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  if (h->kernel_family == 1) {  // one warp per 32 columns: reported as 32 threads x 1 row, variant + 3
    if (threads_theta) *threads_theta = 32;
    if (rows_per_block) *rows_per_block = 1;
    if (variant) *variant = 3 + h->kernel_variant;
    return TEUK_OK;
  }
  int tx, ty;
  teuk::row_block_shape(h, tx, ty);
  if (h->kernel_family == 4) {  // fused iterations: reported as variant 10 with R full-step rows
    teuk::fused_shape(h, tx, ty);
    if (threads_theta) *threads_theta = tx;
    if (rows_per_block) *rows_per_block = ty;
    if (variant) *variant = 10;
    return TEUK_OK;
  }
  if (h->kernel_family == 3) {  // the persistent kernel's block (see persist_impl)
    ty = h->rows_per_block;
    tx = std::min(((h->n_th + 31) / 32) * 32, 256 / ty);
    if (h->threads_theta > 0 && h->threads_theta < tx) tx = h->threads_theta;
  }
  if (threads_theta) *threads_theta = tx;
  if (rows_per_block) *rows_per_block = ty;
  // balanced kernels are reported as variant + 6, the persistent kernel as 9
  if (variant) *variant = h->kernel_family == 3 ? 9 : (h->kernel_family == 2 ? 6 : 0) + h->kernel_variant;
  return TEUK_OK;
}

int teuk_set_launch_shape(teuk_t h, int threads_theta, int rows_per_block, int variant) {
  if (!h || variant < 0 || (variant > 8 && variant != 10)) return TEUK_ERR_INVALID_ARG;
  if (h->engine == 1 && variant >= 3)
    return invalid(h, "launch shape: the integer engine has the rows-per-block kernels only (variants 0..2)");
  if (variant == 10) {
    if (h->is_slab()) return invalid(h, "launch shape: fused iterations are not for slabs");
    if (threads_theta < 32 || threads_theta % 32 != 0 || threads_theta > 128 || rows_per_block < 1 ||
        threads_theta * (rows_per_block + 1) > 256)
      return invalid(h, "launch shape: fused iterations need threads_theta a multiple of 32 up to 128 and "
                        "threads_theta * (rows + 1) <= 256");
    if (!fused_smem_fits(h, rows_per_block))
      return invalid(h, "launch shape: the fused block's rows need more shared memory than a block can have");
    TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
    int rc = settle_state(h);
    if (rc == TEUK_OK) rc = ensure_u2(h);
    if (rc != TEUK_OK) return rc;
    h->kernel_family = 4;
    h->kernel_variant = 0;
    h->threads_theta = threads_theta;
    h->rows_per_block = rows_per_block;
    drop_graph(h);
    return TEUK_OK;
  }
  if (variant >= 6) {
    if (threads_theta < 32 || threads_theta % 32 != 0 || threads_theta > 256)
      return invalid(h, "launch shape: threads_theta a multiple of 32, at most 256");
    h->kernel_family = 2;
    h->kernel_variant = variant - 6;
    h->threads_theta = threads_theta;
    h->rows_per_block = 1;
  } else if (variant < 3) {
    if (threads_theta < 32 || threads_theta % 32 != 0 || rows_per_block < 1 ||
        threads_theta * rows_per_block > 256)
      return invalid(h, "launch shape: threads_theta a multiple of 32, threads_theta * rows <= 256");
    if (h->engine == 1 && !ix_shape_fits(h, rows_per_block))
      return invalid(h, "launch shape: the integer engine's rows need more shared memory than a block can have");
    h->kernel_family = 0;
    h->kernel_variant = variant;
    h->threads_theta = threads_theta;
    h->rows_per_block = rows_per_block;
  } else {
    h->kernel_family = 1;
    h->kernel_variant = variant - 3;
  }
  drop_graph(h);
  return TEUK_OK;
}

int teuk_timing(teuk_t h, int enable) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  drain_timing(h);
  if (h->timing != (enable != 0)) drop_graph(h);  // the graph is captured with or without events
  h->timing = enable != 0;
  h->ms[0] = h->ms[1] = 0;
  h->n_timed[0] = h->n_timed[1] = 0;
  return TEUK_OK;
}

int teuk_kernel_times(teuk_t h, double* ms_half, double* ms_full, int64_t* n_half, int64_t* n_full) {
  if (!h) return TEUK_ERR_INVALID_ARG;
  drain_timing(h);
  if (ms_half) *ms_half = h->ms[0];
  if (ms_full) *ms_full = h->ms[1];
  if (n_half) *n_half = h->n_timed[0];
  if (n_full) *n_full = h->n_timed[1];
  h->ms[0] = h->ms[1] = 0;
  h->n_timed[0] = h->n_timed[1] = 0;
  return TEUK_OK;
}

int teuk_fp64_peak(double* ops_per_second) {
  if (!ops_per_second) return TEUK_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TEUK_ERR_NO_DEVICE;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8, iters = 4096;
  double* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)threads * blocks * sizeof(double)) != cudaSuccess) return TEUK_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    fp64_peak_kernel<<<blocks, threads>>>(buf, 0.999999, 1e-7, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return TEUK_ERR_CUDA;
  *ops_per_second = (double)threads * blocks * iters * 8 / (best * 1e-3);
  return TEUK_OK;
}

int teuk_mw_eval(int op, int words, int device, const double* a, const double* b, double* out, int64_t n) {
  if (!a || !b || !out || n < 0 || op < 0 || op > 12) return TEUK_ERR_INVALID_ARG;
  switch (words) {
    case 1: return teuk::mw_eval_w1(op, device, a, b, out, n);
    case 2: return teuk::mw_eval_w2(op, device, a, b, out, n);
    case 4: return teuk::mw_eval_w4(op, device, a, b, out, n);
    default: return TEUK_ERR_INVALID_ARG;
  }
}

}  // extern "C"
