// Batched execution of many teuk problems in one cooperative launch (include/teuk.h,
// teuk_batch_*): members of uneven size, theta resolution and substep count advance their
// outer steps together; see batch_kernel in teuk_kernels.cuh, and batch_ix_kernel in
// teuk_ix.cuh for members on the integer engine.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "teuk_internal.h"
#include "teuk_kernels.cuh"

struct teuk_batch_s {
  int W = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<teuk_s*> members;               // sorted by k, descending
  std::vector<teuk::BatchMember> host_members;
  teuk::BatchMember* d_members = nullptr;
  int engine = 0;                             // the members' arithmetic engine (all the same)
  std::vector<teuk::IxArgs> host_ix;          // engine 1: the members' engine arguments
  teuk::IxArgs* d_ix = nullptr;
  int* d_item_member = nullptr;
  int* d_active = nullptr;
  int k_max = 0;
  int n_items = 0;
  int grid = 0;
  size_t smem = 0;
  int64_t points_per_outer = 0;
  int64_t launches = 0;
  std::string last_error;
};

namespace {

constexpr int kThreads = 256;
constexpr int64_t kStepsPerLaunch = 200;  // outer steps covered by one cooperative launch

teuk::StepArgs member_args(const teuk_s* h) {
  teuk::StepArgs sa{};
  sa.g = teuk::Geom{h->n_r, h->n_th, h->pitch, h->parity};
  sa.u_in = h->u;
  sa.u_out = h->u;
  sa.uh = h->uh;
  sa.cn = h->cn;
  sa.ch = h->ch;
  sa.wts = h->wts;
  std::memcpy(sa.h4, h->h4_w, sizeof(sa.h4));
  std::memcpy(sa.h2, h->h2_w, sizeof(sa.h2));
  sa.radius = h->radius;
  sa.record = 0;
  sa.i_obs = h->i_obs;
  sa.ring_slot = 0;
  sa.ring_counter = nullptr;
  sa.ring_cap = h->ring_cap;
  sa.ring = h->ring;
  sa.status = h->status;
  return sa;
}

const void* kernel_for(int W) {
  switch (W) {
    case 1: return (const void*)teuk::batch_kernel<1>;
    case 2: return (const void*)teuk::batch_kernel<2>;
    default: return (const void*)teuk::batch_kernel<4>;
  }
}

teuk::IxArgs member_ix_args(const teuk_s* h) {
  const int U = h->W / 2;  // uint4 per engine mantissa: 1 (dd), 2 (qd)
  const size_t ncn = (size_t)teuk::kIxPlanes * h->n_r * h->pitch;
  return teuk::IxArgs{member_args(h), h->ix_m, h->ix_e, h->ix_m + U * ncn, h->ix_e + ncn, 0, 20, -1};
}

void free_batch(teuk_batch_s* b) {
  if (b->d_ix) cudaFree(b->d_ix);
  b->d_ix = nullptr;
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_item_member) cudaFree(b->d_item_member);
  if (b->d_active) cudaFree(b->d_active);
  b->d_members = nullptr;
  b->d_item_member = nullptr;
  b->d_active = nullptr;
}

}  // namespace

extern "C" {

int teuk_batch_create(teuk_batch_t* out, const teuk_t* members, int n_members) {
  if (!out || !members || n_members < 1) return TEUK_ERR_INVALID_ARG;
  *out = nullptr;
  teuk_batch_s* b = new (std::nothrow) teuk_batch_s;
  if (!b) return TEUK_ERR_OOM;
  for (int i = 0; i < n_members; ++i) {
    if (!members[i]) { delete b; return TEUK_ERR_INVALID_ARG; }
    b->members.push_back(members[i]);
  }
  b->W = b->members[0]->W;
  b->device = b->members[0]->device;
  b->stream = b->members[0]->stream;
  b->engine = b->members[0]->engine;
  for (teuk_s* h : b->members)
    if (h->W != b->W || h->device != b->device || h->dissipating() || h->is_slab() || h->engine != b->engine ||
        (h->engine == 1 && !h->ix_m)) {
      delete b;
      return TEUK_ERR_INVALID_ARG;
    }
  // members with more iterations per outer step first: the active items of round q are a prefix
  std::stable_sort(b->members.begin(), b->members.end(), [](const teuk_s* x, const teuk_s* y) { return x->k > y->k; });
  std::vector<int> item_member;
  size_t smem = 0;
  for (size_t idx = 0; idx < b->members.size(); ++idx) {
    teuk_s* h = b->members[idx];
    teuk::BatchMember M{};
    M.a = member_args(h);
    M.k = h->k;
    M.tx = std::min(kThreads, ((h->n_th + 31) / 32) * 32);
    M.rows = std::max(1, kThreads / M.tx);
    M.item_begin = (int)item_member.size();
    const int n_items = (h->n_r - 1 + M.rows - 1) / M.rows;
    for (int t = 0; t < n_items; ++t) item_member.push_back((int)idx);
    b->host_members.push_back(M);
    const int gs = h->n_th + 2 * h->radius;
    if (b->engine == 1) {
      smem = std::max(smem, b->W == 2 ? teuk::ix_row_smem_w2(M.rows, gs) : teuk::ix_row_smem_w4(M.rows, gs));
      b->host_ix.push_back(member_ix_args(h));
    } else {
      smem = std::max(smem, (size_t)M.rows * 2 * b->W * gs * sizeof(double));
    }
    b->k_max = std::max(b->k_max, h->k);
    b->points_per_outer += (int64_t)h->k * h->n_r * h->n_th;
  }
  b->n_items = (int)item_member.size();
  std::vector<int> active(b->k_max, 0);
  for (int q = 0; q < b->k_max; ++q)
    for (const auto& M : b->host_members)
      if (M.k > q) active[q] = std::max(active[q], M.item_begin + (int)((M.a.g.n_r - 1 + M.rows - 1) / M.rows));
  b->smem = smem;
  auto fail = [&](cudaError_t e, const char* what) {
    free_batch(b);
    delete b;
    return teuk::cuda_fail(nullptr, e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_members, b->host_members.size() * sizeof(teuk::BatchMember))) != cudaSuccess)
    return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&b->d_item_member, item_member.size() * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&b->d_active, active.size() * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc");
  cudaMemcpy(b->d_item_member, item_member.data(), item_member.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_active, active.data(), active.size() * sizeof(int), cudaMemcpyHostToDevice);
  int per_sm = 0, sms = 0;
  if (b->engine == 1) {
    if ((e = cudaMalloc(&b->d_ix, b->host_ix.size() * sizeof(teuk::IxArgs))) != cudaSuccess)
      return fail(e, "cudaMalloc");
    e = b->W == 2 ? teuk::batch_ix_occupancy_w2(&per_sm, smem) : teuk::batch_ix_occupancy_w4(&per_sm, smem);
    if (e != cudaSuccess) return fail(e, "batch kernel occupancy");
  } else {
    const void* fn = kernel_for(b->W);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return fail(e, "cudaFuncSetAttribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem)) != cudaSuccess)
      return fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->grid = per_sm * sms;
  if (b->grid < 1) return fail(cudaErrorInvalidConfiguration, "batch kernel does not fit on an SM");
  *out = b;
  return TEUK_OK;
}

int teuk_batch_step(teuk_batch_t b, int64_t n_outer_steps) {
  if (!b || n_outer_steps < 0) return TEUK_ERR_INVALID_ARG;
  // the members' own streams must have finished their earlier work; their engine is the batch's
  for (teuk_s* h : b->members) {
    if (h->engine != b->engine) {
      b->last_error = "a member's arithmetic engine changed after the batch was made";
      return TEUK_ERR_INVALID_ARG;
    }
    if (h->stream != b->stream) cudaStreamSynchronize(h->stream);
  }
  int64_t done = 0;
  while (done < n_outer_steps) {
    const int64_t chunk = std::min(kStepsPerLaunch, n_outer_steps - done);
    for (size_t idx = 0; idx < b->members.size(); ++idx) {
      teuk_s* h = b->members[idx];
      teuk::BatchMember& M = b->host_members[idx];
      M.a = member_args(h);
      M.ring_cap = h->ring ? h->ring_cap : 0;
      M.ring_base = h->n_recorded;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_members, b->host_members.data(),
                                    b->host_members.size() * sizeof(teuk::BatchMember), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e != cudaSuccess) { b->last_error = cudaGetErrorString(e); return TEUK_ERR_CUDA; }
    teuk::BatchArgs args{b->d_members, b->d_item_member, b->d_active, b->k_max, (int)chunk};
    if (b->engine == 1) {
      for (size_t idx = 0; idx < b->members.size(); ++idx) b->host_ix[idx] = member_ix_args(b->members[idx]);
      e = cudaMemcpyAsync(b->d_ix, b->host_ix.data(), b->host_ix.size() * sizeof(teuk::IxArgs),
                          cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess)
        e = b->W == 2 ? teuk::batch_ix_launch_w2(args, b->d_ix, b->grid, b->smem, b->stream)
                      : teuk::batch_ix_launch_w4(args, b->d_ix, b->grid, b->smem, b->stream);
    } else {
      void* params[] = {&args};
      e = cudaLaunchCooperativeKernel(kernel_for(b->W), dim3(b->grid), dim3(kThreads), params, b->smem, b->stream);
    }
    if (e != cudaSuccess) { b->last_error = std::string("cooperative launch: ") + cudaGetErrorString(e); return TEUK_ERR_CUDA; }
    ++b->launches;
    for (teuk_s* h : b->members) {
      h->substeps_done += chunk * h->k;
      if (h->ring) h->n_recorded += chunk;
    }
    done += chunk;
  }
  return TEUK_OK;
}

int teuk_batch_sync(teuk_batch_t b) {
  if (!b) return TEUK_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) { b->last_error = cudaGetErrorString(e); return TEUK_ERR_CUDA; }
  for (teuk_s* h : b->members) {
    int rc = teuk_sync(h);
    if (rc != TEUK_OK) return rc;
  }
  return TEUK_OK;
}

int teuk_batch_info(teuk_batch_t b, int* grid_blocks, int* k_max, int64_t* points_per_outer_step,
                    int64_t* launches) {
  if (!b) return TEUK_ERR_INVALID_ARG;
  if (grid_blocks) *grid_blocks = b->grid;
  if (k_max) *k_max = b->k_max;
  if (points_per_outer_step) *points_per_outer_step = b->points_per_outer;
  if (launches) *launches = b->launches;
  return TEUK_OK;
}

int teuk_batch_destroy(teuk_batch_t b) {
  if (!b) return TEUK_ERR_INVALID_ARG;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
  return TEUK_OK;
}

}  // extern "C"
