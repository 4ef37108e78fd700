// Integer-engine kernels of one precision (built once for double-double, once for
// quad-double: TEUK_WORDS = 2 or 4), in a unit of their own so that they compile in parallel
// with the FP64-transform kernels of teuk_prec.cu: conversion of the coefficient tables, the
// step's two kernels per Lax-Wendroff iteration (Eqs. lw1, lw2) and the batched executor.
#include <cstring>

#include "teuk_internal.h"
#include "teuk_kernels.cuh"
#include "teuk_ix.cuh"

#if TEUK_WORDS != 2 && TEUK_WORDS != 4
#error "teuk_ixk.cu is built for TEUK_WORDS = 2 or 4"
#endif

#define TEUK_CAT2(a, b) a##b
#define TEUK_CAT(a, b) TEUK_CAT2(a, b)
#define TEUK_SUFFIX(name) TEUK_CAT(name, TEUK_WORDS)

namespace teuk {
namespace TEUK_SUFFIX(ixk_w) {

constexpr int W = TEUK_WORDS;
constexpr int U = IxT<W>::kU4;

// The engine's coefficient tables, converted once from the folded multi-word tables (planes
// 0..7), then plane 5 -> (H5 A2, H5 A1 cot theta_j) as planes 5 and 8 (ix_fold_kernel).
int tables(teuk_s* h) {
  const size_t ws = (size_t)h->n_r * h->pitch, hs = (size_t)(h->n_r - 1) * h->pitch;
  const size_t ncn = (size_t)kIxPlanes * ws, nch = (size_t)kIxPlanes * hs, total = ncn + nch;
  TEUK_CUDA(h, cudaMalloc(&h->ix_m, total * U * sizeof(uint4)));
  TEUK_CUDA(h, cudaMalloc(&h->ix_e, total * sizeof(int)));
  ix_table_kernel<W><<<(unsigned)((8 * ws + 255) / 256), 256, 0, h->stream>>>(h->cn, ws, ws, 8 * ws, h->ix_m, h->ix_e);
  ix_table_kernel<W><<<(unsigned)((8 * hs + 255) / 256), 256, 0, h->stream>>>(h->ch, hs, hs, 8 * hs,
                                                                             h->ix_m + U * ncn, h->ix_e + ncn);
  ix_fold_kernel<W><<<(unsigned)((ws + 255) / 256), 256, 0, h->stream>>>(h->ix_m, h->ix_e, ws, h->pitch, h->n_th,
                                                                        h->lfac);
  ix_fold_kernel<W><<<(unsigned)((hs + 255) / 256), 256, 0, h->stream>>>(h->ix_m + U * ncn, h->ix_e + ncn, hs,
                                                                        h->pitch, h->n_th, h->lfac);
  TEUK_CUDA(h, cudaGetLastError());
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

// The half and full kernels of register-budget variant V for the block shape blk: rows of
// the row family, shared rows in the engine's format.
template <int V>
int launch_pair(teuk_s* h, const StepArgs& sa, dim3 blk) {
  const int nh = h->n_r - 1, nf = h->n_r - 2;
  const size_t ncn = (size_t)kIxPlanes * h->n_r * h->pitch;
  const int gs = h->n_th + 2 * h->radius;
  const long long key = ((long long)V << 40) | ((long long)blk.x << 20) | blk.y;
  if (h->ix_stage_key != key) {
    // stage in shared memory as much as keeps as many blocks per SM resident: nothing (0), the
    // table rows (1), the table and state rows (3); the full step's footprint is the larger
    const int opts[3] = {0, 1, 3};
    int occ[3] = {0, 0, 0}, dev = 0, optin = 0;
    TEUK_CUDA(h, cudaGetDevice(&dev));
    TEUK_CUDA(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (int k = 0; k < 3; ++k) {
      const size_t b = ix_smem_bytes<W>((int)blk.y, gs, h->pitch, opts[k], true);
      if (b > (size_t)optin) continue;
      TEUK_CUDA(h, cudaFuncSetAttribute(full_ix_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[k], full_ix_kernel<W, V>, (int)(blk.x * blk.y), b) !=
          cudaSuccess) {
        cudaGetLastError();
        occ[k] = 0;
      }
    }
    h->ix_stage = 0;
    for (int k = 1; k < 3; ++k)
      if (occ[k] > 0 && occ[k] >= occ[0]) h->ix_stage = opts[k];
    h->ix_stage_key = key;
  }
  // the give-up test needs the copies: it stages the table rows at least
  const int stage = h->test_stall_block >= 0 && h->ix_stage == 0 ? 1 : h->ix_stage;
  IxArgs x{sa, h->ix_m, h->ix_e, h->ix_m + U * ncn, h->ix_e + ncn, stage, h->wait_log2, h->test_stall_block};
  const size_t ism_h = ix_smem_bytes<W>((int)blk.y, gs, h->pitch, stage, false);
  const size_t ism_f = ix_smem_bytes<W>((int)blk.y, gs, h->pitch, stage, true);
  {
    int dev = 0, optin = 0;
    TEUK_CUDA(h, cudaGetDevice(&dev));
    TEUK_CUDA(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (ism_f > (size_t)optin) {
      h->last_error = "launch shape: the engine's rows need more shared memory than a block can have";
      return TEUK_ERR_INVALID_ARG;
    }
  }
  TEUK_CUDA(h, cudaFuncSetAttribute(half_ix_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism_h));
  TEUK_CUDA(h, cudaFuncSetAttribute(full_ix_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism_f));
  cudaEvent_t ev = nullptr;
  time_begin(h, &ev);
  half_ix_kernel<W, V><<<(nh + blk.y - 1) / blk.y, blk, ism_h, h->stream>>>(x);
  time_end(h, 0, ev);
  time_begin(h, &ev);
  full_ix_kernel<W, V><<<(nf + blk.y - 1) / blk.y, blk, ism_f, h->stream>>>(x);
  time_end(h, 1, ev);
  h->launches += 2;
  TEUK_CUDA(h, cudaGetLastError());
  return TEUK_OK;
}

}  // namespace ixk_wN
using namespace TEUK_SUFFIX(ixk_w);

int TEUK_SUFFIX(ix_tables_w)(teuk_s* h) { return tables(h); }
int TEUK_SUFFIX(ix_launch_pair_w)(teuk_s* h, const StepArgs& sa, dim3 blk, int variant) {
  switch (variant) {
    case 1: return launch_pair<1>(h, sa, blk);
    case 2: return launch_pair<2>(h, sa, blk);
    default: return launch_pair<0>(h, sa, blk);
  }
}

// Shared memory of `rows` engine rows without staged tables (launch-shape checks, batches);
// resident blocks per SM and the cooperative launch of batch_ix_kernel (teuk_batch.cu).
size_t TEUK_SUFFIX(ix_row_smem_w)(int rows, int gstride) { return ix_smem_bytes<W>(rows, gstride, 0, 0, true); }
cudaError_t TEUK_SUFFIX(batch_ix_occupancy_w)(int* per_sm, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(batch_ix_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_ix_kernel<W>, 256, smem);
  return e;
}
cudaError_t TEUK_SUFFIX(batch_ix_launch_w)(const BatchArgs& args, const IxArgs* d_ix, int grid, size_t smem,
                                           cudaStream_t st) {
  BatchArgs a = args;
  const IxArgs* p = d_ix;
  void* params[] = {&a, &p};
  return cudaLaunchCooperativeKernel((const void*)batch_ix_kernel<W>, dim3(grid), dim3(256), params, smem, st);
}

}  // namespace teuk

#if TEUK_WORDS == 2
namespace {
// Throughput of the integer engine's product window (ix::mul_window: 10 partial products of
// 32-bit limbs, each a mad.lo.cc / madc.hi.cc pair with its carry), the work unit of the
// engine's roofline: every thread runs 4 independent windows per iteration, each fed back
// into the next so that none can be hoisted.
__global__ void ix_window_peak_kernel(uint32_t* out, uint32_t seed, int iters) {
  uint32_t a[4][4], b[4][4], p[4][5];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[c][k] = seed * (2654435761u + 97u * c + k) + threadIdx.x;
      b[c][k] = seed ^ (40503u * (c + 1) + 7u * k + blockIdx.x);
    }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      ix::mul_window(a[c], b[c], p[c]);
      a[c][0] ^= p[c][4];
      a[c][1] += p[c][3];
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) x ^= p[c][0] ^ p[c][1] ^ p[c][2] ^ p[c][3] ^ p[c][4];
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}
}  // namespace

extern "C" int teuk_int_peak(double* pairs_per_second) {
  if (!pairs_per_second) return TEUK_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TEUK_ERR_NO_DEVICE;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TEUK_ERR_CUDA;
  const int threads = 256, blocks = sms * 8, iters = 2048;
  uint32_t* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)threads * blocks * sizeof(uint32_t)) != cudaSuccess) return TEUK_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    ix_window_peak_kernel<<<blocks, threads>>>(buf, 12345u + rep, iters);
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
  // 4 windows of 10 partial products per iteration and thread
  *pairs_per_second = (double)threads * blocks * iters * 4 * 10 / (best * 1e-3);
  return TEUK_OK;
}
#endif
