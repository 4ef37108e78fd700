// Lax-Wendroff iterations for callers that must not allocate device memory.
//
// The regular path keeps the half-step rows of every iteration in a buffer that
// teuk_create allocates per handle. Some callers cannot let a library allocate while they
// step: applications whose device memory is owned by a pool of their own (a framework's
// caching allocator, a fixed budget carved out at start-up), and latency-sensitive loops
// that cannot afford cudaMalloc / cudaFree, which may synchronise the whole device and stall
// every other stream. teuk_substep_noalloc serves them: the caller passes the input and
// output state buffers it owns, the constant tables come from an existing handle, and the
// half-step rows live in one fixed array in this file, which every GPU that loads the
// library holds until the process exits. Nothing is allocated per call.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "teuk_internal.h"

namespace {

// Room for the half-step rows: 4 components x w words x (n_r - 1) rows x pitch doubles.
constexpr size_t kScratchDoubles = size_t(1) << 21;  // 16 MiB per GPU
static __device__ __align__(256) double g_halfstep_rows[kScratchDoubles];

// Device address of g_halfstep_rows, looked up on the first call on each device.
constexpr int kMaxDevices = 128;
double* g_rows_ptr[kMaxDevices] = {};
std::mutex g_rows_mutex;

int rows_on_current_device(teuk_s* h, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return teuk::cuda_fail(h, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    h->last_error = "teuk_substep_noalloc: device index out of range";
    return TEUK_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_rows_mutex);
  if (!g_rows_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_halfstep_rows);
    if (e != cudaSuccess) return teuk::cuda_fail(h, e, "cudaGetSymbolAddress(g_halfstep_rows)");
    g_rows_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_rows_ptr[dev];
  return TEUK_OK;
}

}  // namespace

extern "C" int teuk_substep_noalloc(teuk_t h, const double* u_in, double* u_out, int64_t n_iterations) {
  if (!h || !u_in || !u_out || n_iterations < 0) return TEUK_ERR_INVALID_ARG;
  if (h->is_slab() && n_iterations > 1) {
    h->last_error = "teuk_substep_noalloc: a slab takes one iteration per call (halo rows between iterations)";
    return TEUK_ERR_INVALID_ARG;
  }
  if (h->dissipating()) {
    h->last_error = "teuk_substep_noalloc: the outer-step dissipation or theta filter needs the handle's own buffers";
    return TEUK_ERR_INVALID_ARG;
  }
  const size_t needed = (size_t)4 * h->W * (size_t)(h->n_r - 1) * h->pitch;
  if (needed > kScratchDoubles) {
    h->last_error = "teuk_substep_noalloc: the half-step rows need " + std::to_string(needed) +
                    " doubles, more than the fixed " + std::to_string(kScratchDoubles) +
                    " (4 * words * (n_r - 1) * pitch must not exceed 2^21)";
    return TEUK_ERR_INVALID_ARG;
  }
  // The integer engine copies rows of u_in into shared memory with bulk asynchronous copies,
  // which need 16-byte aligned sources; rows are multiples of 128 bytes, so the base pointers
  // decide. Refused here instead of faulting inside a kernel.
  if (((uintptr_t)u_in | (uintptr_t)u_out) & 15u) {
    h->last_error = "teuk_substep_noalloc: u_in and u_out must be 16-byte aligned";
    return TEUK_ERR_INVALID_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return teuk::cuda_fail(h, e, "cudaGetDevice");
  if (dev != h->device) {
    h->last_error = "teuk_substep_noalloc: the handle's device must be current";
    return TEUK_ERR_INVALID_ARG;
  }
  double* rows = nullptr;
  int rc = rows_on_current_device(h, &rows);
  if (rc != TEUK_OK) return rc;
  // Phi = Pi = 0 on the first and last r* rows of the output (Sec. 3.B): the kernels never
  // write them, so a separate output buffer gets them here.
  const size_t row_bytes = (size_t)h->pitch * sizeof(double);
  const size_t plane_bytes = (size_t)h->n_r * row_bytes;
  const int planes = 4 * h->W;
  TEUK_CUDA(h, cudaMemset2DAsync(u_out, plane_bytes, 0, row_bytes, planes, h->stream));
  TEUK_CUDA(h, cudaMemset2DAsync(u_out + (size_t)(h->n_r - 1) * h->pitch, plane_bytes, 0, row_bytes, planes,
                                 h->stream));
  const double* src = u_in;
  for (int64_t t = 0; t < n_iterations; ++t) {
    switch (h->W) {
      case 1: rc = teuk::substep_buffers_w1(h, src, u_out, rows); break;
      case 2: rc = teuk::substep_buffers_w2(h, src, u_out, rows); break;
      default: rc = teuk::substep_buffers_w4(h, src, u_out, rows); break;
    }
    if (rc != TEUK_OK) return rc;
    src = u_out;  // later iterations run in place on the output
  }
  return TEUK_OK;
}
