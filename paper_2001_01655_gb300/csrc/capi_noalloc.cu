// Allocation-free variant of the FP32 level-0 operator apply (tomg_fine_apply_f32_noalloc).
//
// Who needs it: callers that must not allocate device memory on the path where they apply the
// operator - code whose device memory is owned by another allocator or a fixed arena, latency-
// critical loops that cannot afford the device-wide synchronisation cudaFree implies, and code
// that runs between other asynchronous work it must not stall.  The regular tomg_level_apply
// stages its FP32 vectors in library-allocated buffers; this variant stages them in one
// fixed-size array that lives in the library's own device image instead.
//
// The staging array is a file-scope __device__ array: every GPU that loads the library holds
// it (8 MiB) until the process exits.  Host code cannot use the array's name as an address, so
// the device address is looked up with cudaGetSymbolAddress once per device (on the first call
// on that device, with that device current) and passed to the kernels.
#include <mutex>
#include <new>

#include "solver.h"

namespace tomg {
namespace {

constexpr int64_t kNoallocMaxDofs = int64_t(1) << 20;  // 1,048,576 DOFs
constexpr int kMaxDevices = 64;

// x (FP32) in [0, n), A x (FP32) in [kNoallocMaxDofs, kNoallocMaxDofs + n)
static __device__ __align__(256) float g_noalloc_scratch[2 * kNoallocMaxDofs];

std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[kMaxDevices] = {nullptr};

float* scratch_for_current_device(int device) {
  if (device < 0 || device >= kMaxDevices)
    TOMG_THROW(TOMG_E_INVALID, "device %d outside the supported range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      TOMG_THROW(TOMG_E_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
                 cudaGetErrorString(e));
    g_noalloc_ptr[device] = static_cast<float*>(p);
  }
  return g_noalloc_ptr[device];
}

}  // namespace
}  // namespace tomg

extern "C" tomg_status tomg_fine_apply_f32_noalloc(tomg_problem* P, const double* x, double* y) {
  // as at every entry point: a non-sticky error left behind by another library's runtime call
  // in this thread would otherwise surface at the first launch check of this call
  (void)cudaGetLastError();
  try {
    if (!P || !x || !y) TOMG_THROW(TOMG_E_INVALID, "null argument");
    if (!P->have_density) TOMG_THROW(TOMG_E_INVALID, "no density set");
    if (P->n > tomg::kNoallocMaxDofs)
      TOMG_THROW(TOMG_E_INVALID,
                 "problem has %lld DOFs; the allocation-free apply supports at most %lld",
                 (long long)P->n, (long long)tomg::kNoallocMaxDofs);
    CK(cudaSetDevice(P->ctx->device));
    float* s = tomg::scratch_for_current_device(P->ctx->device);
    float* x32 = s;
    float* y32 = s + tomg::kNoallocMaxDofs;
    cudaStream_t st = P->ctx->stream;
    // every scratch entry the apply reads is written first by the cast, so nothing is cleared
    tomg::cast_f64_f32(st, x, x32, P->n);
    const tomg::Ebe op{P->dim, P->nx, P->ny, P->nz, P->Ke32.p, P->E32.p, P->mask.p, 0,
                       P->Ke32_host.data()};
    tomg::ebe_op<float>(st, tomg::MODE_APPLY, op, x32, y32, nullptr, nullptr, 0.0, nullptr, nullptr);
    tomg::cast_f32_f64(st, y32, y, P->n);
    return TOMG_OK;
  } catch (const tomg::Error& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    tomg::set_error("host allocation failed");
    return TOMG_E_OOM;
  } catch (...) {
    tomg::set_error("unexpected internal error");
    return TOMG_E_CUDA;
  }
}
