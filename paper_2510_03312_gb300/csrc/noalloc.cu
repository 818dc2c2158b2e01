// noalloc.cu -- forward rendering without any device allocation.
//
// Some callers cannot allocate device memory at the point where they render:
// plugin hosts and embedded renderers that hand out no allocator, processes
// that run under a pre-sized memory pool where a cudaMalloc would fail or
// fragment it, and real-time loops that forbid allocation after start-up.
// For them this file provides ubs_render_fwd_static: the same preprocess ->
// bin_sort -> render_fwd sequence as the regular entry points, with the
// workspace taken from a fixed array in the library's own device memory
// instead of a caller-supplied buffer.
//
// The array (kStaticScratchBytes = 32 MiB) is a file-scope __device__
// variable: every GPU on which the library's module for this file is loaded
// holds it until the process exits.  Its device address is looked up once
// per device (cudaGetSymbolAddress with that device current) on the first
// call made on that device, so that first call should happen before any
// stream capture begins.  All calls on a device share the one array and it
// keeps the previous call's contents; the steps reset what must start at
// zero themselves.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array.  The cached address
// is never looked up again, so a device reset (cudaDeviceReset) after the
// first call on that device is not supported.
//
// What the device-side steps report (an instance capacity too small for the
// scene, with the count it needs) sits in the array's status header, which
// ubs_read_status_static copies out, as ubs_read_status does for a
// caller-owned workspace.
#include <atomic>

#include "ubs.h"
#include <cuda_runtime.h>

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_ubs_static_scratch[kStaticScratchBytes];

std::atomic<void*> g_scratch_addr[kMaxDevices];  // device address, per device ordinal

void* scratch_for_current_device(ubs_status* st) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *st = UBS_ERR_CUDA;
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *st = UBS_ERR_INVALID_ARG;
    return nullptr;
  }
  void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (p) return p;
  // the array's name is a host-side stand-in: its device address must be
  // looked up with this device current
  const cudaError_t e = cudaGetSymbolAddress(&p, g_ubs_static_scratch);
  if (e != cudaSuccess || p == nullptr) {
    *st = UBS_ERR_CUDA;
    return nullptr;
  }
  g_scratch_addr[dev].store(p, std::memory_order_release);
  return p;
}

}  // namespace

extern "C" ubs_status ubs_render_fwd_static(const ubs_problem* problem, float* image, cudaStream_t stream) {
  if (!problem || !image) return UBS_ERR_INVALID_ARG;
  const size_t need = ubs_workspace_size(problem);
  if (need == 0) return UBS_ERR_INVALID_ARG;
  if (need > kStaticScratchBytes) return UBS_ERR_WORKSPACE;  // the problem is larger than the fixed scratch
  ubs_status st = UBS_OK;
  void* ws = scratch_for_current_device(&st);
  if (!ws) return st;
  st = ubs_preprocess(problem, ws, kStaticScratchBytes, stream);
  if (st != UBS_OK) return st;
  st = ubs_bin_sort(problem, ws, kStaticScratchBytes, stream);
  if (st != UBS_OK) return st;
  return ubs_render_fwd(problem, ws, kStaticScratchBytes, image, stream);
}

extern "C" ubs_status ubs_read_status_static(const ubs_problem* problem, ubs_device_status* out,
                                             cudaStream_t stream) {
  if (!problem || !out) return UBS_ERR_INVALID_ARG;
  const size_t need = ubs_workspace_size(problem);
  if (need == 0) return UBS_ERR_INVALID_ARG;
  if (need > kStaticScratchBytes) return UBS_ERR_WORKSPACE;
  ubs_status st = UBS_OK;
  void* ws = scratch_for_current_device(&st);
  if (!ws) return st;
  return ubs_read_status(problem, ws, kStaticScratchBytes, out, stream);
}
