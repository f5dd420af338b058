// Allocation-free variant of the LSQML epoch.
//
// Some callers cannot allocate device memory themselves: acquisition-side
// plugins and other host applications that reserve the whole device memory
// budget up front through their own allocator, or real-time pipelines that
// must not call cudaMalloc because it can synchronise the device and stall
// the streams they are feeding. ptycho_lsqml_epoch_static serves them by
// taking its scratch from a fixed file-scope device array instead of a caller
// workspace.
//
// The array is PTYCHO_STATIC_WS_BYTES bytes per device; every GPU that loads
// this part of the library keeps it until the process exits. Its name is only
// a host-side stand-in in host code, so the device address is looked up once
// per device with cudaGetSymbolAddress (the first call on each device does
// that set-up; make it before any stream capture) and handed to the ordinary
// epoch as its workspace.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ptycho.h"

namespace ptycho {
namespace {

__device__ __align__(256) unsigned char g_static_scratch[PTYCHO_STATIC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices];

// Device address of g_static_scratch on the current device (looked up once).
ptycho_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PTYCHO_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PTYCHO_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PTYCHO_OK;
}

}  // namespace
}  // namespace ptycho

extern "C" ptycho_status ptycho_lsqml_epoch_static(const ptycho_dims* dims, float* object, float* probe,
                                                   float* pos, const float* meas, const int32_t* order,
                                                   const ptycho_lsqml_opts* opts, double* loss, double* alpha,
                                                   void* stream) {
  if (!dims || !opts || opts->batch < 1) return PTYCHO_ERR_ARG;
  if (ptycho_workspace_bytes(dims, opts->batch) == 0) return PTYCHO_ERR_UNSUPPORTED;
  const size_t need = ptycho_workspace_bytes_opts(dims, opts);
  if (need == 0) return PTYCHO_ERR_ARG;   // the dimensions are supported: the options are not valid
  if (!object || !probe || (dims->J > 0 && (!pos || !meas))) return PTYCHO_ERR_ARG;
  if (need > (size_t)PTYCHO_STATIC_WS_BYTES) return PTYCHO_ERR_TOO_LARGE;
  void* ws = nullptr;
  ptycho_status st = ptycho::static_scratch(&ws);
  if (st != PTYCHO_OK) return st;
  // the array keeps the previous call's contents: clear its status word first
  // (the epoch itself zeroes every accumulator it reads)
  if ((st = ptycho_workspace_init(ws, need, stream)) != PTYCHO_OK) return st;
  // graph capture would let the driver allocate for the executable graph: run eagerly
  ptycho_lsqml_opts o = *opts;
  o.flags &= ~(int32_t)PTYCHO_FLAG_GRAPH;
  if ((st = ptycho_lsqml_epoch(dims, object, probe, pos, meas, order, &o, loss, alpha, ws, need, stream)) !=
      PTYCHO_OK)
    return st;
  return ptycho_status_read(ws, stream);
}
