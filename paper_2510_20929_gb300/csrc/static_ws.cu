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
// a host-side stand-in in host code, so the device address is looked up with
// cudaGetSymbolAddress once per device and CUDA context (the first call on
// each device does that set-up, and the first call after the context was
// destroyed and created again repeats it, since the module and its array are
// loaded afresh; make that call before any stream capture) and handed to the
// ordinary epoch as its workspace.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ptycho.h"
#include "internal.h"

namespace ptycho {
namespace {

__device__ __align__(256) unsigned char g_static_scratch[PTYCHO_STATIC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];   // id of the context the address belongs to

// Unique id of the current CUDA context (0 when there is none), through the
// driver entry points the runtime hands out (no link-time driver dependency).
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return 0;
    get_current = (GetCurrent)f1;
    get_id = (GetId)f2;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_static_scratch in the current device's context (looked
// up once per context).
ptycho_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PTYCHO_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  unsigned long long ctx = current_context_id();
  if (!ctx || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;   // the lookup also makes the device's primary context current
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PTYCHO_ERR_CUDA;
    if (!ctx) ctx = current_context_id();
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = ctx;
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
  // the argument checks of ptycho_lsqml_epoch, with the same statuses
  ptycho_status st = ptycho::check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if ((st = ptycho::check_opts(opts)) != PTYCHO_OK) return st;
  if ((st = ptycho::check_precision(dims->N, opts->precision, meas)) != PTYCHO_OK) return st;
  if (!object || !probe || (dims->J > 0 && (!pos || !meas))) return PTYCHO_ERR_ARG;
  const size_t need = ptycho_workspace_bytes_opts(dims, opts);
  if (need == 0) return PTYCHO_ERR_ARG;
  if (need > (size_t)PTYCHO_STATIC_WS_BYTES) return PTYCHO_ERR_TOO_LARGE;
  void* ws = nullptr;
  st = ptycho::static_scratch(&ws);
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
