// Batched serving of several independent reconstructions, and the stream and
// CUDA-graph plumbing shared with the single-reconstruction epoch.
//
// Each reconstruction of a batched call gets its own section of the workspace
// and runs its epoch on one of the device's worker streams; the caller's stream
// forks to the workers and joins them again, so the minibatch kernels of
// different reconstructions overlap on the GPU and fill the SMs that one
// reconstruction's minibatch leaves idle. With PTYCHO_FLAG_GRAPH the whole
// fork/join launch sequence is captured once into a CUDA graph and replayed as
// a single graph launch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.h"
#include "ptycho.h"

namespace ptycho {
namespace {

constexpr int kMaxDevices = 64;
constexpr int kWorkers = 16;
constexpr int kMaxGraphs = 16;

struct DeviceStreams {
  bool ready = false;
  cudaStream_t origin = nullptr;
  cudaStream_t workers[kWorkers] = {};
};

std::mutex g_mu;
DeviceStreams g_dev[kMaxDevices];

struct GraphEntry {
  int dev;
  std::vector<unsigned char> key;
  cudaGraphExec_t exec;
  unsigned long long last_use;
};
std::vector<GraphEntry> g_graphs;
unsigned long long g_clock = 0;

ptycho_status device_streams(DeviceStreams** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PTYCHO_ERR_UNSUPPORTED;
  DeviceStreams& d = g_dev[dev];
  if (!d.ready) {
    if (cudaStreamCreateWithFlags(&d.origin, cudaStreamNonBlocking) != cudaSuccess) return PTYCHO_ERR_CUDA;
    for (int i = 0; i < kWorkers; ++i)
      if (cudaStreamCreateWithFlags(&d.workers[i], cudaStreamNonBlocking) != cudaSuccess) return PTYCHO_ERR_CUDA;
    d.ready = true;
  }
  *out = &d;
  return PTYCHO_OK;
}

}  // namespace

ptycho_status worker_streams(cudaStream_t** out, int* count) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceStreams* d = nullptr;
  ptycho_status st = device_streams(&d);
  if (st != PTYCHO_OK) return st;
  *out = d->workers;
  *count = kWorkers;
  return PTYCHO_OK;
}

ptycho_status capture_origin(cudaStream_t* origin) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceStreams* d = nullptr;
  ptycho_status st = device_streams(&d);
  if (st != PTYCHO_OK) return st;
  *origin = d->origin;
  return PTYCHO_OK;
}

ptycho_status graph_lookup(const GraphKey& key, cudaGraphExec_t* exec) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& e : g_graphs)
    if (e.dev == dev && e.key == key.bytes) {
      e.last_use = ++g_clock;
      *exec = e.exec;
      return PTYCHO_OK;
    }
  *exec = nullptr;
  return PTYCHO_OK;
}

ptycho_status graph_store(const GraphKey& key, cudaGraphExec_t exec) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_graphs.size() >= kMaxGraphs) {
    // evict the least recently used graph; its launches are stream-ordered and
    // destroying an executable graph with launches in flight is allowed
    size_t v = 0;
    for (size_t i = 1; i < g_graphs.size(); ++i)
      if (g_graphs[i].last_use < g_graphs[v].last_use) v = i;
    cudaGraphExecDestroy(g_graphs[v].exec);
    g_graphs.erase(g_graphs.begin() + v);
  }
  g_graphs.push_back({dev, key.bytes, exec, ++g_clock});
  return PTYCHO_OK;
}

// Runs run(i, section_i, worker stream) for every reconstruction, forked from
// and joined back into `origin`; section i of `ws` has section(i) bytes and
// its status word is cleared first.
template <class Section, class Run>
static ptycho_status run_sections(int n, void* ws, cudaStream_t origin, Section&& section, Run&& run) {
  cudaStream_t* workers = nullptr;
  int nw = 0;
  ptycho_status rs = worker_streams(&workers, &nw);
  if (rs != PTYCHO_OK) return rs;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins((size_t)(n < nw ? n : nw), nullptr);
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return PTYCHO_ERR_CUDA;
  for (auto& e : joins)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rs = PTYCHO_ERR_CUDA;
  if (rs == PTYCHO_OK && cudaEventRecord(fork, origin) != cudaSuccess) rs = PTYCHO_ERR_CUDA;
  for (int k = 0; rs == PTYCHO_OK && k < (int)joins.size(); ++k)
    if (cudaStreamWaitEvent(workers[k], fork, 0) != cudaSuccess) rs = PTYCHO_ERR_CUDA;
  char* base = (char*)ws;
  for (int i = 0; rs == PTYCHO_OK && i < n; ++i) {
    if (cudaMemsetAsync(base, 0, 256, workers[i % nw]) != cudaSuccess) {
      rs = PTYCHO_ERR_CUDA;
      break;
    }
    rs = run(i, (void*)base, workers[i % nw]);
    base += section(i);
  }
  for (int k = 0; rs == PTYCHO_OK && k < (int)joins.size(); ++k)
    if (cudaEventRecord(joins[k], workers[k]) != cudaSuccess || cudaStreamWaitEvent(origin, joins[k], 0) != cudaSuccess)
      rs = PTYCHO_ERR_CUDA;
  cudaEventDestroy(fork);
  for (auto& e : joins)
    if (e) cudaEventDestroy(e);
  return rs;
}

}  // namespace ptycho

using namespace ptycho;

extern "C" {

size_t ptycho_workspace_bytes_batched(int32_t n, const ptycho_dims* dims, const ptycho_lsqml_opts* opts) {
  if (n < 1 || !dims || !opts) return 0;
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    if (check_dims(&dims[i]) != PTYCHO_OK || opts[i].batch < 1) return 0;
    if (check_opts(&opts[i]) != PTYCHO_OK) return 0;
    total += layout_for(dims[i], opts[i]).total;
  }
  return total;
}

ptycho_status ptycho_lsqml_epoch_batched(int32_t n, const ptycho_dims* dims, float* const* objects,
                                         float* const* probes, float* const* pos, const float* const* meas,
                                         const int32_t* const* orders, const ptycho_lsqml_opts* opts,
                                         double* losses, void* ws, size_t ws_bytes, void* stream) {
  if (n < 1 || !dims || !objects || !probes || !pos || !meas || !opts) return PTYCHO_ERR_ARG;
  ptycho_status st;
  for (int i = 0; i < n; ++i) {
    if ((st = check_dims(&dims[i])) != PTYCHO_OK) return st;
    if ((st = check_opts(&opts[i])) != PTYCHO_OK) return st;
    if ((st = check_precision(dims[i].N, opts[i].precision, meas[i])) != PTYCHO_OK) return st;
    if (!objects[i] || !probes[i] || (dims[i].J > 0 && (!pos[i] || !meas[i]))) return PTYCHO_ERR_ARG;
  }
  const size_t need = ptycho_workspace_bytes_batched(n, dims, opts);
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < need) return PTYCHO_ERR_WORKSPACE;
  auto section = [&](int i) { return layout_for(dims[i], opts[i]).total; };
  auto run = [&](int i, void* base, cudaStream_t s) {
    ptycho_lsqml_opts oi = opts[i];
    oi.flags = 0;
    return run_epoch(dims[i], (float2*)objects[i], (float2*)probes[i], pos[i], meas[i],
                     orders ? orders[i] : nullptr, oi, losses ? losses + i : nullptr, nullptr, base, s);
  };
  auto body = [&](cudaStream_t origin) { return run_sections(n, ws, origin, section, run); };
  bool graph = true;
  for (int i = 0; i < n; ++i) graph = graph && (opts[i].flags & PTYCHO_FLAG_GRAPH);
  if (!graph) return body((cudaStream_t)stream);
  GraphKey key;
  key.add(n).add(ws).add(losses).add(orders != nullptr);
  for (int i = 0; i < n; ++i)
    key.add(dims[i]).add(opts[i]).add(objects[i]).add(probes[i]).add(pos[i]).add(meas[i]).add(orders ? orders[i] : nullptr);
  return run_graphed(key, (cudaStream_t)stream, body);
}

size_t ptycho_workspace_bytes_opr_batched(int32_t n, const ptycho_dims* dims, const ptycho_opr_opts* opr,
                                          const ptycho_lsqml_opts* opts) {
  if (n < 1 || !dims || !opr || !opts) return 0;
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    const size_t b = ptycho_workspace_bytes_opr(&dims[i], opr[i].K, opts[i].batch);
    if (b == 0) return 0;
    total += b;
  }
  return total;
}

ptycho_status ptycho_lsqml_epoch_opr_batched(int32_t n, const ptycho_dims* dims, const ptycho_opr_opts* opr,
                                             float* const* objects, float* const* U, float* const* w,
                                             float* const* P_rest, const float* const* pos,
                                             const float* const* meas, const int32_t* const* orders,
                                             const ptycho_lsqml_opts* opts, double* losses, void* ws,
                                             size_t ws_bytes, void* stream) {
  if (n < 1 || !dims || !opr || !objects || !U || !w || !pos || !meas || !opts) return PTYCHO_ERR_ARG;
  ptycho_status st;
  for (int i = 0; i < n; ++i) {
    if ((st = check_dims(&dims[i])) != PTYCHO_OK) return st;
    if ((st = check_opr_opts(&opr[i])) != PTYCHO_OK) return st;
    if ((st = check_opts(&opts[i])) != PTYCHO_OK) return st;
    if (opts[i].update_positions || opts[i].object_per_epoch || opts[i].precision != PTYCHO_PRECISION_FP32)
      return PTYCHO_ERR_UNSUPPORTED;
    if (!objects[i] || !U[i] || (dims[i].M > 1 && (!P_rest || !P_rest[i])) ||
        (dims[i].J > 0 && (!pos[i] || !meas[i] || !w[i])))
      return PTYCHO_ERR_ARG;
  }
  const size_t need = ptycho_workspace_bytes_opr_batched(n, dims, opr, opts);
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < need) return PTYCHO_ERR_WORKSPACE;
  auto section = [&](int i) { return make_layout(dims[i], opts[i].batch, opr[i].K).total; };
  auto run = [&](int i, void* base, cudaStream_t s) {
    ptycho_lsqml_opts oi = opts[i];
    oi.flags = 0;
    return run_epoch_opr(dims[i], opr[i], (float2*)objects[i], (float2*)U[i], w[i],
                         P_rest ? (float2*)P_rest[i] : nullptr, pos[i], meas[i], orders ? orders[i] : nullptr, oi,
                         losses ? losses + i : nullptr, nullptr, base, s);
  };
  auto body = [&](cudaStream_t origin) { return run_sections(n, ws, origin, section, run); };
  bool graph = true;
  for (int i = 0; i < n; ++i) graph = graph && (opts[i].flags & PTYCHO_FLAG_GRAPH);
  if (!graph) return body((cudaStream_t)stream);
  GraphKey key;
  key.add(n).add(ws).add(losses).add(orders != nullptr).add(P_rest != nullptr);
  for (int i = 0; i < n; ++i)
    key.add(dims[i]).add(opr[i]).add(opts[i]).add(objects[i]).add(U[i]).add(w[i])
        .add(P_rest ? P_rest[i] : nullptr).add(pos[i]).add(meas[i]).add(orders ? orders[i] : nullptr);
  return run_graphed(key, (cudaStream_t)stream, body);
}

}  // extern "C"
