// Internal interfaces shared by the translation units of libptycho (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "ptycho.h"

namespace ptycho {

struct Layout {
  size_t hdr, acc, psi, o, g, h, dPacc, Dp, dP, Sp, Cp, Sdp, valid, total;
};

size_t align256(size_t b);
Layout make_layout(const ptycho_dims& d, int B);
ptycho_status check_dims(const ptycho_dims* d);
ptycho_status check_opts(const ptycho_lsqml_opts* o);
// One LSQML epoch on stream s with workspace ws (arguments already validated).
ptycho_status run_epoch(const ptycho_dims& d, float2* obj, float2* probe, const float* pos, const float* meas,
                        const int32_t* order, const ptycho_lsqml_opts& o, double* loss, double* alpha, void* ws,
                        cudaStream_t s);

// Byte-exact key of a captured launch sequence (dimensions, options, pointers).
struct GraphKey {
  std::vector<unsigned char> bytes;
  template <class T>
  GraphKey& add(const T& v) {
    const unsigned char* p = (const unsigned char*)&v;
    bytes.insert(bytes.end(), p, p + sizeof(T));
    return *this;
  }
};

// Worker streams of the current device (created on first use, never destroyed).
ptycho_status worker_streams(cudaStream_t** out, int* count);

// Captures body(origin) into a CUDA graph on the first call with this key
// (on an internal origin stream), then launches the cached executable graph
// on `caller`. Later calls with the same key only launch the graph.
template <class F>
ptycho_status run_graphed(const GraphKey& key, cudaStream_t caller, F&& body);

ptycho_status graph_lookup(const GraphKey& key, cudaGraphExec_t* exec);
ptycho_status graph_store(const GraphKey& key, cudaGraphExec_t exec);
ptycho_status capture_origin(cudaStream_t* origin);

template <class F>
ptycho_status run_graphed(const GraphKey& key, cudaStream_t caller, F&& body) {
  cudaGraphExec_t exec = nullptr;
  if (graph_lookup(key, &exec) == PTYCHO_OK && exec)
    return cudaGraphLaunch(exec, caller) == cudaSuccess ? PTYCHO_OK : PTYCHO_ERR_CUDA;
  cudaStream_t origin = nullptr;
  ptycho_status st = capture_origin(&origin);
  if (st != PTYCHO_OK) return st;
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PTYCHO_ERR_CUDA;
  st = body(origin);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(origin, &graph);
  if (st != PTYCHO_OK || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return st != PTYCHO_OK ? st : PTYCHO_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return PTYCHO_ERR_CUDA;
  if ((st = graph_store(key, exec)) != PTYCHO_OK) {
    cudaGraphExecDestroy(exec);
    return st;
  }
  return cudaGraphLaunch(exec, caller) == cudaSuccess ? PTYCHO_OK : PTYCHO_ERR_CUDA;
}

}  // namespace ptycho
