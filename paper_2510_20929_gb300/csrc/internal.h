// Internal interfaces shared by the translation units of libptycho (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "ptycho.h"

namespace ptycho {

struct Layout {
  size_t hdr, acc, psi, o, g, h, dPacc, Dp, dP, Sp, Cp, Sdp, valid;
  size_t p0, dUacc, Du, dU, gram;   // orthogonal probe relaxation (K > 0) only
  size_t possum;                     // position-correction sums [B, 5] (FP64)
  size_t p2part;                     // partial step-size sums [B, P2_CHUNKS, 5] (FP64)
  size_t dOe;                        // epoch object accumulator [H, W] (object_per_epoch) or 0
  size_t dft;                        // DFT-matrix chunks of the split-BF16 DFT-GEMM (N <= 128) or 0
  size_t total;
};

// Device pointers of the workspace regions.
struct Ptrs {
  struct WsHeader* hdr;
  float4* acc;
  float2 *psi, *o, *g, *h, *dPacc, *dP, *Cp;
  float *Dp, *Sp, *Sdp;
  int* valid;
  float2 *p0, *dUacc, *dU;
  float* Du;
  double* gram;
  double* possum;
  double* p2part;
  float2* dOe;
  void* dft;
};

size_t align256(size_t b);
// Workspace regions for a minibatch of B positions; K > 0 adds the regions of
// the relaxed primary probe mode with K eigenmodes.
Layout make_layout(const ptycho_dims& d, int B, int K = 0, bool epoch_object = false);
// The layout one LSQML epoch with these options uses.
Layout layout_for(const ptycho_dims& d, const ptycho_lsqml_opts& o);
Ptrs carve(void* ws, const Layout& L);
ptycho_status check_dims(const ptycho_dims* d);
ptycho_status check_opts(const ptycho_lsqml_opts* o);
ptycho_status check_ws(void* ws, size_t have, size_t need);
ptycho_status cuda_status(cudaError_t e);
int grid_for(size_t n, int threads, int cap);
// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

struct BatchArgs;
struct Pass2Args;
struct BatchScalars;
// Launch wrappers (profiled) shared by the entry points.
cudaError_t pass1(int N, const BatchArgs& a, cudaStream_t s, int variant = 0);
cudaError_t pass2(int N, const Pass2Args& a, cudaStream_t s, int variant = 0);
// True when the split-BF16 DFT-GEMM form is built for window N.
bool dft_gemm_supported(int N);
// PTYCHO_OK, or the error for an unknown precision or a measured-intensity
// array that is not 16-byte aligned under BF16X3 (ARG), or a precision not
// built for N (UNSUPPORTED).
ptycho_status check_precision(int N, int precision, const void* meas);
// Fills the DFT chunks of the workspace (once per call of an entry point).
cudaError_t dft_planes(int N, void* dft, cudaStream_t s);
// The per-position pass with the far field on the tensor cores: exit waves,
// k_far_tc, then (unless the mode is the forward model) the overlap-add part.
cudaError_t pass1_dft(int N, const BatchArgs& a, const void* dft, cudaStream_t s);
// The probe-reduction variant used without tuning: the minibatch split over
// four threads per pixel pair, eight positions in flight each (the fastest
// candidate on every workload measured, by up to 2.3x at small windows).
constexpr int kReduceDefault = 3;
// Batch sums of h over the Mc modes starting at plane k0 of each slot (slots
// hold Ms planes), Dp = sum |o|^2 and the illumination maximum. The patch of
// slot i starts at o_s + i * o_stride (complex elements; 0: N * N).
cudaError_t probe_reduce(int NN, int k0, int Mc, int Ms, int nb, const float2* h_s, const float2* o_s,
                         const int* valid, float2* dPacc, int accumulate, float* Dp, const float4* acc, int HW,
                         BatchScalars* sc, cudaStream_t s, int o_stride = 0, int variant = kReduceDefault);
cudaError_t norm_probe(int NN, int M, const float2* dPacc, const float* Dp, const float2* probe, float delta_p,
                       int update_probe, const BatchScalars* sc, float2* dP, float2* Cp, float* Sdp,
                       cudaStream_t s);
cudaError_t probe_update(int NN, int M, float2* probe, const float2* dP, float* Sp, int update_probe,
                         const BatchScalars* sc, BatchScalars* sc_next, cudaStream_t s, float4* clear = nullptr,
                         size_t nclear = 0);
cudaError_t init_epoch(int NN, int M, const float2* probe, float* Sp, struct WsHeader* hdr, cudaStream_t s);
// True when a minibatch's object tiles are cheaper to visit than the whole
// object plane: the illumination maximum then scans only those tiles
// (tile_illum_max) and the accumulator is cleared tile by tile (clear_acc).
bool tiles_cheaper(int nb, int N, int H, int W);
cudaError_t tile_illum_max(const ptycho_dims& d, int nb, int b0, const float* pos, const int32_t* order,
                           const int* valid, const float4* acc, BatchScalars* sc, cudaStream_t s);
cudaError_t clear_acc(bool tiles, const ptycho_dims& d, int nb, int b0, const float* pos, const int32_t* order,
                      const int* valid, float4* acc, cudaStream_t s);
// One LSQML epoch on stream s with workspace ws (arguments already validated).
// Measured intensities that arrive during the epoch: minibatch b waits for
// ready[b] (its positions' intensities are in `meas` from then on) and reads
// `meas` instead of the epoch's own pointer.
struct MeasSwitch {
  const float* meas = nullptr;
  const cudaEvent_t* ready = nullptr;   // one per minibatch
};
ptycho_status run_epoch(const ptycho_dims& d, float2* obj, float2* probe, float* pos, const float* meas,
                        const int32_t* order, const ptycho_lsqml_opts& o, double* loss, double* alpha, void* ws,
                        cudaStream_t s, const MeasSwitch* later = nullptr);

// One LSQML epoch with orthogonal probe relaxation (arguments already validated).
ptycho_status run_epoch_opr(const ptycho_dims& d, const ptycho_opr_opts& r, float2* obj, float2* U, float* wts,
                            float2* P_rest, const float* pos, const float* meas, const int32_t* order,
                            const ptycho_lsqml_opts& o, double* loss, double* alpha, void* ws, cudaStream_t s);
ptycho_status check_opr_opts(const ptycho_opr_opts* r);

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
