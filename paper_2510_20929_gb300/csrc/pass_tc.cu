// The split-BF16 DFT-GEMM form of the per-position pass (windows 32, 64 and
// 128): the exit-wave part of k_pass1, the tensor-core far-field stage
// k_far_tc, and the overlap-add part of k_pass1, plus the DFT-matrix fill.
#include "kernels.cuh"
#include "kernels_tc.cuh"
#include "launch.h"

namespace ptycho {

template <int N>
size_t dft_plane_bytes() {
  return FarTc<N>::dft_bytes;
}

template <int N>
cudaError_t launch_dft_planes(void* dft, cudaStream_t s) {
  constexpr int n = FarTc<N>::NCH * FarTc<N>::MT * 16;
  k_dft_planes<N><<<(n + 255) / 256, 256, 0, s>>>((uint16_t*)dft);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_pass1_part(const BatchArgs& a, cudaStream_t s, int part) {
  constexpr int T = Threads<N>::T;
  if (a.opr_U) return part == 1 ? launch_pass1_t<N, T, true, 1>(a, s) : launch_pass1_t<N, T, true, 2>(a, s);
  return part == 1 ? launch_pass1_t<N, T, false, 1>(a, s) : launch_pass1_t<N, T, false, 2>(a, s);
}

// Persistent: as many CTAs as fit at once (one per SM at N = 128), at most one per position.
template <int N>
cudaError_t launch_far_tc(const BatchArgs& b, const void* dft, cudaStream_t s) {
  using C = FarTc<N>;
  static unsigned long long done = 0;
  cudaError_t e = smem_optin(k_far_tc<N>, C::bytes, &done);
  if (e != cudaSuccess) return e;
  if (b.nb <= 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_far_tc<N>, C::T, C::bytes)) != cudaSuccess)
    return e;
  const int grid = b.nb < sms * (per_sm > 0 ? per_sm : 1) ? b.nb : sms * (per_sm > 0 ? per_sm : 1);
  FarArgs a;
  a.H = b.H; a.W = b.W; a.M = b.M; a.J = b.J;
  a.pos = b.pos; a.order = b.order; a.b0 = b.b0; a.nb = b.nb; a.mode = b.mode; a.eps = b.eps;
  a.meas = b.meas; a.psi_s = b.psi_s; a.dft = (const uint16_t*)dft;
  a.ipred = b.ipred; a.loss = b.loss; a.status = b.status;
  return launch_pdl(k_far_tc<N>, dim3(grid), dim3(C::T), C::bytes, s, a);
}

#define PTYCHO_TC_INSTANCES(N)                                                     \
  template size_t dft_plane_bytes<N>();                                           \
  template cudaError_t launch_dft_planes<N>(void*, cudaStream_t);                 \
  template cudaError_t launch_pass1_part<N>(const BatchArgs&, cudaStream_t, int); \
  template cudaError_t launch_far_tc<N>(const BatchArgs&, const void*, cudaStream_t);
PTYCHO_TC_INSTANCES(32)
PTYCHO_TC_INSTANCES(64)
PTYCHO_TC_INSTANCES(128)

}  // namespace ptycho
