// The split-BF16 DFT-GEMM form of the per-position pass (windows 32, 64 and
// 128): the exit-wave part of k_pass1, the tensor-core far-field stage
// k_far_tc, and the overlap-add part of k_pass1, plus the DFT-matrix fill.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>

#include "kernels.cuh"
#include "kernels_tc.cuh"
#include "launch.h"
#include "ptycho.h"

namespace ptycho {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// Tensor map of a float32 [d2][d1][d0] array, tiles of b1 rows x b0 floats
// (b0 * 4 = 128 bytes) written to shared memory with the 128-byte swizzle.
static bool encode_tiles(TmaDesc* out, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
                         uint32_t b1) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * 4, d0 * d1 * 4};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUtensorMap m;
  static_assert(sizeof(CUtensorMap) == sizeof(TmaDesc), "tensor map size");
  if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  memcpy(out, &m, sizeof(m));
  return true;
}

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

// Tensor map of the object as 8-byte elements [H][W], tiles of (N + 1) rows
// x (N + 2) elements, no swizzle; needs W even and a 16-byte aligned base.
static bool encode_object(TmaDesc* out, const void* base, int H, int W, int N) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)W * 8};
  const cuuint32_t box[2] = {(cuuint32_t)(N + 2), (cuuint32_t)(N + 1)};
  const cuuint32_t es[2] = {1, 1};
  CUtensorMap m;
  if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, const_cast<void*>(base), dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  memcpy(out, &m, sizeof(m));
  return true;
}

template <int N, bool OPR>
static cudaError_t launch_exit_tma(const BatchArgs& a, const TmaDesc& t, cudaStream_t s) {
  using C = ExitTma<N>;
  static unsigned long long done = 0;
  cudaError_t e = smem_optin(k_exit_tma<N, OPR>, C::bytes, &done);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_exit_tma<N, OPR>, dim3(a.nb), dim3(C::T), C::bytes, s, a, t);
}

template <int N>
cudaError_t launch_pass1_part(const BatchArgs& a, cudaStream_t s, int part) {
  if (part == 1 && a.nb > 0 && ((uintptr_t)a.obj & 15) == 0 && a.W % 2 == 0) {
    // the exit waves from object tiles staged by tensor copies (rows of 8-byte
    // elements need a 16-byte row pitch: even widths only)
    TmaDesc t;
    if (!encode_object(&t, a.obj, a.H, a.W, N)) return cudaErrorInvalidValue;
    return a.opr_U ? launch_exit_tma<N, true>(a, t, s) : launch_exit_tma<N, false>(a, t, s);
  }
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
  // exit-wave tiles: 16 complex columns x N rows of image slot * M + k;
  // measured-intensity tiles: 32 columns x N rows of position j
  TmaDesc tpsi, tmeas;
  memset(&tmeas, 0, sizeof(tmeas));
  if (!encode_tiles(&tpsi, b.psi_s, 2 * N, N, (uint64_t)b.nb * b.M, 32, N)) return cudaErrorInvalidValue;
  if (b.mode != MODE_FWD && !encode_tiles(&tmeas, b.meas, N, N, (uint64_t)b.J, 32, N)) return cudaErrorInvalidValue;
  return launch_pdl(k_far_tc<N>, dim3(grid), dim3(C::T), C::bytes, s, a, tpsi, tmeas);
}

// Diagnostic: one warp waits (bounded, about 2^26 SM cycles) on an mbarrier
// that nothing arrives on, then records the timeout status as the tensor-core
// kernels do when a wait gives up.
__global__ void k_selftest_wait(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  const bool done = tc::mbar_wait(&bar, 0, 1ll << 26);
  if (threadIdx.x == 0 && !done) atomicOr(status, FLAG_TIMEOUT);
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

extern "C" ptycho_status ptycho_selftest_wait_timeout(void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < sizeof(ptycho::WsHeader)) return PTYCHO_ERR_WORKSPACE;
  ptycho::k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>(&((ptycho::WsHeader*)ws)->status);
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ERR_CUDA;
}
