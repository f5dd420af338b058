// Device-side helpers shared by the LSQML kernels: argument blocks, bilinear
// sub-pixel sampling (the object's patch extraction / update routine, Pty-Chi
// Sec. 2.1), status flags and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace ptycho {

// Status bits written by kernels into the workspace header (atomicOr).
enum : int {
  FLAG_BOUNDS = 1,     // a position's bilinear tile leaves the object, or an order entry is out of range
  FLAG_NONFINITE = 2,  // a measured intensity is negative or not finite
  FLAG_TIMEOUT = 4,    // a bounded wait on the tensor-core pipeline gave up
};

// What the per-position pass computes after the forward model.
enum : int {
  MODE_FWD = 0,          // intensities only
  MODE_LSQML_GAUSS = 1,  // exit-wave change chi for LSQML, amplitude data term
  MODE_LSQML_POISSON = 2,
  MODE_GRAD_GAUSS = 3,   // gradient of the amplitude data term
  MODE_GRAD_POISSON = 4,
  MODE_VJP = 5,          // gradient given dL/dI
};

// Per-batch scalars (two sets, alternated by batch parity so that one batch's
// update kernel can clear the next batch's set without a race).
struct BatchScalars {
  unsigned int max_illum;  // float bits of max(illumination) (non-negative)
  int count;               // positions whose step sizes were solved
  double sum_alpha_p;      // sum of alpha_P over the batch
  unsigned int max_dp;     // float bits of max(sum_j |o_j|^2) (non-negative)
  int pad0;
  double pad[1];
};

struct WsHeader {
  int status;
  int pad[3];
  BatchScalars sc[2];
};

struct BatchArgs {
  int H, W, M, J;
  const float2* obj;
  const float2* probe;
  const float* pos;
  const float* meas;   // measured intensities, or dL/dI in MODE_VJP
  const int* order;    // may be null: identity
  int b0, nb;          // first entry of `order` in this batch, positions in the batch
  int mode;
  float eps;
  float2* psi_s;       // [B, M, N, N] far fields (unitary scale)
  float2* o_s;         // [B, N, N] object patches
  float2* g_s;         // [B, N, N] sum_k conj(P_k) chi_k
  float2* h_s;         // [B, M, N, N] conj(o) chi_k
  int* valid;          // [B]
  const float* Sp;     // [N, N] sum_k |P_k|^2 (illumination scatter)
  float4* acc;         // [H, W] (dO_acc.re, dO_acc.im, illum, unused) or null
  float2* gobj;        // [H, W] gradient accumulator or null
  float* ipred;        // [J, N, N] predicted intensities or null
  float* gpos;         // [J, 2] position gradient or null
  double* loss;        // scalar accumulator or null
  int* status;
  // Orthogonal probe relaxation: when opr_U is set, the primary mode of
  // position j is sum_m opr_w[j][m] opr_U[m] and `probe` holds the M - 1
  // shared modes; p0_s receives the synthesised primary mode per slot.
  const float2* opr_U; // [K, N, N] or null
  const float* opr_w;  // [J, K]
  int K;
  float2* p0_s;        // [B, N, N] (null in the forward mode)
  // Position correction (LSQML): per slot the sums A11, A12, A22, b1, b2 of
  // the least-squares shift, FP64, accumulated with atomics (or null).
  double* possum;      // [B, 5]
  // Gradient modes: evaluate the forward model and the data term (loss) only,
  // without the back-propagation.
  int loss_only;
};

struct Pass2Args {
  int H, W, M, J;
  const float* pos;
  const int* order;
  int b0, nb;
  const float2* o_s;
  const float2* g_s;
  const float2* h_s;
  const int* valid;
  const float4* acc;
  const float* Sp;
  const float2* Cp;
  const float* Sdp;
  const float2* dP;
  float2* obj;         // object, updated in place by the alpha-weighted scatter
  double* alpha_out;   // [J, 2] or null
  BatchScalars* sc;
  float delta_o;       // relative preconditioner damping
  double lam;
  int update_object, update_probe;
  // Orthogonal probe relaxation (Cp, Sp, Sdp, dP then cover the shared modes)
  const float2* opr_dU; // [K, N, N] eigenmode directions, or null
  const float* opr_w;   // [J, K]
  int K;
  const float2* p0_s;   // [B, N, N] primary mode of each slot
  // Split form (k_pass2_sums + k_pass2_update): partial sums of the five
  // step-size terms per slot and chunk, FP64 [B, P2_CHUNKS, 5]; null selects
  // the single-kernel form.
  double* part;
};

constexpr int P2_CHUNKS = 8;   // chunks of a position's pixels and h planes in the split step-size pass

// Arguments of the multislice per-position pass (kernels_ms.cuh).
// Incident wave of slice s (1..S-1) of mode k in the slot's scratch: kept per
// mode by the forward pass, or one mode's at a time when recomputed.
__device__ __forceinline__ size_t ms_inc_offset(bool recompute, size_t slotNN, int M, int S, int k, int s, int NN) {
  return (recompute ? slotNN * (S - 1) : (slotNN * M + (size_t)k * NN) * (S - 1)) + (size_t)(s - 1) * NN;
}

struct MsArgs {
  int H, W, M, J, S;
  const float2* obj;    // [S, H, W]
  const float2* probe;  // [M, N, N]
  const float* pos;
  const float* meas;    // measured intensities, or dL/dI in MODE_VJP
  int b0, nb, mode;
  float eps;
  const float2* Hf;     // [N, N] propagator, FFT order
  float2* psi_s;        // [B, M, N, N] far fields (unitary scale)
  float2* o_s;          // [B, S, N, N] slice patches
  float2* in_s;         // [B, M, S - 1, N, N] incident waves of slices 1..S-1, or
                        // [B, S - 1, N, N] of one mode when they are recomputed
  int recompute;        // 1: the backward pass recomputes each mode's incident waves
  float2* go_s;         // [B, S, N, N] per-slice object gradients (patch frame)
  float2* h_s;          // [B, M, N, N] probe gradient of each position
  int* valid;           // [B]
  float2* gobj;         // [S, H, W] gradient accumulator, or null
  float* ipred;         // [J, N, N] or null
  float* gpos;          // [J, 2] or null
  double* loss;
  int* status;
  // LSQML (MODE_LSQML_*): minibatch order (null: identity), the per-slice
  // object-frame accumulators, each slice's illumination sum_k |inc|^2 per
  // slot (slices 1..S-1; slice 0 uses Sp = sum_k |P_k|^2)
  const int* order;
  float4* acc;          // [S, H, W] (dO_acc.re, dO_acc.im, illum, unused)
  float* w_s;           // [B, S - 1, N, N]
  const float* Sp;      // [N, N]
};

// Arguments of the multislice LSQML tangent pass (k_step_ms): per slot the
// first-order changes of the exit waves when every slice moves along its
// direction (u) and when the probe moves along its direction (v), reduced to
// the Gram entries |u|^2, Re<u, v>, |v|^2 of the step-size system.
struct MsStepArgs {
  int H, W, M, J, S;
  const int* order;
  int b0, nb;
  const float2* probe;   // [M, N, N]
  const float2* Hf;      // [N, N]
  const float2* o_s;     // [B, S, N, N] slice patches
  float2* in_s;          // [B, M, S - 1, N, N] incident waves of slices 1..S-1, or
                         // [B, S - 1, N, N] scratch for one mode's (recompute)
  int recompute;         // 1: each mode's incident waves are recomputed here first
  const float2* d_s;     // [B, S, N, N] each slice's direction at the slot's position
  const float2* dP;      // [M, N, N] probe direction
  float2* u_s;           // [B, N, N] the object tangent of one mode at the exit plane
  const int* valid;
  double* part;          // [B, Q, 3] Gram partials per CTA of a slot (Q CTAs per position)
};

constexpr int OPR_KMAX = 8;   // eigenmodes of the relaxed primary probe mode

// Shared probe mode k, or null for the synthesised primary mode (OPR).
template <bool OPR>
__device__ __forceinline__ const float2* shared_mode(const BatchArgs& a, int k, int NN) {
  if (OPR) return k == 0 ? nullptr : a.probe + (size_t)(k - 1) * NN;
  return a.probe + (size_t)k * NN;
}

// sum_m wj[m] V_m at the pixel pair starting at p (V: [K, N, N], 16-byte pairs).
__device__ __forceinline__ float4 opr_pair(const float2* __restrict__ V, const float* wj, int K, int NN, int p) {
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4   // four independent loads in flight
  for (int m = 0; m < K; ++m) {
    const float4 u = __ldg((const float4*)(V + (size_t)m * NN + p));
    const float w = wj[m];
    s.x = fmaf(w, u.x, s.x); s.y = fmaf(w, u.y, s.y); s.z = fmaf(w, u.z, s.z); s.w = fmaf(w, u.w, s.w);
  }
  return s;
}

// sum_m wj[m] V_m at one pixel.
__device__ __forceinline__ float2 opr_pixel(const float2* __restrict__ V, const float* wj, int K, int NN, int p) {
  float2 s = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int m = 0; m < K; ++m) {
    const float2 u = __ldg(V + (size_t)m * NN + p);
    s.x = fmaf(wj[m], u.x, s.x); s.y = fmaf(wj[m], u.y, s.y);
  }
  return s;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream serialization attribute may start while its predecessor on the
// stream drains; it waits here, before its first global memory access, until
// the predecessor has completed and its writes are visible (a no-op for a
// kernel launched without the attribute).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Launches `kernel` with the programmatic stream serialization attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Asynchronous prefetch of `bytes` (a multiple of 16) at a 16-byte aligned
// global address into L2; no-op for a misaligned address.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  if (((uintptr_t)p & 15) == 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// max(0, illumination) over the elements t, t + nt, t + 2 nt, ... < n of an
// accumulator plane (component .z), U loads in flight per thread (a plane
// scan that waits on one load at a time runs at a fraction of HBM speed).
template <int U>
__device__ __forceinline__ float illum_max_share(const float4* __restrict__ p, size_t n, size_t t, size_t nt) {
  float m = 0.f;
  size_t i = t;
  for (; i + (U - 1) * nt < n; i += U * nt) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = __ldcs(&p[i + u * nt].z);
#pragma unroll
    for (int u = 0; u < U; ++u) m = fmaxf(m, v[u]);
  }
  for (; i < n; i += nt) m = fmaxf(m, __ldcs(&p[i].z));
  return m;
}

// Tile origin and fraction of a probe-centre position; false if the bilinear
// (N+1)^2 tile is not inside the object or the value is not finite.
__device__ __forceinline__ bool tile_of(float py, float px, int N, int H, int W, int& ty, int& tx,
                                        float& fy, float& fx) {
  const float sy = py - 0.5f * (float)N, sx = px - 0.5f * (float)N;
  // floor(s) >= 0 and floor(s) + N + 1 <= extent  <=>  0 <= s < extent - N (NaN fails)
  if (!(sy >= 0.f && sy < (float)(H - N) && sx >= 0.f && sx < (float)(W - N))) return false;
  const float fly = floorf(sy), flx = floorf(sx);
  ty = (int)fly;
  tx = (int)flx;
  fy = sy - fly;
  fx = sx - flx;
  return true;
}

// o = (1-fy)(1-fx) O[y][x] + (1-fy) fx O[y][x+1] + fy (1-fx) O[y+1][x] + fy fx O[y+1][x+1]
__device__ __forceinline__ float2 bilinear(const float2* __restrict__ O, int W, int y, int x, float fy,
                                           float fx) {
  const float2* p = O + (size_t)y * W + x;
  const float2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + W), d = __ldg(p + W + 1);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  return make_float2(w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x,
                     w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y);
}

// Two horizontally adjacent bilinear samples (columns x and x+1): six corner loads.
__device__ __forceinline__ void bilinear2(const float2* __restrict__ O, int W, int y, int x, float fy, float fx,
                                          float2& o0, float2& o1) {
  const float2* p = O + (size_t)y * W + x;
  const float2 a0 = __ldg(p), a1 = __ldg(p + 1), a2 = __ldg(p + 2);
  const float2 b0 = __ldg(p + W), b1 = __ldg(p + W + 1), b2 = __ldg(p + W + 2);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  o0 = make_float2(w00 * a0.x + w01 * a1.x + w10 * b0.x + w11 * b1.x,
                   w00 * a0.y + w01 * a1.y + w10 * b0.y + w11 * b1.y);
  o1 = make_float2(w00 * a1.x + w01 * a2.x + w10 * b1.x + w11 * b2.x,
                   w00 * a1.y + w01 * a2.y + w10 * b1.y + w11 * b2.y);
}

// Block-wide sum of NV per-thread FP32 partials (passed as doubles, which
// hold them exactly); result valid in thread 0. `red` holds 32*NV doubles. A
// shuffle tree in FP32 within each warp, then warp 0 adds the warps' sums with
// a second shuffle tree in FP64. FP64 runs at about 1/64 of the FP32 rate on
// this part, so an FP64 tree over every thread of a 1024-thread CTA cost
// microseconds; the FP32 warp tree adds five roundings to each thread's own
// partial sum.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float f[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    f[q] = (float)v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f[q] += __shfl_down_sync(0xffffffffu, f[q], o);
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[warp * NV + q] = (double)f[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? red[lane * NV + q] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[q] = s;
    }
  }
}

__device__ __forceinline__ float block_max(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) v = fmaxf(v, red[w]);
  if (threadIdx.x == 0) red[0] = v;
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

}  // namespace ptycho
