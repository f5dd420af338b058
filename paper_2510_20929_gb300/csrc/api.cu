// C-ABI entry points of libptycho and the object/probe-frame kernels of the
// LSQML minibatch (probe direction, preconditioner maxima, probe update).
//
// Per minibatch the epoch runs: k_pass1 (per position: forward model, data
// term, chi, scatter of the object direction and illumination), k_probe_reduce
// (batch sums of conj(o_j) chi_jk and |o_j|^2 per probe pixel, and the maxima
// used by the relative dampings), k_norm_probe (preconditioned probe direction
// and the per-pixel planes of the step solve), k_pass2 (per position: FP64 step
// sizes and the alpha-weighted, preconditioned object update), a memset of the
// object-frame accumulator, and k_probe_update.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "ptycho.h"
#include "common.cuh"
#include "launch.h"
#include "profile.h"
#include "internal.h"

namespace ptycho {

// ---------------------------------------------------------------------------
// Object/probe-frame kernels (window size is a runtime argument here).
// ---------------------------------------------------------------------------
__global__ void k_init_epoch(int NN, int M, const float2* probe, float* Sp, WsHeader* hdr) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NN; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < M; ++k) s += cabs2(probe[(size_t)k * NN + p]);
    Sp[p] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) memset(hdr->sc, 0, sizeof(hdr->sc));
}

// Batch sums of the probe-direction numerator and of the patch intensity:
// item (k, q) with k < Mc sums conj(o_j) chi_j,k0+k over the batch (pixel pair q,
// into dPacc_k, added to its previous value when `accumulate`; each slot holds
// Ms planes), and k == Mc sums |o_j|^2 into Dp and reports max(Dp). Blocks
// with blockIdx.y == 1 scan the illumination plane for its maximum. U
// positions are loaded per iteration; with PG > 1 the batch is split into PG
// consecutive ranges, each summed by its own thread of the block (PG times the
// loads in flight), and the block adds the PG partial sums in range order.
template <int U, int PG>
__global__ void k_probe_reduce(int NN, int k0, int Mc, int Ms, int nb, const float2* __restrict__ h_s,
                               const float2* __restrict__ o_s, const int* __restrict__ valid, float2* dPacc,
                               int accumulate, float* Dp, const float4* __restrict__ acc, int HW,
                               BatchScalars* sc, int o_stride) {
  constexpr int IPB = 256 / PG;   // items per block (blockDim.x == 256)
  __shared__ float red[32];
  __shared__ float4 part[PG][IPB];
  wait_prior_grid();
  if (blockIdx.y == 1) {
    if (!acc) return;
    float m = illum_max_share<8>(acc, (size_t)HW, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                                 (size_t)gridDim.x * blockDim.x);
    m = block_max(m, red);
    if (threadIdx.x == 0) atomicMax(&sc->max_illum, __float_as_uint(m));
    return;
  }
  const int NP = NN / 2;
  const int g = (int)threadIdx.x / IPB, li = (int)threadIdx.x % IPB;
  const int t = blockIdx.x * IPB + li;
  const int k = t / NP, q = t % NP;
  const int i_lo = (int)((long long)nb * g / PG), i_hi = (int)((long long)nb * (g + 1) / PG);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);   // dPacc: the pixel pair; Dp: (d.x, d.y, -, -)
  const bool num = k < Mc && dPacc, den = k == Mc && Dp;
  if (num) {
    const float4* h = (const float4*)h_s + (size_t)(k0 + k) * NP + q;
    const size_t stride = (size_t)Ms * NP;
    for (int i = i_lo; i < i_hi; i += U) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        v[u] = (i + u < i_hi && valid[i + u]) ? __ldcs(h + (size_t)(i + u) * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        s.x += v[u].x; s.y += v[u].y; s.z += v[u].z; s.w += v[u].w;
      }
    }
  } else if (den) {
    const float4* o = (const float4*)o_s + q;
    const size_t ostep = o_stride ? (size_t)o_stride / 2 : (size_t)NP;   // float4 per slot
    for (int i = i_lo; i < i_hi; i += U) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        v[u] = (i + u < i_hi && valid[i + u]) ? __ldg(o + (size_t)(i + u) * ostep) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        s.x += v[u].x * v[u].x + v[u].y * v[u].y;
        s.y += v[u].z * v[u].z + v[u].w * v[u].w;
      }
    }
  }
  if constexpr (PG > 1) {
    part[g][li] = s;
    __syncthreads();
    if (g == 0)
#pragma unroll
      for (int r = 1; r < PG; ++r) {
        const float4 v = part[r][li];
        s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
      }
  }
  float dmax = 0.f;
  if (g == 0 && num) {
    float4* out = (float4*)dPacc + (size_t)k * NP + q;
    if (accumulate) {
      const float4 o = *out;
      s.x += o.x; s.y += o.y; s.z += o.z; s.w += o.w;
    }
    *out = s;
  } else if (g == 0 && den) {
    ((float2*)Dp)[q] = make_float2(s.x, s.y);
    dmax = fmaxf(s.x, s.y);
  }
  if (Dp) {
    dmax = block_max(dmax, red);
    if (threadIdx.x == 0) atomicMax(&sc->max_dp, __float_as_uint(dmax));
  }
}

// dP_k = dPacc_k / (Dp + delta_p max(Dp)); Cp = sum_k conj(P_k) dP_k; Sdp = sum_k |dP_k|^2.
// The loads of up to KB modes are issued together (one L2 round trip per KB
// modes instead of one per mode); the sums run over k in order.
constexpr int kModeChunk = 8;
__global__ void k_norm_probe(int NN, int M, const float2* __restrict__ dPacc, const float* __restrict__ Dp,
                             const float2* __restrict__ probe, float delta_p, int update_probe,
                             const BatchScalars* sc, float2* __restrict__ dP, float2* __restrict__ Cp,
                             float* __restrict__ Sdp) {
  constexpr int KB = kModeChunk;
  wait_prior_grid();
  const float damp = delta_p * __uint_as_float(sc->max_dp);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NN; p += gridDim.x * blockDim.x) {
    float2 c = make_float2(0.f, 0.f);
    float sd = 0.f;
    const float inv = update_probe ? 1.f / (Dp[p] + damp) : 0.f;
    for (int k0 = 0; k0 < M; k0 += KB) {
      float2 a[KB], P[KB];
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const size_t q = (size_t)(k0 + u) * NN + p;
        a[u] = (k0 + u < M && update_probe) ? dPacc[q] : make_float2(0.f, 0.f);
        P[u] = (k0 + u < M) ? probe[q] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < KB; ++u)
        if (k0 + u < M) {
          const float2 v = cscale(a[u], inv);
          dP[(size_t)(k0 + u) * NN + p] = v;
          c = cadd(c, cmulc(P[u], v));
          sd += cabs2(v);
        }
    }
    Cp[p] = c;
    Sdp[p] = sd;
  }
}

// P_k += mean_j(alpha_P) dP_k; refresh Sp = sum_k |P_k|^2 (when Sp is set); clear the next
// batch's scalars. Loads of up to KB modes at a time, as in k_norm_probe.
__global__ void k_probe_update(int NN, int M, float2* __restrict__ probe, const float2* __restrict__ dP,
                               float* __restrict__ Sp, int update_probe, const BatchScalars* sc,
                               BatchScalars* sc_next, float4* __restrict__ clear, size_t nclear) {
  constexpr int KB = kModeChunk;
  wait_prior_grid();
  const float mean_ap = sc->count > 0 ? (float)(sc->sum_alpha_p / (double)sc->count) : 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NN; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k0 = 0; k0 < M; k0 += KB) {
      float2 v[KB], d[KB];
#pragma unroll
      for (int u = 0; u < KB; ++u) {
        const size_t q = (size_t)(k0 + u) * NN + p;
        v[u] = (k0 + u < M) ? probe[q] : make_float2(0.f, 0.f);
        d[u] = (k0 + u < M && update_probe) ? dP[q] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < KB; ++u)
        if (k0 + u < M) {
          if (update_probe) {
            v[u].x = fmaf(mean_ap, d[u].x, v[u].x);
            v[u].y = fmaf(mean_ap, d[u].y, v[u].y);
            probe[(size_t)(k0 + u) * NN + p] = v[u];
          }
          s += cabs2(v[u]);
        }
    }
    if (Sp) Sp[p] = s;
  }
  // (when given) the minibatch's object-frame accumulator plane is zeroed in
  // the same launch: both only have to follow the step-size pass
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < nclear; p += (size_t)gridDim.x * blockDim.x)
    clear[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (blockIdx.x == 0 && threadIdx.x == 0) memset(sc_next, 0, sizeof(BatchScalars));
}

// Object tile of the batch's slot blockIdx.y (false: the slot was skipped by
// pass 1). Blocks blockIdx.x walk its (N+1)^2 pixels.
__device__ __forceinline__ bool slot_tile(int N, int H, int W, int J, const float* pos, const int* order, int b0,
                                          const int* valid, int& ty, int& tx) {
  const int slot = blockIdx.y;
  if (!valid[slot]) return false;
  const int e = b0 + slot;
  const int j = order ? order[e] : e;
  float fy, fx;
  return tile_of(pos[2 * j], pos[2 * j + 1], N, H, W, ty, tx, fy, fx);
}

// max(illumination) over the tiles of the batch (all non-zero illumination
// of the minibatch lies in them).
__global__ void k_tile_illum_max(int N, int H, int W, int J, const float* pos, const int* order, int b0,
                                 const int* valid, const float4* __restrict__ acc, BatchScalars* sc) {
  __shared__ float red[32];
  int ty, tx;
  if (!slot_tile(N, H, W, J, pos, order, b0, valid, ty, tx)) return;
  // (the launch gives each thread about four elements of the tile: all four
  // loads are issued before the first use)
  constexpr int U = 4;
  const int N1 = N + 1, n = N1 * N1, nt = gridDim.x * blockDim.x;
  float m = 0.f;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < n; i += U * nt) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = i + u * nt;
      v[u] = k < n ? __ldcs(&acc[(size_t)(ty + k / N1) * W + tx + k % N1].z) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) m = fmaxf(m, v[u]);
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(&sc->max_illum, __float_as_uint(m));
}

// Zeroes the batch's tiles of the accumulator.
__global__ void k_tile_clear(int N, int H, int W, int J, const float* pos, const int* order, int b0,
                             const int* valid, float4* acc) {
  int ty, tx;
  if (!slot_tile(N, H, W, J, pos, order, b0, valid, ty, tx)) return;
  const int N1 = N + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N1 * N1; i += gridDim.x * blockDim.x)
    acc[(size_t)(ty + i / N1) * W + tx + i % N1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Position correction: one thread per slot solves the least-squares shift
// from its five sums (FP64, the damping and fallbacks of the step sizes),
// clamps each component to +-max_shift, moves the position by step times it
// and keeps it inside the bounds rule, at most extent - N/2 - 1/64.
__global__ void k_pos_apply(int nb, int b0, const int* __restrict__ order, const int* __restrict__ valid,
                            const double* __restrict__ possum, float* pos, int N, int H, int W, double lam,
                            double step, double max_shift) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nb || !valid[slot]) return;
  const int e = b0 + slot;
  const int j = order ? order[e] : e;
  const double* v = possum + (size_t)slot * 5;
  const double a11 = v[0], a12 = v[1], a22 = v[2], r1 = v[3], r2 = v[4];
  const double tr = 0.5 * (a11 + a22);
  const double d11 = a11 + lam * tr, d22 = a22 + lam * tr;
  const double det = d11 * d22 - a12 * a12;
  double dy, dx;
  if (det > 0.0) {
    dy = (d22 * r1 - a12 * r2) / det;
    dx = (d11 * r2 - a12 * r1) / det;
  } else {
    dy = d11 > 0.0 ? r1 / d11 : 0.0;
    dx = d22 > 0.0 ? r2 / d22 : 0.0;
  }
  dy = fmin(fmax(dy, -max_shift), max_shift);
  dx = fmin(fmax(dx, -max_shift), max_shift);
  const double lo = 0.5 * N, margin = 1.0 / 64.0;
  const double y = fmin(fmax((double)pos[2 * j] + step * dy, lo), (double)H - lo - margin);
  const double x = fmin(fmax((double)pos[2 * j + 1] + step * dx, lo), (double)W - lo - margin);
  pos[2 * j] = (float)y;
  pos[2 * j + 1] = (float)x;
}

// Zeroes n float4 (the object-frame accumulator of one minibatch).
__global__ void k_clear_plane(size_t n, float4* acc) {
  wait_prior_grid();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// O += dO (the epoch's accumulated object update).
__global__ void k_add_plane(size_t n, float2* O, const float2* __restrict__ dO) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    O[p] = cadd(O[p], dO[p]);
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

Layout make_layout(const ptycho_dims& d, int B, int K, bool epoch_object) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t HW = (size_t)d.H * d.W, NN = (size_t)d.N * d.N, M = d.M;
  L.hdr = take(sizeof(WsHeader));
  L.acc = take(HW * sizeof(float4));
  L.psi = take((size_t)B * M * NN * sizeof(float2));
  L.o = take((size_t)B * NN * sizeof(float2));
  L.g = take((size_t)B * NN * sizeof(float2));
  L.h = take((size_t)B * M * NN * sizeof(float2));
  L.dPacc = take(M * NN * sizeof(float2));
  L.Dp = take(NN * sizeof(float));
  L.dP = take(M * NN * sizeof(float2));
  L.Sp = take(NN * sizeof(float));
  L.Cp = take(NN * sizeof(float2));
  L.Sdp = take(NN * sizeof(float));
  L.valid = take((size_t)B * sizeof(int));
  L.p0 = L.dUacc = L.Du = L.dU = L.gram = 0;
  if (K > 0) {
    L.p0 = take((size_t)B * NN * sizeof(float2));
    L.dUacc = take((size_t)K * NN * sizeof(float2));
    L.Du = take((size_t)K * NN * sizeof(float));
    L.dU = take((size_t)K * NN * sizeof(float2));
    L.gram = take((size_t)B * (OPR_KMAX * (OPR_KMAX + 1) / 2 + OPR_KMAX) * sizeof(double));   // weight-step sums
  }
  L.possum = take((size_t)B * 5 * sizeof(double));
  L.p2part = take((size_t)B * P2_CHUNKS * 5 * sizeof(double));
  L.dOe = epoch_object ? take(HW * sizeof(float2)) : 0;
  L.dft = 0;
  switch (d.N) {
    case 32: L.dft = take(dft_plane_bytes<32>()); break;
    case 64: L.dft = take(dft_plane_bytes<64>()); break;
    case 128: L.dft = take(dft_plane_bytes<128>()); break;
  }
  L.total = off;
  return L;
}

Layout layout_for(const ptycho_dims& d, const ptycho_lsqml_opts& o) {
  return make_layout(d, o.batch, 0, o.object_per_epoch != 0);
}

static bool supported_N(int N) { return N == 16 || N == 32 || N == 64 || N == 128 || N == 192 || N == 256; }

ptycho_status check_dims(const ptycho_dims* d) {
  if (!d) return PTYCHO_ERR_ARG;
  if (!supported_N(d->N) || d->M < 1 || d->M > 16) return PTYCHO_ERR_UNSUPPORTED;
  if (d->H < d->N + 1 || d->W < d->N + 1 || d->J < 0) return PTYCHO_ERR_ARG;
  if ((int64_t)d->H * d->W > ((int64_t)1 << 31) - 1) return PTYCHO_ERR_ARG;
  return PTYCHO_OK;
}

ptycho_status check_ws(void* ws, size_t have, size_t need) {
  if (!ws || ((uintptr_t)ws & 255) != 0 || have < need) return PTYCHO_ERR_WORKSPACE;
  return PTYCHO_OK;
}

template <class Fn>
static cudaError_t dispatch_N(int N, Fn&& fn) {
  switch (N) {
    case 16: return fn(std::integral_constant<int, 16>());
    case 32: return fn(std::integral_constant<int, 32>());
    case 64: return fn(std::integral_constant<int, 64>());
    case 128: return fn(std::integral_constant<int, 128>());
    case 192: return fn(std::integral_constant<int, 192>());
    case 256: return fn(std::integral_constant<int, 256>());
  }
  return cudaErrorInvalidValue;
}

// Runs `launch` bracketed by the profiler's events for kernel `id` (no-op when off).
template <class F>
static cudaError_t timed(int id, cudaStream_t s, F&& launch) {
  cudaEvent_t e0 = profile_begin(id, s);
  cudaError_t e = launch();
  profile_end(id, e0, s);
  return e;
}

cudaError_t pass1(int N, const BatchArgs& a, cudaStream_t s, int variant) {
  return timed(K_PASS1, s, [&] {
    return dispatch_N(N, [&](auto c) { return launch_pass1<decltype(c)::value>(a, s, variant); });
  });
}

bool dft_gemm_supported(int N) { return N == 32 || N == 64 || N == 128; }

ptycho_status check_precision(int N, int precision, const void* meas) {
  if (precision == PTYCHO_PRECISION_FP32) return PTYCHO_OK;
  if (precision != PTYCHO_PRECISION_BF16X3) return PTYCHO_ERR_ARG;
  if (!dft_gemm_supported(N)) return PTYCHO_ERR_UNSUPPORTED;
  // the measured intensities are read with tensor copies: 16-byte aligned
  return ((uintptr_t)meas & 15) ? PTYCHO_ERR_ARG : PTYCHO_OK;
}

template <class Fn>
static cudaError_t dispatch_tc(int N, Fn&& fn) {
  switch (N) {
    case 32: return fn(std::integral_constant<int, 32>());
    case 64: return fn(std::integral_constant<int, 64>());
    case 128: return fn(std::integral_constant<int, 128>());
  }
  return cudaErrorInvalidValue;
}

cudaError_t dft_planes(int N, void* dft, cudaStream_t s) {
  return timed(K_DFT_PLANES, s, [&] {
    return dispatch_tc(N, [&](auto c) { return launch_dft_planes<decltype(c)::value>(dft, s); });
  });
}

cudaError_t pass1_dft(int N, const BatchArgs& a, const void* dft, cudaStream_t s) {
  cudaError_t e = timed(K_PASS1_EXIT, s, [&] {
    return dispatch_tc(N, [&](auto c) { return launch_pass1_part<decltype(c)::value>(a, s, 1); });
  });
  if (e != cudaSuccess) return e;
  e = timed(K_FAR_TC, s, [&] {
    return dispatch_tc(N, [&](auto c) { return launch_far_tc<decltype(c)::value>(a, dft, s); });
  });
  if (e != cudaSuccess || a.mode == MODE_FWD || a.loss_only) return e;
  return timed(K_PASS1_OVERLAP, s, [&] {
    return dispatch_tc(N, [&](auto c) { return launch_pass1_part<decltype(c)::value>(a, s, 2); });
  });
}

cudaError_t pass2(int N, const Pass2Args& a, cudaStream_t s, int variant) {
  return timed(K_PASS2, s, [&] {
    return dispatch_N(N, [&](auto c) { return launch_pass2<decltype(c)::value>(a, s, variant); });
  });
}

// ---------------------------------------------------------------------------
// Autotuner: CTA-size variants of the two per-position passes, chosen per
// (device, N, M, H, W, B) by timing each candidate on the first minibatch.
// ---------------------------------------------------------------------------
struct TuneKey {
  int dev, N, M, H, W, B;
  bool operator==(const TuneKey& o) const {
    return dev == o.dev && N == o.N && M == o.M && H == o.H && W == o.W && B == o.B;
  }
};
// v[0]: the per-position pass (candidates: pass1_variants(N)), v[1]: the
// step-size pass (candidates: pass2_variants(N): single kernel, split, cluster
// at 4 or 3 CTAs per SM), v[2]: the probe reduction (positions
// in flight per thread: 16, 8, 32, or 8 in each of 4 threads splitting the
// batch); ms[i][c]: candidate c's mean time.
struct TuneEntry {
  TuneKey key;
  int v[PTYCHO_TUNE_KERNELS];
  float ms[PTYCHO_TUNE_KERNELS][PTYCHO_TUNE_MAX];
};

static int pass1_variants(int N) { return N == 128 ? 3 : (N <= 128 ? 2 : 1); }
static int pass2_variants(int N) { return N <= 128 ? 4 : 2; }
static constexpr int kReduceVariants = 4;
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

static bool tune_lookup(const TuneKey& k, TuneEntry* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& e : g_tune)
    if (e.key == k) {
      *out = e;
      return true;
    }
  return false;
}

static void tune_store(const TuneEntry& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& e : g_tune)
    if (e.key == t.key) {
      e = t;
      return;
    }
  g_tune.push_back(t);
}

// Mean time of `reps` runs of launch() on stream s (after one warm-up run).
template <class F>
static float time_launch(cudaStream_t s, int reps, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return 1e30f;
  float ms = 1e30f;
  if (launch() == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = launch() == cudaSuccess;
    if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
      ms /= (float)reps;
    else
      ms = 1e30f;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

cudaError_t probe_reduce(int NN, int k0, int Mc, int Ms, int nb, const float2* h_s, const float2* o_s,
                         const int* valid, float2* dPacc, int accumulate, float* Dp, const float4* acc, int HW,
                         BatchScalars* sc, cudaStream_t s, int o_stride, int variant) {
  cudaEvent_t e0 = profile_begin(K_PROBE_REDUCE, s);
  const int NP = NN / 2;
  const int items = (dPacc ? Mc * NP : 0) + (Dp ? NP : 0);
  const int ipb = variant == 3 ? 256 / 4 : 256;   // items per block
  int bx = (items + ipb - 1) / ipb;
  if (acc && bx < 2 * sm_count()) bx = 2 * sm_count();
  dim3 grid(bx > 0 ? bx : 1, acc ? 2 : 1);
  auto kern = variant == 1 ? k_probe_reduce<8, 1>
            : variant == 2 ? k_probe_reduce<32, 1>
            : variant == 3 ? k_probe_reduce<8, 4> : k_probe_reduce<16, 1>;
  const cudaError_t e = launch_pdl(kern, grid, dim3(256), 0, s, NN, k0, Mc, Ms, nb, h_s, o_s, valid, dPacc,
                                   accumulate, Dp, acc, HW, sc, o_stride);
  profile_end(K_PROBE_REDUCE, e0, s);
  return e;
}

int sm_count() {
  static int cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = __atomic_load_n(&cached[dev], __ATOMIC_RELAXED);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
    __atomic_store_n(&cached[dev], n, __ATOMIC_RELAXED);
  }
  return n;
}

int grid_for(size_t n, int threads, int cap) {
  size_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b > (size_t)cap ? cap : b);
}

cudaError_t norm_probe(int NN, int M, const float2* dPacc, const float* Dp, const float2* probe, float delta_p,
                       int update_probe, const BatchScalars* sc, float2* dP, float2* Cp, float* Sdp,
                       cudaStream_t s) {
  return timed(K_NORM_PROBE, s, [&] {
    return launch_pdl(k_norm_probe, dim3(grid_for(NN, 128, 2 * sm_count())), dim3(128), 0, s, NN, M, dPacc, Dp, probe, delta_p,
                      update_probe, sc, dP, Cp, Sdp);
  });
}

cudaError_t probe_update(int NN, int M, float2* probe, const float2* dP, float* Sp, int update_probe,
                         const BatchScalars* sc, BatchScalars* sc_next, cudaStream_t s, float4* clear, size_t nclear) {
  return timed(K_UPDATE, s, [&] {
    const int g = clear ? grid_for(nclear, 256, 8 * sm_count()) : grid_for(NN, 256, sm_count());
    return launch_pdl(k_probe_update, dim3(g), dim3(256), 0, s, NN, M, probe, dP, Sp, update_probe, sc, sc_next,
                      clear, clear ? nclear : (size_t)0);
  });
}

cudaError_t init_epoch(int NN, int M, const float2* probe, float* Sp, WsHeader* hdr, cudaStream_t s) {
  return timed(K_INIT, s, [&] {
    k_init_epoch<<<grid_for(NN, 256, sm_count()), 256, 0, s>>>(NN, M, probe, Sp, hdr);
    return cudaGetLastError();
  });
}

bool tiles_cheaper(int nb, int N, int H, int W) {
  // a tile row is a run of 16 (N + 1) bytes, which the scan and the clear
  // stream at about the plane's bandwidth (measured on the 192 and 256
  // windows), so the tiles win as soon as they hold fewer elements
  return (size_t)nb * (N + 1) * (N + 1) < (size_t)H * W;
}

static dim3 tile_grid(int nb, int N) {
  const int n1 = (N + 1) * (N + 1);
  return dim3((unsigned)((n1 + 1023) / 1024), (unsigned)nb);
}

cudaError_t tile_illum_max(const ptycho_dims& d, int nb, int b0, const float* pos, const int32_t* order,
                           const int* valid, const float4* acc, BatchScalars* sc, cudaStream_t s) {
  return timed(K_TILE_MAX, s, [&] {
    k_tile_illum_max<<<tile_grid(nb, d.N), 256, 0, s>>>(d.N, d.H, d.W, d.J, pos, order, b0, valid, acc, sc);
    return cudaGetLastError();
  });
}

cudaError_t clear_acc(bool tiles, const ptycho_dims& d, int nb, int b0, const float* pos, const int32_t* order,
                      const int* valid, float4* acc, cudaStream_t s) {
  if (!tiles) {
    const size_t n = (size_t)d.H * d.W;
    return timed(K_CLEAR_PLANE, s, [&] {
      return launch_pdl(k_clear_plane, dim3(grid_for(n, 256, 8 * sm_count())), dim3(256), 0, s, n, acc);
    });
  }
  return timed(K_TILE_CLEAR, s, [&] {
    k_tile_clear<<<tile_grid(nb, d.N), 256, 0, s>>>(d.N, d.H, d.W, d.J, pos, order, b0, valid, acc);
    return cudaGetLastError();
  });
}

Ptrs carve(void* ws, const Layout& L) {
  char* b = (char*)ws;
  Ptrs p;
  p.hdr = (WsHeader*)(b + L.hdr);
  p.acc = (float4*)(b + L.acc);
  p.psi = (float2*)(b + L.psi);
  p.o = (float2*)(b + L.o);
  p.g = (float2*)(b + L.g);
  p.h = (float2*)(b + L.h);
  p.dPacc = (float2*)(b + L.dPacc);
  p.Dp = (float*)(b + L.Dp);
  p.dP = (float2*)(b + L.dP);
  p.Sp = (float*)(b + L.Sp);
  p.Cp = (float2*)(b + L.Cp);
  p.Sdp = (float*)(b + L.Sdp);
  p.valid = (int*)(b + L.valid);
  p.p0 = L.p0 ? (float2*)(b + L.p0) : nullptr;
  p.dUacc = L.dUacc ? (float2*)(b + L.dUacc) : nullptr;
  p.Du = L.Du ? (float*)(b + L.Du) : nullptr;
  p.dU = L.dU ? (float2*)(b + L.dU) : nullptr;
  p.gram = L.gram ? (double*)(b + L.gram) : nullptr;
  p.possum = (double*)(b + L.possum);
  p.p2part = (double*)(b + L.p2part);
  p.dOe = L.dOe ? (float2*)(b + L.dOe) : nullptr;
  p.dft = L.dft ? (void*)(b + L.dft) : nullptr;
  return p;
}

ptycho_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PTYCHO_OK : PTYCHO_ERR_CUDA; }

// Times both CTA-size variants of k_pass1 and k_pass2 on the epoch's first
// minibatch, without side effects on the caller's data: the loss is not
// written, k_pass2's object update goes to the far-field scratch (when it is
// large enough to stand in for the object, else k_pass2 keeps its default),
// and the accumulators and batch scalars are cleared again afterwards.
static ptycho_status autotune(const ptycho_dims& d, float2* obj, float2* probe, const float* pos, const float* meas,
                              const int32_t* order, const ptycho_lsqml_opts& o, const Ptrs& w, const Layout& L,
                              cudaStream_t s, TuneEntry* t) {
  const int B = o.batch, N = d.N, M = d.M, NN = N * N, HW = d.H * d.W;
  const int nb = d.J < B ? d.J : B;
  BatchScalars* sc = &w.hdr->sc[0];
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.H = d.H; a.W = d.W; a.M = M; a.J = d.J;
  a.obj = obj; a.probe = probe; a.pos = pos; a.meas = meas; a.order = order;
  a.b0 = 0; a.nb = nb;
  a.mode = (o.noise == PTYCHO_NOISE_POISSON) ? MODE_LSQML_POISSON : MODE_LSQML_GAUSS;
  a.eps = (float)o.eps;
  a.psi_s = w.h; a.o_s = w.o; a.g_s = w.g; a.h_s = w.h; a.valid = w.valid;   // (far fields under h: see run_epoch)
  a.Sp = w.Sp; a.acc = w.acc; a.loss = nullptr; a.status = &w.hdr->status;
  auto best = [](const float* ms, int n) {
    int b = 0;
    for (int c = 1; c < n; ++c)
      if (ms[c] < ms[b]) b = c;
    return b;
  };
  const int n1 = pass1_variants(N);
  for (int v = 0; v < n1; ++v) t->ms[0][v] = time_launch(s, 3, [&] { return pass1(N, a, s, v); });
  t->v[0] = best(t->ms[0], n1);
  // one clean pass 1 with the chosen variant feeds the other candidates
  if (cudaMemsetAsync(w.acc, 0, (size_t)HW * sizeof(float4), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (pass1(N, a, s, t->v[0]) != cudaSuccess) return PTYCHO_ERR_CUDA;
  for (int v = 0; v < kReduceVariants; ++v)
    t->ms[2][v] = time_launch(s, 3, [&] {
      return probe_reduce(NN, 0, M, M, nb, w.h, w.o, w.valid, o.update_probe ? w.dPacc : nullptr, 0,
                          o.update_probe ? w.Dp : nullptr, w.acc, HW, sc, s, 0, v);
    });
  t->v[2] = best(t->ms[2], kReduceVariants);
  if (norm_probe(NN, M, w.dPacc, w.Dp, probe, (float)o.delta_p, o.update_probe, sc, w.dP, w.Cp, w.Sdp, s) !=
      cudaSuccess)
    return PTYCHO_ERR_CUDA;
  t->v[1] = 0;
  if (L.o - L.psi >= (size_t)HW * sizeof(float2) && o.update_object) {
    Pass2Args q;
    memset(&q, 0, sizeof(q));
    q.H = d.H; q.W = d.W; q.M = M; q.J = d.J;
    q.pos = pos; q.order = order; q.b0 = 0; q.nb = nb;
    q.o_s = w.o; q.g_s = w.g; q.h_s = w.h; q.valid = w.valid;
    q.acc = w.acc; q.Sp = w.Sp; q.Cp = w.Cp; q.Sdp = w.Sdp; q.dP = w.dP;
    q.obj = w.psi;  // stand-in object: the far-field scratch
    q.part = w.p2part;
    q.sc = sc;
    q.delta_o = (float)o.delta_o; q.lam = o.lambda_reg;
    q.update_object = o.update_object; q.update_probe = o.update_probe;
    const int n2 = pass2_variants(N);
    for (int v = 0; v < n2; ++v) t->ms[1][v] = time_launch(s, 3, [&] { return pass2(N, q, s, v); });
    t->v[1] = best(t->ms[1], n2);
  }
  // restore the epoch's starting state of the accumulators and scalars
  if (cudaMemsetAsync(w.acc, 0, (size_t)HW * sizeof(float4), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  return init_epoch(NN, M, probe, w.Sp, w.hdr, s) == cudaSuccess ? PTYCHO_OK : PTYCHO_ERR_CUDA;
}

ptycho_status run_epoch(const ptycho_dims& d, float2* obj, float2* probe, float* pos,
                               const float* meas, const int32_t* order, const ptycho_lsqml_opts& o,
                               double* loss, double* alpha, void* ws, cudaStream_t s, const MeasSwitch* later) {
  const int B = o.batch, N = d.N, M = d.M, NN = N * N, HW = d.H * d.W;
  const Layout L = layout_for(d, o);
  Ptrs w = carve(ws, L);
  cudaError_t e = cudaSuccess;
  if (loss && (e = cudaMemsetAsync(loss, 0, sizeof(double), s)) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if ((e = cudaMemsetAsync(w.acc, 0, (size_t)HW * sizeof(float4), s)) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if ((e = init_epoch(NN, M, probe, w.Sp, w.hdr, s)) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (o.object_per_epoch && (e = cudaMemsetAsync(w.dOe, 0, (size_t)HW * sizeof(float2), s)) != cudaSuccess)
    return PTYCHO_ERR_CUDA;
  const bool tc = o.precision == PTYCHO_PRECISION_BF16X3;
  if (tc && (e = dft_planes(N, w.dft, s)) != cudaSuccess) return PTYCHO_ERR_CUDA;
  int dev = 0;
  cudaGetDevice(&dev);
  if (later && later->meas && d.J > 0) {   // the first minibatch (and the autotuner) read the arriving copy
    if ((e = cudaStreamWaitEvent(s, later->ready[0], 0)) != cudaSuccess) return PTYCHO_ERR_CUDA;
    meas = later->meas;
  }
  TuneEntry tune;
  memset(&tune, 0, sizeof(tune));
  tune.v[2] = kReduceDefault;   // (until tuned or pinned)
  tune.key = {dev, N, M, d.H, d.W, B};
  if (!tc && !tune_lookup(tune.key, &tune) && (o.flags & PTYCHO_FLAG_AUTOTUNE) && d.J > 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      ptycho_status ts = autotune(d, obj, probe, pos, meas, order, o, w, L, s, &tune);
      if (ts != PTYCHO_OK) return ts;
      tune_store(tune);
    }
  }
  const int nbatch = (d.J + B - 1) / B;
  for (int b = 0; b < nbatch; ++b) {
    const int b0 = b * B, nb = (d.J - b0 < B) ? d.J - b0 : B;
    BatchScalars* sc = &w.hdr->sc[b & 1];
    BatchScalars* sc_next = &w.hdr->sc[(b + 1) & 1];
    if (later && later->meas && b > 0 && (e = cudaStreamWaitEvent(s, later->ready[b], 0)) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.H = d.H; a.W = d.W; a.M = M; a.J = d.J;
    a.obj = obj; a.probe = probe; a.pos = pos; a.order = order;
    a.meas = (later && later->meas) ? later->meas : meas;
    a.b0 = b0; a.nb = nb;
    a.mode = (o.noise == PTYCHO_NOISE_POISSON) ? MODE_LSQML_POISSON : MODE_LSQML_GAUSS;
    a.eps = (float)o.eps;
    // FP32: the far field of mode k shares its scratch with h_k, which the
    // pass writes only after the inverse transform of mode k has consumed the
    // far field (same slot, same mode, the same CTA): a far field still in L2
    // is overwritten there instead of being written back to HBM
    a.psi_s = tc ? w.psi : w.h; a.o_s = w.o; a.g_s = w.g; a.h_s = w.h; a.valid = w.valid;
    a.Sp = w.Sp; a.acc = w.acc;
    a.loss = loss; a.status = &w.hdr->status;
    if (o.update_positions) {
      a.possum = w.possum;
      if ((e = cudaMemsetAsync(w.possum, 0, (size_t)nb * 5 * sizeof(double), s)) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
    }
    if ((e = tc ? pass1_dft(N, a, w.dft, s) : pass1(N, a, s, tune.v[0])) != cudaSuccess) return PTYCHO_ERR_CUDA;
    const bool tiles = tiles_cheaper(nb, N, d.H, d.W);
    if ((e = probe_reduce(NN, 0, M, M, nb, w.h, w.o, w.valid, o.update_probe ? w.dPacc : nullptr, 0,
                          o.update_probe ? w.Dp : nullptr, tiles ? nullptr : w.acc, HW, sc, s, 0, tune.v[2])) !=
        cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (tiles && tile_illum_max(d, nb, b0, pos, order, w.valid, w.acc, sc, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if ((e = norm_probe(NN, M, w.dPacc, w.Dp, probe, (float)o.delta_p, o.update_probe, sc, w.dP, w.Cp, w.Sdp,
                        s)) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    Pass2Args q;
    memset(&q, 0, sizeof(q));
    q.H = d.H; q.W = d.W; q.M = M; q.J = d.J;
    q.pos = pos; q.order = order; q.b0 = b0; q.nb = nb;
    q.o_s = w.o; q.g_s = w.g; q.h_s = w.h; q.valid = w.valid;
    q.acc = w.acc; q.Sp = w.Sp; q.Cp = w.Cp; q.Sdp = w.Sdp; q.dP = w.dP;
    q.obj = o.object_per_epoch ? w.dOe : obj; q.alpha_out = alpha; q.sc = sc; q.part = w.p2part;
    q.delta_o = (float)o.delta_o; q.lam = o.lambda_reg;
    q.update_object = o.update_object; q.update_probe = o.update_probe;
    if ((e = pass2(N, q, s, tune.v[1])) != cudaSuccess) return PTYCHO_ERR_CUDA;
    // the whole plane is zeroed by the probe update's launch; tiles by their own kernel
    if (tiles && (e = clear_acc(tiles, d, nb, b0, pos, order, w.valid, w.acc, s)) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if ((e = probe_update(NN, M, probe, w.dP, w.Sp, o.update_probe, sc, sc_next, s, tiles ? nullptr : w.acc,
                          (size_t)HW)) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (o.update_positions) {   // last: pass 2 and the tile clear read this batch's positions
      k_pos_apply<<<(nb + 127) / 128, 128, 0, s>>>(nb, b0, order, w.valid, w.possum, pos, N, d.H, d.W,
                                                   o.lambda_reg, o.pos_step, o.pos_max_shift);
      if ((e = cudaGetLastError()) != cudaSuccess) return PTYCHO_ERR_CUDA;
    }
  }
  if (o.object_per_epoch) {
    k_add_plane<<<grid_for((size_t)HW, 256, 4 * sm_count()), 256, 0, s>>>((size_t)HW, obj, w.dOe);
    if ((e = cudaGetLastError()) != cudaSuccess) return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

ptycho_status check_opts(const ptycho_lsqml_opts* o) {
  if (!o || o->batch < 1 || (o->noise != PTYCHO_NOISE_GAUSSIAN && o->noise != PTYCHO_NOISE_POISSON))
    return PTYCHO_ERR_ARG;
  if (o->precision != PTYCHO_PRECISION_FP32 && o->precision != PTYCHO_PRECISION_BF16X3) return PTYCHO_ERR_ARG;
  if ((o->update_positions != 0 && o->update_positions != 1) || (o->object_per_epoch != 0 && o->object_per_epoch != 1))
    return PTYCHO_ERR_ARG;
  if (!(o->pos_step >= 0.0) || !(o->pos_step < 1e30) || !(o->pos_max_shift >= 0.0) || !(o->pos_max_shift < 1e30))
    return PTYCHO_ERR_ARG;
  if (o->flags & ~(int32_t)(PTYCHO_FLAG_GRAPH | PTYCHO_FLAG_AUTOTUNE)) return PTYCHO_ERR_ARG;
  if (!(o->delta_o >= 0.0) || !(o->delta_p >= 0.0) || !(o->lambda_reg >= 0.0) || !(o->eps >= 0.0))
    return PTYCHO_ERR_ARG;
  return PTYCHO_OK;
}

// Copies the measured intensities of the minibatch positions order[b0 ..
// b0 + nb) from mapped host memory (read over the host link) to their own
// rows of the device copy; entries outside 0..J-1 are left to the epoch's
// checks. The minibatch's nb * NN4 16-byte elements are walked flat, U loads
// in flight per thread: few CTAs can keep the host link busy, and each CTA
// keeps an SM from the per-position pass only for as long as it copies.
template <int U>
__global__ void k_gather_meas(const float4* __restrict__ src, float4* dst, const int* __restrict__ order, int b0,
                              int nb, int J, int NN4) {
  const size_t total = (size_t)nb * NN4, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x; base < total; base += U * stride) {
    float4 v[U];
    size_t at[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t idx = base + u * stride;
      at[u] = ~(size_t)0;
      if (idx < total) {
        const int i = (int)(idx / NN4), off = (int)(idx % NN4);
        const int e = b0 + i;
        const int j = order ? order[e] : e;
        if (j >= 0 && j < J) {
          at[u] = (size_t)j * NN4 + off;
          v[u] = src[at[u]];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (at[u] != ~(size_t)0) dst[at[u]] = v[u];
  }
}

}  // namespace ptycho

using namespace ptycho;

extern "C" {

const char* ptycho_version(void) { return "ptycho-gb300 0.1 (sm_103a)"; }

const char* ptycho_status_string(ptycho_status s) {
  switch (s) {
    case PTYCHO_OK: return "ok";
    case PTYCHO_ERR_ARG: return "invalid argument";
    case PTYCHO_ERR_BOUNDS: return "scan position outside the object (or order entry out of range)";
    case PTYCHO_ERR_NONFINITE: return "negative or non-finite measured intensity";
    case PTYCHO_ERR_CUDA: return "CUDA runtime error";
    case PTYCHO_ERR_TIMEOUT: return "device wait timed out";
    case PTYCHO_ERR_UNSUPPORTED: return "unsupported window size or mode count";
    case PTYCHO_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case PTYCHO_ERR_TOO_LARGE: return "problem needs more scratch than the static array holds";
  }
  return "unknown status";
}

int32_t ptycho_tuning_read(const ptycho_dims* dims, int32_t batch, int32_t* variants, float* ms) {
  if (!dims) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  TuneEntry t;
  if (!tune_lookup({dev, dims->N, dims->M, dims->H, dims->W, batch}, &t)) return 0;
  for (int i = 0; i < PTYCHO_TUNE_KERNELS; ++i) {
    if (variants) variants[i] = t.v[i];
    if (ms)
      for (int c = 0; c < PTYCHO_TUNE_MAX; ++c) ms[i * PTYCHO_TUNE_MAX + c] = t.ms[i][c];
  }
  return 1;
}

ptycho_status ptycho_tuning_set(const ptycho_dims* dims, int32_t batch, const int32_t* variants) {
  ptycho_status st = check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if (batch < 1 || !variants) return PTYCHO_ERR_ARG;
  const int n[PTYCHO_TUNE_KERNELS] = {pass1_variants(dims->N), pass2_variants(dims->N), kReduceVariants};
  for (int i = 0; i < PTYCHO_TUNE_KERNELS; ++i)
    if (variants[i] < 0 || variants[i] >= n[i]) return PTYCHO_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  TuneEntry t;
  memset(&t, 0, sizeof(t));
  t.key = {dev, dims->N, dims->M, dims->H, dims->W, batch};
  for (int i = 0; i < PTYCHO_TUNE_KERNELS; ++i) t.v[i] = variants[i];
  tune_store(t);
  return PTYCHO_OK;
}

ptycho_status ptycho_workspace_init(void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < align256(sizeof(WsHeader))) return PTYCHO_ERR_WORKSPACE;
  return cuda_status(cudaMemsetAsync(ws, 0, sizeof(WsHeader), (cudaStream_t)stream));
}

size_t ptycho_workspace_bytes(const ptycho_dims* dims, int32_t batch) {
  if (check_dims(dims) != PTYCHO_OK || batch < 1) return 0;
  return make_layout(*dims, batch).total;
}

size_t ptycho_workspace_bytes_opts(const ptycho_dims* dims, const ptycho_lsqml_opts* opts) {
  if (check_dims(dims) != PTYCHO_OK || check_opts(opts) != PTYCHO_OK) return 0;
  return layout_for(*dims, *opts).total;
}

ptycho_status ptycho_forward_ex(const ptycho_dims* dims, int32_t precision, int32_t batch, const float* object,
                                const float* probe, const float* pos, float* I_pred, void* ws, size_t ws_bytes,
                                void* stream) {
  ptycho_status st = check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if ((st = check_precision(dims->N, precision, nullptr)) != PTYCHO_OK) return st;
  if (batch < 1) return PTYCHO_ERR_ARG;
  if (!object || !probe || (dims->J > 0 && (!pos || !I_pred))) return PTYCHO_ERR_ARG;
  const bool tc = precision == PTYCHO_PRECISION_BF16X3;
  const Layout L = make_layout(*dims, batch);
  if ((st = check_ws(ws, ws_bytes, tc ? L.total : align256(sizeof(WsHeader)))) != PTYCHO_OK) return st;
  if (dims->J == 0) return PTYCHO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.H = dims->H; a.W = dims->W; a.M = dims->M; a.J = dims->J;
  a.obj = (const float2*)object; a.probe = (const float2*)probe; a.pos = pos;
  a.mode = MODE_FWD;
  a.ipred = I_pred; a.status = &((WsHeader*)ws)->status;
  if (!tc) {
    a.b0 = 0; a.nb = dims->J;
    return cuda_status(pass1(dims->N, a, s));
  }
  Ptrs w = carve(ws, L);
  if (dft_planes(dims->N, w.dft, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  a.psi_s = w.psi; a.valid = w.valid;
  for (int b0 = 0; b0 < dims->J; b0 += batch) {
    a.b0 = b0;
    a.nb = (dims->J - b0 < batch) ? dims->J - b0 : batch;
    if (pass1_dft(dims->N, a, w.dft, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

ptycho_status ptycho_forward(const ptycho_dims* dims, const float* object, const float* probe, const float* pos,
                             float* I_pred, void* ws, size_t ws_bytes, void* stream) {
  return ptycho_forward_ex(dims, PTYCHO_PRECISION_FP32, 1, object, probe, pos, I_pred, ws, ws_bytes, stream);
}

ptycho_status ptycho_adjoint_ex(const ptycho_dims* dims, int32_t precision, const float* object, const float* probe,
                                const float* pos, const float* meas, int32_t noise, double eps, int32_t batch,
                                float* g_object, float* g_probe, float* g_pos, double* loss, void* ws,
                                size_t ws_bytes, void* stream) {
  ptycho_status st = check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if ((st = check_precision(dims->N, precision, meas)) != PTYCHO_OK) return st;
  if (batch < 1 || !(eps >= 0.0)) return PTYCHO_ERR_ARG;
  if (noise != PTYCHO_NOISE_GAUSSIAN && noise != PTYCHO_NOISE_POISSON && noise != PTYCHO_NOISE_VJP)
    return PTYCHO_ERR_ARG;
  // no gradient buffer at all (and a loss): the forward model and data term only
  const bool loss_only = !g_object && !g_probe && !g_pos;
  if (!object || !probe) return PTYCHO_ERR_ARG;
  if (loss_only ? (!loss || noise == PTYCHO_NOISE_VJP) : (!g_object || !g_probe)) return PTYCHO_ERR_ARG;
  if (dims->J > 0 && (!pos || !meas)) return PTYCHO_ERR_ARG;
  const Layout L = make_layout(*dims, batch);
  if ((st = check_ws(ws, ws_bytes, L.total)) != PTYCHO_OK) return st;
  Ptrs w = carve(ws, L);
  cudaStream_t s = (cudaStream_t)stream;
  const int NN = dims->N * dims->N;
  const bool tc = precision == PTYCHO_PRECISION_BF16X3;
  if (tc && dims->J > 0 && dft_planes(dims->N, w.dft, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  for (int b0 = 0; b0 < dims->J; b0 += batch) {
    const int nb = (dims->J - b0 < batch) ? dims->J - b0 : batch;
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.H = dims->H; a.W = dims->W; a.M = dims->M; a.J = dims->J;
    a.obj = (const float2*)object; a.probe = (const float2*)probe; a.pos = pos; a.meas = meas;
    a.b0 = b0; a.nb = nb;
    a.mode = noise == PTYCHO_NOISE_GAUSSIAN ? MODE_GRAD_GAUSS
             : noise == PTYCHO_NOISE_POISSON ? MODE_GRAD_POISSON : MODE_VJP;
    a.eps = (float)eps;
    a.psi_s = w.psi; a.o_s = w.o; a.g_s = w.g; a.h_s = w.h; a.valid = w.valid;
    a.gobj = (float2*)g_object; a.gpos = g_pos; a.loss = loss; a.status = &w.hdr->status;
    a.loss_only = loss_only ? 1 : 0;
    if ((tc ? pass1_dft(dims->N, a, w.dft, s) : pass1(dims->N, a, s)) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (loss_only) continue;
    if (probe_reduce(NN, 0, dims->M, dims->M, nb, w.h, w.o, w.valid, (float2*)g_probe, 1, nullptr, nullptr, 0,
                     nullptr, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

ptycho_status ptycho_adjoint(const ptycho_dims* dims, const float* object, const float* probe, const float* pos,
                             const float* meas, int32_t noise, double eps, int32_t batch, float* g_object,
                             float* g_probe, float* g_pos, double* loss, void* ws, size_t ws_bytes,
                             void* stream) {
  return ptycho_adjoint_ex(dims, PTYCHO_PRECISION_FP32, object, probe, pos, meas, noise, eps, batch, g_object,
                           g_probe, g_pos, loss, ws, ws_bytes, stream);
}

ptycho_status ptycho_lsqml_epoch(const ptycho_dims* dims, float* object, float* probe, float* pos,
                                 const float* meas, const int32_t* order, const ptycho_lsqml_opts* opts,
                                 double* loss, double* alpha, void* ws, size_t ws_bytes, void* stream) {
  ptycho_status st = check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if ((st = check_opts(opts)) != PTYCHO_OK) return st;
  if ((st = check_precision(dims->N, opts->precision, meas)) != PTYCHO_OK) return st;
  if (!object || !probe || (dims->J > 0 && (!pos || !meas))) return PTYCHO_ERR_ARG;
  const Layout L = layout_for(*dims, *opts);
  if ((st = check_ws(ws, ws_bytes, L.total)) != PTYCHO_OK) return st;
  auto body = [&](cudaStream_t s) {
    return run_epoch(*dims, (float2*)object, (float2*)probe, pos, meas, order, *opts, loss, alpha, ws, s);
  };
  if (!(opts->flags & PTYCHO_FLAG_GRAPH)) return body((cudaStream_t)stream);
  GraphKey key;
  key.add(*dims).add(object).add(probe).add(pos).add(meas).add(order).add(*opts).add(loss).add(alpha).add(ws);
  return run_graphed(key, (cudaStream_t)stream, body);
}

static size_t host_extra(const ptycho_dims& d) {  // device staging of the host buffers
  const size_t HW = (size_t)d.H * d.W, NN = (size_t)d.N * d.N;
  return align256(HW * 8) + align256((size_t)d.M * NN * 8) + align256((size_t)d.J * 8) +
         align256((size_t)d.J * NN * 4) + align256((size_t)d.J * 4) + align256(8);
}

size_t ptycho_host_workspace_bytes(const ptycho_dims* dims, int32_t batch) {
  if (check_dims(dims) != PTYCHO_OK || batch < 1) return 0;
  return make_layout(*dims, batch).total + host_extra(*dims);
}

size_t ptycho_host_workspace_bytes_opts(const ptycho_dims* dims, const ptycho_lsqml_opts* opts) {
  if (check_dims(dims) != PTYCHO_OK || check_opts(opts) != PTYCHO_OK) return 0;
  return layout_for(*dims, *opts).total + host_extra(*dims);
}

ptycho_status ptycho_lsqml_epoch_host(const ptycho_dims* dims, float* object, float* probe, float* pos,
                                      const float* meas, const int32_t* order, const ptycho_lsqml_opts* opts,
                                      double* loss, void* ws, size_t ws_bytes, void* stream) {
  ptycho_status st = check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if ((st = check_opts(opts)) != PTYCHO_OK) return st;
  // (the device copy of the host intensities sits at a 256-byte boundary)
  if ((st = check_precision(dims->N, opts->precision, nullptr)) != PTYCHO_OK) return st;
  if (!object || !probe || (dims->J > 0 && (!pos || !meas))) return PTYCHO_ERR_ARG;
  const Layout L = layout_for(*dims, *opts);
  if ((st = check_ws(ws, ws_bytes, L.total + host_extra(*dims))) != PTYCHO_OK) return st;
  const ptycho_dims& d = *dims;
  const size_t HW = (size_t)d.H * d.W, NN = (size_t)d.N * d.N;
  char* b = (char*)ws + L.total;
  float2* dobj = (float2*)b; b += align256(HW * 8);
  float2* dprobe = (float2*)b; b += align256((size_t)d.M * NN * 8);
  float* dpos = (float*)b; b += align256((size_t)d.J * 8);
  float* dmeas = (float*)b; b += align256((size_t)d.J * NN * 4);
  int32_t* dorder = (int32_t*)b; b += align256((size_t)d.J * 4);
  double* dloss = (double*)b;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t n, cudaMemcpyKind k) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, k, s);
  };
  // the order first: the intensity gather below needs it, and it runs while
  // the object, probe and positions are copied
  if (order) cp(dorder, order, (size_t)d.J * 4, cudaMemcpyHostToDevice);
  // The measured intensities, the bulk of the input: pinned host memory that is
  // mapped into the device's address space is gathered into the workspace
  // during the epoch (below), so the transfer overlaps the compute; other host
  // memory (and the tensor-copy form) is staged first.
  const float* mdev = nullptr;
  if (opts->precision == PTYCHO_PRECISION_FP32 && d.J > 0) {
    void* mapped = nullptr;
    if (cudaHostGetDevicePointer(&mapped, (void*)meas, 0) == cudaSuccess)
      mdev = (const float*)mapped;
    else
      (void)cudaGetLastError();   // not mapped pinned memory: clear the error and stage it
  }
  // Mapped intensities: a gather kernel on a worker stream copies them into the
  // workspace copy minibatch by minibatch, in the epoch's order, reading them
  // over the host link; minibatch b waits only for its own positions, so
  // after the first minibatch's copy the transfer runs under the compute.
  MeasSwitch later;
  std::vector<cudaEvent_t> ready;
  cudaStream_t cs = nullptr;
  const int B = opts->batch, nbatch = (d.J + B - 1) / B;
  if (mdev) {
    cudaStream_t* workers = nullptr;
    int nw = 0;
    if ((st = worker_streams(&workers, &nw)) != PTYCHO_OK) return st;
    cs = workers[0];
    ready.assign((size_t)nbatch + 1, nullptr);   // [nbatch]: the fork from the caller's stream
    for (auto& ev : ready)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ready[nbatch], s);   // the order is on the device
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready[nbatch], 0);
    for (int b = 0; b < nbatch && e == cudaSuccess; ++b) {
      const int b0 = b * B, nb = (d.J - b0 < B) ? d.J - b0 : B;
      // the first minibatch precedes all compute: a wide grid; the later ones
      // run under it on two CTAs
      if (b == 0)
        k_gather_meas<4><<<2 * sm_count(), 256, 0, cs>>>((const float4*)mdev, (float4*)dmeas,
                                                         order ? dorder : nullptr, b0, nb, d.J, (int)(NN / 4));
      else
        k_gather_meas<8><<<2, 1024, 0, cs>>>((const float4*)mdev, (float4*)dmeas, order ? dorder : nullptr, b0, nb,
                                             d.J, (int)(NN / 4));
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(ready[b], cs);
    }
    later.meas = dmeas;
    later.ready = ready.data();
  } else {
    cp(dmeas, meas, (size_t)d.J * NN * 4, cudaMemcpyHostToDevice);
    mdev = dmeas;
  }
  cp(dobj, object, HW * 8, cudaMemcpyHostToDevice);
  cp(dprobe, probe, (size_t)d.M * NN * 8, cudaMemcpyHostToDevice);
  cp(dpos, pos, (size_t)d.J * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    st = run_epoch(d, dobj, dprobe, dpos, mdev, order ? dorder : nullptr, *opts, dloss, nullptr, ws, s,
                   later.meas ? &later : nullptr);
  else
    st = PTYCHO_ERR_CUDA;
  if (!ready.empty()) {
    // on success the epoch waited for every gather; on an error they may
    // still be running into the workspace: let them finish
    if (st != PTYCHO_OK) cudaStreamSynchronize(cs);
    for (auto ev : ready)
      if (ev) cudaEventDestroy(ev);
  }
  if (st != PTYCHO_OK) return st;
  cp(object, dobj, HW * 8, cudaMemcpyDeviceToHost);
  cp(probe, dprobe, (size_t)d.M * NN * 8, cudaMemcpyDeviceToHost);
  if (opts->update_positions) cp(pos, dpos, (size_t)d.J * 8, cudaMemcpyDeviceToHost);
  if (loss) cp(loss, dloss, 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return PTYCHO_ERR_CUDA;
  return cuda_status(cudaStreamSynchronize(s));
}

ptycho_status ptycho_status_read(void* ws, void* stream) {
  if (!ws) return PTYCHO_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  WsHeader* hdr = (WsHeader*)ws;
  int h = 0;
  if (cudaMemcpyAsync(&h, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PTYCHO_ERR_CUDA;
  if (cudaMemsetAsync(&hdr->status, 0, sizeof(int), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (h & FLAG_TIMEOUT) return PTYCHO_ERR_TIMEOUT;
  if (h & FLAG_BOUNDS) return PTYCHO_ERR_BOUNDS;
  if (h & FLAG_NONFINITE) return PTYCHO_ERR_NONFINITE;
  return PTYCHO_OK;
}

}  // extern "C"
