// Orthogonal probe relaxation (Pty-Chi Sec. 2.1: scan-point-specific probes).
//
// The primary probe mode of position j is P_j0 = sum_m w_jm U_m over K
// eigenmodes U [K, N, N] with real weights w [J, K]; the other M - 1
// incoherent modes are shared. The per-position kernels (k_pass1, k_pass2)
// synthesise P_j0 on chip from the eigenmodes and the position's weights;
// this file holds the eigenmode and weight kernels and the entry points:
//   gradient form: dL/dU_m = sum_j w_jm h_j0 and dL/dw_jm = Re<U_m, h_j0>,
//     with h_j0 = conj(o_j) times the gradient with respect to psi_j0;
//   LSQML form: eigenmode directions dU_m = sum_j w_jm h_j0 / (D_m + delta_P),
//     D_m = sum_j w_jm^2 |o_j|^2, which enter the per-position step sizes
//     through dP_j0 = sum_m w_jm dU_m and follow the probe step, and a
//     per-position least-squares weight update that fits the primary mode's
//     exit-wave change chi_j0 with the eigenmodes' exit waves U_m o_j.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "ptycho.h"
#include "common.cuh"
#include "profile.h"
#include "internal.h"

namespace ptycho {

// Batch sums of the relaxed primary mode per probe pixel pair q. Block row
// blockIdx.y takes slots [chunk * y, chunk * (y + 1)) of the batch and adds,
// with vector atomics, dUacc_m += sum_j w_jm h_j0 and (when D is set)
// D_m += sum_j w_jm^2 |o_j|^2. The slots' validity and weights are staged in
// shared memory, RS slots at a time, so that the loop over the slots waits
// only on the h and o loads, two slots' loads in flight (added in slot order).
template <int KM>
__global__ void __launch_bounds__(256) k_opr_reduce(int NN, int M, int K, int nb, int chunk, int b0,
                                                    const int* __restrict__ order, const float* __restrict__ w,
                                                    const float2* __restrict__ h_s, const float2* __restrict__ o_s,
                                                    const int* __restrict__ valid, float2* dUacc, float* D) {
  constexpr int RS = 64;
  __shared__ int ok_s[RS];
  __shared__ float w_s[RS][KM];
  const int NP = NN / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = blockIdx.y * chunk, i1 = min(nb, i0 + chunk);
  float4 s[KM];
  float2 d[KM];
#pragma unroll
  for (int m = 0; m < KM; ++m) {
    s[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    d[m] = make_float2(0.f, 0.f);
  }
  auto add = [&](int r, const float4& h, const float4& o) {
    const float oa0 = o.x * o.x + o.y * o.y, oa1 = o.z * o.z + o.w * o.w;
#pragma unroll
    for (int m = 0; m < KM; ++m) {
      if (m < K) {
        const float wm = w_s[r][m], w2 = wm * wm;
        s[m].x = fmaf(wm, h.x, s[m].x); s[m].y = fmaf(wm, h.y, s[m].y);
        s[m].z = fmaf(wm, h.z, s[m].z); s[m].w = fmaf(wm, h.w, s[m].w);
        d[m].x = fmaf(w2, oa0, d[m].x); d[m].y = fmaf(w2, oa1, d[m].y);
      }
    }
  };
  for (int t0 = i0; t0 < i1; t0 += RS) {
    const int n = min(RS, i1 - t0);
    __syncthreads();   // the previous round's staging is consumed
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int i = t0 + r;
      const int ok = valid[i];   // (an invalid slot's position index may be out of range)
      ok_s[r] = ok;
      if (ok) {
        const int e = b0 + i;
        const int j = order ? order[e] : e;
        for (int m = 0; m < K; ++m) w_s[r][m] = __ldg(w + (size_t)j * K + m);
      }
    }
    __syncthreads();
    if (q < NP) {
      int r = 0;
      for (; r + 1 < n; r += 2) {
        const bool v0 = ok_s[r] != 0, v1 = ok_s[r + 1] != 0;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const size_t i = (size_t)(t0 + r);
        const float4 h0 = v0 ? __ldg((const float4*)(h_s + i * M * NN) + q) : z;
        const float4 h1 = v1 ? __ldg((const float4*)(h_s + (i + 1) * M * NN) + q) : z;
        const float4 o0 = (v0 && D) ? __ldg((const float4*)(o_s + i * NN) + q) : z;
        const float4 o1 = (v1 && D) ? __ldg((const float4*)(o_s + (i + 1) * NN) + q) : z;
        if (v0) add(r, h0, o0);
        if (v1) add(r + 1, h1, o1);
      }
      if (r < n && ok_s[r]) {
        const size_t i = (size_t)(t0 + r);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        add(r, __ldg((const float4*)(h_s + i * M * NN) + q), D ? __ldg((const float4*)(o_s + i * NN) + q) : z);
      }
    }
  }
  if (q >= NP) return;
#pragma unroll
  for (int m = 0; m < KM; ++m) {
    if (m < K) {
      atomicAdd((float4*)(dUacc + (size_t)m * NN) + q, s[m]);
      if (D) atomicAdd((float2*)(D + (size_t)m * NN) + q, d[m]);
    }
  }
}

// Maximum of a non-negative plane into *out (float bits, atomicMax).
__global__ void k_plane_max(const float* __restrict__ v, size_t n, unsigned int* out) {
  __shared__ float red[32];
  float m = 0.f;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, v[p]);
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(out, __float_as_uint(m));
}

// dU_m = dUacc_m / (D_m + delta_p max) (zero when the probe is not updated).
__global__ void k_norm_opr(size_t n, const float2* dUacc, const float* D, int update_probe, float delta_p,
                           const BatchScalars* sc, float2* dU) {
  const float damp = delta_p * __uint_as_float(sc->max_dp);
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    dU[p] = update_probe ? cscale(dUacc[p], 1.f / (D[p] + damp)) : make_float2(0.f, 0.f);
}

// Per-slot sums of the weight step (FP64 atomics into gram[slot]):
// gram[NA + m] = b_m = Re<U_m, h_j0>, and with `ls`
// gram[t(m, n)] = A_mn = sum |o_j|^2 Re(conj(U_m) U_n) for m <= n.
// A CTA takes GRAM_SLOTS slots (one warp each) and the pixel range
// [blockIdx.x * span, +span) in chunks of GRAM_CHUNK pixels. Each chunk's
// eigenmode values, h_j0 and o_j are copied into shared memory with cp.async
// (double-buffered: the next chunk is in flight while this one is summed), so
// that U is fetched once per CTA instead of once per slot. span and the
// window area are multiples of GRAM_CHUNK.
constexpr int GRAM_SLOTS = 8, GRAM_CHUNK = 256;

template <int KM>
struct GramSmem {
  float2 u[2][KM][GRAM_CHUNK];
  float2 h[2][GRAM_SLOTS][GRAM_CHUNK];
  float2 o[2][GRAM_SLOTS][GRAM_CHUNK];
};

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

template <int KM>
__global__ void __launch_bounds__(32 * GRAM_SLOTS, 2) k_opr_gram(int N, int M, int K, int ls, int nb, int span,
                                                                 const int* __restrict__ valid,
                                                                 const float2* __restrict__ U,
                                                                 const float2* __restrict__ h_s,
                                                                 const float2* __restrict__ o_s, double* gram) {
  constexpr int NA = KM * (KM + 1) / 2, NV = NA + KM;
  extern __shared__ __align__(16) unsigned char gsm[];
  GramSmem<KM>& sm = *(GramSmem<KM>*)gsm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot0 = blockIdx.y * GRAM_SLOTS;
  const int slot = slot0 + warp;
  const bool active = slot < nb && valid[slot];
  const int NN = N * N;
  const int p0 = blockIdx.x * span, p1 = min(NN, p0 + span);
  // eigenmode rows m >= K are never copied: zero them once
  for (int i = threadIdx.x; i < 2 * KM * GRAM_CHUNK; i += blockDim.x) {
    const int b = i / (KM * GRAM_CHUNK), m = (i / GRAM_CHUNK) % KM, q = i % GRAM_CHUNK;
    if (m >= K) sm.u[b][m][q] = make_float2(0.f, 0.f);
  }
  auto stage = [&](int c0, int b) {
    for (int i = threadIdx.x; i < K * GRAM_CHUNK; i += blockDim.x) {
      const int m = i / GRAM_CHUNK, q = i % GRAM_CHUNK;
      cp_async8(&sm.u[b][m][q], U + (size_t)m * NN + c0 + q);
    }
    for (int i = threadIdx.x; i < GRAM_SLOTS * GRAM_CHUNK; i += blockDim.x) {
      const int sl = i / GRAM_CHUNK, q = i % GRAM_CHUNK, sg = slot0 + sl;
      if (sg < nb) {
        cp_async8(&sm.h[b][sl][q], h_s + (size_t)sg * M * NN + c0 + q);
        if (ls) cp_async8(&sm.o[b][sl][q], o_s + (size_t)sg * NN + c0 + q);
      }
    }
    cp_async_commit();
  };
  float acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0.f;
  stage(p0, 0);
  int b = 0;
  for (int c0 = p0; c0 < p1; c0 += GRAM_CHUNK, b ^= 1) {
    if (c0 + GRAM_CHUNK < p1) {
      stage(c0 + GRAM_CHUNK, b ^ 1);
      cp_async_wait<1>();   // this chunk's group has landed (the next may be in flight)
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (active) {
      for (int q = lane; q < GRAM_CHUNK; q += 32) {
        const float2 hv = sm.h[b][warp][q];
        float2 u[KM];
#pragma unroll
        for (int m = 0; m < KM; ++m) u[m] = sm.u[b][m][q];
#pragma unroll
        for (int m = 0; m < KM; ++m) acc[NA + m] += u[m].x * hv.x + u[m].y * hv.y;   // Re(conj(U_m) h)
        if (ls) {
          const float2 ov = sm.o[b][warp][q];
          const float c = ov.x * ov.x + ov.y * ov.y;
          int t = 0;
#pragma unroll
          for (int m = 0; m < KM; ++m) {
            const float cx = c * u[m].x, cy = c * u[m].y;
#pragma unroll
            for (int n = m; n < KM; ++n, ++t) acc[t] = fmaf(cx, u[n].x, fmaf(cy, u[n].y, acc[t]));
          }
        }
      }
    }
    __syncthreads();   // buffer b is refilled by the stage two chunks ahead
  }
  if (!active) return;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    float x = acc[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0 && (ls || t >= NA)) atomicAdd(gram + (size_t)slot * NV + t, (double)x);
  }
}

// In-register FP64 solve of (A + dmp I) x = b for K unknowns (Cholesky on the
// packed upper triangle a[t(m, n)], m <= n); false if not positive definite.
template <int K, int KM>
__device__ __forceinline__ bool chol_solve(const double* v, double lam, double (&x)[KM]) {
  constexpr int NA = KM * (KM + 1) / 2;
  double L[K][K];
  double tr = 0.0;
#pragma unroll
  for (int m = 0; m < K; ++m) tr += v[m * KM - m * (m - 1) / 2];   // A_mm
  const double dmp = lam * tr / (double)K;
#pragma unroll
  for (int r = 0; r < K; ++r) {
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double sum = v[c * KM - c * (c - 1) / 2 + (r - c)] + (r == c ? dmp : 0.0);   // A_cr, c <= r
#pragma unroll
      for (int k = 0; k < c; ++k) sum -= L[r][k] * L[c][k];
      if (r == c) {
        if (!(sum > 0.0)) return false;
        L[r][r] = sqrt(sum);
      } else {
        L[r][c] = sum / L[c][c];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < K; ++r) {   // L y = b
    double sum = v[NA + r];
#pragma unroll
    for (int k = 0; k < r; ++k) sum -= L[r][k] * x[k];
    x[r] = sum / L[r][r];
  }
#pragma unroll
  for (int r = K - 1; r >= 0; --r) {   // L^T x = y
    double sum = x[r];
#pragma unroll
    for (int k = r + 1; k < K; ++k) sum -= L[k][r] * x[k];
    x[r] = sum / L[r][r];
  }
  return true;
}

// One thread per slot. Gradient form (gw set): dL/dw_j += b. Otherwise the
// damped normal equations (A + lam tr(A)/K I) dw = b are solved in FP64
// (Cholesky; no update if the system is not positive definite) and
// w_j += step dw.
template <int KM>
__global__ void k_opr_solve(int nb, int K, int b0, const int* __restrict__ order, const int* __restrict__ valid,
                            const double* __restrict__ gram, float* w, float* gw, double lam, float step) {
  constexpr int NA = KM * (KM + 1) / 2, NV = NA + KM;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nb || !valid[slot]) return;
  const int e = b0 + slot;
  const int j = order ? order[e] : e;
  const double* v = gram + (size_t)slot * NV;
  if (gw) {
    for (int m = 0; m < K; ++m) gw[(size_t)j * K + m] += (float)v[NA + m];
    return;
  }
  double x[KM];
  bool ok = false;
  switch (K) {
    case 1: ok = chol_solve<1, KM>(v, lam, x); break;
    case 2: ok = chol_solve<2, KM>(v, lam, x); break;
    case 3: ok = chol_solve<3, KM>(v, lam, x); break;
    case 4: ok = chol_solve<4, KM>(v, lam, x); break;
    case 5: ok = chol_solve<5, KM>(v, lam, x); break;
    case 6: ok = chol_solve<6, KM>(v, lam, x); break;
    case 7: ok = chol_solve<7, KM>(v, lam, x); break;
    case 8: ok = chol_solve<8, KM>(v, lam, x); break;
  }
  if (!ok) return;   // not positive definite: no weight update
  for (int m = 0; m < K; ++m) w[(size_t)j * K + m] += (float)(step * x[m]);
}

constexpr int OPR_NV = OPR_KMAX * (OPR_KMAX + 1) / 2 + OPR_KMAX;   // sums per slot of the weight step

// Opts a kernel into more than 48 KB of dynamic shared memory, once per device.
template <class Kern>
static cudaError_t smem_optin_once(Kern kernel, size_t bytes, unsigned long long* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) __atomic_fetch_or(done_mask, bit, __ATOMIC_ACQ_REL);
  return e;
}

static cudaError_t opr_reduce(int NN, int M, int K, int nb, int b0, const int* order, const float* w,
                              const float2* h_s, const float2* o_s, const int* valid, float2* dUacc, float* D,
                              cudaStream_t s) {
  // pixel pairs across blockIdx.x, the batch split into enough chunks for two CTAs per SM
  const int NP = NN / 2;
  const int bx = (NP + 255) / 256;
  int chunks = (2 * sm_count() + bx - 1) / bx;
  if (chunks > nb) chunks = nb;
  if (chunks < 1) chunks = 1;
  const int chunk = (nb + chunks - 1) / chunks;
  chunks = (nb + chunk - 1) / chunk;
  cudaEvent_t e0 = profile_begin(K_OPR_REDUCE, s);
  k_opr_reduce<OPR_KMAX><<<dim3(bx, chunks), 256, 0, s>>>(NN, M, K, nb, chunk, b0, order, w, h_s, o_s, valid,
                                                          dUacc, D);
  profile_end(K_OPR_REDUCE, e0, s);
  return cudaGetLastError();
}

// Weight gradient (gw set) or least-squares weight update of the batch's
// positions; `gram` is the per-slot scratch of OPR_NV doubles.
static cudaError_t opr_weights(int N, int M, int K, int nb, int b0, const int* order, const int* valid,
                               const float2* U, const float2* h_s, const float2* o_s, float* w, float* gw,
                               double* gram, double lam, float step, cudaStream_t s) {
  cudaEvent_t e0 = profile_begin(K_OPR_WEIGHTS, s);
  cudaError_t e = cudaMemsetAsync(gram, 0, (size_t)nb * OPR_NV * sizeof(double), s);
  if (e == cudaSuccess) {
    // pixel spans of whole chunks, enough CTAs for two per SM
    const int NN = N * N, groups = (nb + GRAM_SLOTS - 1) / GRAM_SLOTS;
    int parts = (2 * sm_count() + groups - 1) / groups;
    const int max_parts = (NN + GRAM_CHUNK - 1) / GRAM_CHUNK;
    if (parts > max_parts) parts = max_parts;
    const int span = ((NN + parts - 1) / parts + GRAM_CHUNK - 1) / GRAM_CHUNK * GRAM_CHUNK;
    parts = (NN + span - 1) / span;
    static unsigned long long done = 0;
    e = smem_optin_once(k_opr_gram<OPR_KMAX>, sizeof(GramSmem<OPR_KMAX>), &done);
    if (e == cudaSuccess)
      k_opr_gram<OPR_KMAX><<<dim3(parts, groups), 32 * GRAM_SLOTS, sizeof(GramSmem<OPR_KMAX>), s>>>(
          N, M, K, gw ? 0 : 1, nb, span, valid, U, h_s, o_s, gram);
    k_opr_solve<OPR_KMAX><<<(nb + 31) / 32, 32, 0, s>>>(nb, K, b0, order, valid, gram, w, gw, lam, step);
    e = cudaGetLastError();
  }
  profile_end(K_OPR_WEIGHTS, e0, s);
  return e;
}

static ptycho_status check_opr_dims(const ptycho_dims* d, int32_t K) {
  const ptycho_status st = check_dims(d);
  if (st != PTYCHO_OK) return st;
  if (K < 1 || K > OPR_KMAX) return PTYCHO_ERR_UNSUPPORTED;
  return PTYCHO_OK;
}

ptycho_status check_opr_opts(const ptycho_opr_opts* r) {
  if (!r) return PTYCHO_ERR_ARG;
  if (r->K < 1 || r->K > OPR_KMAX) return PTYCHO_ERR_UNSUPPORTED;
  if ((r->update_weights != 0 && r->update_weights != 1) || r->reserved[0] != 0 || r->reserved[1] != 0)
    return PTYCHO_ERR_ARG;
  if (!(r->weight_step >= 0.0) || !(r->weight_step < 1e30)) return PTYCHO_ERR_ARG;
  return PTYCHO_OK;
}

static void opr_args(BatchArgs& a, const ptycho_dims& d, int K, const float* object, const float* U,
                     const float* w, const float* P_rest, const float* pos) {
  memset(&a, 0, sizeof(a));
  a.H = d.H; a.W = d.W; a.M = d.M; a.J = d.J;
  a.obj = (const float2*)object; a.probe = (const float2*)P_rest; a.pos = pos;
  a.opr_U = (const float2*)U; a.opr_w = w; a.K = K;
}

ptycho_status run_epoch_opr(const ptycho_dims& d, const ptycho_opr_opts& r, float2* obj, float2* U, float* wts,
                            float2* P_rest, const float* pos, const float* meas, const int32_t* order,
                            const ptycho_lsqml_opts& o, double* loss, double* alpha, void* ws, cudaStream_t s) {
  const int B = o.batch, N = d.N, M = d.M, NN = N * N, HW = d.H * d.W, K = r.K;
  const Layout L = make_layout(d, B, K);
  Ptrs w = carve(ws, L);
  if (loss && cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (cudaMemsetAsync(w.acc, 0, (size_t)HW * sizeof(float4), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (init_epoch(NN, M - 1, P_rest, w.Sp, w.hdr, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  const size_t KNN = (size_t)K * NN;
  const int nbatch = (d.J + B - 1) / B;
  for (int b = 0; b < nbatch; ++b) {
    const int b0 = b * B, nb = (d.J - b0 < B) ? d.J - b0 : B;
    BatchScalars* sc = &w.hdr->sc[b & 1];
    BatchScalars* sc_next = &w.hdr->sc[(b + 1) & 1];
    BatchArgs a;
    opr_args(a, d, K, (const float*)obj, (const float*)U, wts, (const float*)P_rest, pos);
    a.meas = meas; a.order = order; a.b0 = b0; a.nb = nb;
    a.mode = (o.noise == PTYCHO_NOISE_POISSON) ? MODE_LSQML_POISSON : MODE_LSQML_GAUSS;
    a.eps = (float)o.eps;
    a.psi_s = w.psi; a.o_s = w.o; a.g_s = w.g; a.h_s = w.h; a.valid = w.valid; a.p0_s = w.p0;
    a.Sp = w.Sp; a.acc = w.acc; a.loss = loss; a.status = &w.hdr->status;
    if (pass1(N, a, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    const bool tiles = tiles_cheaper(nb, N, d.H, d.W);
    if (probe_reduce(NN, 1, M - 1, M, nb, w.h, w.o, w.valid, o.update_probe ? w.dPacc : nullptr, 0,
                     o.update_probe ? w.Dp : nullptr, tiles ? nullptr : w.acc, HW, sc, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (tiles && tile_illum_max(d, nb, b0, pos, order, w.valid, w.acc, sc, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (o.update_probe) {
      if (cudaMemsetAsync(w.dUacc, 0, KNN * sizeof(float2), s) != cudaSuccess ||
          cudaMemsetAsync(w.Du, 0, KNN * sizeof(float), s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      if (opr_reduce(NN, M, K, nb, b0, order, wts, w.h, w.o, w.valid, w.dUacc, w.Du, s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      k_plane_max<<<grid_for(KNN, 256, 2 * sm_count()), 256, 0, s>>>(w.Du, KNN, &sc->max_dp);
      if (cudaGetLastError() != cudaSuccess) return PTYCHO_ERR_CUDA;
    }
    if (norm_probe(NN, M - 1, w.dPacc, w.Dp, P_rest, (float)o.delta_p, o.update_probe, sc, w.dP, w.Cp, w.Sdp,
                   s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    k_norm_opr<<<grid_for(KNN, 256, 2 * sm_count()), 256, 0, s>>>(KNN, w.dUacc, w.Du, o.update_probe, (float)o.delta_p,
                                                             sc, w.dU);
    if (cudaGetLastError() != cudaSuccess) return PTYCHO_ERR_CUDA;
    Pass2Args q;
    memset(&q, 0, sizeof(q));
    q.H = d.H; q.W = d.W; q.M = M; q.J = d.J;
    q.pos = pos; q.order = order; q.b0 = b0; q.nb = nb;
    q.o_s = w.o; q.g_s = w.g; q.h_s = w.h; q.valid = w.valid;
    q.acc = w.acc; q.Sp = w.Sp; q.Cp = w.Cp; q.Sdp = w.Sdp; q.dP = w.dP;
    q.obj = obj; q.alpha_out = alpha; q.sc = sc;
    q.delta_o = (float)o.delta_o; q.lam = o.lambda_reg;
    q.update_object = o.update_object; q.update_probe = o.update_probe;
    q.opr_dU = w.dU; q.opr_w = wts; q.K = K; q.p0_s = w.p0; q.part = w.p2part;
    if (pass2(N, q, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (r.update_weights && opr_weights(N, M, K, nb, b0, order, w.valid, U, w.h, w.o, wts, nullptr, w.gram,
                                        o.lambda_reg, (float)r.weight_step, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (clear_acc(tiles, d, nb, b0, pos, order, w.valid, w.acc, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (probe_update(NN, M - 1, P_rest, w.dP, w.Sp, o.update_probe, sc, sc_next, s) != cudaSuccess ||
        probe_update(NN, K, U, w.dU, nullptr, o.update_probe, sc, sc_next, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

}  // namespace ptycho

using namespace ptycho;

extern "C" {

size_t ptycho_workspace_bytes_opr(const ptycho_dims* dims, int32_t K, int32_t batch) {
  if (check_opr_dims(dims, K) != PTYCHO_OK || batch < 1) return 0;
  return make_layout(*dims, batch, K).total;
}

ptycho_status ptycho_forward_opr(const ptycho_dims* dims, int32_t K, const float* object, const float* U,
                                 const float* w, const float* P_rest, const float* pos, float* I_pred, void* ws,
                                 size_t ws_bytes, void* stream) {
  ptycho_status st = check_opr_dims(dims, K);
  if (st != PTYCHO_OK) return st;
  if (!object || !U || (dims->M > 1 && !P_rest) || (dims->J > 0 && (!pos || !I_pred || !w))) return PTYCHO_ERR_ARG;
  if ((st = check_ws(ws, ws_bytes, align256(sizeof(WsHeader)))) != PTYCHO_OK) return st;
  if (dims->J == 0) return PTYCHO_OK;
  BatchArgs a;
  opr_args(a, *dims, K, object, U, w, P_rest, pos);
  a.b0 = 0; a.nb = dims->J; a.mode = MODE_FWD;
  a.ipred = I_pred; a.status = &((WsHeader*)ws)->status;
  return cuda_status(pass1(dims->N, a, (cudaStream_t)stream));
}

ptycho_status ptycho_adjoint_opr(const ptycho_dims* dims, int32_t K, const float* object, const float* U,
                                 const float* w, const float* P_rest, const float* pos, const float* meas,
                                 int32_t noise, double eps, int32_t batch, float* g_object, float* g_U, float* g_w,
                                 float* g_P_rest, float* g_pos, double* loss, void* ws, size_t ws_bytes,
                                 void* stream) {
  ptycho_status st = check_opr_dims(dims, K);
  if (st != PTYCHO_OK) return st;
  if (batch < 1 || !(eps >= 0.0)) return PTYCHO_ERR_ARG;
  if (noise != PTYCHO_NOISE_GAUSSIAN && noise != PTYCHO_NOISE_POISSON && noise != PTYCHO_NOISE_VJP)
    return PTYCHO_ERR_ARG;
  if (!object || !U || !g_object || !g_U || (dims->M > 1 && (!P_rest || !g_P_rest))) return PTYCHO_ERR_ARG;
  if (dims->J > 0 && (!pos || !meas || !w)) return PTYCHO_ERR_ARG;
  const Layout L = make_layout(*dims, batch, K);
  if ((st = check_ws(ws, ws_bytes, L.total)) != PTYCHO_OK) return st;
  Ptrs wp = carve(ws, L);
  cudaStream_t s = (cudaStream_t)stream;
  const int N = dims->N, M = dims->M, NN = N * N;
  for (int b0 = 0; b0 < dims->J; b0 += batch) {
    const int nb = (dims->J - b0 < batch) ? dims->J - b0 : batch;
    BatchArgs a;
    opr_args(a, *dims, K, object, U, w, P_rest, pos);
    a.meas = meas; a.b0 = b0; a.nb = nb;
    a.mode = noise == PTYCHO_NOISE_GAUSSIAN ? MODE_GRAD_GAUSS
             : noise == PTYCHO_NOISE_POISSON ? MODE_GRAD_POISSON : MODE_VJP;
    a.eps = (float)eps;
    a.psi_s = wp.psi; a.o_s = wp.o; a.g_s = wp.g; a.h_s = wp.h; a.valid = wp.valid; a.p0_s = wp.p0;
    a.gobj = (float2*)g_object; a.gpos = g_pos; a.loss = loss; a.status = &wp.hdr->status;
    if (pass1(N, a, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (M > 1 && probe_reduce(NN, 1, M - 1, M, nb, wp.h, wp.o, wp.valid, (float2*)g_P_rest, 1, nullptr, nullptr, 0,
                              nullptr, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (opr_reduce(NN, M, K, nb, b0, nullptr, w, wp.h, wp.o, wp.valid, (float2*)g_U, nullptr, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (g_w && opr_weights(N, M, K, nb, b0, nullptr, wp.valid, (const float2*)U, wp.h, wp.o, nullptr, g_w,
                           wp.gram, 0.0, 0.f, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

ptycho_status ptycho_lsqml_epoch_opr(const ptycho_dims* dims, const ptycho_opr_opts* opr, float* object, float* U,
                                     float* w, float* P_rest, const float* pos, const float* meas,
                                     const int32_t* order, const ptycho_lsqml_opts* opts, double* loss,
                                     double* alpha, void* ws, size_t ws_bytes, void* stream) {
  ptycho_status st = check_dims(dims);
  if (st != PTYCHO_OK) return st;
  if ((st = check_opr_opts(opr)) != PTYCHO_OK) return st;
  if ((st = check_opts(opts)) != PTYCHO_OK) return st;
  if (opts->update_positions || opts->object_per_epoch || opts->precision != PTYCHO_PRECISION_FP32)
    return PTYCHO_ERR_UNSUPPORTED;
  if (!object || !U || (dims->M > 1 && !P_rest) || (dims->J > 0 && (!pos || !meas || !w))) return PTYCHO_ERR_ARG;
  const Layout L = make_layout(*dims, opts->batch, opr->K);
  if ((st = check_ws(ws, ws_bytes, L.total)) != PTYCHO_OK) return st;
  auto body = [&](cudaStream_t s) {
    return run_epoch_opr(*dims, *opr, (float2*)object, (float2*)U, w, (float2*)P_rest, pos, meas, order, *opts,
                         loss, alpha, ws, s);
  };
  if (!(opts->flags & PTYCHO_FLAG_GRAPH)) return body((cudaStream_t)stream);
  GraphKey key;
  key.add(*dims).add(*opr).add(object).add(U).add(w).add(P_rest).add(pos).add(meas).add(order).add(*opts);
  key.add(loss).add(alpha).add(ws);
  return run_graphed(key, (cudaStream_t)stream, body);
}

}  // extern "C"
