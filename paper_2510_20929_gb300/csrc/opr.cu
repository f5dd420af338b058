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
// D_m += sum_j w_jm^2 |o_j|^2.
template <int KM>
__global__ void __launch_bounds__(256) k_opr_reduce(int NN, int M, int K, int nb, int chunk, int b0,
                                                    const int* __restrict__ order, const float* __restrict__ w,
                                                    const float2* __restrict__ h_s, const float2* __restrict__ o_s,
                                                    const int* __restrict__ valid, float2* dUacc, float* D) {
  const int NP = NN / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NP) return;
  const int i0 = blockIdx.y * chunk, i1 = min(nb, i0 + chunk);
  float4 s[KM];
  float2 d[KM];
#pragma unroll
  for (int m = 0; m < KM; ++m) {
    s[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    d[m] = make_float2(0.f, 0.f);
  }
  for (int i = i0; i < i1; ++i) {
    if (!valid[i]) continue;
    const int e = b0 + i;
    const int j = order ? order[e] : e;
    const float4 h = __ldg((const float4*)(h_s + (size_t)i * M * NN) + q);
    float oa0 = 0.f, oa1 = 0.f;
    if (D) {
      const float4 o = __ldg((const float4*)(o_s + (size_t)i * NN) + q);
      oa0 = o.x * o.x + o.y * o.y;
      oa1 = o.z * o.z + o.w * o.w;
    }
#pragma unroll
    for (int m = 0; m < KM; ++m) {
      if (m < K) {
        const float wm = __ldg(w + (size_t)j * K + m), w2 = wm * wm;
        s[m].x = fmaf(wm, h.x, s[m].x); s[m].y = fmaf(wm, h.y, s[m].y);
        s[m].z = fmaf(wm, h.z, s[m].z); s[m].w = fmaf(wm, h.w, s[m].w);
        d[m].x = fmaf(w2, oa0, d[m].x); d[m].y = fmaf(w2, oa1, d[m].y);
      }
    }
  }
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

// One CTA per slot of the batch. b_m = Re<U_m, h_j0>; in gradient form
// (gw set) b is added to dL/dw_j. Otherwise the damped normal equations
// (A + lam tr(A)/K I) dw = b with A_mn = sum |o_j|^2 Re(conj(U_m) U_n) are
// solved in FP64 (Cholesky; no update if the system is not positive
// definite) and w_j += step dw.
template <int KM>
__global__ void __launch_bounds__(256) k_opr_weights(int N, int M, int K, int b0, const int* __restrict__ order,
                                                     const int* __restrict__ valid, const float2* __restrict__ U,
                                                     const float2* __restrict__ h_s, const float2* __restrict__ o_s,
                                                     float* w, float* gw, double lam, float step) {
  constexpr int NA = KM * (KM + 1) / 2, NV = NA + KM;
  __shared__ double red[32 * NV];
  const int slot = blockIdx.x;
  if (!valid[slot]) return;
  const int e = b0 + slot;
  const int j = order ? order[e] : e;
  const int NN = N * N, NP = NN / 2;
  const bool ls = (gw == nullptr);
  const float4* h = (const float4*)(h_s + (size_t)slot * M * NN);
  const float4* o = (const float4*)(o_s + (size_t)slot * NN);
  float acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0.f;
  for (int q = threadIdx.x; q < NP; q += blockDim.x) {
    const float4 hv = __ldg(h + q);
    float4 u[KM];
#pragma unroll
    for (int m = 0; m < KM; ++m)
      u[m] = m < K ? __ldg((const float4*)(U + (size_t)m * NN) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int m = 0; m < KM; ++m)   // Re(conj(U_m) h) at both pixels
      acc[NA + m] += u[m].x * hv.x + u[m].y * hv.y + u[m].z * hv.z + u[m].w * hv.w;
    if (ls) {
      const float4 ov = __ldg(o + q);
      const float oa0 = ov.x * ov.x + ov.y * ov.y, oa1 = ov.z * ov.z + ov.w * ov.w;
      int t = 0;
#pragma unroll
      for (int m = 0; m < KM; ++m)
#pragma unroll
        for (int n = m; n < KM; ++n, ++t)
          acc[t] += oa0 * (u[m].x * u[n].x + u[m].y * u[n].y) + oa1 * (u[m].z * u[n].z + u[m].w * u[n].w);
    }
  }
  double v[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = (double)acc[t];
  block_sum<NV>(v, red);
  if (threadIdx.x != 0) return;
  if (!ls) {
    for (int m = 0; m < K; ++m) atomicAdd(gw + (size_t)j * K + m, (float)v[NA + m]);
    return;
  }
  double A[KM][KM], L[KM][KM], y[KM];
  int t = 0;
  for (int m = 0; m < KM; ++m)
    for (int n = m; n < KM; ++n, ++t) A[m][n] = A[n][m] = v[t];
  double tr = 0.0;
  for (int m = 0; m < K; ++m) tr += A[m][m];
  const double dmp = lam * tr / (double)K;
  for (int r = 0; r < K; ++r) {
    for (int c = 0; c <= r; ++c) {
      double sum = A[r][c] + (r == c ? dmp : 0.0);
      for (int k = 0; k < c; ++k) sum -= L[r][k] * L[c][k];
      if (r == c) {
        if (!(sum > 0.0)) return;   // not positive definite: no weight update
        L[r][r] = sqrt(sum);
      } else {
        L[r][c] = sum / L[c][c];
      }
    }
  }
  for (int r = 0; r < K; ++r) {    // L y = b
    double sum = v[NA + r];
    for (int k = 0; k < r; ++k) sum -= L[r][k] * y[k];
    y[r] = sum / L[r][r];
  }
  for (int r = K - 1; r >= 0; --r) {   // L^T x = y (x stored in y)
    double sum = y[r];
    for (int k = r + 1; k < K; ++k) sum -= L[k][r] * y[k];
    y[r] = sum / L[r][r];
  }
  for (int m = 0; m < K; ++m) w[(size_t)j * K + m] += (float)(step * y[m]);
}

static cudaError_t opr_reduce(int NN, int M, int K, int nb, int b0, const int* order, const float* w,
                              const float2* h_s, const float2* o_s, const int* valid, float2* dUacc, float* D,
                              cudaStream_t s) {
  // pixel pairs across blockIdx.x, the batch split into enough chunks for two CTAs per SM
  const int NP = NN / 2;
  const int bx = (NP + 255) / 256;
  int chunks = (2 * 152 + bx - 1) / bx;
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

static cudaError_t opr_weights(int N, int M, int K, int nb, int b0, const int* order, const int* valid,
                               const float2* U, const float2* h_s, const float2* o_s, float* w, float* gw,
                               double lam, float step, cudaStream_t s) {
  cudaEvent_t e0 = profile_begin(K_OPR_WEIGHTS, s);
  k_opr_weights<OPR_KMAX><<<nb, 256, 0, s>>>(N, M, K, b0, order, valid, U, h_s, o_s, w, gw, lam, step);
  profile_end(K_OPR_WEIGHTS, e0, s);
  return cudaGetLastError();
}

static ptycho_status check_opr_dims(const ptycho_dims* d, int32_t K) {
  const ptycho_status st = check_dims(d);
  if (st != PTYCHO_OK) return st;
  if (K < 1 || K > OPR_KMAX) return PTYCHO_ERR_UNSUPPORTED;
  return PTYCHO_OK;
}

static ptycho_status check_opr_opts(const ptycho_opr_opts* r) {
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
    if (probe_reduce(NN, 1, M - 1, M, nb, w.h, w.o, w.valid, o.update_probe ? w.dPacc : nullptr, 0,
                     o.update_probe ? w.Dp : nullptr, w.acc, HW, sc, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (o.update_probe) {
      if (cudaMemsetAsync(w.dUacc, 0, KNN * sizeof(float2), s) != cudaSuccess ||
          cudaMemsetAsync(w.Du, 0, KNN * sizeof(float), s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      if (opr_reduce(NN, M, K, nb, b0, order, wts, w.h, w.o, w.valid, w.dUacc, w.Du, s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      k_plane_max<<<grid_for(KNN, 256, 2 * 152), 256, 0, s>>>(w.Du, KNN, &sc->max_dp);
      if (cudaGetLastError() != cudaSuccess) return PTYCHO_ERR_CUDA;
    }
    if (norm_probe(NN, M - 1, w.dPacc, w.Dp, P_rest, (float)o.delta_p, o.update_probe, sc, w.dP, w.Cp, w.Sdp,
                   s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    k_norm_opr<<<grid_for(KNN, 256, 2 * 152), 256, 0, s>>>(KNN, w.dUacc, w.Du, o.update_probe, (float)o.delta_p,
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
    q.opr_dU = w.dU; q.opr_w = wts; q.K = K; q.p0_s = w.p0;
    if (pass2(N, q, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (r.update_weights && opr_weights(N, M, K, nb, b0, order, w.valid, U, w.h, w.o, wts, nullptr, o.lambda_reg,
                                        (float)r.weight_step, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
    if (cudaMemsetAsync(w.acc, 0, (size_t)HW * sizeof(float4), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
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
    if (g_w && opr_weights(N, M, K, nb, b0, nullptr, wp.valid, (const float2*)U, wp.h, wp.o, nullptr, g_w, 0.0,
                           0.f, s) != cudaSuccess)
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
