// Multislice entry points (Pty-Chi Sec. 1 and Sec. 2.1: multislice modelling):
// the angular-spectrum propagator, the forward model and the adjoint of the
// multislice per-position pass (kernels_ms.cuh; kernels_ms_cluster.cuh for the
// 192 and 256 windows).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "ptycho.h"
#include "common.cuh"
#include "internal.h"
#include "launch.h"
#include "profile.h"
#include "kernels.cuh"

namespace ptycho {

// H[ky][kx] = exp(i 2 pi dz (sqrt(1/lambda^2 - |f|^2) - 1/lambda)) on the FFT
// grid f = k / (N pixel) (k = 0..N/2-1, -N/2..-1), evanescent frequencies 0;
// the bracket is evaluated as -|f|^2 / (sqrt(1/lambda^2 - |f|^2) + 1/lambda)
// in FP64 so that the large constant 1/lambda cancels exactly.
__global__ void k_asm_propagator(int N, double pixel, double wavelength, double dz, float2* Hf) {
  const int NN = N * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NN; i += gridDim.x * blockDim.x) {
    const int ky = i / N, kx = i % N;
    const double fy = (double)(ky < N / 2 ? ky : ky - N) / (N * pixel);
    const double fx = (double)(kx < N / 2 ? kx : kx - N) / (N * pixel);
    const double f2 = fy * fy + fx * fx, inv_l = 1.0 / wavelength, inv_l2 = inv_l * inv_l;
    float2 h = make_float2(0.f, 0.f);
    if (f2 < inv_l2) {
      const double ph = 2.0 * 3.14159265358979323846 * dz * (-f2 / (sqrt(inv_l2 - f2) + inv_l));
      double sn, cs;
      sincos(ph, &sn, &cs);
      h = make_float2((float)cs, (float)sn);
    }
    Hf[i] = h;
  }
}

namespace {

struct MsLayout {
  size_t hdr, Hf, psi, o, in, go, h, valid, total;
};

MsLayout ms_layout(const ptycho_dims& d, int S, int B, bool recompute) {
  MsLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t NN = (size_t)d.N * d.N, M = d.M;
  L.hdr = take(sizeof(WsHeader));
  L.Hf = take(NN * sizeof(float2));
  L.psi = take((size_t)B * M * NN * sizeof(float2));
  L.o = take((size_t)B * S * NN * sizeof(float2));
  // incident waves: every mode's kept by the forward pass, or one mode's at a time
  L.in = take((size_t)B * (recompute ? 1 : M) * (S > 1 ? S - 1 : 0) * NN * sizeof(float2));
  L.go = take((size_t)B * S * NN * sizeof(float2));
  L.h = take((size_t)B * M * NN * sizeof(float2));
  L.valid = take((size_t)B * sizeof(int));
  L.total = off;
  return L;
}

ptycho_status check_ms(const ptycho_dims* d, const ptycho_multislice* ms) {
  const ptycho_status st = check_dims(d);
  if (st != PTYCHO_OK) return st;
  if (!ms || (ms->recompute != 0 && ms->recompute != 1)) return PTYCHO_ERR_ARG;
  if (ms->S < 1 || ms->S > 16) return PTYCHO_ERR_UNSUPPORTED;
  if (!(ms->wavelength > 0.0) || !(ms->pixel_size > 0.0) || !(fabs(ms->dz) < 1e300)) return PTYCHO_ERR_ARG;
  if ((int64_t)ms->S * d->H * d->W > ((int64_t)1 << 31) - 1) return PTYCHO_ERR_ARG;
  return PTYCHO_OK;
}

cudaError_t pass1_ms(int N, const MsArgs& a, cudaStream_t s) {
  cudaEvent_t e0 = profile_begin(K_PASS1_MS, s);
  cudaError_t e = cudaErrorInvalidValue;
  switch (N) {
    case 16: e = launch_pass1_ms<16>(a, s); break;
    case 32: e = launch_pass1_ms<32>(a, s); break;
    case 64: e = launch_pass1_ms<64>(a, s); break;
    case 128: e = launch_pass1_ms<128>(a, s); break;
    case 192: e = launch_pass1_ms<192>(a, s); break;
    case 256: e = launch_pass1_ms<256>(a, s); break;
  }
  profile_end(K_PASS1_MS, e0, s);
  return e;
}

// ---------------------------------------------------------------------------
// LSQML with a multislice object. Per slice s the exit-plane change carried
// back through the slices gives the direction numerator g_js (go_s) and the
// illumination sum_k |inc_jsk|^2 (w_s; slice 0: Sp); every slice has its own
// object-frame accumulator and preconditioner damping; slice 0 shares the 2x2
// step-size system with the probe, later slices have 1x1 fits.
// ---------------------------------------------------------------------------
struct MsLsqmlLayout {
  MsLayout base;
  size_t acc, w, dPacc, Dp, dP, Sp, Cp, Sdp, smax, d, u, part, dsum, total;
};

MsLsqmlLayout ms_lsqml_layout(const ptycho_dims& d, int S, int B, bool recompute) {
  MsLsqmlLayout L;
  L.base = ms_layout(d, S, B, recompute);
  size_t off = L.base.total;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t NN = (size_t)d.N * d.N, M = d.M, HW = (size_t)d.H * d.W;
  L.acc = take((size_t)S * HW * sizeof(float4));
  L.w = take((size_t)B * (S > 1 ? S - 1 : 0) * NN * sizeof(float));
  L.dPacc = take(M * NN * sizeof(float2));
  L.Dp = take(NN * sizeof(float));
  L.dP = take(M * NN * sizeof(float2));
  L.Sp = take(NN * sizeof(float));
  L.Cp = take(NN * sizeof(float2));
  L.Sdp = take(NN * sizeof(float));
  L.smax = take(16 * sizeof(unsigned int));
  L.d = take((size_t)B * S * NN * sizeof(float2));        // the slices' directions at each slot's position
  L.u = take((size_t)B * NN * sizeof(float2));            // one mode's object tangent per slot
  L.part = take((size_t)B * 8 * 3 * sizeof(double));      // Gram partials, up to 8 CTAs per position
  L.dsum = take((size_t)B * S * 2 * sizeof(double));      // right-hand-side partials per slot and slice
  L.total = off;
  return L;
}

struct MsPass2Args {
  int H, W, M, J, S;
  const float* pos;
  const int* order;
  int b0, nb;
  const float2* o_s;          // [B, S, N, N]
  const float2* go_s;         // [B, S, N, N] direction numerators
  const float2* h_s;          // [B, M, N, N]
  const float* w_s;           // [B, S - 1, N, N]
  const int* valid;
  const float4* acc;          // [S, H, W]
  const unsigned int* smax;   // [S] float bits of each slice's maximum illumination
  const float* Sp;
  const float2* Cp;
  const float* Sdp;
  const float2* dP;
  float2* obj;                // [S, H, W], updated in place
  double* alpha_out;          // [J, 2] or null
  BatchScalars* sc;
  float delta_o;
  double lam;
  int update_object, update_probe;
  float2* d_s;                // [B, S, N, N] directions at the slots' positions (written by k_ms_dir)
  double* dsum;               // [B, S, 2]: Re<d_s, g_s> per slice; slice 0 also Re sum_k <dP_k, h_k>
  const double* part;         // [B, Q, 3] Gram partials of the tangents (k_step_ms)
  int Q;                      // CTAs per position of the tangent pass
};

// max over the illumination component of each slice's accumulator
__global__ void k_ms_illum_max(size_t HW, const float4* __restrict__ acc, unsigned int* smax) {
  __shared__ float red[32];
  const float4* a = acc + (size_t)blockIdx.y * HW;
  float m = illum_max_share<8>(a, HW, blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(smax + blockIdx.y, __float_as_uint(m));
}

// One CTA per (position, slice): the slice's preconditioned direction at the
// position, d_s = S_j(dO_acc_s / (illum_s + delta_O,s)) (bilinear, the
// quotient taken per corner), into scratch for the tangent pass, and the
// right-hand-side term Re<d_s, g_s>; the slice-0 CTA adds the probe's
// Re sum_k <dP_k, h_k>.
template <int N>
__global__ void __launch_bounds__(512, 1) k_ms_dir(MsPass2Args a) {
  constexpr int NN = N * N, T = 512;
  __shared__ double red[32 * 2];
  const int slot = blockIdx.x, s = blockIdx.y, tid = threadIdx.x, S = a.S;
  double* out = a.dsum + ((size_t)slot * S + s) * 2;
  if (!a.valid[slot]) {
    if (tid < 2) out[tid] = 0.0;
    return;
  }
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  int ty, tx;
  float fy, fx;
  tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  const size_t HW = (size_t)a.H * a.W;
  const float4* acc = a.acc + s * HW;
  const float damp = a.delta_o * __uint_as_float(a.smax[s]);
  const float2* g_s = a.go_s + ((size_t)slot * S + s) * NN;
  float2* d_s = a.d_s + ((size_t)slot * S + s) * NN;
  float b1 = 0.f, b2 = 0.f;
#pragma unroll 1
  for (int p = tid; p < NN; p += T) {
    const int r = p / N, c = p % N;
    float2 d = make_float2(0.f, 0.f);
    if (a.update_object) d = dohat(acc + (size_t)(ty + r) * a.W + (tx + c), a.W, w00, w01, w10, w11, damp);
    d_s[p] = d;
    const float2 g = __ldcs(g_s + p);
    b1 += d.x * g.x + d.y * g.y;             // Re(conj(d) g)
  }
  if (s == 0 && a.update_probe) {
    const float4* h4 = (const float4*)(a.h_s + (size_t)slot * a.M * NN);
    const float4* d4 = (const float4*)a.dP;
    const int Qp = a.M * NN / 2;
    for (int q = tid; q < Qp; q += T) {
      const float4 dp = __ldg(d4 + q);
      const float4 h = __ldcs(h4 + q);
      b2 += dp.x * h.x + dp.y * h.y + dp.z * h.z + dp.w * h.w;   // Re(conj(dP_k) h_k)
    }
  }
  double v[2] = {b1, b2};
  block_sum<2>(v, red);
  if (tid == 0) {
    out[0] = v[0];
    out[1] = v[1];
  }
}

// One CTA per (position, slice): the 2x2 step-size system of the position
// (Gram entries of the tangents, right-hand sides from the slices' and the
// probe's numerators, summed in a fixed order), the FP64 solve (the same in
// every slice's CTA), and the slice's update O_s += alpha_O S_j^T g_s /
// (illum_s + delta_O,s); the slice-0 CTA records alpha and adds alpha_P to
// the minibatch's mean.
template <int N>
__global__ void __launch_bounds__(512, 2) k_ms_update(MsPass2Args a) {
  constexpr int NN = N * N, T = 512;
  __shared__ double alpha_sh;
  const int slot = blockIdx.x, s = blockIdx.y, tid = threadIdx.x, S = a.S;
  if (!a.valid[slot]) return;
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  if (tid == 0) {
    double a11 = 0.0, a12 = 0.0, a22 = 0.0, r1 = 0.0;
    for (int q = 0; q < a.Q; ++q) {
      const double* pp = a.part + ((size_t)slot * a.Q + q) * 3;
      a11 += pp[0];
      a12 += pp[1];
      a22 += pp[2];
    }
    for (int t = 0; t < S; ++t) r1 += a.dsum[((size_t)slot * S + t) * 2];
    const double r2 = a.dsum[(size_t)slot * S * 2 + 1];
    const double tr = 0.5 * (a11 + a22);
    const double d11 = a11 + a.lam * tr, d22 = a22 + a.lam * tr;
    const double det = d11 * d22 - a12 * a12;
    double aO, aP;
    if (det > 0.0) {
      aO = (d22 * r1 - a12 * r2) / det;
      aP = (d11 * r2 - a12 * r1) / det;
    } else {
      aO = d11 > 0.0 ? r1 / d11 : 0.0;
      aP = d22 > 0.0 ? r2 / d22 : 0.0;
    }
    if (s == 0) {
      atomicAdd(&a.sc->sum_alpha_p, aP);
      atomicAdd(&a.sc->count, 1);
      if (a.alpha_out) {
        a.alpha_out[2 * j] = aO;
        a.alpha_out[2 * j + 1] = aP;
      }
    }
    alpha_sh = aO;
  }
  __syncthreads();
  if (!a.update_object) return;
  int ty, tx;
  float fy, fx;
  tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  const size_t HW = (size_t)a.H * a.W;
  const float4* acc = a.acc + s * HW;
  const float damp = a.delta_o * __uint_as_float(a.smax[s]);
  const float2* g_s = a.go_s + ((size_t)slot * S + s) * NN;
  const float aO = (float)alpha_sh;
  const float c00 = aO * (1.f - fy) * (1.f - fx), c01 = aO * (1.f - fy) * fx;
  const float c10 = aO * fy * (1.f - fx), c11 = aO * fy * fx;
  float2* obj = a.obj + s * HW;
  constexpr int N1 = N + 1;
  for (int q = tid; q < N1 * N1; q += T) {
    const int y = q / N1, x = q % N1;
    float2 sacc = make_float2(0.f, 0.f);
    if (y < N && x < N) { const float2 g = g_s[y * N + x]; sacc.x += c00 * g.x; sacc.y += c00 * g.y; }
    if (y < N && x > 0) { const float2 g = g_s[y * N + x - 1]; sacc.x += c01 * g.x; sacc.y += c01 * g.y; }
    if (y > 0 && x < N) { const float2 g = g_s[(y - 1) * N + x]; sacc.x += c10 * g.x; sacc.y += c10 * g.y; }
    if (y > 0 && x > 0) { const float2 g = g_s[(y - 1) * N + x - 1]; sacc.x += c11 * g.x; sacc.y += c11 * g.y; }
    const size_t oi = (size_t)(ty + y) * a.W + (tx + x);
    const float inv = 1.f / (__ldg(&acc[oi].z) + damp);
    atomicAdd(obj + oi, make_float2(sacc.x * inv, sacc.y * inv));
  }
}

template <class Fn>
cudaError_t dispatch_ms_N(int N, Fn&& fn) {
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

// The step-size pass of the multislice LSQML minibatch: directions at the
// positions and the right-hand sides (k_ms_dir), the tangents' Gram entries
// (k_step_ms), then the solve and the slices' updates (k_ms_update).
cudaError_t pass2_ms(int N, const MsPass2Args& a, const MsStepArgs& t, cudaStream_t s) {
  if (a.nb <= 0) return cudaSuccess;
  const dim3 grid((unsigned)a.nb, (unsigned)a.S);
  cudaEvent_t e0 = profile_begin(K_PASS2, s);
  cudaError_t e = dispatch_ms_N(N, [&](auto c) {
    constexpr int NC = decltype(c)::value;
    k_ms_dir<NC><<<grid, 512, 0, s>>>(a);
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    if ((r = launch_step_ms<NC>(t, s)) != cudaSuccess) return r;
    k_ms_update<NC><<<grid, 512, 0, s>>>(a);
    return cudaGetLastError();
  });
  profile_end(K_PASS2, e0, s);
  return e;
}

// Fills the propagator and the common arguments; returns the layout.
MsLayout ms_setup(const ptycho_dims& d, const ptycho_multislice& ms, int batch, void* ws, MsArgs& a, cudaStream_t s,
                  cudaError_t* err) {
  const MsLayout L = ms_layout(d, ms.S, batch, ms.recompute != 0);
  char* b = (char*)ws;
  memset(&a, 0, sizeof(a));
  a.H = d.H; a.W = d.W; a.M = d.M; a.J = d.J; a.S = ms.S;
  a.Hf = (const float2*)(b + L.Hf);
  a.psi_s = (float2*)(b + L.psi);
  a.o_s = (float2*)(b + L.o);
  a.in_s = ms.S > 1 ? (float2*)(b + L.in) : nullptr;
  a.recompute = ms.recompute;
  a.go_s = (float2*)(b + L.go);
  a.h_s = (float2*)(b + L.h);
  a.valid = (int*)(b + L.valid);
  a.status = &((WsHeader*)ws)->status;
  k_asm_propagator<<<grid_for((size_t)d.N * d.N, 256, sm_count()), 256, 0, s>>>(d.N, ms.pixel_size, ms.wavelength, ms.dz,
                                                                          (float2*)(b + L.Hf));
  *err = cudaGetLastError();
  return L;
}

}  // namespace
}  // namespace ptycho

using namespace ptycho;

extern "C" {

size_t ptycho_workspace_bytes_ms(const ptycho_dims* dims, const ptycho_multislice* ms, int32_t batch) {
  if (check_ms(dims, ms) != PTYCHO_OK || batch < 1) return 0;
  return ms_layout(*dims, ms->S, batch, ms->recompute != 0).total;
}

ptycho_status ptycho_forward_ms(const ptycho_dims* dims, const ptycho_multislice* ms, const float* object,
                                const float* probe, const float* pos, float* I_pred, int32_t batch, void* ws,
                                size_t ws_bytes, void* stream) {
  ptycho_status st = check_ms(dims, ms);
  if (st != PTYCHO_OK) return st;
  if (batch < 1 || !object || !probe || (dims->J > 0 && (!pos || !I_pred))) return PTYCHO_ERR_ARG;
  if ((st = check_ws(ws, ws_bytes, ms_layout(*dims, ms->S, batch, ms->recompute != 0).total)) != PTYCHO_OK)
    return st;
  if (dims->J == 0) return PTYCHO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  MsArgs a;
  cudaError_t e = cudaSuccess;
  ms_setup(*dims, *ms, batch, ws, a, s, &e);
  if (e != cudaSuccess) return PTYCHO_ERR_CUDA;
  a.obj = (const float2*)object; a.probe = (const float2*)probe; a.pos = pos;
  a.mode = MODE_FWD; a.ipred = I_pred;
  for (int b0 = 0; b0 < dims->J; b0 += batch) {
    a.b0 = b0;
    a.nb = (dims->J - b0 < batch) ? dims->J - b0 : batch;
    if (pass1_ms(dims->N, a, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

ptycho_status ptycho_adjoint_ms(const ptycho_dims* dims, const ptycho_multislice* ms, const float* object,
                                const float* probe, const float* pos, const float* meas, int32_t noise, double eps,
                                int32_t batch, float* g_object, float* g_probe, float* g_pos, double* loss, void* ws,
                                size_t ws_bytes, void* stream) {
  ptycho_status st = check_ms(dims, ms);
  if (st != PTYCHO_OK) return st;
  if (batch < 1 || !(eps >= 0.0)) return PTYCHO_ERR_ARG;
  if (noise != PTYCHO_NOISE_GAUSSIAN && noise != PTYCHO_NOISE_POISSON && noise != PTYCHO_NOISE_VJP)
    return PTYCHO_ERR_ARG;
  if (!object || !probe || !g_object || !g_probe || (dims->J > 0 && (!pos || !meas))) return PTYCHO_ERR_ARG;
  if ((st = check_ws(ws, ws_bytes, ms_layout(*dims, ms->S, batch, ms->recompute != 0).total)) != PTYCHO_OK)
    return st;
  if (dims->J == 0) return PTYCHO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  MsArgs a;
  cudaError_t e = cudaSuccess;
  ms_setup(*dims, *ms, batch, ws, a, s, &e);
  if (e != cudaSuccess) return PTYCHO_ERR_CUDA;
  a.obj = (const float2*)object; a.probe = (const float2*)probe; a.pos = pos; a.meas = meas;
  a.mode = noise == PTYCHO_NOISE_GAUSSIAN ? MODE_GRAD_GAUSS : noise == PTYCHO_NOISE_POISSON ? MODE_GRAD_POISSON
                                                                                          : MODE_VJP;
  a.eps = (float)eps;
  a.gobj = (float2*)g_object; a.gpos = g_pos; a.loss = loss;
  const int NN = dims->N * dims->N;
  for (int b0 = 0; b0 < dims->J; b0 += batch) {
    a.b0 = b0;
    a.nb = (dims->J - b0 < batch) ? dims->J - b0 : batch;
    if (pass1_ms(dims->N, a, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (probe_reduce(NN, 0, dims->M, dims->M, a.nb, a.h_s, a.o_s, a.valid, (float2*)g_probe, 1, nullptr, nullptr, 0,
                     nullptr, s) != cudaSuccess)
      return PTYCHO_ERR_CUDA;
  }
  return PTYCHO_OK;
}

size_t ptycho_workspace_bytes_lsqml_ms(const ptycho_dims* dims, const ptycho_multislice* ms,
                                        const ptycho_lsqml_opts* opts) {
  if (check_ms(dims, ms) != PTYCHO_OK || check_opts(opts) != PTYCHO_OK) return 0;
  return ms_lsqml_layout(*dims, ms->S, opts->batch, ms->recompute != 0).total;
}

ptycho_status ptycho_lsqml_epoch_ms(const ptycho_dims* dims, const ptycho_multislice* ms, float* object, float* probe,
                                    const float* pos, const float* meas, const int32_t* order,
                                    const ptycho_lsqml_opts* opts, double* loss, double* alpha, void* ws,
                                    size_t ws_bytes, void* stream) {
  ptycho_status st = check_ms(dims, ms);
  if (st != PTYCHO_OK) return st;
  if ((st = check_opts(opts)) != PTYCHO_OK) return st;
  if (opts->precision != PTYCHO_PRECISION_FP32 || opts->update_positions || opts->object_per_epoch)
    return PTYCHO_ERR_UNSUPPORTED;
  if (!object || !probe || (dims->J > 0 && (!pos || !meas))) return PTYCHO_ERR_ARG;
  const MsLsqmlLayout L = ms_lsqml_layout(*dims, ms->S, opts->batch, ms->recompute != 0);
  if ((st = check_ws(ws, ws_bytes, L.total)) != PTYCHO_OK) return st;
  auto body = [&](cudaStream_t s) -> ptycho_status {
    const ptycho_dims& d = *dims;
    const int S = ms->S, B = opts->batch, M = d.M, NN = d.N * d.N;
    const size_t HW = (size_t)d.H * d.W;
    char* b = (char*)ws;
    WsHeader* hdr = (WsHeader*)ws;
    float4* acc = (float4*)(b + L.acc);
    float2* dPacc = (float2*)(b + L.dPacc);
    float* Dp = (float*)(b + L.Dp);
    float2* dP = (float2*)(b + L.dP);
    float* Sp = (float*)(b + L.Sp);
    float2* Cp = (float2*)(b + L.Cp);
    float* Sdp = (float*)(b + L.Sdp);
    unsigned int* smax = (unsigned int*)(b + L.smax);
    MsArgs a;
    cudaError_t e = cudaSuccess;
    ms_setup(d, *ms, B, ws, a, s, &e);
    if (e != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (cudaMemsetAsync(acc, 0, (size_t)S * HW * sizeof(float4), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    if (init_epoch(NN, M, (const float2*)probe, Sp, hdr, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
    a.obj = (const float2*)object; a.probe = (const float2*)probe; a.pos = pos; a.meas = meas; a.order = order;
    a.mode = opts->noise == PTYCHO_NOISE_POISSON ? MODE_LSQML_POISSON : MODE_LSQML_GAUSS;
    a.eps = (float)opts->eps;
    a.loss = loss;
    a.acc = acc;
    a.w_s = (float*)(b + L.w);
    a.Sp = Sp;
    const int nbatch = (d.J + B - 1) / B;
    for (int bi = 0; bi < nbatch; ++bi) {
      BatchScalars* sc = &hdr->sc[bi & 1];
      BatchScalars* sc_next = &hdr->sc[(bi + 1) & 1];
      a.b0 = bi * B;
      a.nb = (d.J - a.b0 < B) ? d.J - a.b0 : B;
      if (pass1_ms(d.N, a, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
      if (probe_reduce(NN, 0, M, M, a.nb, a.h_s, a.o_s, a.valid, opts->update_probe ? dPacc : nullptr, 0,
                       opts->update_probe ? Dp : nullptr, nullptr, 0, sc, s, S * NN) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      if (cudaMemsetAsync(smax, 0, (size_t)S * sizeof(unsigned int), s) != cudaSuccess) return PTYCHO_ERR_CUDA;
      k_ms_illum_max<<<dim3((unsigned)grid_for(HW, 256, 2 * sm_count()), (unsigned)S), 256, 0, s>>>(HW, acc, smax);
      if (cudaGetLastError() != cudaSuccess) return PTYCHO_ERR_CUDA;
      if (norm_probe(NN, M, dPacc, Dp, (const float2*)probe, (float)opts->delta_p, opts->update_probe, sc, dP, Cp,
                     Sdp, s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      MsPass2Args q;
      memset(&q, 0, sizeof(q));
      q.H = d.H; q.W = d.W; q.M = M; q.J = d.J; q.S = S;
      q.pos = pos; q.order = order; q.b0 = a.b0; q.nb = a.nb;
      q.o_s = a.o_s; q.go_s = a.go_s; q.h_s = a.h_s; q.w_s = a.w_s; q.valid = a.valid;
      q.acc = acc; q.smax = smax; q.Sp = Sp; q.Cp = Cp; q.Sdp = Sdp; q.dP = dP;
      q.obj = (float2*)object; q.alpha_out = alpha; q.sc = sc;
      q.delta_o = (float)opts->delta_o; q.lam = opts->lambda_reg;
      q.update_object = opts->update_object; q.update_probe = opts->update_probe;
      q.d_s = (float2*)(b + L.d); q.dsum = (double*)(b + L.dsum); q.part = (double*)(b + L.part);
      q.Q = ms_cluster_ctas(d.N);
      MsStepArgs t;
      memset(&t, 0, sizeof(t));
      t.H = d.H; t.W = d.W; t.M = M; t.J = d.J; t.S = S;
      t.order = order; t.b0 = a.b0; t.nb = a.nb;
      t.probe = (const float2*)probe; t.Hf = a.Hf; t.o_s = a.o_s; t.in_s = a.in_s; t.d_s = q.d_s; t.dP = dP;
      t.recompute = a.recompute;
      t.u_s = (float2*)(b + L.u); t.valid = a.valid; t.part = (double*)(b + L.part);
      if (pass2_ms(d.N, q, t, s) != cudaSuccess) return PTYCHO_ERR_CUDA;
      if (clear_acc(false, ptycho_dims{(int32_t)(S * d.H), d.W, d.N, d.M, d.J}, a.nb, a.b0, pos, order, a.valid, acc,
                    s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
      if (probe_update(NN, M, (float2*)probe, dP, Sp, opts->update_probe, sc, sc_next, s) != cudaSuccess)
        return PTYCHO_ERR_CUDA;
    }
    return PTYCHO_OK;
  };
  if (!(opts->flags & PTYCHO_FLAG_GRAPH)) return body((cudaStream_t)stream);
  GraphKey key;
  key.add(*dims).add(*ms).add(object).add(probe).add(pos).add(meas).add(order).add(*opts).add(loss).add(alpha).add(ws);
  return run_graphed(key, (cudaStream_t)stream, body);
}

}  // extern "C"
