// Multislice entry points (Pty-Chi Sec. 1 and Sec. 2.1: multislice modelling):
// the angular-spectrum propagator, the forward model and the adjoint of the
// multislice per-position pass (kernels_ms.cuh; kernels_ms_cluster.cuh for the
// 192 and 256 windows).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "ptycho.h"
#include "common.cuh"
#include "internal.h"
#include "launch.h"
#include "profile.h"

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

MsLayout ms_layout(const ptycho_dims& d, int S, int B) {
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
  L.in = take((size_t)B * M * (S > 1 ? S - 1 : 0) * NN * sizeof(float2));
  L.go = take((size_t)B * S * NN * sizeof(float2));
  L.h = take((size_t)B * M * NN * sizeof(float2));
  L.valid = take((size_t)B * sizeof(int));
  L.total = off;
  return L;
}

ptycho_status check_ms(const ptycho_dims* d, const ptycho_multislice* ms) {
  const ptycho_status st = check_dims(d);
  if (st != PTYCHO_OK) return st;
  if (!ms || ms->reserved != 0) return PTYCHO_ERR_ARG;
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

// Fills the propagator and the common arguments; returns the layout.
MsLayout ms_setup(const ptycho_dims& d, const ptycho_multislice& ms, int batch, void* ws, MsArgs& a, cudaStream_t s,
                  cudaError_t* err) {
  const MsLayout L = ms_layout(d, ms.S, batch);
  char* b = (char*)ws;
  memset(&a, 0, sizeof(a));
  a.H = d.H; a.W = d.W; a.M = d.M; a.J = d.J; a.S = ms.S;
  a.Hf = (const float2*)(b + L.Hf);
  a.psi_s = (float2*)(b + L.psi);
  a.o_s = (float2*)(b + L.o);
  a.in_s = ms.S > 1 ? (float2*)(b + L.in) : nullptr;
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
  return ms_layout(*dims, ms->S, batch).total;
}

ptycho_status ptycho_forward_ms(const ptycho_dims* dims, const ptycho_multislice* ms, const float* object,
                                const float* probe, const float* pos, float* I_pred, int32_t batch, void* ws,
                                size_t ws_bytes, void* stream) {
  ptycho_status st = check_ms(dims, ms);
  if (st != PTYCHO_OK) return st;
  if (batch < 1 || !object || !probe || (dims->J > 0 && (!pos || !I_pred))) return PTYCHO_ERR_ARG;
  if ((st = check_ws(ws, ws_bytes, ms_layout(*dims, ms->S, batch).total)) != PTYCHO_OK) return st;
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
  if ((st = check_ws(ws, ws_bytes, ms_layout(*dims, ms->S, batch).total)) != PTYCHO_OK) return st;
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

}  // extern "C"
