// Far-field stage of the per-position pass with the 2-D DFT evaluated as
// dense complex GEMMs on the 5th-generation tensor cores, in split BF16:
// every FP32 operand x is carried as x_hi + x_lo (x_hi = bf16(x),
// x_lo = bf16(x - x_hi)), and each real product keeps the three terms
// A_hi B_hi + A_lo B_hi + A_hi B_lo, accumulated in FP32 in tensor memory.
//
// The unitary 2-D DFT of an N x N tile X is F X F^T with F[m][c] =
// exp(-2 pi i m c / N) / sqrt(N) (Sec. 2.1, Eq. 4's far-field propagator).
// With D[m][n] = sum_c A[m][c] B[n][c] (A and B both K-major) it is two
// passes with the DFT matrix as A:
//   pass 1: D1[f][r] = sum_c F[f][c] X[r][c]       (B = X: rows r, K = columns c)
//   pass 2: D2[f'][f] = sum_r F[f'][r] D1[f][r]    (B = D1: rows f, K = r)
// so D2 = F X F^T with the row index in the TMEM lane and no transpose in
// between: the thread that owns TMEM lane f after pass 1 writes row f of the
// next B operand. The inverse uses conj(F). A complex product is four real
// products on separate re/im planes, the sign of the Fi terms chosen by the
// instruction descriptor's negate-A bit.
//
// k_far_tc: per minibatch position (persistent CTAs, 8 warps): the exit waves
// psi_jk (written by the first part of the per-position pass) are
// transformed mode by mode; the far fields overwrite them in the scratch and
// their intensities accumulate per thread; the data term (Eq. 1 amplitude
// loss or the Poisson likelihood) gives the loss and the far-field factor;
// every mode is then scaled and transformed back, and chi_jk = F^-1[(rho - 1)
// Psi_jk] overwrites the scratch for the overlap-add part of the pass.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace ptycho {

template <int N>
struct FarTc {
  static_assert(N == 32 || N == 64 || N == 128, "DFT-GEMM windows");
  static constexpr int T = 256;                  // 8 warps: TMEM lane quarter w % 4, column half w / 4
  static constexpr int HALF = N / 2;
  static constexpr int NCH = N / 16;             // K-steps of one pass (= DFT chunks)
  static constexpr int NS = 4;                   // ring slots of DFT chunks
  static constexpr int MT = 128;                 // MMA tile rows (DFT rows beyond N are zero)
  static constexpr uint32_t APLANE = MT * 16 * 2;            // one 128 x 16 BF16 plane of a chunk
  static constexpr uint32_t CHUNK = 4 * APLANE;              // Fr_hi, Fr_lo, Fi_hi, Fi_lo
  static constexpr uint32_t ASBO = 256;                      // 8-row groups of a 16-wide K slice
  static constexpr uint32_t BPLANE = (uint32_t)N * N * 2;    // one N x N BF16 operand plane
  static constexpr uint32_t BSBO = (uint32_t)(N / 8) * 128;  // 8-row groups of a full-K plane
  static constexpr size_t planes = 0;                        // Xr_hi, Xr_lo, Xi_hi, Xi_lo
  static constexpr size_t ring = planes + 4 * (size_t)BPLANE;
  static constexpr size_t bars = ring + (size_t)NS * CHUNK;  // full[NS], empty[NS], done
  static constexpr size_t red = bars + 128;
  static constexpr size_t misc = red + 32 * sizeof(double);
  static constexpr size_t bytes = misc + 16;
  static constexpr uint32_t COLS = 2 * N;                    // TMEM: D_re [0, N), D_im [N, 2N)
  static constexpr size_t dft_bytes = (size_t)NCH * CHUNK;
};

struct FarArgs {
  int H, W, M, J;
  const float* pos;
  const int* order;
  int b0, nb, mode;
  float eps;
  const float* meas;      // measured intensities, or dL/dI in MODE_VJP
  float2* psi_s;          // [B, M, N, N]: exit waves in, chi out (natural layout)
  const uint16_t* dft;    // DFT chunks written by k_dft_planes
  float* ipred;           // [J, N, N] or null
  double* loss;           // or null
  int* status;
};

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
// x = hi + lo + O(2^-18 |x|)
__device__ __forceinline__ void split_bf16(float v, uint16_t& hi, uint16_t& lo) {
  hi = bf16_bits(v);
  lo = bf16_bits(v - bf16_value(hi));
}

// The DFT matrix of one pass as NCH chunks (one per 16-wide K slice), each the
// four planes Fr_hi, Fr_lo, Fi_hi, Fi_lo of 128 rows x 16 BF16 in the
// operand's shared-memory image (core matrices of 8 rows x 16 bytes, K-adjacent
// ones 128 bytes apart, 8-row groups 256 bytes apart). F[m][c] =
// exp(-2 pi i m c / N), rows m >= N zero; evaluated in FP64 from m c mod N.
template <int N>
__global__ void k_dft_planes(uint16_t* out) {
  using C = FarTc<N>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C::NCH * C::MT * 16) return;
  const int s = idx / (C::MT * 16), m = (idx / 16) % C::MT, kk = idx % 16, c = 16 * s + kk;
  double re = 0.0, im = 0.0;
  if (m < N) {
    const int r = (int)(((long long)m * c) % N);
    double sn, cs;
    sincospi(2.0 * (double)r / (double)N, &sn, &cs);
    re = cs;
    im = -sn;
  }
  const size_t e = (size_t)s * (C::CHUNK / 2) + (size_t)(m / 8) * (C::ASBO / 2) + (kk / 8) * 64 + (m % 8) * 8 + (kk % 8);
  constexpr size_t P = C::APLANE / 2;
  const float reh = (float)re, imh = (float)im;
  const uint16_t rh = bf16_bits(reh), ih = bf16_bits(imh);
  out[e] = rh;
  out[e + P] = bf16_bits((float)(re - (double)bf16_value(rh)));
  out[e + 2 * P] = ih;
  out[e + 3 * P] = bf16_bits((float)(im - (double)bf16_value(ih)));
}

// Eight consecutive K values (k0 % 8 == 0) of operand row `row` into the four
// planes (hi/lo of the real and imaginary parts).
template <int N>
__device__ __forceinline__ void put8(unsigned char* planes, int row, int k0, const float* re, const float* im) {
  using C = FarTc<N>;
  uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint16_t a0, b0, a1, b1;
    split_bf16(re[2 * q], a0, b0);
    split_bf16(re[2 * q + 1], a1, b1);
    rh[q] = (uint32_t)a0 | ((uint32_t)a1 << 16);
    rl[q] = (uint32_t)b0 | ((uint32_t)b1 << 16);
    split_bf16(im[2 * q], a0, b0);
    split_bf16(im[2 * q + 1], a1, b1);
    ih[q] = (uint32_t)a0 | ((uint32_t)a1 << 16);
    il[q] = (uint32_t)b0 | ((uint32_t)b1 << 16);
  }
  unsigned char* p = planes + (size_t)(row / 8) * C::BSBO + (size_t)(k0 / 8) * 128 + (row % 8) * 16;
  *(uint4*)p = make_uint4(rh[0], rh[1], rh[2], rh[3]);
  *(uint4*)(p + C::BPLANE) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
  *(uint4*)(p + 2 * C::BPLANE) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
  *(uint4*)(p + 3 * C::BPLANE) = make_uint4(il[0], il[1], il[2], il[3]);
}

// Row `row`, columns [c0, c0 + N/2) of an N x N complex image in global
// memory (times the per-column factor f when SCALE) into the operand planes.
template <int N, bool SCALE>
__device__ __forceinline__ void rows_to_planes(unsigned char* planes, const float2* src, int row, int c0,
                                               const float (&f)[N / 2]) {
  // 16 columns (eight 16-byte loads) in flight per step
#pragma unroll
  for (int g = 0; g < N / 16; g += 2) {
    const float4* s = (const float4*)(src + (size_t)row * N + c0 + 8 * g);
    float4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcg(s + q);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float re[8], im[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        re[2 * q] = v[4 * h + q].x; im[2 * q] = v[4 * h + q].y;
        re[2 * q + 1] = v[4 * h + q].z; im[2 * q + 1] = v[4 * h + q].w;
      }
      if (SCALE) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          re[i] *= f[8 * (g + h) + i];
          im[i] *= f[8 * (g + h) + i];
        }
      }
      put8<N>(planes, row, c0 + 8 * (g + h), re, im);
    }
  }
}

// The pass result in TMEM (this thread's lane = operand row) into the planes
// as the next pass's B operand.
template <int N>
__device__ __forceinline__ void tmem_to_planes(unsigned char* planes, uint32_t trow, int row, int c0) {
  constexpr int G = N / 32 < 2 ? N / 32 : 2;   // 16-column groups per TMEM round trip
#pragma unroll 1
  for (int g = 0; g < N / 32; g += G) {
    float re[G][16], im[G][16];
#pragma unroll
    for (int h = 0; h < G; ++h) {
      tc::tmem_ld16(trow + c0 + 16 * (g + h), re[h]);
      tc::tmem_ld16(trow + N + c0 + 16 * (g + h), im[h]);
    }
    tc::tmem_wait_ld();
#pragma unroll
    for (int h = 0; h < G; ++h) {
      put8<N>(planes, row, c0 + 16 * (g + h), re[h], im[h]);
      put8<N>(planes, row, c0 + 16 * (g + h) + 8, re[h] + 8, im[h] + 8);
    }
  }
}

// The pass result (row `row`, columns [c0, c0 + N/2)) times `scale` into
// global memory; with ACC its squared modulus is added to (or, when `first`,
// stored into) `acc`.
template <int N, bool ACC>
__device__ __forceinline__ void tmem_to_global(float2* dst, uint32_t trow, int row, int c0, float scale,
                                               float (&acc)[N / 2], bool first) {
  constexpr int G = N / 32 < 2 ? N / 32 : 2;   // 16-column groups per TMEM round trip
#pragma unroll
  for (int g = 0; g < N / 32; g += G) {
    float re[G][16], im[G][16];
#pragma unroll
    for (int h = 0; h < G; ++h) {
      tc::tmem_ld16(trow + c0 + 16 * (g + h), re[h]);
      tc::tmem_ld16(trow + N + c0 + 16 * (g + h), im[h]);
    }
    tc::tmem_wait_ld();
#pragma unroll
    for (int h = 0; h < G; ++h) {
      float4* d = (float4*)(dst + (size_t)row * N + c0 + 16 * (g + h));
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const float x0 = re[h][i] * scale, y0 = im[h][i] * scale;
        const float x1 = re[h][i + 1] * scale, y1 = im[h][i + 1] * scale;
        d[i / 2] = make_float4(x0, y0, x1, y1);
        if (ACC) {
          const int c = 16 * (g + h) + i;
          const float a0 = fmaf(x0, x0, y0 * y0), a1 = fmaf(x1, x1, y1 * y1);
          acc[c] = first ? a0 : acc[c] + a0;
          acc[c + 1] = first ? a1 : acc[c + 1] + a1;
        }
      }
    }
  }
}

template <int N>
__global__ void __launch_bounds__(256, 1) k_far_tc(FarArgs a) {
  using C = FarTc<N>;
  constexpr int NN = N * N, HALF = C::HALF;
  extern __shared__ __align__(16) unsigned char smem[];
  wait_prior_grid();
  unsigned char* planes = smem + C::planes;
  unsigned char* ring = smem + C::ring;
  uint64_t* full = (uint64_t*)(smem + C::bars);
  uint64_t* empty = full + C::NS;
  uint64_t* done = empty + C::NS;
  double* red = (double*)(smem + C::red);
  uint32_t* holder = (uint32_t*)(smem + C::misc);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane;   // TMEM lane = operand row
  const int c0 = (warp >> 2) * HALF;        // this thread's column half
  const bool act = row < N;                 // warp-uniform (N is a multiple of 32)

  if (tid == 0) {
    for (int s = 0; s < C::NS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(holder, C::COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *holder;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const unsigned char* dft = (const unsigned char*)a.dft;

  // Ring of DFT chunks: chunk q of the (periodic) sequence 0..NCH-1, 0.. lives
  // in slot q % NS; `full` completes when its bytes have landed, `empty` when
  // the MMAs reading it have completed. Only thread 0 uses these counters.
  long long qc = 0, issued = 0;
  if (tid == 0) {
    for (int s = 0; s < C::NS; ++s) {
      tc::mbar_expect_tx(&full[s], C::CHUNK);
      tc::bulk_g2s(ring + (size_t)s * C::CHUNK, dft + (size_t)(s % C::NCH) * C::CHUNK, C::CHUNK, &full[s]);
    }
    issued = C::NS;
  }

  constexpr uint32_t I_POS = tc::idesc_bf16(C::MT, N, false), I_NEG = tc::idesc_bf16(C::MT, N, true);
  // One pass: NCH K-steps of 12 MMAs (3 split terms x 4 real products), then
  // a commit to `done`. Thread 0 only; false if a wait gave up.
  auto issue_pass = [&](bool inverse) -> bool {
    const uint32_t pb = tc::smem_u32(planes);
    const uint32_t i_re = inverse ? I_POS : I_NEG;   // Fi Xi into D_re: minus forward, plus inverse
    const uint32_t i_im = inverse ? I_NEG : I_POS;   // Fi Xr into D_im: plus forward, minus inverse
    const uint32_t dre = tmem, dim = tmem + N;
    for (int s = 0; s < C::NCH; ++s, ++qc) {
      const int sl = (int)(qc % C::NS);
      if (!tc::mbar_wait(&full[sl], (uint32_t)((qc / C::NS) & 1))) return false;
      const uint32_t sa = tc::smem_u32(ring + (size_t)sl * C::CHUNK);
      const uint64_t aRh = tc::sdesc(sa, 128, C::ASBO), aRl = tc::sdesc(sa + C::APLANE, 128, C::ASBO);
      const uint64_t aIh = tc::sdesc(sa + 2 * C::APLANE, 128, C::ASBO);
      const uint64_t aIl = tc::sdesc(sa + 3 * C::APLANE, 128, C::ASBO);
      const uint32_t bo = pb + 256u * (uint32_t)s;
      const uint64_t bRh = tc::sdesc(bo, 128, C::BSBO), bRl = tc::sdesc(bo + C::BPLANE, 128, C::BSBO);
      const uint64_t bIh = tc::sdesc(bo + 2 * C::BPLANE, 128, C::BSBO);
      const uint64_t bIl = tc::sdesc(bo + 3 * C::BPLANE, 128, C::BSBO);
      const uint32_t acc0 = s > 0 ? 1u : 0u;
      tc::mma_bf16(dre, aRh, bRh, I_POS, acc0);
      tc::mma_bf16(dre, aRl, bRh, I_POS, 1u);
      tc::mma_bf16(dre, aRh, bRl, I_POS, 1u);
      tc::mma_bf16(dre, aIh, bIh, i_re, 1u);
      tc::mma_bf16(dre, aIl, bIh, i_re, 1u);
      tc::mma_bf16(dre, aIh, bIl, i_re, 1u);
      tc::mma_bf16(dim, aRh, bIh, I_POS, acc0);
      tc::mma_bf16(dim, aRl, bIh, I_POS, 1u);
      tc::mma_bf16(dim, aRh, bIl, I_POS, 1u);
      tc::mma_bf16(dim, aIh, bRh, i_im, 1u);
      tc::mma_bf16(dim, aIl, bRh, i_im, 1u);
      tc::mma_bf16(dim, aIh, bRl, i_im, 1u);
      tc::mma_commit(&empty[sl]);
      if (qc >= 1) {   // refill the previous chunk's slot once its MMAs are done
        const long long qp = qc - 1, qn = qp + C::NS;
        const int sp = (int)(qp % C::NS);
        if (!tc::mbar_wait(&empty[sp], (uint32_t)((qp / C::NS) & 1))) return false;
        tc::mbar_expect_tx(&full[sp], C::CHUNK);
        tc::bulk_g2s(ring + (size_t)sp * C::CHUNK, dft + (size_t)(qn % C::NCH) * C::CHUNK, C::CHUNK, &full[sp]);
        ++issued;
      }
    }
    tc::mma_commit(done);
    return true;
  };

  uint32_t npass = 0;
  // All threads: publish the planes, issue one pass, wait for it. False (on
  // every thread) if any wait gave up.
  auto run_pass = [&](bool inverse) -> bool {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!issue_pass(inverse)) atomicOr(a.status, FLAG_TIMEOUT);
    }
    const bool ok = tc::mbar_wait(done, npass & 1u);
    ++npass;
    tc::fence_after_sync();
    return !__syncthreads_or(!ok);
  };

  const float invN = 1.0f / (float)N;
  constexpr uint32_t IMG = (uint32_t)NN * sizeof(float2);
  // L2 prefetch of an image this CTA reads next (thread 0)
  auto prefetch = [&](const float2* p) {
    if (tid == 0) tc::prefetch_l2(p, IMG);
  };
  bool alive = true;
  if (blockIdx.x < a.nb) prefetch(a.psi_s + (size_t)blockIdx.x * a.M * NN);
  for (int slot = blockIdx.x; slot < a.nb && alive; slot += gridDim.x) {
    const int e = a.b0 + slot;
    const int j = a.order ? a.order[e] : e;
    int ty, tx;
    float fy, fx;
    if (!(j >= 0 && j < a.J) || !tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx))
      continue;   // flagged by the first part of the pass
    float2* psi = a.psi_s + (size_t)slot * a.M * NN;
    if (tid == 0 && a.meas && a.mode != MODE_FWD) tc::prefetch_l2(a.meas + (size_t)j * NN, (uint32_t)NN * 4);
    const bool more = slot + (int)gridDim.x < a.nb;
    float2* next_slot = more ? a.psi_s + (size_t)(slot + gridDim.x) * a.M * NN : nullptr;
    float acc[HALF];
#pragma unroll
    for (int i = 0; i < HALF; ++i) acc[i] = 0.f;

    // ---- forward: Psi_k = F psi_k F^T / N, I = sum_k |Psi_k|^2 ----------------------
    for (int k = 0; k < a.M && alive; ++k) {
      if (k + 1 < a.M) prefetch(psi + (size_t)(k + 1) * NN);
      else if (a.mode == MODE_FWD && next_slot) prefetch(next_slot);
      if (act) rows_to_planes<N, false>(planes, psi + (size_t)k * NN, row, c0, acc);
      if (!(alive = run_pass(false))) break;
      if (act) tmem_to_planes<N>(planes, trow, row, c0);
      if (!(alive = run_pass(false))) break;
      if (act) tmem_to_global<N, true>(psi + (size_t)k * NN, trow, row, c0, invN, acc, k == 0);
    }
    if (!alive) break;

    // ---- data term: loss and the far-field factor (times 1/N for the inverse) --------
    float lsum = 0.f;
    bool bad = false;
    if (act) {
      const float* meas = a.meas ? a.meas + (size_t)j * NN + (size_t)row * N + c0 : nullptr;
      float* ip = a.ipred ? a.ipred + (size_t)j * NN + (size_t)row * N + c0 : nullptr;
#pragma unroll
      for (int i = 0; i < HALF; ++i) {
        const float I = acc[i];
        if (ip) ip[i] = I;
        if (a.mode == MODE_FWD) continue;
        const float Im = __ldg(meas + i);
        float fac;
        if (a.mode == MODE_VJP) {
          bad |= !isfinite(Im);
          fac = 2.f * Im;
        } else {
          bad |= !(Im >= 0.f) || !isfinite(Im);
          const float Ie = I + a.eps;
          if (a.mode == MODE_LSQML_GAUSS || a.mode == MODE_GRAD_GAUSS) {
            const float sIe = sqrtf(Ie), sIm = sqrtf(Im);
            const float d = sIe - sIm;
            lsum = fmaf(d, d, lsum);
            const float rho = sIm / sIe;
            fac = (a.mode == MODE_LSQML_GAUSS) ? rho - 1.f : 2.f * (1.f - rho);
          } else {
            lsum += I - Im * logf(Ie);
            const float q = Im / Ie;
            fac = (a.mode == MODE_LSQML_POISSON) ? 0.5f * (q - 1.f) : 2.f * (1.f - q);
          }
        }
        acc[i] = fac * invN;
      }
    }
    if (bad) atomicOr(a.status, FLAG_NONFINITE);
    if (a.loss && a.mode != MODE_FWD && a.mode != MODE_VJP) {
      double v[1] = {(double)lsum};
      block_sum<1>(v, red);
      if (tid == 0) atomicAdd(a.loss, v[0]);
    }
    if (a.mode == MODE_FWD) continue;

    // ---- back-propagation: chi_k = conj(F) (fac Psi_k) conj(F)^T -------------------
    for (int k = a.M - 1; k >= 0 && alive; --k) {
      if (k > 0) prefetch(psi + (size_t)(k - 1) * NN);
      else if (next_slot) prefetch(next_slot);
      if (act) rows_to_planes<N, true>(planes, psi + (size_t)k * NN, row, c0, acc);
      if (!(alive = run_pass(true))) break;
      if (act) tmem_to_planes<N>(planes, trow, row, c0);
      if (!(alive = run_pass(true))) break;
      if (act) tmem_to_global<N, false>(psi + (size_t)k * NN, trow, row, c0, 1.f, acc, false);
    }
  }
  if (!alive && tid == 0) atomicOr(a.status, FLAG_TIMEOUT);

  // Copies still in flight land before the CTA exits; then TMEM is released.
  if (tid == 0) {
    for (; qc < issued; ++qc)
      if (!tc::mbar_wait(&full[(int)(qc % C::NS)], (uint32_t)((qc / C::NS) & 1))) {
        atomicOr(a.status, FLAG_TIMEOUT);
        break;
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, C::COLS);
}

}  // namespace ptycho
