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
// k_exit_tma (below) writes the exit waves psi_jk of a minibatch to the
// scratch from object tiles staged by tensor copies (objects of odd width go
// through the first part of the per-position pass instead).
//
// k_far_tc: per minibatch position (persistent CTAs): the exit waves psi_jk
// are transformed mode by mode; the far fields overwrite them in the scratch and their intensities
// accumulate per thread; the data term (Eq. 1 amplitude loss or the Poisson
// likelihood) gives the loss and the far-field factor; every mode is then
// scaled and transformed back, and chi_jk = F^-1[(rho - 1) Psi_jk] overwrites
// the scratch for the overlap-add part of the pass.
//
// Warp roles: eight producer warps write the B operand of every K step (a
// 16-wide K slice of four BF16 planes) into a ring of shared-memory slots;
// one MMA warp streams the DFT-matrix chunks and issues the MMAs as slices
// land; one TMA warp stages the exit waves and the measured intensities from
// global memory into a second ring with tiled tensor copies (128-byte
// swizzle). Pass-1 slices come from the staged exit waves, from the last
// forward far field still in TMEM (the first inverse transform) or from the
// far fields in L2 (the other inverse transforms); pass-2 slices from the
// pass-1 accumulator in TMEM. Pass 1 accumulates in TMEM buffer A, pass 2 in
// buffer B, so an image's pass-2 result drains while the next image's pass 1
// runs.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace ptycho {

template <int N>
struct FarTc {
  static_assert(N == 32 || N == 64 || N == 128, "DFT-GEMM windows");
  static constexpr int PW = 8;                    // producer warps: TMEM lane quarter w % 4, column set w / 4
  static constexpr int T = 32 * (PW + 2);         // and the MMA warp (PW) and the TMA warp (PW + 1)
  static constexpr int HALF = N / 2;              // columns per producer thread: 16 s + 8 (w / 4) + [0, 8)
  static constexpr int NCH = N / 16;              // K steps of one pass (= DFT chunks)
  static constexpr int NSF = 4;                   // ring slots of DFT chunks
  static constexpr int NSB = 6;                   // ring slots of B slices
  static constexpr int NSS = 4;                   // ring slots of staged tiles
  static constexpr int MT = 128;                  // MMA tile rows (DFT rows beyond N are zero)
  static constexpr uint32_t APLANE = MT * 16 * 2;            // one 128 x 16 BF16 plane of a chunk
  static constexpr uint32_t CHUNK = 4 * APLANE;              // Fr_hi, Fr_lo, Fi_hi, Fi_lo
  static constexpr uint32_t ASBO = 256;                      // 8-row groups of a 16-wide K slice
  static constexpr uint32_t BPLANE = (uint32_t)N * 16 * 2;   // one N x 16 BF16 plane of a B slice
  static constexpr uint32_t SLICE = 4 * BPLANE;              // Xr_hi, Xr_lo, Xi_hi, Xi_lo
  static constexpr uint32_t BSBO = 256;
  static constexpr uint32_t SSLOT = 128u * N;                // a staged tile: N rows x 32 floats
  static constexpr size_t fring = 0;
  static constexpr size_t sring = fring + (size_t)NSF * CHUNK;   // 1024-byte aligned (swizzled tiles)
  static constexpr size_t bring = sring + (size_t)NSS * SSLOT;
  static constexpr size_t bars = bring + (size_t)NSB * SLICE;
  static constexpr int NBAR = 2 * NSF + 2 * NSB + 2 * NSS + 3;   // F, B and staging rings, p1, p2, drained
  static constexpr size_t misc = bars + 8 * (size_t)NBAR;
  static constexpr size_t bytes = misc + 16 + 1024;             // + alignment of the base to 1024 bytes
  static constexpr uint32_t COLS = 4 * N;                    // buffer A [0, 2N), buffer B [2N, 4N)
  static constexpr size_t dft_bytes = (size_t)NCH * CHUNK;
  static_assert(bytes <= 232448, "shared memory per CTA");
  static_assert(COLS >= 32 && COLS <= 512 && (COLS & (COLS - 1)) == 0, "TMEM allocation: a power of two <= 512");
  static_assert(sring % 1024 == 0 && SSLOT % 1024 == 0, "128-byte swizzled tiles need 1024-byte alignment");
  static_assert(CHUNK % 16 == 0 && SLICE % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// An encoded tensor map (CUtensorMap), passed by value as a kernel parameter.
struct alignas(64) TmaDesc {
  unsigned long long v[16];
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

// Exit waves of the split-BF16 form: per position the object tile (rows
// ty..ty+N, columns xs..xs+N+1 with xs = tx rounded down to an even column,
// so that the copy starts on a 16-byte boundary) lands in shared memory with
// one tiled tensor copy; the bilinear patch o_j = S_j(O) (Sec. 2.1, the same
// weights and expression as the per-position pass) is interpolated from it,
// and o_j and psi_jk = P_k o_j of every mode go to the scratch.
template <int N>
struct ExitTma {
  static constexpr int T = 512;
  static constexpr int TW = N + 2, TH = N + 1;   // staged tile: TH rows of TW complex values
  static constexpr uint32_t TILE_BYTES = (uint32_t)TW * TH * 8;
  static constexpr size_t tile = 0;
  static constexpr size_t bar = ((size_t)TILE_BYTES + 127) / 128 * 128;
  static constexpr size_t wsh = bar + 16;        // eigenmode weights of the position (OPR)
  static constexpr size_t bytes = wsh + 4 * 8 + 128;   // + alignment of the base to 128 bytes
  static_assert(TW <= 256 && TH <= 256, "tensor-copy box dimensions");
  static_assert((TW * 8) % 16 == 0, "tensor-copy box rows are multiples of 16 bytes");
  static_assert(bytes <= 232448, "shared memory per CTA");
};

template <int N, bool OPR>
__global__ void __launch_bounds__(512, 1) k_exit_tma(BatchArgs a, const __grid_constant__ TmaDesc tm_obj) {
  using C = ExitTma<N>;
  constexpr int NN = N * N, T = C::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  wait_prior_grid();
  unsigned char* smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  const float2* tile = (const float2*)(smem + C::tile);
  uint64_t* bar = (uint64_t*)(smem + C::bar);
  float* wj = (float*)(smem + C::wsh);
  const int slot = blockIdx.x, tid = threadIdx.x;
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  int ty = 0, tx = 0;
  float fy = 0.f, fx = 0.f;
  bool ok = (j >= 0 && j < a.J);
  if (ok) ok = tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  if (!ok) {
    if (tid == 0) {
      atomicOr(a.status, FLAG_BOUNDS);
      if (a.valid) a.valid[slot] = 0;
    }
    return;
  }
  const int xs = tx & ~1, d = tx - xs;
  if (tid == 0) {
    if (a.valid) a.valid[slot] = 1;
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    tc::mbar_expect_tx(bar, C::TILE_BYTES);
    tc::tma_load_2d(smem + C::tile, &tm_obj, xs, ty, bar);
  }
  if (OPR && tid < a.K) wj[tid] = a.opr_w[(size_t)j * a.K + tid];
  __syncthreads();
  if (!__syncthreads_and(tc::mbar_wait(bar, 0))) {
    if (tid == 0) atomicOr(a.status, FLAG_TIMEOUT);
    return;
  }
  const int M = a.M;
  const size_t slotNN = (size_t)slot * NN;
  float2* o_s = a.o_s ? a.o_s + slotNN : nullptr;
  float2* psi = a.psi_s + slotNN * M;
  float2* p0 = (OPR && a.p0_s) ? a.p0_s + slotNN : nullptr;
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
#pragma unroll 2
  for (int q = tid; q < NN / 2; q += T) {   // pixel pairs (r, c), (r, c + 1)
    const int p = 2 * q, r = p / N, c = p % N;
    const float2* t0 = tile + r * C::TW + c + d;
    const float2* t1 = t0 + C::TW;
    const float2 a0 = t0[0], a1 = t0[1], a2 = t0[2], b0 = t1[0], b1 = t1[1], b2 = t1[2];
    const float2 o0 = make_float2(w00 * a0.x + w01 * a1.x + w10 * b0.x + w11 * b1.x,
                                  w00 * a0.y + w01 * a1.y + w10 * b0.y + w11 * b1.y);
    const float2 o1 = make_float2(w00 * a1.x + w01 * a2.x + w10 * b1.x + w11 * b2.x,
                                  w00 * a1.y + w01 * a2.y + w10 * b1.y + w11 * b2.y);
    if (o_s) *(float4*)(o_s + p) = make_float4(o0.x, o0.y, o1.x, o1.y);
    for (int k = 0; k < M; ++k) {
      const float2* Pk = shared_mode<OPR>(a, k, NN);
      float4 P2;
      if (!OPR || Pk) {
        P2 = __ldg((const float4*)(Pk + p));
      } else {   // relaxed primary mode of this position
        P2 = opr_pair(a.opr_U, wj, a.K, NN, p);
        if (p0) *(float4*)(p0 + p) = P2;
      }
      const float2 x0 = cmul(make_float2(P2.x, P2.y), o0), x1 = cmul(make_float2(P2.z, P2.w), o1);
      *(float4*)(psi + (size_t)k * NN + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
    }
  }
}

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
// x = hi + lo to within 2^-16 |x| (BF16 keeps 8 significant bits)
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

// Eight consecutive K values (K offset 8 h of a 16-wide slice) of operand
// row `row` into the four planes of a B slice (hi/lo of re and im).
template <int N>
__device__ __forceinline__ void put8(unsigned char* slice, int row, int h, const float* re, const float* im) {
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
  unsigned char* p = slice + (size_t)(row / 8) * C::BSBO + h * 128 + (row % 8) * 16;
  *(uint4*)p = make_uint4(rh[0], rh[1], rh[2], rh[3]);
  *(uint4*)(p + C::BPLANE) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
  *(uint4*)(p + 2 * C::BPLANE) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
  *(uint4*)(p + 3 * C::BPLANE) = make_uint4(il[0], il[1], il[2], il[3]);
}

// Bounded wait that also gives up when another role has aborted; the
// outcome is made uniform over the warp.
__device__ __forceinline__ bool role_wait(uint64_t* b, uint32_t parity, volatile int* abort_s) {
  bool ok = tc::mbar_try_wait(b, parity);
  if (!ok) {
    const long long t0 = clock64();
    while (!(ok = tc::mbar_try_wait(b, parity))) {
      if (*abort_s) break;
      if (clock64() - t0 > (1ll << 31)) {
        *abort_s = 1;
        break;
      }
    }
  }
  return !__any_sync(0xffffffffu, !ok);
}

// Staged-tile element of row `row`, 16-byte chunk `c` (of 8), in the
// 128-byte swizzle the tensor copies write: chunk c of row r sits at c ^ (r % 8).
__device__ __forceinline__ float4 staged_chunk(const unsigned char* tile, int row, int c) {
  return *(const float4*)(tile + (size_t)row * 128 + ((c ^ (row & 7)) << 4));
}

template <int N>
__global__ void __launch_bounds__(FarTc<N>::T, 1)
    k_far_tc(FarArgs a, const __grid_constant__ TmaDesc tm_psi, const __grid_constant__ TmaDesc tm_meas) {
  using C = FarTc<N>;
  constexpr int NN = N * N, HALF = C::HALF, NCH = C::NCH, NSB = C::NSB, NSS = C::NSS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  wait_prior_grid();
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* fring = smem + C::fring;
  unsigned char* sring = smem + C::sring;
  unsigned char* bring = smem + C::bring;
  uint64_t* fullF = (uint64_t*)(smem + C::bars);
  uint64_t* emptyF = fullF + C::NSF;
  uint64_t* fullB = emptyF + C::NSF;
  uint64_t* emptyB = fullB + NSB;
  uint64_t* fullS = emptyB + NSB;
  uint64_t* emptyS = fullS + NSS;
  uint64_t* p1done = emptyS + NSS;
  uint64_t* p2done = p1done + 1;
  uint64_t* drained = p2done + 1;
  uint32_t* holder = (uint32_t*)(smem + C::misc);
  volatile int* abort_s = (volatile int*)(holder + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < C::NSF; ++s) {
      tc::mbar_init(&fullF[s], 1);
      tc::mbar_init(&emptyF[s], 1);
    }
    for (int s = 0; s < NSB; ++s) {
      tc::mbar_init(&fullB[s], C::PW);
      tc::mbar_init(&emptyB[s], 1);
    }
    for (int s = 0; s < NSS; ++s) {
      tc::mbar_init(&fullS[s], 1);
      tc::mbar_init(&emptyS[s], C::PW);
    }
    tc::mbar_init(p1done, 1);
    tc::mbar_init(p2done, 1);
    tc::mbar_init(drained, C::PW);
    *abort_s = 0;
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
  const uint32_t bufA = tmem, bufB = tmem + 2 * N;

  // The image sequence every role walks: per valid slot, M forward transforms,
  // then (unless only intensities are wanted) M inverse ones.
  auto slot_j = [&](int slot) -> int {
    const int e = a.b0 + slot;
    const int j = a.order ? a.order[e] : e;
    int ty, tx;
    float fy, fx;
    if (!(j >= 0 && j < a.J) || !tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx)) return -1;
    return j;   // an invalid slot is flagged by the first part of the pass
  };
  const bool backward = a.mode != MODE_FWD;

  if (warp == C::PW) {
    // ================================ MMA warp ====================================
    if (lane == 0) {
      const unsigned char* dft = (const unsigned char*)a.dft;
      uint32_t qc = 0, issued = 0, cb = 0;
      int64_t last_mma = -1;   // the last chunk whose MMAs were issued (and committed)
      for (int s = 0; s < C::NSF; ++s) {
        tc::mbar_expect_tx(&fullF[s], C::CHUNK);
        tc::bulk_g2s(fring + (size_t)s * C::CHUNK, dft + (size_t)(s % NCH) * C::CHUNK, C::CHUNK, &fullF[s]);
      }
      issued = C::NSF;
      constexpr uint32_t I_POS = tc::idesc_bf16(C::MT, N, false), I_NEG = tc::idesc_bf16(C::MT, N, true);
      bool ok = true;
      // one pass into the accumulator at `d` (re at d, im at d + N)
      auto pass = [&](uint32_t d, bool inverse, uint64_t* done) {
        const uint32_t i_re = inverse ? I_POS : I_NEG;   // Fi Xi into D_re: minus forward, plus inverse
        const uint32_t i_im = inverse ? I_NEG : I_POS;   // Fi Xr into D_im: plus forward, minus inverse
        for (int s = 0; s < NCH && ok; ++s, ++qc, ++cb) {
          const int sf = (int)(qc % C::NSF), sb = (int)(cb % NSB);
          if (!tc::mbar_wait(&fullF[sf], (uint32_t)((qc / C::NSF) & 1)) ||
              !tc::mbar_wait(&fullB[sb], (uint32_t)((cb / NSB) & 1))) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(fring + (size_t)sf * C::CHUNK);
          const uint64_t aRh = tc::sdesc(sa, 128, C::ASBO), aRl = tc::sdesc(sa + C::APLANE, 128, C::ASBO);
          const uint64_t aIh = tc::sdesc(sa + 2 * C::APLANE, 128, C::ASBO);
          const uint64_t aIl = tc::sdesc(sa + 3 * C::APLANE, 128, C::ASBO);
          const uint32_t sbase = tc::smem_u32(bring + (size_t)sb * C::SLICE);
          const uint64_t bRh = tc::sdesc(sbase, 128, C::BSBO), bRl = tc::sdesc(sbase + C::BPLANE, 128, C::BSBO);
          const uint64_t bIh = tc::sdesc(sbase + 2 * C::BPLANE, 128, C::BSBO);
          const uint64_t bIl = tc::sdesc(sbase + 3 * C::BPLANE, 128, C::BSBO);
          const uint32_t acc0 = s > 0 ? 1u : 0u, dre = d, dim = d + N;
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
          tc::mma_commit(&emptyF[sf]);
          tc::mma_commit(&emptyB[sb]);
          last_mma = qc;
          if (qc >= 1) {   // refill the previous chunk's slot once its MMAs are done
            const uint32_t qp = qc - 1, qn = qp + C::NSF;
            const int sp = (int)(qp % C::NSF);
            if (!tc::mbar_wait(&emptyF[sp], (uint32_t)((qp / C::NSF) & 1))) {
              ok = false;
              break;
            }
            tc::mbar_expect_tx(&fullF[sp], C::CHUNK);
            tc::bulk_g2s(fring + (size_t)sp * C::CHUNK, dft + (size_t)(qn % NCH) * C::CHUNK, C::CHUNK,
                         &fullF[sp]);
            ++issued;
          }
        }
        if (ok) tc::mma_commit(done);
      };
      uint32_t n = 0;
      for (int slot = blockIdx.x; slot < a.nb && ok && !*abort_s; slot += gridDim.x) {
        if (slot_j(slot) < 0) continue;
        for (int t = 0; t < (backward ? 2 * a.M : a.M) && ok && !*abort_s; ++t, ++n) {
          const bool inverse = t >= a.M;
          pass(bufA, inverse, p1done);
          if (ok && n >= 1 && !tc::mbar_wait(drained, (uint32_t)((n - 1) & 1))) ok = false;
          if (ok) pass(bufB, inverse, p2done);
        }
      }
      if (!ok) *abort_s = 1;
      // copies still in flight land before the CTA exits
      for (; qc < issued; ++qc)
        if (!tc::mbar_wait(&fullF[(int)(qc % C::NSF)], (uint32_t)((qc / C::NSF) & 1))) {
          *abort_s = 1;
          break;
        }
      // after an abort, the MMAs already issued finish (their last commit
      // completes) before the tensor memory is released
      if (*abort_s && last_mma >= 0)
        tc::mbar_wait(&emptyF[(int)(last_mma % C::NSF)], (uint32_t)((last_mma / C::NSF) & 1));
    }
  } else if (warp == C::PW + 1) {
    // ================================ TMA warp ====================================
    // Stages, in the order the producers consume them, the exit waves of the
    // forward transforms (N x 32-float tiles, 16 complex columns each) and
    // the measured intensities of the data term (N x 32-float tiles).
    if (lane == 0) {
      uint32_t ps = 0;
      bool ok = true;
      auto stage = [&](const TmaDesc* map, int x, int z) {
        const int sl = (int)(ps % NSS);
        if (ps >= NSS && !tc::mbar_wait(&emptyS[sl], (uint32_t)(((ps / NSS) - 1) & 1))) {
          ok = false;
          return;
        }
        tc::mbar_expect_tx(&fullS[sl], C::SSLOT);
        tc::tma_load_3d(sring + (size_t)sl * C::SSLOT, map, x, 0, z, &fullS[sl]);
        ++ps;
      };
      for (int slot = blockIdx.x; slot < a.nb && ok && !*abort_s; slot += gridDim.x) {
        const int j = slot_j(slot);
        if (j < 0) continue;
        for (int k = 0; k < a.M && ok; ++k)
          for (int s = 0; s < NCH && ok; ++s) stage(&tm_psi, 32 * s, slot * a.M + k);
        if (backward)
          for (int b = 0; b < (NCH + 1) / 2 && ok; ++b) stage(&tm_meas, 32 * b, j);
      }
      if (!ok) *abort_s = 1;
      // tiles still in flight land before the CTA exits (the last fill of each slot)
      for (uint32_t p = ps - (ps < (uint32_t)NSS ? ps : (uint32_t)NSS); p < ps; ++p)
        if (!tc::mbar_wait(&fullS[(int)(p % NSS)], (uint32_t)((p / NSS) & 1))) {
          *abort_s = 1;
          break;
        }
    }
  } else {
    // ============================= producer warps =================================
    const int q4 = warp & 3, h = warp >> 2;
    const int row = 32 * q4 + lane;           // TMEM lane = operand row
    const bool act = row < N;                  // warp-uniform
    const uint32_t lrow = (uint32_t)(32 * q4) << 16;
    const float invN = 1.0f / (float)N;
    uint32_t pb = 0, ps = 0, n = 0, nd = 0;
    float acc[HALF];                           // I, then the far-field factor, of columns 16 s + 8 h + [0, 8)
#pragma unroll
    for (int i = 0; i < HALF; ++i) acc[i] = 0.f;
    bool alive = true;

    // takes B slot pb (waiting for it to be free), fills it, publishes it
    auto publish = [&](auto&& fill) {
      const int sb = (int)(pb % NSB);
      if (pb >= NSB && !role_wait(&emptyB[sb], (uint32_t)(((pb / NSB) - 1) & 1), abort_s)) {
        alive = false;
        return;
      }
      if (act) fill(bring + (size_t)sb * C::SLICE);
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&fullB[sb]);
      ++pb;
    };
    // waits for staged tile ps; returns it (null if a wait gave up)
    auto staged = [&]() -> const unsigned char* {
      const int sl = (int)(ps % NSS);
      if (!role_wait(&fullS[sl], (uint32_t)((ps / NSS) & 1), abort_s)) {
        alive = false;
        return nullptr;
      }
      return sring + (size_t)sl * C::SSLOT;
    };
    auto release_staged = [&]() {
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&emptyS[(int)(ps % NSS)]);
      ++ps;
    };
    // pass-1 slices of a forward transform from the staged exit wave
    auto produce_staged = [&]() {
#pragma unroll 1
      for (int s = 0; s < NCH; ++s) {
        const unsigned char* tile = staged();
        if (!alive) break;
        float4 v[4];
        if (act) {
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = staged_chunk(tile, row, 4 * h + i);
        }
        publish([&](unsigned char* slice) {
          float re[8], im[8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            re[2 * i] = v[i].x; im[2 * i] = v[i].y; re[2 * i + 1] = v[i].z; im[2 * i + 1] = v[i].w;
          }
          put8<N>(slice, row, h, re, im);
        });
        if (!alive) break;
        release_staged();
      }
    };
    // pass-1 slices of an inverse transform from a far field in global memory
    // (just written by this CTA, so in L2), times the factors
    auto produce_global = [&](const float2* src) {
      constexpr int G = 2;   // slices of loads in flight
#pragma unroll
      for (int s0 = 0; s0 < NCH; s0 += G) {
        if (!alive) break;
        float4 v[G][4];
        if (act) {
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const float4* p4 = (const float4*)(src + (size_t)row * N + 16 * (s0 + g) + 8 * h);
#pragma unroll
            for (int i = 0; i < 4; ++i) v[g][i] = __ldcg(p4 + i);
          }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (!alive) break;
          publish([&](unsigned char* slice) {
            float re[8], im[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              re[2 * i] = v[g][i].x; im[2 * i] = v[g][i].y; re[2 * i + 1] = v[g][i].z; im[2 * i + 1] = v[g][i].w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              re[i] *= acc[8 * (s0 + g) + i];
              im[i] *= acc[8 * (s0 + g) + i];
            }
            put8<N>(slice, row, h, re, im);
          });
        }
      }
    };
    // slices from an accumulator in TMEM: pass-2 slices from buffer A, or
    // (SCALE) the first inverse transform's pass-1 slices from the last forward
    // far field in buffer B, times 1/N and the factors
    auto produce_tmem = [&](uint32_t buf, bool scale) {
      constexpr int G = NCH < 2 ? NCH : 2;   // slices per TMEM round trip
      if (scale) {
#pragma unroll
        for (int s = 0; s < NCH; ++s) {
          if (!alive) break;
          float re[8], im[8];
          if (act) {
            tc::tmem_ld8(buf + lrow + 16 * s + 8 * h, re);
            tc::tmem_ld8(buf + lrow + N + 16 * s + 8 * h, im);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float f = acc[8 * s + i] * invN;
              re[i] *= f;
              im[i] *= f;
            }
          }
          publish([&](unsigned char* slice) { put8<N>(slice, row, h, re, im); });
        }
        return;
      }
#pragma unroll 1
      for (int s0 = 0; s0 < NCH; s0 += G) {
        if (!alive) break;
        float re[G][8], im[G][8];
        if (act) {
#pragma unroll
          for (int g = 0; g < G; ++g) {
            tc::tmem_ld8(buf + lrow + 16 * (s0 + g) + 8 * h, re[g]);
            tc::tmem_ld8(buf + lrow + N + 16 * (s0 + g) + 8 * h, im[g]);
          }
          tc::tmem_wait_ld();
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (!alive) break;
          publish([&](unsigned char* slice) { put8<N>(slice, row, h, re[g], im[g]); });
        }
      }
    };
    // the pass-2 accumulator (buffer B) times `scale` to global memory (unless
    // dst is null); with `accumulate` its squared modulus is stored into
    // (first) or added to acc
    auto drain = [&](float2* dst, bool accumulate, bool first, float scale) {
      if (act) {
#pragma unroll
        for (int s = 0; s < NCH; ++s) {
          float re[8], im[8];
          tc::tmem_ld8(bufB + lrow + 16 * s + 8 * h, re);
          tc::tmem_ld8(bufB + lrow + N + 16 * s + 8 * h, im);
          tc::tmem_wait_ld();
          float4* d4 = dst ? (float4*)(dst + (size_t)row * N + 16 * s + 8 * h) : nullptr;
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            const float x0 = re[i] * scale, y0 = im[i] * scale, x1 = re[i + 1] * scale, y1 = im[i + 1] * scale;
            if (d4) d4[i / 2] = make_float4(x0, y0, x1, y1);
            if (accumulate) {
              const float a0 = fmaf(x0, x0, y0 * y0), a1 = fmaf(x1, x1, y1 * y1);
              acc[8 * s + i] = first ? a0 : acc[8 * s + i] + a0;
              acc[8 * s + i + 1] = first ? a1 : acc[8 * s + i + 1] + a1;
            }
          }
        }
      }
    };
    auto arrive_drained = [&]() {
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(drained);
    };
    // the data term of position j from the intensities in acc: loss, ipred, and
    // the far-field factor (times 1/N for the unnormalised inverse) into acc;
    // the measured values come from the staged tiles (none in the forward mode)
    auto data_term = [&](int j) {
      float lsum = 0.f;
      bool bad = false;
      float* ip = (a.ipred && act) ? a.ipred + (size_t)j * NN + (size_t)row * N + 8 * h : nullptr;
#pragma unroll
      for (int b = 0; b < (NCH + 1) / 2; ++b) {
        float mv[2][8];
        if (backward) {
          const unsigned char* tile = staged();
          if (!alive) break;
          if (act) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              const float4 m0 = staged_chunk(tile, row, 4 * g + 2 * h), m1 = staged_chunk(tile, row, 4 * g + 2 * h + 1);
              mv[g][0] = m0.x; mv[g][1] = m0.y; mv[g][2] = m0.z; mv[g][3] = m0.w;
              mv[g][4] = m1.x; mv[g][5] = m1.y; mv[g][6] = m1.z; mv[g][7] = m1.w;
            }
          }
          release_staged();
        }
        if (act) {
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const int s = 2 * b + g;
            if (s >= NCH) break;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int c = 16 * s + i, ai = 8 * s + i;
              const float I = acc[ai];
              if (ip) ip[c] = I;
              if (!backward) continue;
              const float Im = mv[g][i];
              float fac;
              if (a.mode == MODE_VJP) {
                bad |= !isfinite(Im);
                fac = 2.f * Im;
              } else {
                bad |= !(Im >= 0.f) || !isfinite(Im);
                const float Ie = I + a.eps;
                if (a.mode == MODE_LSQML_GAUSS || a.mode == MODE_GRAD_GAUSS) {
                  const float sIe = sqrtf(Ie), sIm = sqrtf(Im);
                  const float dd = sIe - sIm;
                  lsum = fmaf(dd, dd, lsum);
                  const float rho = sIm / sIe;
                  fac = (a.mode == MODE_LSQML_GAUSS) ? rho - 1.f : 2.f * (1.f - rho);
                } else {
                  lsum += I - Im * logf(Ie);
                  const float qq = Im / Ie;
                  fac = (a.mode == MODE_LSQML_POISSON) ? 0.5f * (qq - 1.f) : 2.f * (1.f - qq);
                }
              }
              acc[ai] = fac * invN;
            }
          }
        }
      }
      if (bad) atomicOr(a.status, FLAG_NONFINITE);
      if (a.loss && backward && a.mode != MODE_VJP) {
        double v = (double)lsum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(a.loss, v);
      }
    };

    // the previous image, drained once the next image's pass-1 slices are out
    float2* prev_dst = nullptr;
    bool have_prev = false, prev_fwd = false, prev_first = false, prev_last_fwd = false;
    int prev_j = -1;
    auto drain_prev = [&]() {
      if (!role_wait(p2done, (uint32_t)(nd & 1), abort_s)) {
        alive = false;
        return;
      }
      tc::fence_after_sync();
      // forward far fields are kept for the inverse transforms (not needed
      // when only intensities are computed); inverse results are chi
      drain(prev_fwd && !backward ? nullptr : prev_dst, prev_fwd, prev_first, prev_fwd ? invN : 1.f);
      arrive_drained();
      ++nd;
      if (prev_fwd && prev_last_fwd && !backward) data_term(prev_j);
      have_prev = false;
    };

    for (int slot = blockIdx.x; slot < a.nb && alive; slot += gridDim.x) {
      const int j = slot_j(slot);
      if (j < 0) continue;
      float2* psi = a.psi_s + (size_t)slot * a.M * NN;
      for (int t = 0; t < (backward ? 2 * a.M : a.M) && alive; ++t, ++n) {
        const bool fwd = t < a.M;
        const int k = fwd ? t : 2 * a.M - 1 - t;
        float2* io = psi + (size_t)k * NN;
        if (fwd) {
          produce_staged();
          if (have_prev && alive) drain_prev();
        } else if (k == a.M - 1) {
          // first inverse transform: the last forward far field is still in
          // buffer B; its intensities complete I, then the data term gives the
          // factor, then its pass-1 slices come straight from TMEM
          if (!role_wait(p2done, (uint32_t)(nd & 1), abort_s)) {
            alive = false;
            break;
          }
          tc::fence_after_sync();
          drain(nullptr, true, a.M == 1, invN);
          ++nd;
          data_term(j);
          if (alive) produce_tmem(bufB, true);
          arrive_drained();
          have_prev = false;
        } else {
          produce_global(io);
          if (have_prev && alive) drain_prev();
        }
        if (!alive) break;
        if (!role_wait(p1done, (uint32_t)(n & 1), abort_s)) {
          alive = false;
          break;
        }
        tc::fence_after_sync();
        produce_tmem(bufA, false);
        prev_dst = io;
        have_prev = true;
        prev_fwd = fwd;
        prev_first = fwd && k == 0;
        prev_last_fwd = fwd && k == a.M - 1;
        prev_j = j;
      }
    }
    if (alive && have_prev) drain_prev();
    if (!alive) *abort_s = 1;
  }

  if (tid == 0 && *abort_s) atomicOr(a.status, FLAG_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, C::COLS);
}

}  // namespace ptycho
