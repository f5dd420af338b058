// Per-scan-position kernels of the LSQML hot path (templated on the window N).
//
// k_pass1: one CTA per position of a minibatch. For every incoherent probe
//   mode k it extracts the sub-pixel object patch o_j = S_j(O) (bilinear),
//   forms the exit wave psi_jk = P_k o_j (Pty-Chi Sec. 2.1, the psi = p o of
//   Eq. 2), propagates it with the unitary 2-D FFT and accumulates the
//   incoherent intensity I_j = sum_k |Psi_jk|^2 (Eq. 4's forward model). It
//   then applies the data term (Eq. 1 amplitude loss, or the Poisson
//   likelihood), forms the far-field correction factor, back-propagates every
//   mode to chi_jk = F^-1[(rho - 1) Psi_jk] (= psi'_jk - psi_jk of Eq. 2), and
//   reduces g_j = sum_k conj(P_k) chi_jk and h_jk = conj(o_j) chi_jk. Finally
//   it scatter-adds S_j^T g_j and the illumination S_j^T sum_k |P_k|^2 into the
//   object-frame accumulators (the LSQML preconditioner) with vector atomics,
//   or, in gradient mode, S_j^T of the object gradient and the position
//   gradient through the bilinear weights.
// k_pass2: one CTA per position: the five reductions of the per-position
//   least-squares step (LSQML's self-adaptive step sizes, Sec. 2.2), the
//   FP64 2x2 solve, and the alpha-weighted object scatter.
#pragma once
#include <cooperative_groups.h>
#include "common.cuh"
#include "tc.cuh"

namespace ptycho {
namespace cg = cooperative_groups;

// CTA sizes of the per-position pass: the default and the alternative the
// autotuner may pick (the full count of line slots N*R1, or half of it with
// two lines per thread).
template <int N> struct Threads;
template <> struct Threads<16> { static constexpr int T = 64, ALT = 32; };
template <> struct Threads<32> { static constexpr int T = 128, ALT = 64; };
template <> struct Threads<64> { static constexpr int T = 256, ALT = 512; };
template <> struct Threads<128> { static constexpr int T = 1024, ALT = 512; };

template <int N>
struct Pass1Smem {
  static constexpr int RP = N + 16;  // row pitch of the intensity/factor plane (floats)
  static constexpr size_t red = 0;
  static constexpr size_t tile = red + 256 * sizeof(double);
  static constexpr size_t tw = tile + (size_t)N * N * sizeof(float2);
  static constexpr size_t rI = tw + (size_t)Twiddles<N>::COUNT * sizeof(float2);
  static constexpr size_t bytes = rI + (size_t)N * RP * sizeof(float);
};

// 2-D forward transform of the tile (natural layout on entry). Column pass
// first, then rows; `out(row, v)` receives each row's unnormalised transform in
// the line "out" layout: v[m] = X[row][Fft2<N>::out_index(n, m)].
template <int N, int T, class Out>
__device__ __forceinline__ void fft2_forward(float2* tile, const float2* tw, Out&& out) {
  using F = Fft2<N>;
  constexpr int R1 = F::R1, R2 = F::R2, L = T / R1, ITER = N / L;
  const int n = F::line_lane(), gid = F::line_slot();
#pragma unroll 1
  for (int it = 0; it < ITER; ++it) {
    const int col = gid + it * L;
    float2 v[R2];
    F::template load_in<false>(v, tile, col, n);
    F::template line_fwd<false>(v, tile, col, n, tw);
    F::template store_out<false>(v, tile, col, n);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < ITER; ++it) {
    const int row = gid + it * L;
    float2 v[R2];
    F::template load_in<true>(v, tile, row, n);
    F::template line_fwd<true>(v, tile, row, n, tw);
    out(row, v);
  }
}

// 2-D inverse (unnormalised). `in(row, v)` supplies each row in the "out"
// layout; `out(col, v)` receives each column with v[n2] = x[n + R1*n2][col].
// The tile must be free on entry.
template <int N, int T, class In, class Out>
__device__ __forceinline__ void fft2_inverse(float2* tile, const float2* tw, In&& in, Out&& out) {
  using F = Fft2<N>;
  constexpr int R1 = F::R1, R2 = F::R2, L = T / R1, ITER = N / L;
  const int n = F::line_lane(), gid = F::line_slot();
#pragma unroll 1
  for (int it = 0; it < ITER; ++it) {
    const int row = gid + it * L;
    float2 v[R2];
    in(row, v);
    F::template line_inv<true>(v, tile, row, n, tw);
    F::template store_in<true>(v, tile, row, n);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < ITER; ++it) {
    const int col = gid + it * L;
    float2 v[R2];
    F::template load_out<false>(v, tile, col, n);
    F::template line_inv<false>(v, tile, col, n, tw);
    out(col, v);
  }
}

// S_j^T of an N x N patch onto its (N+1)^2 object tile, evaluated separably:
// h_y(x) = (1-fx) p(y, x) + fx p(y, x-1) and out(y, x) = (1-fy) h_y(x) + fy h_{y-1}(x),
// with p = 0 outside the patch. A thread owns one tile column x and a run of
// rows (lanes of a warp emit consecutive x, so the atomics coalesce); each
// output costs two patch reads. `load(y, x)` returns the patch value as a
// float4 (unused components zero), `emit(y, x, v)` consumes the tile value.
template <int N, int T, class Load, class Emit>
__device__ __forceinline__ void bilinear_scatter(float fy, float fx, Load&& load, Emit&& emit) {
  constexpr int N1 = N + 1;
  constexpr int SEG = (T / N1) > 0 ? T / N1 : 1;
  constexpr int RS = (N1 + SEG - 1) / SEG;
  const float gx = 1.f - fx, gy = 1.f - fy;
  for (int item = threadIdx.x; item < N1 * SEG; item += T) {
    const int seg = item / N1, x = item % N1;
    const int y0 = seg * RS, y1 = min(N1, y0 + RS);
    auto hrow = [&](int y) {
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
      if (y < N) {
        if (x < N) {
          const float4 a = load(y, x);
          h = make_float4(gx * a.x, gx * a.y, gx * a.z, gx * a.w);
        }
        if (x > 0) {
          const float4 b = load(y, x - 1);
          h.x = fmaf(fx, b.x, h.x); h.y = fmaf(fx, b.y, h.y);
          h.z = fmaf(fx, b.z, h.z); h.w = fmaf(fx, b.w, h.w);
        }
      }
      return h;
    };
    float4 hp = (y0 > 0) ? hrow(y0 - 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int y = y0; y < y1; ++y) {
      const float4 h = hrow(y);
      emit(y, x, make_float4(fmaf(gy, h.x, fy * hp.x), fmaf(gy, h.y, fy * hp.y), fmaf(gy, h.z, fy * hp.z),
                             fmaf(gy, h.w, fy * hp.w)));
      hp = h;
    }
  }
}

// OPR: the primary probe mode is synthesised per position (a separate
// instantiation, so that the shared-probe kernel carries none of it).
// PART 0 is the whole pass. With the far field evaluated elsewhere (the
// tensor-core DFT-GEMM stage, k_far_tc) it runs in two parts around it:
// PART 1 writes the exit waves psi_jk to the far-field scratch (and the
// patches, the relaxed primary mode and the slot flags) and stops; PART 2
// reads chi_jk from the scratch and does the rest (g, h, the overlap-add, the
// position sums).
template <int N, int T, bool OPR, int PART>
__global__ void __launch_bounds__(T, 1) k_pass1(BatchArgs a) {
  using F = Fft2<N>;
  using SM = Pass1Smem<N>;
  constexpr int R1 = F::R1, R2 = F::R2, NN = N * N, RP = SM::RP;
  extern __shared__ __align__(16) unsigned char smem[];
  wait_prior_grid();
  double* red = (double*)(smem + SM::red);
  float2* tile = (float2*)(smem + SM::tile);
  float2* tw = (float2*)(smem + SM::tw);
  float* rI = (float*)(smem + SM::rI);

  const int slot = blockIdx.x;
  const int tid = threadIdx.x, n = F::line_lane();
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
  if (tid == 0 && a.valid) a.valid[slot] = 1;
  // the measured intensities are first read by the data term, after the forward
  // transforms: fetch them into L2 meanwhile (they may live in host memory)
  if (PART == 0 && tid == 0 && a.meas && a.mode != MODE_FWD)
    prefetch_l2_bulk(a.meas + (size_t)j * N * N, (uint32_t)(N * N * sizeof(float)));
  if (PART == 0) make_twiddles<N>(tw);

  const int M = a.M;
  const float invN = 1.0f / (float)N;
  const size_t slotNN = (size_t)slot * NN;
  float* wj = (float*)(red + 128);   // this position's eigenmode weights (OPR)
  float2* p0 = (OPR && a.p0_s) ? a.p0_s + slotNN : nullptr;
  if (OPR) {
    if (tid < a.K) wj[tid] = a.opr_w[(size_t)j * a.K + tid];
    __syncthreads();
  }
  float2* psi_s = a.psi_s ? a.psi_s + slotNN * M : nullptr;
  float2* o_s = a.o_s ? a.o_s + slotNN : nullptr;

  // Tensor memory as per-thread storage (the whole pass, window 128): the
  // patch o_j and the running sum g_j of the thread's natural-layout pixel
  // pairs stay on chip across the modes instead of making round trips through
  // L2. Warp w reaches TMEM lanes 32 (w % 4) ..+31; the T/128 warps sharing a
  // lane quarter split its 512 columns, CW each: o in the first 4 STEPS
  // columns (pair q at 4q), g in the next 4 STEPS. The CTA holds all 512
  // columns; no other TMEM-allocating CTA fits beside it on the SM (its
  // shared memory alone exceeds half of the SM's), so the allocation never
  // waits.
  constexpr bool TM = (PART == 0 && N == 128);
  constexpr int STEPS = NatPairs<N, T>::STEPS;
  static_assert(!TM || (STEPS % 2 == 0 && 8 * STEPS == 65536 / T), "o and g fill each warp's TMEM columns");
  // (the base address lives in shared memory, beyond the block reductions'
  // 160 doubles; the thread's column base is recomputed where it is used, so
  // that no register is held across the transforms)
  uint32_t* tm_holder = (uint32_t*)(red + 250);
  if constexpr (TM) {
    if ((tid >> 5) == 0) {
      tc::tmem_alloc(tm_holder, 512);
      tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  auto tm_o = [&]() -> uint32_t {   // this thread's patch columns (g follows at + 4 STEPS)
    const int w = (int)(threadIdx.x >> 5);
    return *tm_holder + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((w >> 2) * (65536 / T));
  };
  // releases the tensor memory once every thread's TMEM accesses have completed
  auto tm_release = [&]() {
    if constexpr (TM) {
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(*tm_holder, 512);
    }
  };

  // ---- forward model: I_j = sum_k |F(P_k o_j)|^2 -------------------------------
#pragma unroll 1
  for (int k = 0; k < (PART == 2 ? 0 : M); ++k) {
    const float2* Pk = shared_mode<OPR>(a, k, NN);
    // psi_k = P_k o_j into the tile, two adjacent pixels per thread and iteration
    const NatPairs<N, T> np;
    if constexpr (TM) {
      // groups of two pairs; the patch from TMEM after the first mode; the
      // probe pairs of the next group are loaded (L2) before this group's work
      const uint32_t t_o = tm_o();
      const bool pre = !OPR || Pk;
      float4 Pn[2];
      if (pre)
#pragma unroll
        for (int u = 0; u < 2; ++u) Pn[u] = __ldg((const float4*)(Pk + np.pix(u)));
#pragma unroll 1
      for (int qg = 0; qg < STEPS / 2; ++qg) {
        const float4 Pc[2] = {Pn[0], Pn[1]};
        if (pre && qg + 1 < STEPS / 2)
#pragma unroll
          for (int u = 0; u < 2; ++u) Pn[u] = __ldg((const float4*)(Pk + np.pix(2 * qg + 2 + u)));
        float ov[8];
        if (k == 0) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int q = 2 * qg + u, p = np.pix(q);
            float2 o0, o1;
            bilinear2(a.obj, a.W, ty + np.row(q), tx + np.c, fy, fx, o0, o1);
            if (o_s) *(float4*)(o_s + p) = make_float4(o0.x, o0.y, o1.x, o1.y);
            ov[4 * u] = o0.x; ov[4 * u + 1] = o0.y; ov[4 * u + 2] = o1.x; ov[4 * u + 3] = o1.y;
          }
          tc::tmem_st8(t_o + 8 * qg, ov);
        } else {
          tc::tmem_ld8_wait(t_o + 8 * qg, ov);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int q = 2 * qg + u, p = np.pix(q);
          float4 P2;
          if (pre) {
            P2 = Pc[u];
          } else {
            P2 = opr_pair(a.opr_U, wj, a.K, NN, p);
            if (p0) *(float4*)(p0 + p) = P2;
          }
          const float2 x0 = cmul(make_float2(P2.x, P2.y), make_float2(ov[4 * u], ov[4 * u + 1]));
          const float2 x1 = cmul(make_float2(P2.z, P2.w), make_float2(ov[4 * u + 2], ov[4 * u + 3]));
          store_pair(tile, np.phys(q), x0, x1);
        }
      }
      if (k == 0) tc::tmem_wait_st();
    } else
#pragma unroll 4
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const int r = np.row(q), c = np.c, p = np.pix(q);
      float2 o0, o1;
      if (k == 0 || !o_s) {
        bilinear2(a.obj, a.W, ty + r, tx + c, fy, fx, o0, o1);
        if (k == 0 && o_s) *(float4*)(o_s + p) = make_float4(o0.x, o0.y, o1.x, o1.y);
      } else {
        const float4 o2 = *(const float4*)(o_s + p);
        o0 = make_float2(o2.x, o2.y);
        o1 = make_float2(o2.z, o2.w);
      }
      float4 P2;
      if (!OPR || Pk) {
        P2 = __ldg((const float4*)(Pk + p));
      } else {   // relaxed primary mode of this position
        P2 = opr_pair(a.opr_U, wj, a.K, NN, p);
        if (p0) *(float4*)(p0 + p) = P2;
      }
      const float2 x0 = cmul(make_float2(P2.x, P2.y), o0), x1 = cmul(make_float2(P2.z, P2.w), o1);
      if constexpr (PART == 1)
        *(float4*)(psi_s + (size_t)k * NN + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
      else
        store_pair(tile, np.phys(q), x0, x1);
    }
    if constexpr (PART == 1) continue;
    __syncthreads();
    // the last mode's far field stays in the tile (each row in its own line's
    // storage, free once the row transform is done): the first inverse
    // transform reads it there instead of from the scratch
    const bool keep = (PART == 0) && k == M - 1 && a.mode != MODE_FWD && !a.loss_only;
    fft2_forward<N, T>(tile, tw, [&](int row, float2 (&v)[R2]) {
#pragma unroll
      for (int m = 0; m < R2; ++m) v[m] = cscale(v[m], invN);
      if constexpr (F::S == 2) {
        // registers (2q, 2q+1) hold two adjacent columns: 8-byte intensity and
        // 16-byte far-field accesses
#pragma unroll
        for (int q = 0; q < R2 / 2; ++q) {
          float2* ri = (float2*)(rI + row * RP + F::out_index(n, 2 * q));
          const float2 i2 = make_float2(cabs2(v[2 * q]), cabs2(v[2 * q + 1]));
          *ri = (k == 0) ? i2 : make_float2(ri->x + i2.x, ri->y + i2.y);
        }
      } else {
#pragma unroll
        for (int m = 0; m < R2; ++m) {
          float* ri = rI + row * RP + F::out_index(n, m);
          *ri = (k == 0) ? cabs2(v[m]) : *ri + cabs2(v[m]);
        }
      }
      if (keep) {
        F::template store_out<true>(v, tile, row, n);
      } else if (psi_s) {
        if constexpr (F::S == 2) {
#pragma unroll
          for (int q = 0; q < R2 / 2; ++q)
            *(float4*)(psi_s + (size_t)k * NN + row * N + F::out_index(n, 2 * q)) =
                make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
        } else {
#pragma unroll
          for (int m = 0; m < R2; ++m) psi_s[(size_t)k * NN + row * N + F::out_index(n, m)] = v[m];
        }
      }
    });
    __syncthreads();
  }

  if constexpr (PART == 1) return;
  const int mode = a.mode;
  // ---- data term: loss and the far-field factor (same thread owns each pixel) ----
  if constexpr (PART == 0) {
    const float eps = a.eps;
    const float* meas = a.meas + (size_t)j * NN;
    float lsum = 0.f;
    bool bad = false;
    {
      constexpr int L = T / R1, ITER = N / L;
      const int gid = F::line_slot();
#pragma unroll 1
      for (int it = 0; it < ITER; ++it) {
        const int row = gid + it * L;
        // the row's measured intensities, all loads issued before any use
        // (registers 2q, 2q+1 are adjacent columns when S = 2: 8-byte loads)
        float Imv[R2];
        if (mode != MODE_FWD) {
          if constexpr (F::S == 2) {
#pragma unroll
            for (int q = 0; q < R2 / 2; ++q) {
              const float2 t = __ldg((const float2*)(meas + row * N + F::out_index(n, 2 * q)));
              Imv[2 * q] = t.x;
              Imv[2 * q + 1] = t.y;
            }
          } else {
#pragma unroll
            for (int m = 0; m < R2; ++m) Imv[m] = __ldg(meas + row * N + F::out_index(n, m));
          }
        }
#pragma unroll
        for (int m = 0; m < R2; ++m) {
          const int col = F::out_index(n, m);
          const int pix = row * N + col;
          const float I = rI[row * RP + col];
          if (a.ipred) a.ipred[(size_t)j * NN + pix] = I;
          if (mode == MODE_FWD) continue;
          const float Im = Imv[m];
          float fac;
          if (mode == MODE_VJP) {
            bad |= !isfinite(Im);
            fac = 2.f * Im;
          } else {
            bad |= !(Im >= 0.f) || !isfinite(Im);
            const float Ie = I + eps;
            if (mode == MODE_LSQML_GAUSS || mode == MODE_GRAD_GAUSS) {
              const float sIe = sqrtf(Ie), sIm = sqrtf(Im);
              const float d = sIe - sIm;
              lsum = fmaf(d, d, lsum);
              const float rho = sIm / sIe;
              fac = (mode == MODE_LSQML_GAUSS) ? rho - 1.f : 2.f * (1.f - rho);
            } else {
              lsum += I - Im * logf(Ie);
              const float q = Im / Ie;
              fac = (mode == MODE_LSQML_POISSON) ? 0.5f * (q - 1.f) : 2.f * (1.f - q);
            }
          }
          rI[row * RP + col] = fac * invN;
        }
      }
    }
    if (bad) atomicOr(a.status, FLAG_NONFINITE);
    if (a.loss && mode != MODE_FWD && mode != MODE_VJP) {
      double v[1] = {(double)lsum};
      block_sum<1>(v, red);
      if (tid == 0) atomicAdd(a.loss, v[0]);
    }
    if (mode == MODE_FWD || a.loss_only) {
      tm_release();
      return;
    }
  }

  // ---- back-propagation: chi_k = F^-1[fac Psi_k], g = sum_k conj(P_k) chi_k, h_k ----
  // The modes run last to first: the far fields written last are read first,
  // while they are still in L2.
  float2* g_s = a.g_s + slotNN;
  float2* h_s = a.h_s + slotNN * M;
#pragma unroll 1
  for (int k = M - 1; k >= 0; --k) {
    const float2* Pk = shared_mode<OPR>(a, k, NN);
    if constexpr (PART == 0) {
      __syncthreads();
      fft2_inverse<N, T>(
          tile, tw,
          [&](int row, float2 (&v)[R2]) {
            if (k == M - 1) {   // the last mode's far field was kept in the tile
              F::template load_out<true>(v, tile, row, n);
              __syncwarp();     // every lane of the line has read before the exchange writes
            } else if constexpr (F::S == 2) {
#pragma unroll
              for (int q = 0; q < R2 / 2; ++q) {
                const float4 X = *(const float4*)(psi_s + (size_t)k * NN + row * N + F::out_index(n, 2 * q));
                v[2 * q] = make_float2(X.x, X.y);
                v[2 * q + 1] = make_float2(X.z, X.w);
              }
            } else {
#pragma unroll
              for (int m = 0; m < R2; ++m) v[m] = psi_s[(size_t)k * NN + row * N + F::out_index(n, m)];
            }
            if constexpr (F::S == 2) {
#pragma unroll
              for (int q = 0; q < R2 / 2; ++q) {
                const float2 f = *(const float2*)(rI + row * RP + F::out_index(n, 2 * q));
                v[2 * q] = cscale(v[2 * q], f.x);
                v[2 * q + 1] = cscale(v[2 * q + 1], f.y);
              }
            } else {
#pragma unroll
              for (int m = 0; m < R2; ++m) v[m] = cscale(v[m], rI[row * RP + F::out_index(n, m)]);
            }
          },
          [&](int col, float2 (&v)[R2]) { F::template store_in<false>(v, tile, col, n); });
      __syncthreads();
    }
    // chi_k (natural layout) is in the tile, or in PART 2 in the scratch:
    // g += conj(P_k) chi_k, h_k = conj(o) chi_k
    const NatPairs<N, T> np;
    if constexpr (TM) {
      // o and the running g from TMEM; the last mode's g goes to the scratch
      // (for the step sizes) and over chi in the tile (for the scatter)
      const uint32_t t_o = tm_o(), t_g = t_o + 4 * STEPS;
      // the probe (or primary-mode) pairs of the next group are loaded before
      // this group's work
      // (the primary modes of OPR were written by this kernel: plain loads)
      auto ldP = [&](int p) {
        return (!OPR || Pk) ? __ldg((const float4*)(Pk + p)) : *(const float4*)(p0 + p);
      };
      float4 Pn[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) Pn[u] = ldP(np.pix(u));
#pragma unroll 1
      for (int qg = 0; qg < STEPS / 2; ++qg) {
        const float4 Pc[2] = {Pn[0], Pn[1]};
        if (qg + 1 < STEPS / 2)
#pragma unroll
          for (int u = 0; u < 2; ++u) Pn[u] = ldP(np.pix(2 * qg + 2 + u));
        float ov[8], gv[8];
        if (k < M - 1)
          tc::tmem_ld8x2_wait(t_o + 8 * qg, ov, t_g + 8 * qg, gv);
        else
          tc::tmem_ld8_wait(t_o + 8 * qg, ov);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int q = 2 * qg + u, p = np.pix(q);
          float2 x0, x1;
          load_pair(tile, np.phys(q), x0, x1);
          const float4 P2 = Pc[u];
          float2 g0 = cmulc(make_float2(P2.x, P2.y), x0), g1 = cmulc(make_float2(P2.z, P2.w), x1);
          if (k < M - 1) {
            g0.x += gv[4 * u]; g0.y += gv[4 * u + 1]; g1.x += gv[4 * u + 2]; g1.y += gv[4 * u + 3];
          }
          const float2 h0 = cmulc(make_float2(ov[4 * u], ov[4 * u + 1]), x0);
          const float2 h1 = cmulc(make_float2(ov[4 * u + 2], ov[4 * u + 3]), x1);
          __stcs((float4*)(h_s + (size_t)k * NN + p), make_float4(h0.x, h0.y, h1.x, h1.y));
          if (k > 0) {
            gv[4 * u] = g0.x; gv[4 * u + 1] = g0.y; gv[4 * u + 2] = g1.x; gv[4 * u + 3] = g1.y;
          } else {
            *(float4*)(g_s + p) = make_float4(g0.x, g0.y, g1.x, g1.y);
            store_pair(tile, np.phys(q), g0, g1);
          }
        }
        if (k > 0) tc::tmem_st8(t_g + 8 * qg, gv);
      }
      if (k > 0) tc::tmem_wait_st();
    } else
#pragma unroll 2
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const int p = np.pix(q);
      float2 x0, x1;
      if constexpr (PART == 2) {
        const float4 c = *(const float4*)(psi_s + (size_t)k * NN + p);
        x0 = make_float2(c.x, c.y);
        x1 = make_float2(c.z, c.w);
      } else {
        load_pair(tile, np.phys(q), x0, x1);
      }
      const float4 P2 = (!OPR || Pk) ? __ldg((const float4*)(Pk + p)) : *(const float4*)(p0 + p);
      const float4 o2 = *(const float4*)(o_s + p);
      const float2 g0 = cmulc(make_float2(P2.x, P2.y), x0), g1 = cmulc(make_float2(P2.z, P2.w), x1);
      float4 gv = make_float4(g0.x, g0.y, g1.x, g1.y);
      if (k < M - 1) {
        const float4 gp = *(const float4*)(g_s + p);
        gv = make_float4(gv.x + gp.x, gv.y + gp.y, gv.z + gp.z, gv.w + gp.w);
      }
      *(float4*)(g_s + p) = gv;
      const float2 h0 = cmulc(make_float2(o2.x, o2.y), x0), h1 = cmulc(make_float2(o2.z, o2.w), x1);
      __stcs((float4*)(h_s + (size_t)k * NN + p), make_float4(h0.x, h0.y, h1.x, h1.y));
    }
  }
  __syncthreads();

  // ---- scatter S_j^T g (and the illumination) into the object frame ----------------
  if (!TM) {   // (with TMEM the last mode wrote g into the tile already)
    const NatPairs<N, T> np;
#pragma unroll 1
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const float4 g2 = *(const float4*)(g_s + np.pix(q));
      store_pair(tile, np.phys(q), make_float2(g2.x, g2.y), make_float2(g2.z, g2.w));
    }
  }
  const bool lsqml = (mode == MODE_LSQML_GAUSS || mode == MODE_LSQML_POISSON);
  // LSQML: the probe intensity sum_k |P_k|^2 of every pixel into shared memory
  // (the intensity/factor plane is free by now), so that the scatter's row walk
  // waits on shared memory rather than on L2
  float* spS = rI;
  if (PART != 1 && lsqml) {
    static_assert((size_t)N * RP >= (size_t)NN, "room for the probe intensity");
#pragma unroll 2
    for (int p = 4 * tid; p < NN; p += 4 * T) {
      float4 v = __ldg((const float4*)(a.Sp + p));
      if (OPR && p0) {
        const float4 q0 = *(const float4*)(p0 + p), q1 = *(const float4*)(p0 + p + 2);
        v.x += q0.x * q0.x + q0.y * q0.y; v.y += q0.z * q0.z + q0.w * q0.w;
        v.z += q1.x * q1.x + q1.y * q1.y; v.w += q1.z * q1.z + q1.w * q1.w;
      }
      *(float4*)(spS + p) = v;
    }
  }
  __syncthreads();
  if (lsqml) {
    bilinear_scatter<N, T>(
        fy, fx,
        [&](int y, int x) {
          const float2 g = tile[tix<N>(y, x)];
          return make_float4(g.x, g.y, spS[y * N + x], 0.f);
        },
        [&](int y, int x, float4 v) {
          atomicAdd(a.acc + (size_t)(ty + y) * a.W + (tx + x), make_float4(v.x, v.y, v.z, 0.f));
        });
  } else {
    bilinear_scatter<N, T>(
        fy, fx,
        [&](int y, int x) {
          const float2 g = tile[tix<N>(y, x)];
          return make_float4(g.x, g.y, 0.f, 0.f);
        },
        [&](int y, int x, float4 v) { atomicAdd(a.gobj + (size_t)(ty + y) * a.W + (tx + x), make_float2(v.x, v.y)); });
  }

  // ---- position gradient through the bilinear weights (gradient modes), or the
  // ---- sums of the least-squares position step (LSQML position correction)
  if (a.gpos || a.possum) {
    const bool ls = a.possum != nullptr;
    float gy = 0.f, gx = 0.f, a11 = 0.f, a12 = 0.f, a22 = 0.f;
    for (int p = tid; p < NN; p += T) {
      const int r = p / N, c = p % N;
      const float2* o = a.obj + (size_t)(ty + r) * a.W + (tx + c);
      const float2 O00 = __ldg(o), O01 = __ldg(o + 1), O10 = __ldg(o + a.W), O11 = __ldg(o + a.W + 1);
      const float2 dy = make_float2((1.f - fx) * (O10.x - O00.x) + fx * (O11.x - O01.x),
                                    (1.f - fx) * (O10.y - O00.y) + fx * (O11.y - O01.y));
      const float2 dx = make_float2((1.f - fy) * (O01.x - O00.x) + fy * (O11.x - O10.x),
                                    (1.f - fy) * (O01.y - O00.y) + fy * (O11.y - O10.y));
      const float2 g = tile[tix<N>(r, c)];
      gy += g.x * dy.x + g.y * dy.y;  // Re(conj(g) dy)
      gx += g.x * dx.x + g.y * dx.y;
      if (ls) {   // sum_k abs(P_k)^2 times the derivative products
        const float sp = __ldg(a.Sp + p) + ((OPR && p0) ? cabs2(p0[p]) : 0.f);
        a11 = fmaf(sp, cabs2(dy), a11);
        a12 = fmaf(sp, dy.x * dx.x + dy.y * dx.y, a12);
        a22 = fmaf(sp, cabs2(dx), a22);
      }
    }
    if (ls) {
      double v[5] = {(double)a11, (double)a12, (double)a22, (double)gy, (double)gx};
      block_sum<5>(v, red);
      if (tid == 0)
        for (int q = 0; q < 5; ++q) atomicAdd(a.possum + (size_t)slot * 5 + q, v[q]);
    } else {
      double v[2] = {(double)gy, (double)gx};
      block_sum<2>(v, red);
      if (tid == 0) {
        a.gpos[2 * j] += (float)v[0];
        a.gpos[2 * j + 1] += (float)v[1];
      }
    }
  }
  tm_release();
}


// CTA sizes of the step-size pass (default, alternative).
constexpr int PASS2_T = 512;

// Bilinear sample of dO_hat = dO_acc / (illum + damp) at the patch pixel whose
// four corners start at q (the quotient is taken per corner, then interpolated).
__device__ __forceinline__ float2 dohat(const float4* q, int W, float w00, float w01, float w10, float w11,
                                        float damp) {
  const float4 q00 = __ldg(q), q01 = __ldg(q + 1), q10 = __ldg(q + W), q11 = __ldg(q + W + 1);
  const float i00 = w00 / (q00.z + damp), i01 = w01 / (q01.z + damp);
  const float i10 = w10 / (q10.z + damp), i11 = w11 / (q11.z + damp);
  return make_float2(q00.x * i00 + q01.x * i01 + q10.x * i10 + q11.x * i11,
                     q00.y * i00 + q01.y * i01 + q10.y * i10 + q11.y * i11);
}

template <int N, int T, bool OPR>
__global__ void __launch_bounds__(T, 1024 / T) k_pass2(Pass2Args a) {
  constexpr int NN = N * N;
  wait_prior_grid();
  __shared__ double red[32 * 5];
  __shared__ double alpha_sh;
  const int slot = blockIdx.x, tid = threadIdx.x;
  if (!a.valid[slot]) return;
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  int ty, tx;
  float fy, fx;
  tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  const float damp = a.delta_o * __uint_as_float(a.sc->max_illum);
  const size_t slotNN = (size_t)slot * NN;
  const int M = a.M;
  const float2* g_s = a.g_s + slotNN;
  const float2* o_s = a.o_s + slotNN;
  const float2* h_s = a.h_s + slotNN * M;
  // OPR: the primary mode P_j0 and its direction sum_m w_jm dU_m differ per
  // position; Sp, Cp, Sdp and dP then hold the shared modes only
  constexpr bool opr = OPR;
  __shared__ float wsh[OPR_KMAX];
  if (opr) {
    if (tid < a.K) wsh[tid] = a.opr_w[(size_t)j * a.K + tid];
    __syncthreads();
  }
  const float2* p0 = opr ? a.p0_s + slotNN : nullptr;

  float A11 = 0.f, A12 = 0.f, A22 = 0.f, b1 = 0.f, b2 = 0.f;
  {
    // two adjacent pixels per iteration: 16-byte loads of g, o and Cp, and the
    // six accumulator corners the pair shares (half the trips of this
    // latency-bound loop); with OPR also the pair's primary mode, its
    // direction sum_m w_jm dU_m (K 16-byte loads) and h_j0
#pragma unroll 1
    for (int p = 2 * tid; p < NN; p += 2 * T) {
      const int r = p / N, c = p % N;
      const float4 g2 = __ldg((const float4*)(g_s + p));   // kept in L2: the update reads g again
      const float4 o2 = __ldcs((const float4*)(o_s + p));
      float2 d0 = make_float2(0.f, 0.f), d1 = d0;
      if (a.update_object) {
        const float4* q = a.acc + (size_t)(ty + r) * a.W + (tx + c);
        const float4 qa = __ldg(q), qb = __ldg(q + 1), qc = __ldg(q + 2);
        const float4 qd = __ldg(q + a.W), qe = __ldg(q + a.W + 1), qf = __ldg(q + a.W + 2);
        const float ia = 1.f / (qa.z + damp), ib = 1.f / (qb.z + damp), ic = 1.f / (qc.z + damp);
        const float id = 1.f / (qd.z + damp), ie = 1.f / (qe.z + damp), iF = 1.f / (qf.z + damp);
        // dO_hat at the pixel: each corner's quotient, then the bilinear weights
        d0 = make_float2(w00 * ia * qa.x + w01 * ib * qb.x + w10 * id * qd.x + w11 * ie * qe.x,
                         w00 * ia * qa.y + w01 * ib * qb.y + w10 * id * qd.y + w11 * ie * qe.y);
        d1 = make_float2(w00 * ib * qb.x + w01 * ic * qc.x + w10 * ie * qe.x + w11 * iF * qf.x,
                         w00 * ib * qb.y + w01 * ic * qc.y + w10 * ie * qe.y + w11 * iF * qf.y);
      }
      float2 sp = __ldg((const float2*)(a.Sp + p)), sdp = __ldg((const float2*)(a.Sdp + p));
      float4 cp = __ldg((const float4*)(a.Cp + p));
      if constexpr (OPR) {
        const float4 P2 = *(const float4*)(p0 + p);
        const float2 Pa = make_float2(P2.x, P2.y), Pb = make_float2(P2.z, P2.w);
        sp.x += cabs2(Pa);
        sp.y += cabs2(Pb);
        if (a.update_probe) {
          const float4 D2 = opr_pair(a.opr_dU, wsh, a.K, NN, p);
          const float2 ea = make_float2(D2.x, D2.y), eb = make_float2(D2.z, D2.w);
          const float2 ca = cmulc(Pa, ea), cb = cmulc(Pb, eb);
          cp = make_float4(cp.x + ca.x, cp.y + ca.y, cp.z + cb.x, cp.w + cb.y);
          sdp.x += cabs2(ea);
          sdp.y += cabs2(eb);
          const float4 h2 = __ldcs((const float4*)(h_s + p));
          b2 += ea.x * h2.x + ea.y * h2.y + eb.x * h2.z + eb.y * h2.w;   // Re(conj(dP_j0) h_j0)
        }
      }
      const float2 g0 = make_float2(g2.x, g2.y), g1 = make_float2(g2.z, g2.w);
      const float2 o0 = make_float2(o2.x, o2.y), o1 = make_float2(o2.z, o2.w);
      A11 += cabs2(d0) * sp.x + cabs2(d1) * sp.y;
      const float2 od0 = cmulc(d0, o0), od1 = cmulc(d1, o1);   // conj(d) o
      A12 += od0.x * cp.x - od0.y * cp.y + od1.x * cp.z - od1.y * cp.w;   // Re(conj(d) o Cp)
      A22 += cabs2(o0) * sdp.x + cabs2(o1) * sdp.y;
      b1 += d0.x * g0.x + d0.y * g0.y + d1.x * g1.x + d1.y * g1.y;       // Re(conj(d) g)
    }
  }
  if (a.update_probe) {
    // b2 = Re sum_k <dP_k, h_k> over the shared modes: their planes are
    // contiguous, two pixels per 16-byte load
    const float4* h4 = (const float4*)(h_s + (opr ? NN : 0));
    const float4* d4 = (const float4*)a.dP;
    const int Q = (opr ? M - 1 : M) * NN / 2;
    int q = tid;
    for (; q + 3 * T < Q; q += 4 * T) {      // four independent 16-byte streams per thread
      float4 dp[4], h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        dp[u] = __ldg(d4 + q + u * T);
        h[u] = __ldcs(h4 + q + u * T);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) b2 += dp[u].x * h[u].x + dp[u].y * h[u].y + dp[u].z * h[u].z + dp[u].w * h[u].w;
    }
    for (; q < Q; q += T) {
      const float4 dp = __ldg(d4 + q);
      const float4 h = __ldcs(h4 + q);
      b2 += dp.x * h.x + dp.y * h.y + dp.z * h.z + dp.w * h.w;   // Re(conj(dP_k) h_k)
    }
  }
  double v[5] = {A11, A12, A22, b1, b2};
  block_sum<5>(v, red);
  if (tid == 0) {
    const double a11 = v[0], a12 = v[1], a22 = v[2], r1 = v[3], r2 = v[4];
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
    alpha_sh = aO;
    if (a.alpha_out) {
      a.alpha_out[2 * j] = aO;
      a.alpha_out[2 * j + 1] = aP;
    }
    atomicAdd(&a.sc->sum_alpha_p, aP);
    atomicAdd(&a.sc->count, 1);
  }
  __syncthreads();
  if (!a.update_object) return;
  // O += alpha_O S_j^T g / (illum + delta_O): each object pixel of the (N+1)^2 tile
  // gathers its four patch neighbours and is divided by its own preconditioner
  const float aO = (float)alpha_sh;
  const float c00 = aO * w00, c01 = aO * w01, c10 = aO * w10, c11 = aO * w11;
  constexpr int N1 = N + 1;
  if (((uintptr_t)a.obj & 15) == 0 && (a.W & 1) == 0) {
    // pairs of object pixels at even object columns, one 16-byte vector atomic
    // each (half the atomic operations); per tile row N/2 pairs and one single
    // pixel (the first when tx is odd, else the last)
    constexpr int PR = N / 2 + 1;
    const int odd = tx & 1;
    auto gat = [&](int y, int x) {
      return (y >= 0 && y < N && x >= 0 && x < N) ? g_s[y * N + x] : make_float2(0.f, 0.f);
    };
    for (int i = tid; i < N1 * PR; i += T) {
      const int y = i / PR, k = i % PR;
      const size_t row = (size_t)(ty + y) * a.W + tx;
      if (k < N / 2) {
        const int x = 2 * k + odd;   // pixels x, x + 1 of the tile row
        const float2 gA = gat(y, x - 1), gB = gat(y, x), gC = gat(y, x + 1);
        const float2 hA = gat(y - 1, x - 1), hB = gat(y - 1, x), hC = gat(y - 1, x + 1);
        const float2 s0 = make_float2(c00 * gB.x + c01 * gA.x + c10 * hB.x + c11 * hA.x,
                                      c00 * gB.y + c01 * gA.y + c10 * hB.y + c11 * hA.y);
        const float2 s1 = make_float2(c00 * gC.x + c01 * gB.x + c10 * hC.x + c11 * hB.x,
                                      c00 * gC.y + c01 * gB.y + c10 * hC.y + c11 * hB.y);
        const float i0 = 1.f / (__ldg(&a.acc[row + x].z) + damp);
        const float i1 = 1.f / (__ldg(&a.acc[row + x + 1].z) + damp);
        atomicAdd((float4*)(a.obj + row + x), make_float4(s0.x * i0, s0.y * i0, s1.x * i1, s1.y * i1));
      } else {
        const int x = odd ? 0 : N;
        const float2 gA = gat(y, x - 1), gB = gat(y, x), hA = gat(y - 1, x - 1), hB = gat(y - 1, x);
        const float2 s0 = make_float2(c00 * gB.x + c01 * gA.x + c10 * hB.x + c11 * hA.x,
                                      c00 * gB.y + c01 * gA.y + c10 * hB.y + c11 * hA.y);
        const float i0 = 1.f / (__ldg(&a.acc[row + x].z) + damp);
        atomicAdd(a.obj + row + x, make_float2(s0.x * i0, s0.y * i0));
      }
    }
    return;
  }
  // each object pixel of the (N+1)^2 tile gathers its four patch neighbours
  // (independent outputs keep many global loads in flight)
  for (int q = tid; q < N1 * N1; q += T) {
    const int y = q / N1, x = q % N1;
    float2 sacc = make_float2(0.f, 0.f);
    if (y < N && x < N) { const float2 g = g_s[y * N + x]; sacc.x += c00 * g.x; sacc.y += c00 * g.y; }
    if (y < N && x > 0) { const float2 g = g_s[y * N + x - 1]; sacc.x += c01 * g.x; sacc.y += c01 * g.y; }
    if (y > 0 && x < N) { const float2 g = g_s[(y - 1) * N + x]; sacc.x += c10 * g.x; sacc.y += c10 * g.y; }
    if (y > 0 && x > 0) { const float2 g = g_s[(y - 1) * N + x - 1]; sacc.x += c11 * g.x; sacc.y += c11 * g.y; }
    const size_t oi = (size_t)(ty + y) * a.W + (tx + x);
    const float inv = 1.f / (__ldg(&a.acc[oi].z) + damp);
    atomicAdd(a.obj + oi, make_float2(sacc.x * inv, sacc.y * inv));
  }
}

// Split form of the step-size pass. The five sums of a position are
// independent over its pixels and its h planes, so k_pass2_sums spreads them
// over P2_CHUNKS CTAs per position (every CTA a pure stream of 16-byte loads,
// many CTAs per SM); each writes its FP64 partials without atomics, and
// k_pass2_update adds a position's partials in chunk order (the result does
// not depend on scheduling), solves the 2x2 system and scatters the object
// update.
constexpr int PASS2S_T = 256, PASS2U_T = 512;

template <int N, bool OPR>
__global__ void __launch_bounds__(PASS2S_T, 3) k_pass2_sums(Pass2Args a) {
  constexpr int NN = N * N, T = PASS2S_T, C = P2_CHUNKS;
  static_assert(NN % (2 * C) == 0, "chunks of pixel pairs");
  wait_prior_grid();
  __shared__ double red[32 * 5];
  __shared__ float wsh[OPR_KMAX];
  const int chunk = blockIdx.x, slot = blockIdx.y, tid = threadIdx.x;
  double* out = a.part + ((size_t)slot * C + chunk) * 5;
  if (!a.valid[slot]) {
    if (tid < 5) out[tid] = 0.0;
    return;
  }
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  int ty, tx;
  float fy, fx;
  tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  const float damp = a.delta_o * __uint_as_float(a.sc->max_illum);
  const size_t slotNN = (size_t)slot * NN;
  const int M = a.M;
  const float2* g_s = a.g_s + slotNN;
  const float2* o_s = a.o_s + slotNN;
  const float2* h_s = a.h_s + slotNN * M;
  if (OPR) {
    if (tid < a.K) wsh[tid] = a.opr_w[(size_t)j * a.K + tid];
    __syncthreads();
  }
  const float2* p0 = OPR ? a.p0_s + slotNN : nullptr;

  // pixels [p_lo, p_hi) of the patch
  const int p_lo = chunk * (NN / C), p_hi = p_lo + NN / C;
  float A11 = 0.f, A12 = 0.f, A22 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll 1
  for (int p = p_lo + tid; p < p_hi; p += T) {
    const int r = p / N, c = p % N;
    const float2 g = __ldcs(g_s + p);
    const float2 o = __ldcs(o_s + p);
    float2 d = make_float2(0.f, 0.f);
    if (a.update_object) d = dohat(a.acc + (size_t)(ty + r) * a.W + (tx + c), a.W, w00, w01, w10, w11, damp);
    float sp = __ldg(a.Sp + p), sdp = __ldg(a.Sdp + p);
    float2 cp = __ldg(a.Cp + p);
    if (OPR) {
      const float2 P0 = p0[p];
      sp += cabs2(P0);
      if (a.update_probe) {
        const float2 d0 = opr_pixel(a.opr_dU, wsh, a.K, NN, p);
        cp = cadd(cp, cmulc(P0, d0));
        sdp += cabs2(d0);
        const float2 h0 = __ldcs(h_s + p);
        b2 += d0.x * h0.x + d0.y * h0.y;     // Re(conj(dP_j0) h_j0)
      }
    }
    A11 += cabs2(d) * sp;
    const float2 od = cmulc(d, o);           // conj(d) o
    A12 += od.x * cp.x - od.y * cp.y;        // Re(conj(d) o Cp)
    A22 += cabs2(o) * sdp;
    b1 += d.x * g.x + d.y * g.y;             // Re(conj(d) g)
  }
  if (a.update_probe) {
    // b2 over this chunk of the shared modes' h planes (contiguous pixel pairs)
    const float4* h4 = (const float4*)(h_s + (OPR ? NN : 0));
    const float4* d4 = (const float4*)a.dP;
    const int Q = (OPR ? M - 1 : M) * NN / 2;
    const int q_lo = (int)((long long)Q * chunk / C), q_hi = (int)((long long)Q * (chunk + 1) / C);
    int q = q_lo + tid;
    for (; q + 3 * T < q_hi; q += 4 * T) {      // four independent 16-byte streams per thread
      float4 dp[4], h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        dp[u] = __ldg(d4 + q + u * T);
        h[u] = __ldcs(h4 + q + u * T);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) b2 += dp[u].x * h[u].x + dp[u].y * h[u].y + dp[u].z * h[u].z + dp[u].w * h[u].w;
    }
    for (; q < q_hi; q += T) {
      const float4 dp = __ldg(d4 + q);
      const float4 h = __ldcs(h4 + q);
      b2 += dp.x * h.x + dp.y * h.y + dp.z * h.z + dp.w * h.w;   // Re(conj(dP_k) h_k)
    }
  }
  double v[5] = {A11, A12, A22, b1, b2};
  block_sum<5>(v, red);
  if (tid == 0)
#pragma unroll
    for (int i = 0; i < 5; ++i) out[i] = v[i];
}

template <int N>
__global__ void __launch_bounds__(PASS2U_T, 2) k_pass2_update(Pass2Args a) {
  constexpr int T = PASS2U_T, C = P2_CHUNKS;
  wait_prior_grid();
  __shared__ double alpha_sh;
  const int slot = blockIdx.x, tid = threadIdx.x;
  if (!a.valid[slot]) return;
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  if (tid == 0) {
    const double* pp = a.part + (size_t)slot * C * 5;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] += pp[c * 5 + i];
    const double a11 = v[0], a12 = v[1], a22 = v[2], r1 = v[3], r2 = v[4];
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
    alpha_sh = aO;
    if (a.alpha_out) {
      a.alpha_out[2 * j] = aO;
      a.alpha_out[2 * j + 1] = aP;
    }
    atomicAdd(&a.sc->sum_alpha_p, aP);
    atomicAdd(&a.sc->count, 1);
  }
  __syncthreads();
  if (!a.update_object) return;
  int ty, tx;
  float fy, fx;
  tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  const float damp = a.delta_o * __uint_as_float(a.sc->max_illum);
  const float2* g_s = a.g_s + (size_t)slot * N * N;
  const float aO = (float)alpha_sh;
  const float c00 = aO * (1.f - fy) * (1.f - fx), c01 = aO * (1.f - fy) * fx;
  const float c10 = aO * fy * (1.f - fx), c11 = aO * fy * fx;
  constexpr int N1 = N + 1;
  // O += alpha_O S_j^T g / (illum + delta_O): each object pixel of the (N+1)^2
  // tile gathers its four patch neighbours, divided by its own preconditioner
  for (int q = tid; q < N1 * N1; q += T) {
    const int y = q / N1, x = q % N1;
    float2 sacc = make_float2(0.f, 0.f);
    if (y < N && x < N) { const float2 g = g_s[y * N + x]; sacc.x += c00 * g.x; sacc.y += c00 * g.y; }
    if (y < N && x > 0) { const float2 g = g_s[y * N + x - 1]; sacc.x += c01 * g.x; sacc.y += c01 * g.y; }
    if (y > 0 && x < N) { const float2 g = g_s[(y - 1) * N + x]; sacc.x += c10 * g.x; sacc.y += c10 * g.y; }
    if (y > 0 && x > 0) { const float2 g = g_s[(y - 1) * N + x - 1]; sacc.x += c11 * g.x; sacc.y += c11 * g.y; }
    const size_t oi = (size_t)(ty + y) * a.W + (tx + x);
    const float inv = 1.f / (__ldg(&a.acc[oi].z) + damp);
    atomicAdd(a.obj + oi, make_float2(sacc.x * inv, sacc.y * inv));
  }
}

// Cluster form of the step-size pass (N <= 128): the PASS2C_C CTAs of a
// cluster share one position. CTA q reduces rows [q N/C, (q+1) N/C) of the
// patch and chunk q of the h planes and keeps its rows of g in shared memory;
// the C partial sums meet over distributed shared memory and are added in
// rank order, so every CTA holds the same FP64 totals and solves the 2x2
// system itself; then CTA q scatters the object update of its band of the
// (N+1)^2 tile (rows q N/C .. (q+1) N/C - 1, the last band also row N) from
// its own rows of g and, for its first row, the row above from L2. Against
// one CTA per position: four times the CTAs (the minibatch no longer leaves
// some SMs with one position and others with two), the serial solve of one
// cluster overlaps the streams of the others, and g is read once.
constexpr int PASS2C_T = 256, PASS2C_C = 4;

template <int N, int MINB>
__global__ void __cluster_dims__(PASS2C_C, 1, 1) __launch_bounds__(PASS2C_T, MINB) k_pass2_cluster(Pass2Args a) {
  constexpr int NN = N * N, T = PASS2C_T, C = PASS2C_C, RB = N / C, N1 = N + 1;
  static_assert(N % C == 0 && N <= 128, "bands of whole rows, g band in static shared memory");
  wait_prior_grid();
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ double red[32 * 5];
  __shared__ double part[5];
  __shared__ double alpha_sh;
  __shared__ __align__(16) float2 gsh[RB * N];
  const int q = (int)cluster.block_rank();
  const int slot = blockIdx.x / C, tid = threadIdx.x;
  if (!a.valid[slot]) return;   // the same decision in every CTA of the cluster
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  int ty, tx;
  float fy, fx;
  tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  const float damp = a.delta_o * __uint_as_float(a.sc->max_illum);
  const size_t slotNN = (size_t)slot * NN;
  const int M = a.M;
  const float2* g_s = a.g_s + slotNN;
  const float2* o_s = a.o_s + slotNN;
  const float2* h_s = a.h_s + slotNN * M;

  const int p_lo = q * RB * N;
  float A11 = 0.f, A12 = 0.f, A22 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll 1
  for (int i = tid; i < RB * N; i += T) {
    const int p = p_lo + i, r = p / N, c = p % N;
    const float2 g = __ldcs(g_s + p);
    const float2 o = __ldcs(o_s + p);
    gsh[i] = g;
    float2 d = make_float2(0.f, 0.f);
    if (a.update_object) d = dohat(a.acc + (size_t)(ty + r) * a.W + (tx + c), a.W, w00, w01, w10, w11, damp);
    const float sp = __ldg(a.Sp + p), sdp = __ldg(a.Sdp + p);
    const float2 cp = __ldg(a.Cp + p);
    A11 += cabs2(d) * sp;
    const float2 od = cmulc(d, o);           // conj(d) o
    A12 += od.x * cp.x - od.y * cp.y;        // Re(conj(d) o Cp)
    A22 += cabs2(o) * sdp;
    b1 += d.x * g.x + d.y * g.y;             // Re(conj(d) g)
  }
  if (a.update_probe) {
    // b2 over chunk q of the h planes (contiguous pixel pairs)
    const float4* h4 = (const float4*)h_s;
    const float4* d4 = (const float4*)a.dP;
    const int Q = M * NN / 2;
    const int q_lo = (int)((long long)Q * q / C), q_hi = (int)((long long)Q * (q + 1) / C);
    int k = q_lo + tid;
    for (; k + 3 * T < q_hi; k += 4 * T) {   // four independent 16-byte streams per thread
      float4 dp[4], h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        dp[u] = __ldg(d4 + k + u * T);
        h[u] = __ldcs(h4 + k + u * T);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) b2 += dp[u].x * h[u].x + dp[u].y * h[u].y + dp[u].z * h[u].z + dp[u].w * h[u].w;
    }
    for (; k < q_hi; k += T) {
      const float4 dp = __ldg(d4 + k);
      const float4 h = __ldcs(h4 + k);
      b2 += dp.x * h.x + dp.y * h.y + dp.z * h.z + dp.w * h.w;   // Re(conj(dP_k) h_k)
    }
  }
  double v[5] = {A11, A12, A22, b1, b2};
  block_sum<5>(v, red);
  if (tid == 0)
#pragma unroll
    for (int i = 0; i < 5; ++i) part[i] = v[i];
  cluster.sync();   // every CTA's partials (and its g band) are written
  if (tid == 0) {
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const double* pr = cluster.map_shared_rank(part, r);
#pragma unroll
      for (int i = 0; i < 5; ++i) t[i] += pr[i];
    }
    const double a11 = t[0], a12 = t[1], a22 = t[2], r1 = t[3], r2 = t[4];
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
    alpha_sh = aO;
    if (q == 0) {
      if (a.alpha_out) {
        a.alpha_out[2 * j] = aO;
        a.alpha_out[2 * j + 1] = aP;
      }
      atomicAdd(&a.sc->sum_alpha_p, aP);
      atomicAdd(&a.sc->count, 1);
    }
  }
  cluster.sync();   // no CTA leaves while another reads its partials; alpha_sh is visible
  if (!a.update_object) return;
  const float aO = (float)alpha_sh;
  const float c00 = aO * w00, c01 = aO * w01, c10 = aO * w10, c11 = aO * w11;
  const int y0 = q * RB, y1 = y0 + RB + (q == C - 1 ? 1 : 0);
  // g at patch row yy (y0 - 1 <= yy < y0 + RB): the band from shared memory, the row above from L2
  auto gat = [&](int yy, int xx) { return yy >= y0 ? gsh[(yy - y0) * N + xx] : __ldg(g_s + yy * N + xx); };
  for (int i = tid; i < (y1 - y0) * N1; i += T) {
    const int y = y0 + i / N1, x = i % N1;
    float2 sacc = make_float2(0.f, 0.f);
    if (y < N && x < N) { const float2 g = gat(y, x); sacc.x += c00 * g.x; sacc.y += c00 * g.y; }
    if (y < N && x > 0) { const float2 g = gat(y, x - 1); sacc.x += c01 * g.x; sacc.y += c01 * g.y; }
    if (y > 0 && x < N) { const float2 g = gat(y - 1, x); sacc.x += c10 * g.x; sacc.y += c10 * g.y; }
    if (y > 0 && x > 0) { const float2 g = gat(y - 1, x - 1); sacc.x += c11 * g.x; sacc.y += c11 * g.y; }
    const size_t oi = (size_t)(ty + y) * a.W + (tx + x);
    const float inv = 1.f / (__ldg(&a.acc[oi].z) + damp);
    atomicAdd(a.obj + oi, make_float2(sacc.x * inv, sacc.y * inv));
  }
}

}  // namespace ptycho

namespace ptycho {

// Opts a kernel into more than 48 KB of dynamic shared memory, once per device
// (so that no attribute call happens while a stream is being captured).
template <class K>
cudaError_t smem_optin(K kernel, size_t bytes, unsigned long long* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) __atomic_fetch_or(done_mask, bit, __ATOMIC_ACQ_REL);
  return e;
}

template <int N, int T, bool OPR, int PART = 0>
cudaError_t launch_pass1_t(const BatchArgs& a, cudaStream_t s) {
  constexpr size_t sm = Pass1Smem<N>::bytes;
  static unsigned long long done = 0;
  cudaError_t e = smem_optin(k_pass1<N, T, OPR, PART>, sm, &done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  return launch_pdl(k_pass1<N, T, OPR, PART>, dim3(a.nb), dim3(T), sm, s, a);
}

// variant 0: default CTA size, 1: the alternative (the relaxed-probe form has
// the default only)
template <int N>
cudaError_t launch_pass1(const BatchArgs& a, cudaStream_t s, int variant) {
  if (a.opr_U) return launch_pass1_t<N, Threads<N>::T, true>(a, s);
  return variant == 1 ? launch_pass1_t<N, Threads<N>::ALT, false>(a, s)
                      : launch_pass1_t<N, Threads<N>::T, false>(a, s);
}

// variant 0: the single-kernel form of PASS2_T threads, 1: the split form
// (when the partials buffer is given), 2 and 3: the cluster form at four and
// three CTAs per SM (64 and 80 registers; N <= 128, not OPR)
template <int N>
cudaError_t launch_pass2(const Pass2Args& a, cudaStream_t s, int variant) {
  if (a.nb <= 0) return cudaSuccess;
  if constexpr (N <= 128) {
    if (variant == 2 && !a.opr_dU)
      return launch_pdl(k_pass2_cluster<N, 4>, dim3(PASS2C_C * a.nb), dim3(PASS2C_T), 0, s, a);
    if (variant == 3 && !a.opr_dU)
      return launch_pdl(k_pass2_cluster<N, 3>, dim3(PASS2C_C * a.nb), dim3(PASS2C_T), 0, s, a);
  }
  if (a.part && variant == 1) {
    cudaError_t e = a.opr_dU
        ? launch_pdl(k_pass2_sums<N, true>, dim3(P2_CHUNKS, a.nb), dim3(PASS2S_T), 0, s, a)
        : launch_pdl(k_pass2_sums<N, false>, dim3(P2_CHUNKS, a.nb), dim3(PASS2S_T), 0, s, a);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_pass2_update<N>, dim3(a.nb), dim3(PASS2U_T), 0, s, a);
  }
  if (a.opr_dU) return launch_pdl(k_pass2<N, PASS2_T, true>, dim3(a.nb), dim3(PASS2_T), 0, s, a);
  return launch_pdl(k_pass2<N, PASS2_T, false>, dim3(a.nb), dim3(PASS2_T), 0, s, a);
}

}  // namespace ptycho
