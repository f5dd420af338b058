// Multislice forward model and its adjoint (Pty-Chi Sec. 1 and Sec. 2.1:
// multislice modelling), for windows held by one CTA (N <= 128).
//
// The object has S slices [S, H, W]. For position j and probe mode k the wave
// entering slice 0 is P_k; the wave leaving slice s is (incident_s) o_j^(s)
// with o_j^(s) = S_j(O^(s)); between slices it is carried by the
// angular-spectrum propagator, incident_s = F^-1[H F (leaving_{s-1})]. The
// far field of the last slice's exit wave gives I_j = sum_k |F psi|^2.
//
// k_pass1_ms: one CTA per position. It extracts all slice patches once,
// runs every mode through the slices in shared memory (a propagation is a
// column FFT pass, a fused row pass that transforms, multiplies by H / N^2 and
// transforms back, and an inverse column pass), keeps the incident waves of
// slices 1..S-1 in scratch for the backward pass, and forms the data term as
// the single-slice kernel does. With a.recompute the forward pass keeps no
// incident waves: the backward pass first runs the mode through the slices
// again (2 (S-1) more 2-D transforms) and parks that mode's waves in the
// slot's scratch, where they are read back soon after, mostly from L2. The
// backward pass runs each mode from the far
// field back through the slices (conj(H) propagation), accumulating the
// per-slice object gradients conj(incident_s) g and the probe gradient
// conj(o^(0)) g, then scatters every slice's gradient into its plane and
// sums the position gradient over the slices.
#pragma once
#include "kernels.cuh"

namespace ptycho {

// Propagates the tile (natural layout, spatial domain) to the next slice:
// tile <- F^-1[H F tile] (CONJ: conj(H), the adjoint). Ends synchronised.
template <int N, int T, bool CONJ>
__device__ __forceinline__ void propagate_tile(float2* tile, const float2* tw, const float2* __restrict__ Hf) {
  using F = Fft2<N>;
  constexpr int R1 = F::R1, R2 = F::R2, L = T / R1, ITER = N / L;
  const int n = F::line_lane(), gid = F::line_slot();
  const float s = 1.0f / (float)(N * N);
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
#pragma unroll
    for (int m = 0; m < R2; ++m) {
      float2 h = __ldg(Hf + row * N + F::out_index(n, m));
      if (CONJ) h.y = -h.y;
      v[m] = cscale(cmul(v[m], h), s);
    }
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
    F::template store_in<false>(v, tile, col, n);
  }
  __syncthreads();
}

// Runs probe mode Pk through the slices again and writes the incident waves of
// slices 1..S-1 to inc (S-1 consecutive N x N planes): the same arithmetic as
// the forward pass, so the waves are bitwise those it saw. Leaves the tile
// holding the last incident wave; starts and ends synchronised.
template <int N, int T>
__device__ __forceinline__ void recompute_incident(float2* tile, const float2* tw, const float2* __restrict__ Hf,
                                                   const float2* Pk, const float2* o_s, float2* inc, int S) {
  constexpr int NN = N * N;
  const NatPairs<N, T> np;
  __syncthreads();
#pragma unroll 2
  for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
    const int p = np.pix(q);
    const float4 o2 = *(const float4*)(o_s + p);
    const float4 P2 = __ldg((const float4*)(Pk + p));
    store_pair(tile, np.phys(q), cmul(make_float2(P2.x, P2.y), make_float2(o2.x, o2.y)),
               cmul(make_float2(P2.z, P2.w), make_float2(o2.z, o2.w)));
  }
  __syncthreads();
#pragma unroll 1
  for (int s = 1; s < S; ++s) {
    propagate_tile<N, T, false>(tile, tw, Hf);
    float2* in = inc + (size_t)(s - 1) * NN;
    const bool last = s == S - 1;
#pragma unroll 2
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const int p = np.pix(q);
      float2 x0, x1;
      load_pair(tile, np.phys(q), x0, x1);
      *(float4*)(in + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
      if (!last) {
        const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
        store_pair(tile, np.phys(q), cmul(x0, make_float2(o2.x, o2.y)), cmul(x1, make_float2(o2.z, o2.w)));
      }
    }
    __syncthreads();
  }
}

// LS: the LSQML instantiation (exit-plane changes instead of gradients, the
// slices' illumination, the per-slice accumulators); the gradient form has
// none of it.
template <int N, int T, bool LS>
__global__ void __launch_bounds__(T, 1) k_pass1_ms(MsArgs a) {
  using F = Fft2<N>;
  using SM = Pass1Smem<N>;
  constexpr int R2 = F::R2, NN = N * N, RP = SM::RP;
  extern __shared__ __align__(16) unsigned char smem[];
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
  make_twiddles<N>(tw);

  const int M = a.M, S = a.S;
  const size_t HW = (size_t)a.H * a.W;
  const float invN = 1.0f / (float)N;
  const size_t slotNN = (size_t)slot * NN;
  const int mode = a.mode;
  const bool grad = mode != MODE_FWD;
  constexpr bool lsqml = LS;
  const bool rec = a.recompute != 0, keep = grad && !rec;
  float2* psi_s = grad ? a.psi_s + slotNN * M : nullptr;
  float2* o_s = a.o_s + slotNN * S;
  const NatPairs<N, T> np;

  // ---- slice patches o^(s) = S_j(O^(s)) -------------------------------------------
  for (int s = 0; s < S; ++s) {
#pragma unroll 2
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      float2 o0, o1;
      bilinear2(a.obj + s * HW, a.W, ty + np.row(q), tx + np.c, fy, fx, o0, o1);
      *(float4*)(o_s + (size_t)s * NN + np.pix(q)) = make_float4(o0.x, o0.y, o1.x, o1.y);
    }
  }
  __syncthreads();

  // ---- forward: every mode through the slices, then the far field --------------------
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = a.probe + (size_t)k * NN;
#pragma unroll 2
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const int p = np.pix(q);
      const float4 o2 = *(const float4*)(o_s + p);
      const float4 P2 = __ldg((const float4*)(Pk + p));
      store_pair(tile, np.phys(q), cmul(make_float2(P2.x, P2.y), make_float2(o2.x, o2.y)),
                 cmul(make_float2(P2.z, P2.w), make_float2(o2.z, o2.w)));
    }
    __syncthreads();
#pragma unroll 1
    for (int s = 1; s < S; ++s) {
      propagate_tile<N, T, false>(tile, tw, a.Hf);
      float2* inc = keep ? a.in_s + ms_inc_offset(false, slotNN, M, S, k, s, NN) : nullptr;
      // LSQML: the slice's illumination sum_k |inc_k|^2
      float2* wsl = lsqml ? (float2*)(a.w_s + (slotNN * (S - 1) + (size_t)(s - 1) * NN)) : nullptr;
#pragma unroll 2
      for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
        const int p = np.pix(q);
        float2 x0, x1;
        load_pair(tile, np.phys(q), x0, x1);
        if (keep) *(float4*)(inc + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
        if (lsqml) {
          float2 w2 = make_float2(cabs2(x0), cabs2(x1));
          if (k > 0) {
            const float2 wp = wsl[p / 2];
            w2.x += wp.x;
            w2.y += wp.y;
          }
          wsl[p / 2] = w2;
        }
        const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
        store_pair(tile, np.phys(q), cmul(x0, make_float2(o2.x, o2.y)), cmul(x1, make_float2(o2.z, o2.w)));
      }
      __syncthreads();
    }
    fft2_forward<N, T>(tile, tw, [&](int row, float2 (&v)[R2]) {
#pragma unroll
      for (int m = 0; m < R2; ++m) {
        const int col = F::out_index(n, m);
        const float2 X = cscale(v[m], invN);
        float* ri = rI + row * RP + col;
        *ri = (k == 0) ? cabs2(X) : *ri + cabs2(X);
        if (grad) psi_s[(size_t)k * NN + row * N + col] = X;
      }
    });
    __syncthreads();
  }

  // ---- data term (as in the single-slice pass) ---------------------------------------
  const float eps = a.eps;
  const float* meas = a.meas ? a.meas + (size_t)j * NN : nullptr;
  float lsum = 0.f;
  bool bad = false;
  {
    constexpr int L = T / F::R1, ITER = N / L;
    const int gid = F::line_slot();
#pragma unroll 1
    for (int it = 0; it < ITER; ++it) {
      const int row = gid + it * L;
#pragma unroll
      for (int m = 0; m < R2; ++m) {
        const int col = F::out_index(n, m);
        const int pix = row * N + col;
        const float I = rI[row * RP + col];
        if (a.ipred) a.ipred[(size_t)j * NN + pix] = I;
        if (!grad) continue;
        const float Im = __ldg(meas + pix);
        float fac;
        if (mode == MODE_VJP) {
          bad |= !isfinite(Im);
          fac = 2.f * Im;
        } else {
          bad |= !(Im >= 0.f) || !isfinite(Im);
          const float Ie = I + eps;
          if (mode == MODE_GRAD_GAUSS || mode == MODE_LSQML_GAUSS) {
            const float sIe = sqrtf(Ie), sIm = sqrtf(Im), d = sIe - sIm;
            lsum = fmaf(d, d, lsum);
            const float rho = sIm / sIe;
            fac = (mode == MODE_LSQML_GAUSS) ? rho - 1.f : 2.f * (1.f - rho);
          } else {
            lsum += I - Im * logf(Ie);
            const float qq = Im / Ie;
            fac = (mode == MODE_LSQML_POISSON) ? 0.5f * (qq - 1.f) : 2.f * (1.f - qq);
          }
        }
        rI[row * RP + col] = fac * invN;
      }
    }
  }
  if (bad) atomicOr(a.status, FLAG_NONFINITE);
  if (a.loss && grad && mode != MODE_VJP) {
    double v[1] = {(double)lsum};
    block_sum<1>(v, red);
    if (tid == 0) atomicAdd(a.loss, v[0]);
  }
  if (!grad) return;

  // ---- backward: each mode from the far field back through the slices ---------------
  float2* go_s = a.go_s + slotNN * S;
  float2* h_s = a.h_s + slotNN * M;
  // modes last to first: the far field and incident waves written last are read
  // first, while they are still in L2
#pragma unroll 1
  for (int k = M - 1; k >= 0; --k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    if (rec && S > 1)
      recompute_incident<N, T>(tile, tw, a.Hf, Pk, o_s, a.in_s + ms_inc_offset(true, slotNN, M, S, k, 1, NN), S);
    __syncthreads();
    fft2_inverse<N, T>(
        tile, tw,
        [&](int row, float2 (&v)[R2]) {
#pragma unroll
          for (int m = 0; m < R2; ++m) {
            const int col = F::out_index(n, m);
            v[m] = cscale(psi_s[(size_t)k * NN + row * N + col], rI[row * RP + col]);
          }
        },
        [&](int col, float2 (&v)[R2]) { F::template store_in<false>(v, tile, col, n); });
    __syncthreads();
#pragma unroll 1
    for (int s = S - 1; s >= 1; --s) {
      const float2* inc = a.in_s + ms_inc_offset(rec, slotNN, M, S, k, s, NN);
#pragma unroll 2
      for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
        const int p = np.pix(q);
        float2 g0, g1;
        load_pair(tile, np.phys(q), g0, g1);
        const float4 i2 = *(const float4*)(inc + p);
        const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 a0 = cmulc(make_float2(i2.x, i2.y), g0), a1 = cmulc(make_float2(i2.z, i2.w), g1);
        float4* gp = (float4*)(go_s + (size_t)s * NN + p);
        gv = make_float4(a0.x, a0.y, a1.x, a1.y);
        if (k < M - 1) {
          const float4 prev = *gp;
          gv = make_float4(gv.x + prev.x, gv.y + prev.y, gv.z + prev.z, gv.w + prev.w);
        }
        *gp = gv;
        store_pair(tile, np.phys(q), cmulc(make_float2(o2.x, o2.y), g0), cmulc(make_float2(o2.z, o2.w), g1));
      }
      __syncthreads();
      propagate_tile<N, T, true>(tile, tw, a.Hf);
    }
    // slice 0: object gradient conj(P_k) g, probe gradient conj(o^(0)) g
#pragma unroll 2
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const int p = np.pix(q);
      float2 g0, g1;
      load_pair(tile, np.phys(q), g0, g1);
      const float4 P2 = __ldg((const float4*)(Pk + p));
      const float4 o2 = *(const float4*)(o_s + p);
      const float2 a0 = cmulc(make_float2(P2.x, P2.y), g0), a1 = cmulc(make_float2(P2.z, P2.w), g1);
      float4 gv = make_float4(a0.x, a0.y, a1.x, a1.y);
      float4* gp = (float4*)(go_s + p);
      if (k < M - 1) {
        const float4 prev = *gp;
        gv = make_float4(gv.x + prev.x, gv.y + prev.y, gv.z + prev.z, gv.w + prev.w);
      }
      *gp = gv;
      const float2 h0 = cmulc(make_float2(o2.x, o2.y), g0), h1 = cmulc(make_float2(o2.z, o2.w), g1);
      __stcs((float4*)(h_s + (size_t)k * NN + p), make_float4(h0.x, h0.y, h1.x, h1.y));
    }
  }
  __syncthreads();

  // ---- per slice: scatter S_j^T of its gradient; position gradient over the slices ----
  float gyv = 0.f, gxv = 0.f;
#pragma unroll 1
  for (int s = 0; s < S; ++s) {
#pragma unroll 2
    for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
      const float4 g2 = *(const float4*)(go_s + (size_t)s * NN + np.pix(q));
      store_pair(tile, np.phys(q), make_float2(g2.x, g2.y), make_float2(g2.z, g2.w));
    }
    __syncthreads();
    if (lsqml) {   // S_j^T of the slice's direction numerator and of its illumination
      float4* acc = a.acc + s * HW;
      const float* wsl = s > 0 ? a.w_s + (slotNN * (S - 1) + (size_t)(s - 1) * NN) : a.Sp;
      bilinear_scatter<N, T>(
          fy, fx,
          [&](int y, int x) {
            const float2 g = tile[tix<N>(y, x)];
            return make_float4(g.x, g.y, wsl[y * N + x], 0.f);
          },
          [&](int y, int x, float4 v) {
            atomicAdd(acc + (size_t)(ty + y) * a.W + (tx + x), make_float4(v.x, v.y, v.z, 0.f));
          });
    }
    if (a.gobj) {
      float2* gplane = a.gobj + s * HW;
      bilinear_scatter<N, T>(
          fy, fx,
          [&](int y, int x) {
            const float2 g = tile[tix<N>(y, x)];
            return make_float4(g.x, g.y, 0.f, 0.f);
          },
          [&](int y, int x, float4 v) { atomicAdd(gplane + (size_t)(ty + y) * a.W + (tx + x), make_float2(v.x, v.y)); });
    }
    if (a.gpos) {
      const float2* Os = a.obj + s * HW;
      for (int p = tid; p < NN; p += T) {
        const int r = p / N, c = p % N;
        const float2* o = Os + (size_t)(ty + r) * a.W + (tx + c);
        const float2 O00 = __ldg(o), O01 = __ldg(o + 1), O10 = __ldg(o + a.W), O11 = __ldg(o + a.W + 1);
        const float2 dy = make_float2((1.f - fx) * (O10.x - O00.x) + fx * (O11.x - O01.x),
                                      (1.f - fx) * (O10.y - O00.y) + fx * (O11.y - O01.y));
        const float2 dx = make_float2((1.f - fy) * (O01.x - O00.x) + fy * (O11.x - O10.x),
                                      (1.f - fy) * (O01.y - O00.y) + fy * (O11.y - O10.y));
        const float2 g = tile[tix<N>(r, c)];
        gyv += g.x * dy.x + g.y * dy.y;
        gxv += g.x * dx.x + g.y * dx.y;
      }
    }
    __syncthreads();
  }
  if (a.gpos) {
    double v[2] = {(double)gyv, (double)gxv};
    block_sum<2>(v, red);
    if (tid == 0) {
      a.gpos[2 * j] += (float)v[0];
      a.gpos[2 * j + 1] += (float)v[1];
    }
  }
}

// Tangents of the multislice forward model for the LSQML step sizes (one CTA
// per position): per mode, u starts as P_k d_0 and is carried through the
// slices as u <- H(u) o_s + inc_s d_s, v starts as dP_k o_0 and is carried as
// v <- H(v) o_s; at the exit plane the CTA sums |u|^2, Re(conj(u) v), |v|^2
// over the pixels and modes (u of the mode parked in scratch while v runs).
template <int N, int T>
__global__ void __launch_bounds__(T, 1) k_step_ms(MsStepArgs a) {
  using SM = Pass1Smem<N>;
  constexpr int NN = N * N;
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = (double*)(smem + SM::red);
  float2* tile = (float2*)(smem + SM::tile);
  float2* tw = (float2*)(smem + SM::tw);
  const int slot = blockIdx.x, tid = threadIdx.x;
  double* out = a.part + (size_t)slot * 3;
  if (!a.valid[slot]) {
    if (tid < 3) out[tid] = 0.0;
    return;
  }
  make_twiddles<N>(tw);
  const int M = a.M, S = a.S;
  const size_t slotNN = (size_t)slot * NN;
  const float2* o_s = a.o_s + slotNN * S;
  const float2* d_s = a.d_s + slotNN * S;
  float2* u_s = a.u_s + slotNN;
  const bool rec = a.recompute != 0;
  float2* in_w = rec ? a.in_s + ms_inc_offset(true, slotNN, M, S, 0, 1, NN) : nullptr;
  const NatPairs<N, T> np;
  float A11 = 0.f, A12 = 0.f, A22 = 0.f;
  auto f2 = [](float4 v, int h) { return h ? make_float2(v.z, v.w) : make_float2(v.x, v.y); };
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    const float2* dPk = a.dP + (size_t)k * NN;
    if (rec && S > 1) recompute_incident<N, T>(tile, tw, a.Hf, Pk, o_s, in_w, S);
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {   // t = 0: the object tangent u, 1: the probe tangent v
      __syncthreads();
#pragma unroll 2
      for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
        const int p = np.pix(q);
        const float4 o2 = *(const float4*)(o_s + p);
        const float4 x2 = t == 0 ? __ldg((const float4*)(Pk + p)) : __ldg((const float4*)(dPk + p));
        const float4 y2 = t == 0 ? *(const float4*)(d_s + p) : o2;
        store_pair(tile, np.phys(q), cmul(f2(x2, 0), f2(y2, 0)), cmul(f2(x2, 1), f2(y2, 1)));
      }
      __syncthreads();
#pragma unroll 1
      for (int s = 1; s < S; ++s) {
        propagate_tile<N, T, false>(tile, tw, a.Hf);
        const float2* inc = a.in_s + ms_inc_offset(rec, slotNN, M, S, k, s, NN);
#pragma unroll 2
        for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
          const int p = np.pix(q);
          float2 x0, x1;
          load_pair(tile, np.phys(q), x0, x1);
          const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
          x0 = cmul(x0, f2(o2, 0));
          x1 = cmul(x1, f2(o2, 1));
          if (t == 0) {   // the slice's own direction as a source
            const float4 i2 = *(const float4*)(inc + p);
            const float4 d2 = *(const float4*)(d_s + (size_t)s * NN + p);
            x0 = cadd(x0, cmul(f2(i2, 0), f2(d2, 0)));
            x1 = cadd(x1, cmul(f2(i2, 1), f2(d2, 1)));
          }
          store_pair(tile, np.phys(q), x0, x1);
        }
        __syncthreads();
      }
#pragma unroll 2
      for (int q = 0; q < NatPairs<N, T>::STEPS; ++q) {
        const int p = np.pix(q);
        float2 x0, x1;
        load_pair(tile, np.phys(q), x0, x1);
        if (t == 0) {
          A11 += cabs2(x0) + cabs2(x1);
          *(float4*)(u_s + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
        } else {
          const float4 u2 = *(const float4*)(u_s + p);
          A22 += cabs2(x0) + cabs2(x1);
          A12 += u2.x * x0.x + u2.y * x0.y + u2.z * x1.x + u2.w * x1.y;   // Re(conj(u) v)
        }
      }
    }
  }
  double v[3] = {(double)A11, (double)A12, (double)A22};
  block_sum<3>(v, red);
  if (tid == 0)
    for (int i = 0; i < 3; ++i) out[i] = v[i];
}

template <int N>
cudaError_t launch_step_ms(const MsStepArgs& a, cudaStream_t s) {
  constexpr int T = N == 128 ? 512 : Threads<N>::T;
  constexpr size_t sm = Pass1Smem<N>::bytes;
  static unsigned long long done = 0;
  cudaError_t e = smem_optin(k_step_ms<N, T>, sm, &done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  k_step_ms<N, T><<<a.nb, T, sm, s>>>(a);
  return cudaGetLastError();
}

// CTA size of the multislice pass: the default of the single-slice pass, but
// 512 threads at N = 128 (the slice loops need more than 64 registers).
template <int N>
cudaError_t launch_pass1_ms(const MsArgs& a, cudaStream_t s) {
  constexpr int T = N == 128 ? 512 : Threads<N>::T;
  constexpr size_t sm = Pass1Smem<N>::bytes;
  static unsigned long long done = 0, done_ls = 0;
  const bool ls = a.mode == MODE_LSQML_GAUSS || a.mode == MODE_LSQML_POISSON;
  cudaError_t e = ls ? smem_optin(k_pass1_ms<N, T, true>, sm, &done_ls) : smem_optin(k_pass1_ms<N, T, false>, sm, &done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  if (ls)
    k_pass1_ms<N, T, true><<<a.nb, T, sm, s>>>(a);
  else
    k_pass1_ms<N, T, false><<<a.nb, T, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ptycho
