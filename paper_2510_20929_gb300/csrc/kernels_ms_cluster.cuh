// Multislice per-position pass for the cluster windows (N = 192, 256): the
// model and the phases of k_pass1_ms, with the N x N tile shared by a cluster
// of Q CTAs as in k_pass1_cluster. CTA q holds the spatial rows LR q ..;
// a 2-D transform (cl::fwd2d) leaves it the frequency columns LR q .., so
// a propagation is fwd2d, a multiplication of those columns by H / N^2, and
// cl::inv2d back to the CTA's spatial rows.
#pragma once
#include "kernels_cluster.cuh"

namespace ptycho {
namespace cl {

// tile <- F^-1[H F tile] over the cluster (CONJ: conj(H)); ends synchronised.
template <class C, bool CONJ>
__device__ __forceinline__ void propagate_cluster(cg::cluster_group& cluster, float2* tile, const float2* twr, int q,
                                                  const float2* __restrict__ Hf) {
  constexpr int N = C::N, T = C::T, LNN = C::LNN;
  const float sc = 1.0f / (float)(N * N);
  fwd2d<C>(cluster, tile, twr, q);
#pragma unroll 4
  for (int e = (int)threadIdx.x; e < LNN; e += T) {   // this CTA's frequency columns
    int x, ky;
    C::freq_index(e, x, ky);
    float2 h = __ldg(Hf + (size_t)ky * N + C::LR * q + x);
    if (CONJ) h.y = -h.y;
    const int t = C::tix(x, ky);
    tile[t] = cscale(cmul(tile[t], h), sc);
  }
  __syncthreads();
  inv2d<C>(cluster, tile, twr, q);
}

// recompute_incident over the cluster: CTA q writes its own rows of the
// incident waves of slices 1..S-1 of mode Pk to inc; starts and ends
// synchronised.
template <class C>
__device__ __forceinline__ void recompute_incident_cluster(cg::cluster_group& cluster, float2* tile,
                                                           const float2* twr, int q, const float2* __restrict__ Hf,
                                                           const float2* Pk, const float2* o_s, float2* inc, int S) {
  constexpr int N = C::N, T = C::T, LR = C::LR, NN = C::NN, NAT_STEPS = C::NAT_STEPS;
  const int tid = threadIdx.x, rowbase = LR * q;
  __syncthreads();
#pragma unroll 2
  for (int st = 0; st < NAT_STEPS; ++st) {
    const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
    const int p = (rowbase + r) * N + c;
    const float4 o2 = *(const float4*)(o_s + p);
    const float4 P2 = __ldg((const float4*)(Pk + p));
    store_pair(tile, C::tix(r, c), cmul(make_float2(P2.x, P2.y), make_float2(o2.x, o2.y)),
               cmul(make_float2(P2.z, P2.w), make_float2(o2.z, o2.w)));
  }
  __syncthreads();
#pragma unroll 1
  for (int s = 1; s < S; ++s) {
    propagate_cluster<C, false>(cluster, tile, twr, q, Hf);
    float2* in = inc + (size_t)(s - 1) * NN;
    const bool last = s == S - 1;
#pragma unroll 2
    for (int st = 0; st < NAT_STEPS; ++st) {
      const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
      const int p = (rowbase + r) * N + c;
      float2 x0, x1;
      load_pair(tile, C::tix(r, c), x0, x1);
      *(float4*)(in + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
      if (!last) {
        const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
        store_pair(tile, C::tix(r, c), cmul(x0, make_float2(o2.x, o2.y)), cmul(x1, make_float2(o2.z, o2.w)));
      }
    }
    __syncthreads();
  }
}

// LS: the LSQML instantiation (as in k_pass1_ms).
template <class C, bool LS>
__global__ void __launch_bounds__(C::T, C::MINB) k_pass1_ms_cluster(MsArgs a) {
  constexpr int N = C::N, Q = C::Q, T = C::T, LR = C::LR, NN = C::NN, LNN = C::LNN;
  constexpr int NAT_STEPS = C::NAT_STEPS;
  using SM = typename C::Smem;
  constexpr int RP = SM::RP;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = (double*)(smem + SM::red);
  float2* tile = (float2*)(smem + SM::tile);
  float2* twr = (float2*)(smem + SM::twr);
  float* rI = (float*)(smem + SM::rI);

  const int q = (int)cluster.block_rank();
  const int slot = blockIdx.x / Q;
  const int tid = threadIdx.x;
  const int j = a.order ? a.order[a.b0 + slot] : a.b0 + slot;
  int ty = 0, tx = 0;
  float fy = 0.f, fx = 0.f;
  bool ok = (j >= 0 && j < a.J);
  if (ok) ok = tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  if (!ok) {   // the same decision in every CTA of the cluster
    if (tid == 0 && q == 0) {
      atomicOr(a.status, FLAG_BOUNDS);
      if (a.valid) a.valid[slot] = 0;
    }
    return;
  }
  if (tid == 0 && q == 0 && a.valid) a.valid[slot] = 1;
  make_line_twiddles<N, C::RR1, C::RR2>(twr);

  const int M = a.M, S = a.S, mode = a.mode;
  const bool grad = mode != MODE_FWD;
  constexpr bool lsqml = LS;
  const bool rec = a.recompute != 0, keep = grad && !rec;
  const size_t HW = (size_t)a.H * a.W;
  const float invN = 1.0f / (float)N;
  const size_t slotNN = (size_t)slot * NN;
  const int rowbase = LR * q;
  float2* psi_s = grad ? a.psi_s + slotNN * M : nullptr;
  float2* o_s = a.o_s + slotNN * S;

  // ---- slice patches of this CTA's rows ----------------------------------------------
  for (int s = 0; s < S; ++s) {
#pragma unroll 2
    for (int st = 0; st < NAT_STEPS; ++st) {
      const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
      float2 o0, o1;
      bilinear2(a.obj + s * HW, a.W, ty + rowbase + r, tx + c, fy, fx, o0, o1);
      *(float4*)(o_s + (size_t)s * NN + (rowbase + r) * N + c) = make_float4(o0.x, o0.y, o1.x, o1.y);
    }
  }

  // ---- forward -----------------------------------------------------------------------
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    __syncthreads();
#pragma unroll 2
    for (int st = 0; st < NAT_STEPS; ++st) {
      const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
      const int p = (rowbase + r) * N + c;
      const float4 o2 = *(const float4*)(o_s + p);
      const float4 P2 = __ldg((const float4*)(Pk + p));
      store_pair(tile, C::tix(r, c), cmul(make_float2(P2.x, P2.y), make_float2(o2.x, o2.y)),
                 cmul(make_float2(P2.z, P2.w), make_float2(o2.z, o2.w)));
    }
    __syncthreads();
#pragma unroll 1
    for (int s = 1; s < S; ++s) {
      propagate_cluster<C, false>(cluster, tile, twr, q, a.Hf);
      float2* inc = keep ? a.in_s + ms_inc_offset(false, slotNN, M, S, k, s, NN) : nullptr;
      // LSQML: the slice's illumination sum_k |inc_k|^2
      float2* wsl = lsqml ? (float2*)(a.w_s + (slotNN * (S - 1) + (size_t)(s - 1) * NN)) : nullptr;
#pragma unroll 2
      for (int st = 0; st < NAT_STEPS; ++st) {
        const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
        const int p = (rowbase + r) * N + c;
        float2 x0, x1;
        load_pair(tile, C::tix(r, c), x0, x1);
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
        store_pair(tile, C::tix(r, c), cmul(x0, make_float2(o2.x, o2.y)), cmul(x1, make_float2(o2.z, o2.w)));
      }
      __syncthreads();
    }
    fwd2d<C>(cluster, tile, twr, q);
#pragma unroll 4
    for (int e = tid; e < LNN; e += T) {   // this CTA's far-field columns
      int x, ky;
      C::freq_index(e, x, ky);
      const float2 X = cscale(tile[C::tix(x, ky)], invN);
      float* ri = rI + x * RP + ky;
      *ri = (k == 0) ? cabs2(X) : *ri + cabs2(X);
      if (grad) psi_s[(size_t)k * NN + (size_t)q * LNN + e] = X;
    }
  }

  // ---- data term (this CTA's far-field columns) ---------------------------------------
  const float eps = a.eps;
  const float* meas = a.meas ? a.meas + (size_t)j * NN : nullptr;
  float lsum = 0.f;
  bool bad = false;
  static_assert(LNN % (2 * T) == 0, "data-term loop takes two elements per step");
#pragma unroll 1
  for (int e0 = tid; e0 < LNN; e0 += 2 * T) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = e0 + u * T;
      int x, ky;
      C::freq_index(e, x, ky);
      const int pix = ky * N + LR * q + x;
      float* ri = rI + x * RP + ky;
      const float I = *ri;
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
      *ri = fac * invN;
    }
  }
  if (bad) atomicOr(a.status, FLAG_NONFINITE);
  if (a.loss && grad && mode != MODE_VJP) {
    double v[1] = {(double)lsum};
    block_sum<1>(v, red);
    if (tid == 0) atomicAdd(a.loss, v[0]);
  }
  if (!grad) {
    cluster.sync();   // no CTA leaves while another may still read its tile
    return;
  }

  // ---- backward ----------------------------------------------------------------------
  float2* go_s = a.go_s + slotNN * S;
  float2* h_s = a.h_s + slotNN * M;
  // modes last to first: the far field and incident waves written last are read
  // first, while they are still in L2
#pragma unroll 1
  for (int k = M - 1; k >= 0; --k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    if (rec && S > 1)
      recompute_incident_cluster<C>(cluster, tile, twr, q, a.Hf, Pk, o_s,
                                    a.in_s + ms_inc_offset(true, slotNN, M, S, k, 1, NN), S);
    __syncthreads();
#pragma unroll 4
    for (int e = tid; e < LNN; e += T) {
      int x, ky;
      C::freq_index(e, x, ky);
      tile[C::tix(x, ky)] = cscale(psi_s[(size_t)k * NN + (size_t)q * LNN + e], rI[x * RP + ky]);
    }
    __syncthreads();
    inv2d<C>(cluster, tile, twr, q);
#pragma unroll 1
    for (int s = S - 1; s >= 1; --s) {
      const float2* inc = a.in_s + ms_inc_offset(rec, slotNN, M, S, k, s, NN);
#pragma unroll 2
      for (int st = 0; st < NAT_STEPS; ++st) {
        const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
        const int p = (rowbase + r) * N + c;
        float2 g0, g1;
        load_pair(tile, C::tix(r, c), g0, g1);
        const float4 i2 = *(const float4*)(inc + p);
        const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
        const float2 a0 = cmulc(make_float2(i2.x, i2.y), g0), a1 = cmulc(make_float2(i2.z, i2.w), g1);
        float4 gv = make_float4(a0.x, a0.y, a1.x, a1.y);
        float4* gp = (float4*)(go_s + (size_t)s * NN + p);
        if (k < M - 1) {
          const float4 prev = *gp;
          gv = make_float4(gv.x + prev.x, gv.y + prev.y, gv.z + prev.z, gv.w + prev.w);
        }
        *gp = gv;
        store_pair(tile, C::tix(r, c), cmulc(make_float2(o2.x, o2.y), g0), cmulc(make_float2(o2.z, o2.w), g1));
      }
      __syncthreads();
      propagate_cluster<C, true>(cluster, tile, twr, q, a.Hf);
    }
#pragma unroll 2
    for (int st = 0; st < NAT_STEPS; ++st) {
      const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
      const int p = (rowbase + r) * N + c;
      float2 g0, g1;
      load_pair(tile, C::tix(r, c), g0, g1);
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
  // every CTA's rows of the slice gradients are written (the scatter reads one
  // row of the neighbour); also no CTA leaves while another reads its tile
  cluster.sync();

  // ---- per slice: scatter this CTA's rows (+ row N); position gradient --------------
  float gyv = 0.f, gxv = 0.f;
  const int y0 = rowbase, y1 = rowbase + LR + (q == Q - 1 ? 1 : 0);
  constexpr int N1 = N + 1;
  const float gx = 1.f - fx, gy = 1.f - fy;
#pragma unroll 1
  for (int s = 0; s < S; ++s) {
    const float2* gsl = go_s + (size_t)s * NN;
    if (lsqml) {   // S_j^T of the slice's direction numerator and of its illumination
      float4* acc = a.acc + s * HW;
      const float* wsl = s > 0 ? a.w_s + (slotNN * (S - 1) + (size_t)(s - 1) * NN) : a.Sp;
      auto hrow4 = [&](int y, int x) {
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        if (y >= 0 && y < N) {
          if (x < N) {
            const float2 v = gsl[y * N + x];
            const float w = wsl[y * N + x];
            h = make_float4(gx * v.x, gx * v.y, gx * w, 0.f);
          }
          if (x > 0) {
            const float2 v = gsl[y * N + x - 1];
            const float w = wsl[y * N + x - 1];
            h.x = fmaf(fx, v.x, h.x);
            h.y = fmaf(fx, v.y, h.y);
            h.z = fmaf(fx, w, h.z);
          }
        }
        return h;
      };
      constexpr int SEG = T / N1 > 0 ? T / N1 : 1;
      const int rows = y1 - y0, rs = (rows + SEG - 1) / SEG;
      for (int item = tid; item < N1 * SEG; item += T) {
        const int sg = item / N1, x = item % N1;
        const int ya = y0 + sg * rs, yb = min(y1, ya + rs);
        if (ya >= yb) continue;
        float4 hp = hrow4(ya - 1, x);
        for (int y = ya; y < yb; ++y) {
          const float4 hc = hrow4(y, x);
          atomicAdd(acc + (size_t)(ty + y) * a.W + (tx + x),
                    make_float4(fmaf(gy, hc.x, fy * hp.x), fmaf(gy, hc.y, fy * hp.y), fmaf(gy, hc.z, fy * hp.z),
                                0.f));
          hp = hc;
        }
      }
    }
    if (a.gobj) {
      float2* gplane = a.gobj + s * HW;
      auto hrow = [&](int y, int x) {
        float2 h = make_float2(0.f, 0.f);
        if (y >= 0 && y < N) {
          if (x < N) {
            const float2 v = gsl[y * N + x];
            h = make_float2(gx * v.x, gx * v.y);
          }
          if (x > 0) {
            const float2 v = gsl[y * N + x - 1];
            h.x = fmaf(fx, v.x, h.x);
            h.y = fmaf(fx, v.y, h.y);
          }
        }
        return h;
      };
      constexpr int SEG = T / N1 > 0 ? T / N1 : 1;
      const int rows = y1 - y0, rs = (rows + SEG - 1) / SEG;
      for (int item = tid; item < N1 * SEG; item += T) {
        const int sg = item / N1, x = item % N1;
        const int ya = y0 + sg * rs, yb = min(y1, ya + rs);
        if (ya >= yb) continue;
        float2 hp = hrow(ya - 1, x);
        for (int y = ya; y < yb; ++y) {
          const float2 hc = hrow(y, x);
          atomicAdd(gplane + (size_t)(ty + y) * a.W + (tx + x),
                    make_float2(fmaf(gy, hc.x, fy * hp.x), fmaf(gy, hc.y, fy * hp.y)));
          hp = hc;
        }
      }
    }
    if (a.gpos) {
      const float2* Os = a.obj + s * HW;
      for (int pl = tid; pl < LNN; pl += T) {
        const int r = rowbase + pl / N, c = pl % N;
        const float2* o = Os + (size_t)(ty + r) * a.W + (tx + c);
        const float2 O00 = __ldg(o), O01 = __ldg(o + 1), O10 = __ldg(o + a.W), O11 = __ldg(o + a.W + 1);
        const float2 dy = make_float2((1.f - fx) * (O10.x - O00.x) + fx * (O11.x - O01.x),
                                      (1.f - fx) * (O10.y - O00.y) + fx * (O11.y - O01.y));
        const float2 dx = make_float2((1.f - fy) * (O01.x - O00.x) + fy * (O11.x - O10.x),
                                      (1.f - fy) * (O01.y - O00.y) + fy * (O11.y - O10.y));
        const float2 g = gsl[r * N + c];
        gyv += g.x * dy.x + g.y * dy.y;
        gxv += g.x * dx.x + g.y * dx.y;
      }
    }
  }
  if (a.gpos) {
    double v[2] = {(double)gyv, (double)gxv};
    block_sum<2>(v, red);
    if (tid == 0) {
      atomicAdd(a.gpos + 2 * j, (float)v[0]);
      atomicAdd(a.gpos + 2 * j + 1, (float)v[1]);
    }
  }
}

// The tangent pass of k_step_ms on the cluster windows: CTA q carries its 64
// rows of u and v through the slices (propagate_cluster) and writes its
// partial Gram entries; the step-size kernel adds the Q partials.
template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) k_step_ms_cluster(MsStepArgs a) {
  constexpr int N = C::N, Q = C::Q, T = C::T, LR = C::LR, NN = C::NN;
  constexpr int NAT_STEPS = C::NAT_STEPS;
  using SM = typename C::Smem;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = (double*)(smem + SM::red);
  float2* tile = (float2*)(smem + SM::tile);
  float2* twr = (float2*)(smem + SM::twr);
  const int q = (int)cluster.block_rank();
  const int slot = blockIdx.x / Q;
  const int tid = threadIdx.x;
  double* out = a.part + ((size_t)slot * Q + q) * 3;
  if (!a.valid[slot]) {   // the same decision in every CTA of the cluster
    if (tid < 3) out[tid] = 0.0;
    return;
  }
  make_line_twiddles<N, C::RR1, C::RR2>(twr);
  const int M = a.M, S = a.S, rowbase = LR * q;
  const size_t slotNN = (size_t)slot * NN;
  const float2* o_s = a.o_s + slotNN * S;
  const float2* d_s = a.d_s + slotNN * S;
  float2* u_s = a.u_s + slotNN;
  const bool rec = a.recompute != 0;
  float2* in_w = rec ? a.in_s + ms_inc_offset(true, slotNN, M, S, 0, 1, NN) : nullptr;
  float A11 = 0.f, A12 = 0.f, A22 = 0.f;
  auto f2 = [](float4 v, int h) { return h ? make_float2(v.z, v.w) : make_float2(v.x, v.y); };
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    const float2* dPk = a.dP + (size_t)k * NN;
    if (rec && S > 1) recompute_incident_cluster<C>(cluster, tile, twr, q, a.Hf, Pk, o_s, in_w, S);
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {   // t = 0: the object tangent u, 1: the probe tangent v
      __syncthreads();
#pragma unroll 2
      for (int st = 0; st < NAT_STEPS; ++st) {
        const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
        const int p = (rowbase + r) * N + c;
        const float4 o2 = *(const float4*)(o_s + p);
        const float4 x2 = t == 0 ? __ldg((const float4*)(Pk + p)) : __ldg((const float4*)(dPk + p));
        const float4 y2 = t == 0 ? *(const float4*)(d_s + p) : o2;
        store_pair(tile, C::tix(r, c), cmul(f2(x2, 0), f2(y2, 0)), cmul(f2(x2, 1), f2(y2, 1)));
      }
      __syncthreads();
#pragma unroll 1
      for (int s = 1; s < S; ++s) {
        propagate_cluster<C, false>(cluster, tile, twr, q, a.Hf);
        const float2* inc = a.in_s + ms_inc_offset(rec, slotNN, M, S, k, s, NN);
#pragma unroll 2
        for (int st = 0; st < NAT_STEPS; ++st) {
          const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
          const int p = (rowbase + r) * N + c;
          float2 x0, x1;
          load_pair(tile, C::tix(r, c), x0, x1);
          const float4 o2 = *(const float4*)(o_s + (size_t)s * NN + p);
          x0 = cmul(x0, f2(o2, 0));
          x1 = cmul(x1, f2(o2, 1));
          if (t == 0) {
            const float4 i2 = *(const float4*)(inc + p);
            const float4 d2 = *(const float4*)(d_s + (size_t)s * NN + p);
            x0 = cadd(x0, cmul(f2(i2, 0), f2(d2, 0)));
            x1 = cadd(x1, cmul(f2(i2, 1), f2(d2, 1)));
          }
          store_pair(tile, C::tix(r, c), x0, x1);
        }
        __syncthreads();
      }
#pragma unroll 2
      for (int st = 0; st < NAT_STEPS; ++st) {
        const int pl = 2 * tid + 2 * T * st, r = pl / N, c = pl % N;
        const int p = (rowbase + r) * N + c;
        float2 x0, x1;
        load_pair(tile, C::tix(r, c), x0, x1);
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
  cluster.sync();   // no CTA leaves while another may still read its tile
}

}  // namespace cl

template <class C>
cudaError_t launch_step_ms_cluster(const MsStepArgs& a, cudaStream_t s, unsigned long long* done) {
  cudaError_t e = smem_optin(cl::k_step_ms_cluster<C>, C::Smem::bytes, done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C::Q * a.nb));
  cfg.blockDim = dim3(C::T);
  cfg.dynamicSmemBytes = C::Smem::bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C::Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cl::k_step_ms_cluster<C>, a);
}

template <class C, bool LS>
cudaError_t launch_ms_cluster_t(const MsArgs& a, cudaStream_t s, unsigned long long* done) {
  cudaError_t e = smem_optin(cl::k_pass1_ms_cluster<C, LS>, C::Smem::bytes, done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C::Q * a.nb));
  cfg.blockDim = dim3(C::T);
  cfg.dynamicSmemBytes = C::Smem::bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C::Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cl::k_pass1_ms_cluster<C, LS>, a);
}

// done[0]: the gradient form's shared-memory opt-in, done[1]: the LSQML form's
template <class C>
cudaError_t launch_ms_cluster(const MsArgs& a, cudaStream_t s, unsigned long long* done) {
  if (a.mode == MODE_LSQML_GAUSS || a.mode == MODE_LSQML_POISSON) return launch_ms_cluster_t<C, true>(a, s, done + 1);
  return launch_ms_cluster_t<C, false>(a, s, done);
}

}  // namespace ptycho
