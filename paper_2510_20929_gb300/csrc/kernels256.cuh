// Per-position pass for 256 x 256 windows on a cluster of four CTAs.
//
// The 256 x 256 complex tile (512 KB) does not fit one CTA's shared memory,
// so a cluster of Q = 4 CTAs shares it: CTA q holds the 64 rows 64q .. 64q+63.
// The 2-D DFT runs as
//   * 256-point transforms of the CTA's own rows (shared memory, as in the
//     single-CTA kernel);
//   * the column transform split as 256 = 4 x 64 (decimation in time over the
//     row index R = 64q + r): a 4-point DFT across the cluster for every
//     (r, c), reading the other CTAs' tiles through distributed shared memory,
//     times the twiddle W_256^(r k1), after which CTA k1 holds the inputs of
//     the outputs k = k1 + 4 k2; then 64-point transforms of its local columns;
//   * the inverse mirrors it: local 64-point column inverses, the conjugate
//     twiddle and 4-point inverse DFT across the cluster, local row inverses.
// Everything else (patch gather, data term, back-propagation, scatter, the
// position gradient) follows the single-CTA k_pass1 on the CTA's own rows;
// the far fields of CTA q are the frequency rows q + 4 k2.
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace ptycho {
namespace n256 {

namespace cg = cooperative_groups;

constexpr int N = 256, Q = 4, LR = 64, T = 1024;
constexpr int NN = N * N, LNN = LR * N;

// Local 64 x 256 tile: column bits XOR f(r, c) = ((r << 2) ^ (r >> 1) ^ (c >> 4)) & 15,
// chosen with the same half-warp bank model for 256-point row lines (lanes
// consecutive) and 64-point column lines (lanes interleaved).
__host__ __device__ constexpr int fr(int r) { return ((r << 2) ^ (r >> 1)) & 15; }
__host__ __device__ constexpr int fcb(int c) { return (c >> 4) & 15; }
__device__ __forceinline__ int tix(int r, int c) { return r * N + (c ^ fr(r) ^ fcb(c)); }

struct RectAddr {
  template <bool ROW>
  __device__ __forceinline__ static int addr(int line, int i_rt, int i_ct) {
    if constexpr (ROW) {
      const int base = line * N + (i_rt ^ fr(line) ^ fcb(i_rt));
      return base ^ (i_ct ^ fcb(i_ct));
    } else {
      const int base = i_rt * N + (line ^ fcb(line) ^ fr(i_rt));
      return (base + i_ct * N) ^ fr(i_ct);
    }
  }
};

using RowF = LineFft<16, 16, false, RectAddr>;   // 256-point rows
using ColF = LineFft<8, 8, true, RectAddr>;      // 64-point local columns

struct Smem {
  static constexpr int RP = N + 16;
  static constexpr size_t red = 0;
  static constexpr size_t tile = red + 256 * sizeof(double);
  static constexpr size_t twr = tile + (size_t)LNN * sizeof(float2);
  static constexpr size_t twc = twr + 16 * 17 * sizeof(float2);
  static constexpr size_t tw256 = twc + 8 * 9 * sizeof(float2);
  static constexpr size_t rI = tw256 + 256 * sizeof(float2);
  static constexpr size_t bytes = rI + (size_t)LR * RP * sizeof(float);
};

// a * W4^m (W4 = e^{-2 pi i / 4}); m taken mod 4
__device__ __forceinline__ float2 w4mul(float2 a, int m) {
  switch (m & 3) {
    case 0: return a;
    case 1: return make_float2(a.y, -a.x);
    case 2: return make_float2(-a.x, -a.y);
    default: return make_float2(-a.y, a.x);
  }
}

// Natural local pixel pairs: thread t handles p = 2t + 2T s (s < 8): local row
// p / 256, columns c, c+1.
constexpr int NAT_STEPS = LNN / (2 * T);

// Cross-cluster 4-point DFT of the tiles, in four column quarters.
// Forward: tile_q <- W256^(r q) sum_q' W4^(q' q) tile_q'.
// Inverse: tile_q <- sum_k1 W4^(-q k1) conj(W256^(r k1)) tile_k1.
template <bool FWD>
__device__ __forceinline__ void cross_exchange(cg::cluster_group& cluster, float2* tile, const float2* tw256, int q) {
  float2* src[Q];
#pragma unroll
  for (int qq = 0; qq < Q; ++qq) src[qq] = cluster.map_shared_rank(tile, qq);
#pragma unroll 1
  for (int h = 0; h < 4; ++h) {
    float2 acc[2][2];
    int rr[2], cc[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int p = 2 * (int)threadIdx.x + 2 * T * j;   // within a 64 x 64 quarter: 4096 pixels
      rr[j] = p / 64;
      cc[j] = 64 * h + p % 64;
      acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int qq = 0; qq < Q; ++qq) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float2 x0, x1;
        load_pair(src[qq], tix(rr[j], cc[j]), x0, x1);
        if constexpr (FWD) {
          const int m = qq * q;
          acc[j][0] = cadd(acc[j][0], w4mul(x0, m));
          acc[j][1] = cadd(acc[j][1], w4mul(x1, m));
        } else {
          const float2 t = tw256[(rr[j] * qq) & 255];     // W256^(r k1), conjugated below
          const int m = -(q * qq);
          acc[j][0] = cadd(acc[j][0], w4mul(cmulc(t, x0), m));
          acc[j][1] = cadd(acc[j][1], w4mul(cmulc(t, x1), m));
        }
      }
    }
    cluster.sync();   // every CTA has read this quarter of every tile
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if constexpr (FWD) {
        const float2 t = tw256[(rr[j] * q) & 255];
        store_pair(tile, tix(rr[j], cc[j]), cmul(acc[j][0], t), cmul(acc[j][1], t));
      } else {
        store_pair(tile, tix(rr[j], cc[j]), acc[j][0], acc[j][1]);
      }
    }
  }
  __syncthreads();
}

// 2-D forward DFT (unnormalised) of the cluster's tile; on return CTA q's tile
// holds the frequency rows q + 4 k2 (local row k2), natural layout.
__device__ __forceinline__ void fwd2d(cg::cluster_group& cluster, float2* tile, const float2* twr,
                                      const float2* twc, const float2* tw256, int q) {
  {
    const int n = RowF::line_lane(), row = RowF::line_slot();
    float2 v[16];
    RowF::load_in<true>(v, tile, row, n);
    RowF::line_fwd<true>(v, tile, row, n, twr);
    RowF::store_out<true>(v, tile, row, n);
  }
  cluster.sync();
  cross_exchange<true>(cluster, tile, tw256, q);
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const int n = ColF::line_lane(), col = ColF::line_slot() + 128 * it;
    float2 v[8];
    ColF::load_in<false>(v, tile, col, n);
    ColF::line_fwd<false>(v, tile, col, n, twc);
    ColF::store_out<false>(v, tile, col, n);
  }
  __syncthreads();
}

// 2-D inverse DFT (unnormalised): tile_q holds frequency rows q + 4 k2 on entry
// and the spatial rows 64q + r on return, natural layout.
__device__ __forceinline__ void inv2d(cg::cluster_group& cluster, float2* tile, const float2* twr,
                                      const float2* twc, const float2* tw256, int q) {
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const int n = ColF::line_lane(), col = ColF::line_slot() + 128 * it;
    float2 v[8];
    ColF::load_out<false>(v, tile, col, n);
    ColF::line_inv<false>(v, tile, col, n, twc);
    ColF::store_in<false>(v, tile, col, n);
  }
  __syncthreads();
  cluster.sync();
  cross_exchange<false>(cluster, tile, tw256, q);
  {
    const int n = RowF::line_lane(), row = RowF::line_slot();
    float2 v[16];
    RowF::load_out<true>(v, tile, row, n);
    RowF::line_inv<true>(v, tile, row, n, twr);
    RowF::store_in<true>(v, tile, row, n);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(T, 1) k_pass1_c256(BatchArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = (double*)(smem + Smem::red);
  float2* tile = (float2*)(smem + Smem::tile);
  float2* twr = (float2*)(smem + Smem::twr);
  float2* twc = (float2*)(smem + Smem::twc);
  float2* tw256 = (float2*)(smem + Smem::tw256);
  float* rI = (float*)(smem + Smem::rI);
  constexpr int RP = Smem::RP;

  const int q = (int)cluster.block_rank();
  const int slot = blockIdx.x / Q;
  const int tid = threadIdx.x;
  const int e = a.b0 + slot;
  const int j = a.order ? a.order[e] : e;
  int ty = 0, tx = 0;
  float fy = 0.f, fx = 0.f;
  bool ok = (j >= 0 && j < a.J);
  if (ok) ok = tile_of(a.pos[2 * j], a.pos[2 * j + 1], N, a.H, a.W, ty, tx, fy, fx);
  if (!ok) {   // the same decision in all four CTAs of the cluster
    if (tid == 0 && q == 0) {
      atomicOr(a.status, FLAG_BOUNDS);
      if (a.valid) a.valid[slot] = 0;
    }
    return;
  }
  if (tid == 0 && q == 0 && a.valid) a.valid[slot] = 1;
  make_line_twiddles<256, 16, 16>(twr);
  make_line_twiddles<64, 8, 8>(twc);
  for (int m = tid; m < 256; m += T) {
    float s, c;
    sincospif(2.0f * (float)m / 256.0f, &s, &c);
    tw256[m] = make_float2(c, -s);
  }

  const int M = a.M;
  const float invN = 1.0f / (float)N;
  const size_t slotNN = (size_t)slot * NN;
  float2* psi_s = a.psi_s ? a.psi_s + slotNN * M : nullptr;
  float2* o_s = a.o_s ? a.o_s + slotNN : nullptr;
  const int rowbase = LR * q;   // first spatial row of this CTA

  // ---- forward model --------------------------------------------------------------
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    __syncthreads();
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
      const int p = (rowbase + r) * N + c;
      float2 o0, o1;
      if (k == 0 || !o_s) {
        bilinear2(a.obj, a.W, ty + rowbase + r, tx + c, fy, fx, o0, o1);
        if (k == 0 && o_s) *(float4*)(o_s + p) = make_float4(o0.x, o0.y, o1.x, o1.y);
      } else {
        const float4 o2 = *(const float4*)(o_s + p);
        o0 = make_float2(o2.x, o2.y);
        o1 = make_float2(o2.z, o2.w);
      }
      const float4 P2 = __ldg((const float4*)(Pk + p));
      store_pair(tile, tix(r, c), cmul(make_float2(P2.x, P2.y), o0), cmul(make_float2(P2.z, P2.w), o1));
    }
    __syncthreads();
    fwd2d(cluster, tile, twr, twc, tw256, q);
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;   // r = local frequency row k2
      float2 X0, X1;
      load_pair(tile, tix(r, c), X0, X1);
      X0 = cscale(X0, invN);
      X1 = cscale(X1, invN);
      float2* ri = (float2*)(rI + r * RP + c);
      const float2 i2 = make_float2(cabs2(X0), cabs2(X1));
      *ri = (k == 0) ? i2 : make_float2(ri->x + i2.x, ri->y + i2.y);
      if (psi_s)
        *(float4*)(psi_s + (size_t)k * NN + (q + 4 * r) * N + c) = make_float4(X0.x, X0.y, X1.x, X1.y);
    }
  }

  // ---- data term (frequency rows q + 4 k2) ----------------------------------------
  const int mode = a.mode;
  const float eps = a.eps;
  const float* meas = a.meas + (size_t)j * NN;
  float lsum = 0.f;
  bool bad = false;
#pragma unroll 1
  for (int s = 0; s < NAT_STEPS; ++s) {
    const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
    const int pix = (q + 4 * r) * N + c;
    float* ri = rI + r * RP + c;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float I = ri[u];
      if (a.ipred) a.ipred[(size_t)j * NN + pix + u] = I;
      if (mode == MODE_FWD) continue;
      const float Im = __ldg(meas + pix + u);
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
          const float qq = Im / Ie;
          fac = (mode == MODE_LSQML_POISSON) ? 0.5f * (qq - 1.f) : 2.f * (1.f - qq);
        }
      }
      ri[u] = fac * invN;
    }
  }
  if (bad) atomicOr(a.status, FLAG_NONFINITE);
  if (a.loss && mode != MODE_FWD && mode != MODE_VJP) {
    double v[1] = {(double)lsum};
    block_sum<1>(v, red);
    if (tid == 0) atomicAdd(a.loss, v[0]);
  }
  if (mode == MODE_FWD) {
    cluster.sync();   // no CTA leaves while another may still read its tile
    return;
  }

  // ---- back-propagation -------------------------------------------------------------
  float2* g_s = a.g_s + slotNN;
  float2* h_s = a.h_s + slotNN * M;
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = a.probe + (size_t)k * NN;
    __syncthreads();
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
      const float4 X = *(const float4*)(psi_s + (size_t)k * NN + (q + 4 * r) * N + c);
      const float2 f = *(const float2*)(rI + r * RP + c);
      store_pair(tile, tix(r, c), make_float2(X.x * f.x, X.y * f.x), make_float2(X.z * f.y, X.w * f.y));
    }
    __syncthreads();
    inv2d(cluster, tile, twr, twc, tw256, q);
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
      const int p = (rowbase + r) * N + c;
      float2 x0, x1;
      load_pair(tile, tix(r, c), x0, x1);
      const float4 P2 = __ldg((const float4*)(Pk + p));
      const float4 o2 = *(const float4*)(o_s + p);
      const float2 g0 = cmulc(make_float2(P2.x, P2.y), x0), g1 = cmulc(make_float2(P2.z, P2.w), x1);
      float4 gv = make_float4(g0.x, g0.y, g1.x, g1.y);
      if (k > 0) {
        const float4 gp = *(const float4*)(g_s + p);
        gv = make_float4(gv.x + gp.x, gv.y + gp.y, gv.z + gp.z, gv.w + gp.w);
      }
      *(float4*)(g_s + p) = gv;
      const float2 h0 = cmulc(make_float2(o2.x, o2.y), x0), h1 = cmulc(make_float2(o2.z, o2.w), x1);
      __stcs((float4*)(h_s + (size_t)k * NN + p), make_float4(h0.x, h0.y, h1.x, h1.y));
    }
  }
  // every CTA's rows of g are written (the scatter reads one row of the neighbour)
  cluster.sync();

  // ---- scatter S_j^T g (and the illumination), rows 64q .. 64q+63 (+ row 256) ------
  const bool lsqml = (mode == MODE_LSQML_GAUSS || mode == MODE_LSQML_POISSON);
  {
    const int y0 = rowbase, y1 = rowbase + LR + (q == Q - 1 ? 1 : 0);
    constexpr int N1 = N + 1;
    const float gx = 1.f - fx, gy = 1.f - fy;
    auto loadg = [&](int y, int x) {
      const float2 g = g_s[y * N + x];
      return make_float4(g.x, g.y, lsqml ? __ldg(a.Sp + y * N + x) : 0.f, 0.f);
    };
    auto hrow = [&](int y, int x) {
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
      if (y >= 0 && y < N) {
        if (x < N) {
          const float4 v = loadg(y, x);
          h = make_float4(gx * v.x, gx * v.y, gx * v.z, 0.f);
        }
        if (x > 0) {
          const float4 v = loadg(y, x - 1);
          h.x = fmaf(fx, v.x, h.x); h.y = fmaf(fx, v.y, h.y); h.z = fmaf(fx, v.z, h.z);
        }
      }
      return h;
    };
    constexpr int SEG = T / N1;                       // 3 row segments of the CTA's rows
    const int rows = y1 - y0, rs = (rows + SEG - 1) / SEG;
    for (int item = tid; item < N1 * SEG; item += T) {
      const int sg = item / N1, x = item % N1;
      const int ya = y0 + sg * rs, yb = min(y1, ya + rs);
      if (ya >= yb) continue;
      float4 hp = hrow(ya - 1, x);
      for (int y = ya; y < yb; ++y) {
        const float4 hc = hrow(y, x);
        const float4 v = make_float4(fmaf(gy, hc.x, fy * hp.x), fmaf(gy, hc.y, fy * hp.y),
                                     fmaf(gy, hc.z, fy * hp.z), 0.f);
        const size_t oi = (size_t)(ty + y) * a.W + (tx + x);
        if (lsqml) atomicAdd(a.acc + oi, v);
        else atomicAdd(a.gobj + oi, make_float2(v.x, v.y));
        hp = hc;
      }
    }
  }

  // ---- position gradient (gradient modes), this CTA's rows ----------------------------
  if (a.gpos) {
    float gyv = 0.f, gxv = 0.f;
    for (int pl = tid; pl < LNN; pl += T) {
      const int r = rowbase + pl / N, c = pl % N;
      const float2* o = a.obj + (size_t)(ty + r) * a.W + (tx + c);
      const float2 O00 = __ldg(o), O01 = __ldg(o + 1), O10 = __ldg(o + a.W), O11 = __ldg(o + a.W + 1);
      const float2 dy = make_float2((1.f - fx) * (O10.x - O00.x) + fx * (O11.x - O01.x),
                                    (1.f - fx) * (O10.y - O00.y) + fx * (O11.y - O01.y));
      const float2 dx = make_float2((1.f - fy) * (O01.x - O00.x) + fy * (O11.x - O10.x),
                                    (1.f - fy) * (O01.y - O00.y) + fy * (O11.y - O10.y));
      const float2 g = g_s[r * N + c];
      gyv += g.x * dy.x + g.y * dy.y;
      gxv += g.x * dx.x + g.y * dx.y;
    }
    double v[2] = {(double)gyv, (double)gxv};
    block_sum<2>(v, red);
    if (tid == 0) {
      atomicAdd(a.gpos + 2 * j, (float)v[0]);
      atomicAdd(a.gpos + 2 * j + 1, (float)v[1]);
    }
  }
}

}  // namespace n256

}  // namespace ptycho
