// Per-position pass for windows larger than one CTA's shared memory, on a
// cluster of Q CTAs (N = 256: Q = 4; N = 192: Q = 3).
//
// The N x N complex tile is shared by the cluster: CTA q holds the 64 rows
// 64q .. 64q+63 (N = 64 Q). The 2-D DFT runs as
//   * N-point transforms of the CTA's own rows (shared memory, as in the
//     single-CTA kernel);
//   * the column transform split as N = Q x 64 (decimation in time over the
//     row index R = 64q + r): a Q-point DFT across the cluster for every
//     (r, c), reading the other CTAs' tiles through distributed shared memory,
//     times the twiddle W_N^(r k1), after which CTA k1 holds the inputs of
//     the outputs k = k1 + Q k2; then 64-point transforms of its local columns;
//   * the inverse mirrors it: local 64-point column inverses, the conjugate
//     twiddle and Q-point inverse DFT across the cluster, local row inverses.
// Everything else (patch gather, data term, back-propagation, scatter, the
// position gradient) follows the single-CTA k_pass1 on the CTA's own rows;
// the far fields of CTA q are the frequency rows q + Q k2.
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace ptycho {
namespace cl {

namespace cg = cooperative_groups;

// Swizzles of the local 64 x N tile (column bits XOR f(r, c), linear over
// GF(2)), chosen with the half-warp bank model for the row and column lines.
struct Swz256 {  // f = ((r << 2) ^ (r >> 1) ^ (c >> 4)) & 15
  __host__ __device__ static constexpr int fr(int r) { return ((r << 2) ^ (r >> 1)) & 15; }
  __host__ __device__ static constexpr int fcb(int c) { return (c >> 4) & 15; }
};
struct Swz128 {  // the single-CTA 128 window's swizzle: f = ((r << 3) ^ (r << 1) ^ (r >> 2) ^ (c >> 4)) & 15
  __host__ __device__ static constexpr int fr(int r) { return ((r << 3) ^ (r << 1) ^ (r >> 2)) & 15; }
  __host__ __device__ static constexpr int fcb(int c) { return (c >> 4) & 15; }
};
struct Swz192 {  // f = ((r << 3) ^ (r << 1) ^ (r >> 2) ^ (c >> 6)) & 15
  __host__ __device__ static constexpr int fr(int r) { return ((r << 3) ^ (r << 1) ^ (r >> 2)) & 15; }
  __host__ __device__ static constexpr int fcb(int c) { return (c >> 6) & 15; }
};

// Element i = i_rt + i_ct of a row or column line of the local 64 x N tile.
// For power-of-two N with disjoint bits in i_rt and i_ct the linear swizzle
// splits into a hoisted per-line part XOR a compile-time part; otherwise (N =
// 192, or the S = 3 exchange offsets) the column is formed first.
template <int N, class Z>
struct RectAddr {
  static constexpr bool POW2 = (N & (N - 1)) == 0;
  template <bool ROW>
  __device__ __forceinline__ static int addr(int line, int i_rt, int i_ct) {
    if constexpr (ROW && POW2) {
      const int base = line * N + (i_rt ^ Z::fr(line) ^ Z::fcb(i_rt));
      return base ^ (i_ct ^ Z::fcb(i_ct));
    } else if constexpr (ROW) {
      const int c = i_rt + i_ct;
      return line * N + (c ^ Z::fr(line) ^ Z::fcb(c));
    } else {
      const int base = i_rt * N + (line ^ Z::fcb(line) ^ Z::fr(i_rt));
      return (base + i_ct * N) ^ Z::fr(i_ct);
    }
  }
};

template <int N_, int Q_, int T_, int RR1_, int RR2_, bool RINTER_, bool CINTER_, class Z_, int MINB_ = 1>
struct Cfg {
  static constexpr int N = N_, Q = Q_, T = T_, LR = 64, NN = N * N, LNN = LR * N;
  static constexpr int MINB = MINB_;   // CTAs per SM the launch bounds ask for
  static constexpr int RR1 = RR1_, RR2 = RR2_;
  using Z = Z_;
  using RowF = LineFft<RR1, RR2, RINTER_, RectAddr<N, Z>>;   // N-point rows
  using ColF = LineFft<8, 8, CINTER_, RectAddr<N, Z>>;       // 64-point local columns
  static constexpr int ROW_ITER = LR * RR1 / T, COL_ITER = N * 8 / T;
  static constexpr int NAT_STEPS = LNN / (2 * T);              // natural pixel pairs per thread
  static constexpr int XB = N / 64, XPAIRS = 2048 / T;        // exchange column blocks, pairs per thread
  static_assert(ROW_ITER >= 1 && COL_ITER >= 1 && XPAIRS >= 1, "CTA size");
  __device__ __forceinline__ static int tix(int r, int c) { return r * N + (c ^ Z::fr(r) ^ Z::fcb(c)); }
  struct Smem {
    static constexpr int RP = N + 16;
    static constexpr size_t red = 0;
    static constexpr size_t tile = red + 256 * sizeof(double);
    static constexpr size_t twr = tile + (size_t)LNN * sizeof(float2);
    static constexpr size_t twc = twr + RR1 * (RR2 + 1) * sizeof(float2);
    static constexpr size_t twn = twc + 8 * 9 * sizeof(float2);
    static constexpr size_t twq = twn + N * sizeof(float2);
    static constexpr size_t rI = twq + 8 * sizeof(float2);
    static constexpr size_t bytes = rI + (size_t)LR * RP * sizeof(float);
  };
};

using Cfg256 = Cfg<256, 4, 1024, 16, 16, false, true, Swz256>;
// the 128 window on a pair of CTAs (64 rows each) that fit two to an SM
using Cfg128 = Cfg<128, 2, 512, 8, 16, true, true, Swz128, 2>;
using Cfg192 = Cfg<192, 3, 512, 8, 24, true, false, Swz192>;

// a * W_Q^m (W_Q = e^{-2 pi i / Q}) from the table twq[m mod Q].
template <int Q>
__device__ __forceinline__ float2 wqmul(float2 a, int m, const float2* twq) {
  if constexpr (Q == 4) {
    switch (m & 3) {
      case 0: return a;
      case 1: return make_float2(a.y, -a.x);
      case 2: return make_float2(-a.x, -a.y);
      default: return make_float2(-a.y, a.x);
    }
  } else {
    const int mm = ((m % Q) + Q) % Q;
    return mm == 0 ? a : cmul(a, twq[mm]);
  }
}

// Cross-cluster Q-point DFT of the tiles, in blocks of 64 columns, two blocks
// per cluster barrier when the block count is even (the barrier orders every
// CTA's reads of a block before its owner overwrites it; fewer, larger steps
// halve the barrier latency).
// Forward: tile_q <- W_N^(r q) sum_q' W_Q^(q' q) tile_q'.
// Inverse: tile_q <- sum_k1 W_Q^(-q k1) conj(W_N^(r k1)) tile_k1.
template <class C, bool FWD>
__device__ __forceinline__ void cross_exchange(cg::cluster_group& cluster, float2* tile, const float2* twn,
                                               const float2* twq, int q) {
  constexpr int Q = C::Q, P = C::XPAIRS, XB = C::XB, GB = (XB % 2 == 0 && C::MINB == 1) ? 2 : 1;
  float2* src[Q];
#pragma unroll
  for (int qq = 0; qq < Q; ++qq) src[qq] = cluster.map_shared_rank(tile, qq);
#pragma unroll 1
  for (int h0 = 0; h0 < XB; h0 += GB) {
    float2 acc[GB][P][2];
#pragma unroll
    for (int hh = 0; hh < GB; ++hh) {
      const int h = h0 + hh;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const int p = 2 * (int)threadIdx.x + 2 * C::T * j;   // within a 64 x 64 block: 4096 pixels
        const int rr = p / 64, cc = 64 * h + p % 64;
        acc[hh][j][0] = acc[hh][j][1] = make_float2(0.f, 0.f);
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) {
          float2 x0, x1;
          load_pair(src[qq], C::tix(rr, cc), x0, x1);
          if constexpr (FWD) {
            const int m = qq * q;
            acc[hh][j][0] = cadd(acc[hh][j][0], wqmul<Q>(x0, m, twq));
            acc[hh][j][1] = cadd(acc[hh][j][1], wqmul<Q>(x1, m, twq));
          } else {
            const float2 t = twn[rr * qq];     // W_N^(r k1), conjugated below
            const int m = -(q * qq);
            acc[hh][j][0] = cadd(acc[hh][j][0], wqmul<Q>(cmulc(t, x0), m, twq));
            acc[hh][j][1] = cadd(acc[hh][j][1], wqmul<Q>(cmulc(t, x1), m, twq));
          }
        }
      }
    }
    cluster.sync();   // every CTA has read these blocks of every tile
#pragma unroll
    for (int hh = 0; hh < GB; ++hh) {
      const int h = h0 + hh;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const int p = 2 * (int)threadIdx.x + 2 * C::T * j;
        const int rr = p / 64, cc = 64 * h + p % 64;
        if constexpr (FWD) {
          const float2 t = twn[rr * q];
          store_pair(tile, C::tix(rr, cc), cmul(acc[hh][j][0], t), cmul(acc[hh][j][1], t));
        } else {
          store_pair(tile, C::tix(rr, cc), acc[hh][j][0], acc[hh][j][1]);
        }
      }
    }
  }
  __syncthreads();
}

// 2-D forward DFT (unnormalised) of the cluster's tile; on return CTA q's tile
// holds the frequency rows q + Q k2 (local row k2), natural layout.
template <class C>
__device__ __forceinline__ void fwd2d(cg::cluster_group& cluster, float2* tile, const float2* twr,
                                      const float2* twc, const float2* twn, const float2* twq, int q) {
  using RowF = typename C::RowF;
  using ColF = typename C::ColF;
#pragma unroll 1
  for (int it = 0; it < C::ROW_ITER; ++it) {
    const int n = RowF::line_lane(), row = RowF::line_slot() + (C::T / C::RR1) * it;
    float2 v[C::RR2];
    RowF::template load_in<true>(v, tile, row, n);
    RowF::template line_fwd<true>(v, tile, row, n, twr);
    RowF::template store_out<true>(v, tile, row, n);
  }
  cluster.sync();
  cross_exchange<C, true>(cluster, tile, twn, twq, q);
#pragma unroll 1
  for (int it = 0; it < C::COL_ITER; ++it) {
    const int n = ColF::line_lane(), col = ColF::line_slot() + (C::T / 8) * it;
    float2 v[8];
    ColF::template load_in<false>(v, tile, col, n);
    ColF::template line_fwd<false>(v, tile, col, n, twc);
    ColF::template store_out<false>(v, tile, col, n);
  }
  __syncthreads();
}

// 2-D inverse DFT (unnormalised): tile_q holds frequency rows q + Q k2 on entry
// and the spatial rows 64q + r on return, natural layout.
template <class C>
__device__ __forceinline__ void inv2d(cg::cluster_group& cluster, float2* tile, const float2* twr,
                                      const float2* twc, const float2* twn, const float2* twq, int q) {
  using RowF = typename C::RowF;
  using ColF = typename C::ColF;
#pragma unroll 1
  for (int it = 0; it < C::COL_ITER; ++it) {
    const int n = ColF::line_lane(), col = ColF::line_slot() + (C::T / 8) * it;
    float2 v[8];
    ColF::template load_out<false>(v, tile, col, n);
    ColF::template line_inv<false>(v, tile, col, n, twc);
    ColF::template store_in<false>(v, tile, col, n);
  }
  __syncthreads();
  cluster.sync();
  cross_exchange<C, false>(cluster, tile, twn, twq, q);
#pragma unroll 1
  for (int it = 0; it < C::ROW_ITER; ++it) {
    const int n = RowF::line_lane(), row = RowF::line_slot() + (C::T / C::RR1) * it;
    float2 v[C::RR2];
    RowF::template load_out<true>(v, tile, row, n);
    RowF::template line_inv<true>(v, tile, row, n, twr);
    RowF::template store_in<true>(v, tile, row, n);
  }
  __syncthreads();
}

template <class C, bool OPR>
__global__ void __launch_bounds__(C::T, C::MINB) k_pass1_cluster(BatchArgs a) {
  constexpr int N = C::N, Q = C::Q, T = C::T, LR = C::LR, NN = C::NN, LNN = C::LNN;
  constexpr int NAT_STEPS = C::NAT_STEPS;
  using SM = typename C::Smem;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = (double*)(smem + SM::red);
  float2* tile = (float2*)(smem + SM::tile);
  float2* twr = (float2*)(smem + SM::twr);
  float2* twc = (float2*)(smem + SM::twc);
  float2* twn = (float2*)(smem + SM::twn);
  float2* twq = (float2*)(smem + SM::twq);
  float* rI = (float*)(smem + SM::rI);
  constexpr int RP = SM::RP;

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
  make_line_twiddles<N, C::RR1, C::RR2>(twr);
  make_line_twiddles<64, 8, 8>(twc);
  for (int m = tid; m < N + Q; m += T) {
    float s, c;
    if (m < N) {
      sincospif(2.0f * (float)m / (float)N, &s, &c);
      twn[m] = make_float2(c, -s);
    } else {
      sincospif(2.0f * (float)(m - N) / (float)Q, &s, &c);
      twq[m - N] = make_float2(c, -s);
    }
  }

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
  const int rowbase = LR * q;   // first spatial row of this CTA

  // ---- forward model --------------------------------------------------------------
#pragma unroll 1
  for (int k = 0; k < M; ++k) {
    const float2* Pk = shared_mode<OPR>(a, k, NN);
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
      float4 P2;
      if (!OPR || Pk) {
        P2 = __ldg((const float4*)(Pk + p));
      } else {   // relaxed primary mode of this position
        P2 = opr_pair(a.opr_U, wj, a.K, NN, p);
        if (p0) *(float4*)(p0 + p) = P2;
      }
      store_pair(tile, C::tix(r, c), cmul(make_float2(P2.x, P2.y), o0), cmul(make_float2(P2.z, P2.w), o1));
    }
    __syncthreads();
    fwd2d<C>(cluster, tile, twr, twc, twn, twq, q);
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;   // r = local frequency row k2
      float2 X0, X1;
      load_pair(tile, C::tix(r, c), X0, X1);
      X0 = cscale(X0, invN);
      X1 = cscale(X1, invN);
      float2* ri = (float2*)(rI + r * RP + c);
      const float2 i2 = make_float2(cabs2(X0), cabs2(X1));
      *ri = (k == 0) ? i2 : make_float2(ri->x + i2.x, ri->y + i2.y);
      if (psi_s)
        *(float4*)(psi_s + (size_t)k * NN + (q + Q * r) * N + c) = make_float4(X0.x, X0.y, X1.x, X1.y);
    }
  }

  // ---- data term (frequency rows q + Q k2) ----------------------------------------
  const int mode = a.mode;
  const float eps = a.eps;
  const float* meas = a.meas + (size_t)j * NN;
  float lsum = 0.f;
  bool bad = false;
#pragma unroll 1
  for (int s = 0; s < NAT_STEPS; ++s) {
    const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
    const int pix = (q + Q * r) * N + c;
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
  if (mode == MODE_FWD || a.loss_only) {
    cluster.sync();   // no CTA leaves while another may still read its tile
    return;
  }

  // ---- back-propagation -------------------------------------------------------------
  // modes last to first: the far fields written last are read first (L2)
  float2* g_s = a.g_s + slotNN;
  float2* h_s = a.h_s + slotNN * M;
#pragma unroll 1
  for (int k = M - 1; k >= 0; --k) {
    const float2* Pk = shared_mode<OPR>(a, k, NN);
    __syncthreads();
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
      const float4 X = *(const float4*)(psi_s + (size_t)k * NN + (q + Q * r) * N + c);
      const float2 f = *(const float2*)(rI + r * RP + c);
      store_pair(tile, C::tix(r, c), make_float2(X.x * f.x, X.y * f.x), make_float2(X.z * f.y, X.w * f.y));
    }
    __syncthreads();
    inv2d<C>(cluster, tile, twr, twc, twn, twq, q);
#pragma unroll 2
    for (int s = 0; s < NAT_STEPS; ++s) {
      const int pl = 2 * tid + 2 * T * s, r = pl / N, c = pl % N;
      const int p = (rowbase + r) * N + c;
      float2 x0, x1;
      load_pair(tile, C::tix(r, c), x0, x1);
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
      const float sp = lsqml ? __ldg(a.Sp + y * N + x) + ((OPR && p0) ? cabs2(p0[y * N + x]) : 0.f) : 0.f;
      return make_float4(g.x, g.y, sp, 0.f);
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
    constexpr int SEG = T / N1 > 0 ? T / N1 : 1;      // row segments of the CTA's rows
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

  // ---- position gradient (gradient modes) or the least-squares position-step
  // ---- sums (LSQML position correction), this CTA's rows ----------------------------
  if (a.gpos || a.possum) {
    const bool ls = a.possum != nullptr;
    float gyv = 0.f, gxv = 0.f, a11 = 0.f, a12 = 0.f, a22 = 0.f;
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
      if (ls) {
        const int p = r * N + c;
        const float sp = __ldg(a.Sp + p) + ((OPR && p0) ? cabs2(p0[p]) : 0.f);
        a11 = fmaf(sp, cabs2(dy), a11);
        a12 = fmaf(sp, dy.x * dx.x + dy.y * dx.y, a12);
        a22 = fmaf(sp, cabs2(dx), a22);
      }
    }
    if (ls) {
      double v[5] = {(double)a11, (double)a12, (double)a22, (double)gyv, (double)gxv};
      block_sum<5>(v, red);
      if (tid == 0)
        for (int q = 0; q < 5; ++q) atomicAdd(a.possum + (size_t)slot * 5 + q, v[q]);
    } else {
      double v[2] = {(double)gyv, (double)gxv};
      block_sum<2>(v, red);
      if (tid == 0) {
        atomicAdd(a.gpos + 2 * j, (float)v[0]);
        atomicAdd(a.gpos + 2 * j + 1, (float)v[1]);
      }
    }
  }
}

}  // namespace cl

}  // namespace ptycho
