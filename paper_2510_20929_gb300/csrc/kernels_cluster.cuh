// Per-position pass for windows larger than one CTA's shared memory, on a
// cluster of Q CTAs (N = 256: Q = 8; N = 192: Q = 6; and a pair of CTAs for
// the 128 window).
//
// The N x N complex tile is shared by the cluster: in the spatial domain CTA q
// holds the LR = N / Q rows LR q .. LR q + LR - 1. The 2-D DFT runs as
//   * N-point transforms of the CTA's own rows (shared memory, as in the
//     single-CTA kernel);
//   * a transpose across the cluster: CTA q gathers, from every CTA s, the
//     LR x LR block of s's rows at columns LR q .. LR q + LR - 1 (distributed
//     shared memory), and stores it transposed, so that its local row x now
//     holds column LR q + x of the whole tile (all N rows);
//   * N-point transforms of those local rows, which are the columns.
// CTA q then holds the far-field columns LR q .. (local row x = column LR q +
// x, local column = frequency row). The inverse mirrors it (row inverses, the
// same transpose back, row inverses). Each CTA reads (Q-1)/Q of its tile from
// the other CTAs once per transform (a Q-point DFT across the cluster would
// read every element from every CTA: Q times that).
// Everything else (patch gather, back-propagation, scatter, the position
// gradient) follows the single-CTA k_pass1 on the CTA's own spatial rows; the
// far-field loops (intensity, data term, the inverse's input) walk the CTA's
// columns with consecutive threads on consecutive columns (freq_index), so
// that the measured intensities and the predicted ones are read and written
// coalesced in their natural [k_y][k_x] order.
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace ptycho {
namespace cl {

namespace cg = cooperative_groups;

// Swizzles of the local LR x N tile (column bits XOR f(r, c), linear over
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

// Element i = i_rt + i_ct of a row or column line of the local LR x N tile.
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

// Q CTAs of T threads per position, LR = N / Q rows (and, after a forward
// transform, LR far-field columns) each; MINB CTAs per SM for the launch bounds.
template <int N_, int Q_, int T_, int RR1_, int RR2_, bool RINTER_, class Z_, int MINB_ = 1>
struct Cfg {
  static constexpr int N = N_, Q = Q_, T = T_, LR = N_ / Q_, NN = N * N, LNN = LR * N;
  static_assert(LR * Q == N && (LR == 32 || LR == 64), "rows per CTA");
  static constexpr int MINB = MINB_;   // CTAs per SM the launch bounds ask for
  static constexpr int RR1 = RR1_, RR2 = RR2_;
  using Z = Z_;
  using RowF = LineFft<RR1, RR2, RINTER_, RectAddr<N, Z>>;   // N-point rows
  static constexpr int ROW_ITER = LR * RR1 / T;
  static constexpr int NAT_STEPS = LNN / (2 * T);              // natural pixel pairs per thread
  static_assert(ROW_ITER >= 1 && (LR * LR / 2) % T == 0 && LNN % T == 0, "CTA size");
  __device__ __forceinline__ static int tix(int r, int c) { return r * N + (c ^ Z::fr(r) ^ Z::fcb(c)); }
  // far-field element e (0 .. LNN-1) of CTA q: local row x = e % LR (column
  // LR q + x of the far field), local column ky = e / LR (its row)
  __device__ __forceinline__ static void freq_index(int e, int& x, int& ky) {
    x = e & (LR - 1);
    ky = e / LR;
  }
  // transpose: pixel pairs of one LR x LR block per thread, rounds per cluster
  // barrier (at most 16 values held per thread, a divisor of Q)
  static constexpr int XP = LR * LR / 2 / T;
  static constexpr int XG = (4 / (XP > 0 ? XP : 1) >= 4 && Q % 4 == 0) ? 4
                          : (4 / (XP > 0 ? XP : 1) >= 2 && Q % 2 == 0) ? 2 : 1;
  struct Smem {
    static constexpr int RP = N + 1;   // intensity plane [LR][RP]: the column walk is conflict-free
    static constexpr size_t red = 0;
    static constexpr size_t tile = red + 256 * sizeof(double);
    static constexpr size_t twr = tile + (size_t)LNN * sizeof(float2);
    static constexpr size_t rI = twr + RR1 * (RR2 + 1) * sizeof(float2);
    static constexpr size_t bytes = rI + (size_t)LR * RP * sizeof(float);
  };
};

// 32 rows per CTA, two CTAs per SM (103 KB and 78 KB of shared memory): one
// cluster's CTA computes while another's waits on the exchange (against 64
// rows and one CTA per SM: the spiral256 pass 2.99 -> 2.48 ms per 256
// positions, multislice256 29.5K -> 32.6K patterns/s)
using Cfg256 = Cfg<256, 8, 512, 16, 16, false, Swz256, 2>;
// the 128 window on a pair of CTAs (64 rows each) that fit two to an SM
using Cfg128 = Cfg<128, 2, 512, 8, 16, true, Swz128, 2>;
using Cfg192 = Cfg<192, 6, 256, 8, 24, true, Swz192, 2>;

// The transpose across the cluster: tile[x][LR s + r] <- tile_s[r][LR q + x]
// for every CTA s of the cluster and r, x in 0..LR-1. It runs in Q rounds; in
// round t CTA q trades blocks with CTA s = (t - q) mod Q (a symmetric pairing:
// the two read each other's block and then overwrite the block the other
// has read; s = q transposes its own diagonal block). Block s of CTA q's tile
// is read only by CTA s and overwritten only in the round that pairs the two,
// after the barrier, so XG rounds can share one cluster barrier: their reads
// go to registers first (XG x LR^2 / T pixels per thread), then the barrier,
// then the transposed stores. Ends synchronised.
template <class C>
__device__ __forceinline__ void transpose_exchange(cg::cluster_group& cluster, float2* tile, int q) {
  constexpr int Q = C::Q, T = C::T, G = C::XG, P = C::XP, LR = C::LR, HP = LR / 2;
  static_assert(Q % G == 0 && P >= 1, "rounds and pairs per thread");
#pragma unroll 1
  for (int t0 = 0; t0 < Q; t0 += G) {
    float2 v[G][P][2];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int s = (t0 + g - q + Q) % Q;
      const float2* src = cluster.map_shared_rank(tile, s);
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int p = (int)threadIdx.x + T * i;   // (r, pair of x): LR x LR/2 pairs
        const int r = p / HP, x = 2 * (p % HP);
        load_pair(src, C::tix(r, LR * q + x), v[g][i][0], v[g][i][1]);
      }
    }
    cluster.sync();   // the blocks of these rounds are read in every CTA
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int s = (t0 + g - q + Q) % Q;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int p = (int)threadIdx.x + T * i;
        const int r = p / HP, x = 2 * (p % HP);
        tile[C::tix(x, LR * s + r)] = v[g][i][0];
        tile[C::tix(x + 1, LR * s + r)] = v[g][i][1];
      }
    }
  }
  __syncthreads();
}

// N-point transforms (forward: natural in, natural out) of the CTA's LR local
// rows, in place.
template <class C, bool FWD>
__device__ __forceinline__ void row_pass(float2* tile, const float2* twr) {
  using RowF = typename C::RowF;
#pragma unroll 1
  for (int it = 0; it < C::ROW_ITER; ++it) {
    const int n = RowF::line_lane(), row = RowF::line_slot() + (C::T / C::RR1) * it;
    float2 v[C::RR2];
    if constexpr (FWD) {
      RowF::template load_in<true>(v, tile, row, n);
      RowF::template line_fwd<true>(v, tile, row, n, twr);
      RowF::template store_out<true>(v, tile, row, n);
    } else {
      RowF::template load_out<true>(v, tile, row, n);
      RowF::template line_inv<true>(v, tile, row, n, twr);
      RowF::template store_in<true>(v, tile, row, n);
    }
  }
}

// 2-D forward DFT (unnormalised) of the cluster's tile: CTA q holds the
// spatial rows LR q .. on entry and the far-field columns LR q .. on return
// (local row x = column LR q + x, natural order along it). Ends synchronised.
template <class C>
__device__ __forceinline__ void fwd2d(cg::cluster_group& cluster, float2* tile, const float2* twr, int q) {
  row_pass<C, true>(tile, twr);
  cluster.sync();   // every CTA's rows are transformed before any CTA reads them
  transpose_exchange<C>(cluster, tile, q);
  row_pass<C, true>(tile, twr);
  __syncthreads();
}

// 2-D inverse DFT (unnormalised): the far-field columns LR q .. on entry, the
// spatial rows LR q .. on return. Ends synchronised.
template <class C>
__device__ __forceinline__ void inv2d(cg::cluster_group& cluster, float2* tile, const float2* twr, int q) {
  row_pass<C, false>(tile, twr);
  cluster.sync();
  transpose_exchange<C>(cluster, tile, q);
  row_pass<C, false>(tile, twr);
  __syncthreads();
}

template <class C, bool OPR>
__global__ void __launch_bounds__(C::T, C::MINB) k_pass1_cluster(BatchArgs a) {
  constexpr int N = C::N, Q = C::Q, T = C::T, LR = C::LR, NN = C::NN, LNN = C::LNN;
  constexpr int NAT_STEPS = C::NAT_STEPS;
  static_assert(LNN % (2 * T) == 0, "data-term loop takes two elements per step");
  using SM = typename C::Smem;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = (double*)(smem + SM::red);
  float2* tile = (float2*)(smem + SM::tile);
  float2* twr = (float2*)(smem + SM::twr);
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
  if (!ok) {   // the same decision in every CTA of the cluster
    if (tid == 0 && q == 0) {
      atomicOr(a.status, FLAG_BOUNDS);
      if (a.valid) a.valid[slot] = 0;
    }
    return;
  }
  if (tid == 0 && q == 0 && a.valid) a.valid[slot] = 1;
  make_line_twiddles<N, C::RR1, C::RR2>(twr);

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
    fwd2d<C>(cluster, tile, twr, q);
    // far field of this CTA's columns: the intensity sum and (gradient and
    // LSQML modes) the far field itself, in a CTA-private scratch order
#pragma unroll 4
    for (int e = tid; e < LNN; e += T) {
      int x, ky;
      C::freq_index(e, x, ky);
      const float2 X = cscale(tile[C::tix(x, ky)], invN);
      float* ri = rI + x * RP + ky;
      *ri = (k == 0) ? cabs2(X) : *ri + cabs2(X);
      if (psi_s) psi_s[(size_t)k * NN + (size_t)q * LNN + e] = X;
    }
  }

  // ---- data term (this CTA's far-field columns) ------------------------------------
  const int mode = a.mode;
  const float eps = a.eps;
  const float* meas = a.meas + (size_t)j * NN;
  float lsum = 0.f;
  bool bad = false;
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
      if (mode == MODE_FWD) continue;
      const float Im = __ldg(meas + pix);
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
      *ri = fac * invN;
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
#pragma unroll 4
    for (int e = tid; e < LNN; e += T) {
      int x, ky;
      C::freq_index(e, x, ky);
      tile[C::tix(x, ky)] = cscale(psi_s[(size_t)k * NN + (size_t)q * LNN + e], rI[x * RP + ky]);
    }
    __syncthreads();
    inv2d<C>(cluster, tile, twr, q);
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
      if (k == 0)   // the finished g of this CTA's rows also into its (now free) tile
        store_pair(tile, C::tix(r, c), make_float2(gv.x, gv.y), make_float2(gv.z, gv.w));
      const float2 h0 = cmulc(make_float2(o2.x, o2.y), x0), h1 = cmulc(make_float2(o2.z, o2.w), x1);
      __stcs((float4*)(h_s + (size_t)k * NN + p), make_float4(h0.x, h0.y, h1.x, h1.y));
    }
  }
  const bool lsqml = (mode == MODE_LSQML_GAUSS || mode == MODE_LSQML_POISSON);
  // LSQML: the probe intensity of this CTA's rows into the free intensity/factor
  // plane, so that the scatter reads its own rows from shared memory
  float* spS = rI;
  if (lsqml) {
    static_assert(LR * RP >= LNN, "room for the probe intensity");
    for (int e = 4 * tid; e < LNN; e += 4 * T) {
      const int p = rowbase * N + e;
      float4 v = __ldg((const float4*)(a.Sp + p));
      if (OPR && p0) {
        const float4 q0 = *(const float4*)(p0 + p), q1 = *(const float4*)(p0 + p + 2);
        v.x += q0.x * q0.x + q0.y * q0.y; v.y += q0.z * q0.z + q0.w * q0.w;
        v.z += q1.x * q1.x + q1.y * q1.y; v.w += q1.z * q1.z + q1.w * q1.w;
      }
      *(float4*)(spS + e) = v;
    }
  }
  // every CTA's rows of g are written (the scatter reads one row of the neighbour)
  cluster.sync();

  // ---- scatter S_j^T g (and the illumination), this CTA's rows (+ row N) ----------
  {
    const int y0 = rowbase, y1 = rowbase + LR + (q == Q - 1 ? 1 : 0);
    constexpr int N1 = N + 1;
    const float gx = 1.f - fx, gy = 1.f - fy;
    auto loadg = [&](int y, int x) {
      if (y >= y0 && y < y0 + LR) {   // this CTA's rows: shared memory
        const float2 g = tile[C::tix(y - y0, x)];
        return make_float4(g.x, g.y, lsqml ? spS[(y - y0) * N + x] : 0.f, 0.f);
      }
      const float2 g = g_s[y * N + x];   // the row above, from the neighbour's rows in L2
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
