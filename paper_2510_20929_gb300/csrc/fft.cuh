// Shared-memory 2-D FFT for one N x N complex64 tile per CTA (sm_103a).
//
// The far-field propagator of the ptychographic forward model (Pty-Chi,
// Sec. 2.1; Eq. 4's F(o, p, Lambda)) is a unitary 2-D DFT of each exit wave.
// This header implements it as two passes of 1-D transforms over the rows and
// columns of a tile held in shared memory:
//
//   * a line (row or column) of N = R1 * R2 points is owned by R1 consecutive
//     lanes of one warp; lane n holds R2 points x[n + R1*n2] in registers;
//   * stage 1 is an R2-point DFT in registers, followed by the twiddles
//     W_N^(n*k2); the lanes then exchange through the line's own storage in
//     the tile (warp-synchronous, no block barrier) and stage 2 runs R1-point
//     DFTs, leaving lane n with X[S*(n + R1*k1) + s], S = R2/R1;
//   * the inverse runs the same stages mirrored (decimation in frequency), so
//     it consumes the forward's output layout and returns the forward's input
//     layout.
//
// The tile is stored row-major with an XOR swizzle of the low four column
// bits, chosen (by an offline bank-conflict model of every access family
// used here) so that the strided row, column and exchange accesses of a warp
// hit distinct 8-byte bank slots. The swizzle is linear over GF(2), so every
// address splits into a per-thread part (hoisted out of the unrolled loops)
// XOR a compile-time part.
//
// All transforms here are unnormalised; callers apply the 1/N of the unitary
// 2-D transform where it folds into other arithmetic.
#pragma once
#include <cuda_runtime.h>

namespace ptycho {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// a * exp(DIR * i * pi / 2): DIR = -1 multiplies by -i (forward), +1 by +i.
template <int DIR>
__device__ __forceinline__ float2 rot90(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// cos(m*pi/8), sin(m*pi/8) for m = 0..4 (the only irrational twiddles of the
// 8- and 16-point kernels below).
#define PT_C1 0.92387953251128674f  // cos(pi/8)
#define PT_S1 0.38268343236508978f  // sin(pi/8)
#define PT_C2 0.70710678118654752f  // cos(pi/4)

// a * exp(DIR * i * m * pi / 8), m compile-time in [0, 16).
template <int DIR, int m>
__device__ __forceinline__ float2 tw16(float2 a) {
  constexpr int mm = m & 15;
  if constexpr (mm == 0) return a;
  else if constexpr (mm == 4) return rot90<DIR>(a);
  else if constexpr (mm == 8) return make_float2(-a.x, -a.y);
  else if constexpr (mm == 12) return rot90<-DIR>(a);
  else {
    // cos and sin of mm*pi/8 from the first-octant constants
    constexpr float cs[16] = {1.f, PT_C1, PT_C2, PT_S1, 0.f, -PT_S1, -PT_C2, -PT_C1,
                              -1.f, -PT_C1, -PT_C2, -PT_S1, 0.f, PT_S1, PT_C2, PT_C1};
    constexpr float sn[16] = {0.f, PT_S1, PT_C2, PT_C1, 1.f, PT_C1, PT_C2, PT_S1,
                              0.f, -PT_S1, -PT_C2, -PT_C1, -1.f, -PT_C1, -PT_C2, -PT_S1};
    const float c = cs[mm], s = DIR < 0 ? -sn[mm] : sn[mm];
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// In-register DFTs of size R (natural order in and out), sign DIR.
template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<1, DIR> {
  template <class V> __device__ __forceinline__ static void run(V&) {}
};

template <int DIR> struct Dft<2, DIR> {
  template <class V> __device__ __forceinline__ static void run(V& v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR> struct Dft<4, DIR> {
  template <class V> __device__ __forceinline__ static void run(V& v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = rot90<DIR>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <int DIR> struct Dft<8, DIR> {
  template <class V> __device__ __forceinline__ static void run(V& v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, DIR>::run(e);
    Dft<4, DIR>::run(o);
    o[1] = tw16<DIR, 2>(o[1]);
    o[2] = tw16<DIR, 4>(o[2]);
    o[3] = tw16<DIR, 6>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <int DIR> struct Dft<16, DIR> {
  // n = b + 4a, k = k1 + 4k2: X[k] = sum_b W16^(b k1) W4^(b k2) sum_a W4^(a k1) v[b + 4a]
  template <class V> __device__ __forceinline__ static void run(V& v) {
    float2 y[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float2 t[4] = {v[b], v[b + 4], v[b + 8], v[b + 12]};
      Dft<4, DIR>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) y[b][k1] = t[k1];
    }
    y[1][1] = tw16<DIR, 1>(y[1][1]);
    y[1][2] = tw16<DIR, 2>(y[1][2]);
    y[1][3] = tw16<DIR, 3>(y[1][3]);
    y[2][1] = tw16<DIR, 2>(y[2][1]);
    y[2][2] = tw16<DIR, 4>(y[2][2]);
    y[2][3] = tw16<DIR, 6>(y[2][3]);
    y[3][1] = tw16<DIR, 3>(y[3][1]);
    y[3][2] = tw16<DIR, 6>(y[3][2]);
    y[3][3] = tw16<DIR, 9>(y[3][3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4, DIR>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
  }
};

// a * exp(DIR * i * m * pi / 12), m compile-time (the 24-point twiddles).
template <int DIR, int m>
__device__ __forceinline__ float2 tw24(float2 a) {
  constexpr int mm = m % 24;
  if constexpr (mm == 0) return a;
  else if constexpr (mm == 6) return rot90<DIR>(a);
  else if constexpr (mm == 12) return make_float2(-a.x, -a.y);
  else if constexpr (mm == 18) return rot90<-DIR>(a);
  else {
    // cos and sin of multiples of 15 degrees
    constexpr float c15 = 0.96592582628906829f, s15 = 0.25881904510252076f;
    constexpr float c30 = 0.86602540378443865f, c45 = 0.70710678118654752f;
    constexpr float cs[24] = {1.f,  c15,  c30,  c45,  0.5f,  s15,  0.f, -s15, -0.5f, -c45, -c30, -c15,
                              -1.f, -c15, -c30, -c45, -0.5f, -s15, 0.f, s15,  0.5f,  c45,  c30,  c15};
    constexpr float sn[24] = {0.f,  s15,  0.5f,  c45,  c30,  c15,  1.f,  c15,  c30,  c45,  0.5f,  s15,
                              0.f, -s15, -0.5f, -c45, -c30, -c15, -1.f, -c15, -c30, -c45, -0.5f, -s15};
    const float c = cs[mm], s = DIR < 0 ? -sn[mm] : sn[mm];
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

template <int DIR> struct Dft<3, DIR> {
  // X0 = v0 + (v1 + v2); X1,2 = v0 - (v1 + v2)/2 +- i DIR sin(2 pi / 3) (v1 - v2)
  template <class V> __device__ __forceinline__ static void run(V& v) {
    constexpr float s3 = 0.86602540378443865f;
    const float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const float2 m = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
    const float2 r = make_float2(-DIR * s3 * t2.y, DIR * s3 * t2.x);   // i DIR s3 t2
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <int DIR> struct Dft<24, DIR> {
  // n = b + 3a, k = k1 + 8k2: X[k] = sum_b W3^(b k2) W24^(b k1) sum_a W8^(a k1) v[b + 3a]
  template <class V> __device__ __forceinline__ static void run(V& v) {
    float2 y[3][8];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 t[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) t[a] = v[b + 3 * a];
      Dft<8, DIR>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) y[b][k1] = t[k1];
    }
    y[1][1] = tw24<DIR, 1>(y[1][1]); y[1][2] = tw24<DIR, 2>(y[1][2]); y[1][3] = tw24<DIR, 3>(y[1][3]);
    y[1][4] = tw24<DIR, 4>(y[1][4]); y[1][5] = tw24<DIR, 5>(y[1][5]); y[1][6] = tw24<DIR, 6>(y[1][6]);
    y[1][7] = tw24<DIR, 7>(y[1][7]);
    y[2][1] = tw24<DIR, 2>(y[2][1]); y[2][2] = tw24<DIR, 4>(y[2][2]); y[2][3] = tw24<DIR, 6>(y[2][3]);
    y[2][4] = tw24<DIR, 8>(y[2][4]); y[2][5] = tw24<DIR, 10>(y[2][5]); y[2][6] = tw24<DIR, 12>(y[2][6]);
    y[2][7] = tw24<DIR, 14>(y[2][7]);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      float2 t[3] = {y[0][k1], y[1][k1], y[2][k1]};
      Dft<3, DIR>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) v[k1 + 8 * k2] = t[k2];
    }
  }
};

// Per-size line split and tile swizzle. The swizzle XORs the low four column
// bits with f(r, c) = fr(r) ^ fc(c >> 4), shift-XOR maps that are linear over
// GF(2). The maps and the lane assignment (INTER: the R1 lanes of a line are
// interleaved across the warp rather than consecutive) come from a search over
// a bank model in which 8-byte accesses are served per half-warp and 16-byte
// accesses per quarter-warp; with them every shared access family used here
// needs the minimum 2 (8-byte) or 4 (16-byte) wavefronts per warp instruction.
template <int N> struct FftCfg;
template <> struct FftCfg<16> {
  static constexpr int R1 = 4, R2 = 4;
  static constexpr bool INTER = false;
  __host__ __device__ static constexpr int fr(int r) { return ((r << 2) ^ r) & 15; }
  __host__ __device__ static constexpr int fc(int) { return 0; }
};
template <> struct FftCfg<32> {
  static constexpr int R1 = 4, R2 = 8;
  static constexpr bool INTER = true;
  __host__ __device__ static constexpr int fr(int r) { return ((r << 3) ^ (r << 2) ^ r) & 15; }
  __host__ __device__ static constexpr int fc(int) { return 0; }
};
template <> struct FftCfg<64> {
  static constexpr int R1 = 8, R2 = 8;
  static constexpr bool INTER = true;
  __host__ __device__ static constexpr int fr(int r) { return ((r << 2) ^ (r >> 1)) & 15; }
  __host__ __device__ static constexpr int fc(int cb) { return (cb << 1) & 15; }
};
template <> struct FftCfg<128> {
  static constexpr int R1 = 8, R2 = 16;
  static constexpr bool INTER = true;
  __host__ __device__ static constexpr int fr(int r) { return ((r << 3) ^ (r << 1) ^ (r >> 2)) & 15; }
  __host__ __device__ static constexpr int fc(int cb) { return cb & 15; }
};

// Physical float2 index of tile element (r, c) for runtime r, c.
template <int N>
__device__ __forceinline__ int tix(int r, int c) {
  return r * N + (c ^ FftCfg<N>::fr(r) ^ FftCfg<N>::fc(c >> 4));
}

// Natural-layout traversal of the tile by pixel pairs: thread t handles the
// pairs (r, c), (r, c+1) with p = 2t + 2T q, c even. The swizzle moves a pair as
// a unit (it only flips the low column bits), possibly swapping its halves, so
// every pair is one 16-byte shared-memory access.
template <int N, int T>
struct NatPairs {
  using C = FftCfg<N>;
  static constexpr int RS = 2 * T / N;           // rows advanced per step (power of two)
  static constexpr int STEPS = N * N / (2 * T);
  static_assert(RS >= 1, "needs 2T >= N");
  int r0, c, xr;
  __device__ __forceinline__ NatPairs() {
    const int p = 2 * (int)threadIdx.x;
    r0 = p / N;
    c = p % N;
    xr = c ^ C::fr(r0) ^ C::fc(c >> 4);
  }
  __device__ __forceinline__ int row(int q) const { return r0 + RS * q; }
  __device__ __forceinline__ int pix(int q) const { return row(q) * N + c; }
  // physical index of pixel (row(q), c); pixel c+1 sits at phys ^ 1
  __device__ __forceinline__ int phys(int q) const { return row(q) * N + (xr ^ C::fr(RS * q)); }
};

__device__ __forceinline__ void store_pair(float2* tile, int ph, float2 a, float2 b) {
  float4* p = (float4*)(tile + (ph & ~1));
  *p = (ph & 1) ? make_float4(b.x, b.y, a.x, a.y) : make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void load_pair(const float2* tile, int ph, float2& a, float2& b) {
  const float4 v = *(const float4*)(tile + (ph & ~1));
  if (ph & 1) {
    a = make_float2(v.z, v.w);
    b = make_float2(v.x, v.y);
  } else {
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  }
}

// Addressing of a square N x N tile with the FftCfg<N> swizzle: element i
// (= i_rt | i_ct, disjoint bits, i_ct compile-time) of a row or column line.
template <int N>
struct SquareAddr {
  using C = FftCfg<N>;
  template <bool ROW>
  __device__ __forceinline__ static int addr(int line, int i_rt, int i_ct) {
    if constexpr (ROW) {
      // (r = line, c = i): c ^ fr(r) ^ fc(c >> 4), split over the disjoint parts of c
      const int base = line * N + (i_rt ^ C::fr(line) ^ C::fc(i_rt >> 4));
      return base ^ (i_ct ^ C::fc(i_ct >> 4));
    } else {
      // (r = i, c = line): r*N + (c ^ fr(r) ^ fc(c >> 4)), split over the parts of r
      const int base = i_rt * N + (line ^ C::fc(line >> 4) ^ C::fr(i_rt));
      return (base + i_ct * N) ^ C::fr(i_ct);
    }
  }
};

// Line transforms of length R1*R2 on lines of a shared tile addressed by Addr.
template <int R1_, int R2_, bool INTER_, class Addr>
struct LineFft {
  static constexpr int R1 = R1_, R2 = R2_, S = R2 / R1, G = 32 / R1;
  static constexpr bool INTER = INTER_;

  // Lane n (0..R1-1) within its line and the thread's line slot: the G lines
  // of a warp are consecutive; the R1 lanes of a line are G lanes apart
  // (INTER) or consecutive.
  __device__ __forceinline__ static int line_lane() {
    return INTER ? (int)(threadIdx.x & 31) / G : (int)threadIdx.x % R1;
  }
  __device__ __forceinline__ static int line_slot() {
    return INTER ? (int)(threadIdx.x >> 5) * G + (int)(threadIdx.x & 31) % G : (int)threadIdx.x / R1;
  }

  template <bool ROW>
  __device__ __forceinline__ static int addr(int line, int i_rt, int i_ct) {
    return Addr::template addr<ROW>(line, i_rt, i_ct);
  }

  // Twiddles W_N^(n k2), k2 = 1..R2-1, for lane n: W^1..W^4 from the table,
  // the rest as W^(4a) W^b (W^8 = W^4 W^4, W^12 = W^8 W^4): at most three
  // roundings per twiddle and four shared loads instead of R2-1.
  __device__ __forceinline__ static void twiddles(float2 (&t)[R2], const float2* tw, int n) {
    t[0] = make_float2(1.f, 0.f);
    constexpr int L4 = R2 - 1 < 4 ? R2 - 1 : 4;
#pragma unroll
    for (int k = 1; k <= L4; ++k) t[k] = tw[n * (R2 + 1) + k];
#pragma unroll
    for (int k = 5; k < R2; ++k) {
      const int a = k & ~3, b = k & 3;
      if (b == 0) t[k] = cmul(t[a - 4], t[4]);
      else t[k] = cmul(t[a], t[b]);
    }
  }

  // Forward line transform (sign -1). In: v[n2] = x[n + R1*n2].
  // Out: v[k1*S + s] = X[S*(n + R1*k1) + s]. The line's storage is used for the exchange.
  template <bool ROW>
  __device__ __forceinline__ static void line_fwd(float2 (&v)[R2], float2* tile, int line, int n,
                                                  const float2* tw) {
    Dft<R2, -1>::run(v);
    {
      float2 t[R2];
      twiddles(t, tw, n);
#pragma unroll
      for (int k2 = 1; k2 < R2; ++k2) v[k2] = cmul(v[k2], t[k2]);
    }
    // exchange: lane n writes Y[n][k2]; lane t reads Y[n1][S*t + s]
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) tile[addr<ROW>(line, n, R1 * k2)] = v[k2];
    __syncwarp();
    float2 w[S][R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1)
#pragma unroll
      for (int s = 0; s < S; ++s) w[s][n1] = tile[addr<ROW>(line, R1 * S * n, n1 + R1 * s)];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < S; ++s) Dft<R1, -1>::run(w[s]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
      for (int s = 0; s < S; ++s) v[k1 * S + s] = w[s][k1];
  }

  // Inverse line transform (sign +1, unnormalised: returns N * x).
  // In: v[k1*S + s] = X[S*(n + R1*k1) + s]. Out: v[n2] = x[n + R1*n2].
  template <bool ROW>
  __device__ __forceinline__ static void line_inv(float2 (&v)[R2], float2* tile, int line, int n,
                                                  const float2* tw) {
    float2 w[S][R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
      for (int s = 0; s < S; ++s) w[s][k1] = v[k1 * S + s];
#pragma unroll
    for (int s = 0; s < S; ++s) Dft<R1, 1>::run(w[s]);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1)
#pragma unroll
      for (int s = 0; s < S; ++s) tile[addr<ROW>(line, R1 * S * n, n1 + R1 * s)] = w[s][n1];
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k2] = tile[addr<ROW>(line, n, R1 * k2)];
    __syncwarp();
    {
      float2 t[R2];
      twiddles(t, tw, n);
#pragma unroll
      for (int k2 = 1; k2 < R2; ++k2) v[k2] = cmulc(t[k2], v[k2]);
    }
    Dft<R2, 1>::run(v);
  }

  // Load / store a line in the "in" layout (x[n + R1*n2]) or the "out" layout
  // (X[S*(n + R1*k1) + s] in register k1*S + s).
  template <bool ROW>
  __device__ __forceinline__ static void load_in(float2 (&v)[R2], const float2* tile, int line, int n) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = tile[addr<ROW>(line, n, R1 * n2)];
  }
  template <bool ROW>
  __device__ __forceinline__ static void store_in(const float2 (&v)[R2], float2* tile, int line, int n) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) tile[addr<ROW>(line, n, R1 * n2)] = v[n2];
  }
  template <bool ROW>
  __device__ __forceinline__ static void load_out(float2 (&v)[R2], const float2* tile, int line, int n) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
      for (int s = 0; s < S; ++s) v[k1 * S + s] = tile[addr<ROW>(line, S * n, S * R1 * k1 + s)];
  }
  template <bool ROW>
  __device__ __forceinline__ static void store_out(const float2 (&v)[R2], float2* tile, int line, int n) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
      for (int s = 0; s < S; ++s) tile[addr<ROW>(line, S * n, S * R1 * k1 + s)] = v[k1 * S + s];
  }

  // Index (within the line) of register m in the "out" layout, and in the "in" layout.
  __device__ __forceinline__ static int out_index(int n, int m) { return S * (n + R1 * (m / S)) + (m % S); }
  __device__ __forceinline__ static int in_index(int n, int m) { return n + R1 * m; }
};

template <int N>
struct Fft2 : LineFft<FftCfg<N>::R1, FftCfg<N>::R2, FftCfg<N>::INTER, SquareAddr<N>> {};

// Twiddle table tw[n*(R2+1) + k2] = exp(-2 pi i n k2 / N) for n < R1, k2 <= R2
// (the padding column makes the per-k2 reads of the R1 lanes of a line hit
// distinct banks). Written by the whole CTA.
template <int N>
struct Twiddles {
  static constexpr int R1 = FftCfg<N>::R1, R2 = FftCfg<N>::R2, COUNT = R1 * (R2 + 1);
};
template <int L, int R1, int R2>
__device__ __forceinline__ void make_line_twiddles(float2* tw) {
  for (int m = threadIdx.x; m < R1 * (R2 + 1); m += blockDim.x) {
    const int n = m / (R2 + 1), k2 = m % (R2 + 1);
    float s, c;
    sincospif(2.0f * (float)(n * k2) / (float)L, &s, &c);
    tw[m] = make_float2(c, -s);
  }
}

template <int N>
__device__ __forceinline__ void make_twiddles(float2* tw) {
  make_line_twiddles<N, FftCfg<N>::R1, FftCfg<N>::R2>(tw);
}

}  // namespace ptycho
