// Per-thread bodies of the mixed-precision kernels of mg_mixed.cu (see
// mg_bodies64.cuh for the convention).
#pragma once

#include "mg_common.cuh"

namespace mg {

// The FP32 root change with every rounding spelled out (no contraction left to
// the compiler), so that the per-colour kernels and the one-launch sweep, which
// evaluates two cells per packed FP32x2 instruction, give the same bits.
// Both forms are evaluated and one is selected (no branch): 2 du / (s0 + s1) where
// both discriminants are non-negative, k2 (s1 - s0) of the guarded roots otherwise.
__device__ __forceinline__ float root_change32(float q0, float q1, float du, const OpConst32& c) {
  const float s0 = q0 > 0.f ? __fmul_rn(q0, rsqrtf(q0)) : 0.f;
  const float s1 = q1 > 0.f ? __fmul_rn(q1, rsqrtf(q1)) : 0.f;
  const float den = __fadd_rn(s0, s1);
  const float conj = den > 0.f ? __fdividef(__fmul_rn(c.sigma2, du), den) : 0.f;
  const float diff = __fmul_rn(c.sk2, __fsub_rn(s1, s0));
  return (q0 >= 0.f && q1 >= 0.f) ? conj : diff;
}

__device__ __forceinline__ float dD32(const StencilT<float>& se, const StencilT<float>& sp,
                                      float q0, const OpConst32& c) {
  if (c.linear) return 0.f;
  const float a1e = __fsub_rn(se.sx, se.sy), a2e = __fsub_rn(se.sx, se.sz),
              a3e = __fsub_rn(se.sy, se.sz);
  const float a1p = __fsub_rn(sp.sx, sp.sy), a2p = __fsub_rn(sp.sx, sp.sz),
              a3p = __fsub_rn(sp.sy, sp.sz);
  const float dA = __fmaf_rn(a3e, __fmaf_rn(2.f, a3p, a3e),
                             __fmaf_rn(a2e, __fmaf_rn(2.f, a2p, a2e),
                                       __fmul_rn(a1e, __fmaf_rn(2.f, a1p, a1e))));
  const float dB = __fmaf_rn(se.cyz, __fmaf_rn(2.f, sp.cyz, se.cyz),
                             __fmaf_rn(se.cxz, __fmaf_rn(2.f, sp.cxz, se.cxz),
                                       __fmul_rn(se.cxy, __fmaf_rn(2.f, sp.cxy, se.cxy))));
  const float du = __fmaf_rn(c.g2, dB, __fmul_rn(c.g1, dA));
  return root_change32(q0, __fmaf_rn(c.c3, du, q0), du, c);
}

// Gauss-Seidel value of one cell of N(e) = g + mu: (face sum - h^2 (dD + g + mu)) / 6.
__device__ __forceinline__ float gs_value32(const StencilT<float>& se, float dd, float g, float mu,
                                            const OpConst32& c) {
  return __fmul_rn(__fmaf_rn(-c.h2, __fadd_rn(dd, __fadd_rn(g, mu)),
                             __fadd_rn(__fadd_rn(se.sx, se.sy), se.sz)),
                   1.f / 6.f);
}

// Two cells of one colour per thread (packed FP32x2 arithmetic, lane x = the
// first cell, lane y = the second): the same operations lane by lane as the
// scalar forms above, so the same bits.
__device__ __forceinline__ float2 ld2(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once: fma(b, -1, a) is the IEEE difference
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

struct Stencil2 {
  float2 sx, sy, sz, cxy, cxz, cyz;
};

// dD32 on two cells at once (same operations, lane by lane).
__device__ __forceinline__ float2 dD2(const Stencil2& se, const Stencil2& sp, float2 q0,
                                      const OpConst32& c) {
  const float2 two = splat(2.f);
  const float2 a1e = sub2(se.sx, se.sy), a2e = sub2(se.sx, se.sz), a3e = sub2(se.sy, se.sz);
  const float2 a1p = sub2(sp.sx, sp.sy), a2p = sub2(sp.sx, sp.sz), a3p = sub2(sp.sy, sp.sz);
  const float2 dA = fma2(a3e, fma2(two, a3p, a3e),
                         fma2(a2e, fma2(two, a2p, a2e), mul2(a1e, fma2(two, a1p, a1e))));
  const float2 dB = fma2(se.cyz, fma2(two, sp.cyz, se.cyz),
                         fma2(se.cxz, fma2(two, sp.cxz, se.cxz),
                              mul2(se.cxy, fma2(two, sp.cxy, se.cxy))));
  const float2 du = fma2(splat(c.g2), dB, mul2(splat(c.g1), dA));
  const float2 q1 = fma2(splat(c.c3), du, q0);
  return make_float2(root_change32(q0.x, q1.x, du.x, c), root_change32(q0.y, q1.y, du.y, c));
}

// The FP64 residual of the outer defect correction and its hand-off to the FP32
// inner problem.  Each thread takes kHandoffCells cells (a block covers
// 256 kHandoffCells consecutive cells, coalesced per step), so the block's norm
// reduction, about 15 FP64 warp instructions, is shared by several cells.
// Index of cell (i,j,k) of an n^3 grid in colour order: the cells of colour
// c = ((i+k)&1) + 2((j+k)&1) fill block c of n^3/4 entries, in the order in which
// the threads of a colour stage visit them (x fastest, then y, then z), so that a
// colour stage reads its own cells' values contiguously.
__device__ __forceinline__ long long colour_index(int i, int j, int k, int n) {
  const int colour = ((i + k) & 1) + 2 * ((j + k) & 1);
  const long long hn = n >> 1;
  return colour * (hn * hn * n) + ((long long)k * hn + (j >> 1)) * hn + (i >> 1);
}

// With q0c / gc (may be null) the hand-off also stores q0 and g in colour order
// (colour_index) for the colour stages of the finest level.
__device__ __forceinline__ void b_residual_handoff64(
    int n, const double* __restrict__ phi, const double* __restrict__ src, OpConst64 c,
    const LevelScalars* __restrict__ sc, float* __restrict__ g, float* __restrict__ q0,
    float* __restrict__ phi0, float* __restrict__ e, Partial* __restrict__ partials,
    long long blk, float* __restrict__ gc = nullptr, float* __restrict__ q0c = nullptr) {
  const long long cells = (long long)n * n * n;
  Partial p;
  partial_init(p);
  const double lam = sc->lambda;
#pragma unroll 1
  for (int r = 0; r < kHandoffCells; ++r) {
    const long long t = ((long long)blk * kHandoffCells + r) * blockDim.x + threadIdx.x;
    if (t >= cells) break;
    int i, j, k;
    split3((unsigned)t, n, i, j, k);
    const StencilT<double> s = gather_periodic(phi, i, j, k, n);
    double q = 1.0, D;
    bool guard = false;
    if (c.mode == OP_LINEAR) {
      D = src[t];
    } else {
      const double A2 = half_A(s);
      const double B = fma(s.cxy, s.cxy, fma(s.cxz, s.cxz, s.cyz * s.cyz));
      if (c.mode == OP_SQRT) {
        q = fma(c.e1h, A2, fma(c.e2, B, src[t]));
        D = fma(c.k2s, sqrt_clamped(q), -c.k2);
      } else {
        const double u = fma(c.c1h, A2, fma(c.c2, B, src[t]));
        q = fma(c.c3, u, 1.0);
        D = (q < 0.0) ? -c.k2 : (2.0 * u) / (1.0 + sqrt(q));
      }
      guard = neg_guard(q);
    }
    const double ctr = phi[t];
    const double lap = (s.sx + s.sy + s.sz) - 6.0 * ctr;
    const double d = fma(lap, c.inv_h2, -D);
    partial_add(p, d, guard);
    g[t] = (float)(lam - d);
    q0[t] = (float)q;
    phi0[t] = (float)ctr;
    e[t] = 0.f;
    if (gc) {
      const long long ci = colour_index(i, j, k, n);
      gc[ci] = (float)(lam - d);
      q0c[ci] = (float)q;
    }
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blk] = p;
}

__device__ __forceinline__ void b_update64(long long cells, double* __restrict__ phi,
                                                  const float* __restrict__ e,
    long long blk) {
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  if (t < cells) phi[t] += (double)e[t];
}

__device__ __forceinline__ void b_restrict32(int nc, const float* __restrict__ fine,
                                                    float* __restrict__ coarse,
    long long blk) {
  const int nf = nc << 1;
  const long long cells = (long long)nc * nc * nc;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  int I, J, K;
  split3((unsigned)t, nc, I, J, K);
  float s = 0.f;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    s += fine[lidx(2 * I + (ch & 1), 2 * J + ((ch >> 1) & 1), 2 * K + (ch >> 2), nf)];
  coarse[t] = s * 0.125f;
}

__device__ __forceinline__ void b_q0_prep32(int n, const float* __restrict__ phi0,
                                                   const double* __restrict__ delta,
                                                   OpConst32 c, float kappa, int floor,
                                                   float* __restrict__ q0,
    long long blk) {
  const long long cells = (long long)n * n * n;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  if (c.linear) {
    q0[t] = 1.f;
    return;
  }
  int i, j, k;
  split3((unsigned)t, n, i, j, k);
  const StencilT<float> s = gather_periodic(phi0, i, j, k, n);
  const float a1 = s.sx - s.sy, a2 = s.sx - s.sz, a3 = s.sy - s.sz;
  const float A = a1 * a1 + a2 * a2 + a3 * a3;
  const float B = s.cxy * s.cxy + s.cxz * s.cxz + s.cyz * s.cyz;
  float qs = fmaf(c.c3 * kappa, (float)delta[t], 1.f);
  if (floor && qs < 0.f) qs = 0.f;
  q0[t] = fmaf(c.c3, c.g1 * A + c.g2 * B, qs);
}

// One cell of an FP32 colour stage: t indexes the colour's n^3/4 cells; t >= n^3/4
// does nothing.  mu is the level's lambda in FP32.
// The update of cell (i,j,k) (linear index id) given its q0 and g.
__device__ __forceinline__ void cell_smooth32_at(int n, float* __restrict__ e,
                                                 const float* __restrict__ phi0, float q0v,
                                                 float gv, float mu, const OpConst32& c, int i,
                                                 int j, int k, long long id) {
  const NbrOff o = nbr_offsets(i, j, k, n);
  const StencilT<float> se = gather_at(e + id, o);
  float dd = 0.f;
  if (!c.linear) dd = dD32(se, gather_at(phi0 + id, o), q0v, c);
  e[id] = gs_value32(se, dd, gv, mu, c);
}

__device__ __forceinline__ void cell_smooth32(int n, float* __restrict__ e,
                                              const float* __restrict__ phi0,
                                              const float* __restrict__ q0,
                                              const float* __restrict__ g, float mu,
                                              const OpConst32& c, int colour, long long t) {
  const int hn = n >> 1;
  const long long total = (long long)hn * hn * n;
  if (t >= total) return;
  int m, jj, k;
  split3((unsigned)t, hn, m, jj, k);
  const int i = 2 * m + ((colour ^ k) & 1);
  const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
  const long long id = lidx(i, j, k, n);
  cell_smooth32_at(n, e, phi0, q0[id], g[id], mu, c, i, j, k, id);
}

// Face sums and cross differences around the cell at c0, for a side N known at
// compile time and a cell off the y and z boundaries, with 8-byte loads of
// x-adjacent pairs.  A warp's cells of one colour sit at every other x of one row,
// all with the x parity P, so in each row that the stencil reads at x - 1, x and
// x + 1 two aligned pairs hold all three values:
//   P = 0: (x-2, x-1) and (x, x+1);   P = 1: (x-1, x) and (x+1, x+2).
// lo / hi are the offsets of those pairs from the cell (the x wrap folded in: the
// pair holding x - 1 of x = 0 is (N-2, N-1), the pair holding x + 1 of x = N - 1 is
// (0, 1)).  The centre row, the two y rows and the two z rows take two pair loads
// each and the four yz rows one scalar load: 14 loads instead of 18, with the same
// sums in the same order as gather_at.
template <int N, int P>
__device__ __forceinline__ StencilT<float> gather_n2(const float* c0, int lo, int hi) {
  constexpr int Y = N, Z = N * N;
  auto pair = [&](int off) { return *reinterpret_cast<const float2*>(c0 + off); };
  // x - 1, x, x + 1 of the row at offset r
  auto row = [&](int r, float& vm, float& v0, float& vp) {
    const float2 a = pair(lo + r), b = pair(hi + r);
    if (P == 0) {
      vm = a.y;
      v0 = b.x;
      vp = b.y;
    } else {
      vm = a.x;
      v0 = a.y;
      vp = b.x;
    }
  };
  float cm, c_, cp, ypm, yp0, ypp, ymm, ym0, ymp, zpm, zp0, zpp, zmm, zm0, zmp;
  row(0, cm, c_, cp);
  row(Y, ypm, yp0, ypp);
  row(-Y, ymm, ym0, ymp);
  row(Z, zpm, zp0, zpp);
  row(-Z, zmm, zm0, zmp);
  StencilT<float> s;
  s.sx = cp + cm;
  s.sy = yp0 + ym0;
  s.sz = zp0 + zm0;
  s.cxy = (ypp + ymm) - (ymp + ypm);
  s.cxz = (zpp + zmm) - (zmp + zpm);
  s.cyz = (c0[Y + Z] + c0[-Y - Z]) - (c0[Y - Z] + c0[-Y + Z]);
  return s;
}

// gather_n2 for two cells of one colour at the same x and y on planes k (at c0) and
// k + 2 (the parities repeat every two planes): the row (j, k+1) is the z + 1 row of
// the first cell and the z - 1 row of the second, and the yz rows (j±1, k+1) are
// shared the same way, so the two stencils take 24 loads instead of 28.  The sums
// are gather_n2's, in the same order.
template <int N, int P>
__device__ __forceinline__ void gather_n2_z2(const float* c0, int lo, int hi,
                                             StencilT<float>& sa, StencilT<float>& sb) {
  constexpr int Y = N, Z = N * N;
  auto pair = [&](int off) { return *reinterpret_cast<const float2*>(c0 + off); };
  auto row = [&](int r, float& vm, float& v0, float& vp) {
    const float2 a = pair(lo + r), b = pair(hi + r);
    if (P == 0) {
      vm = a.y;
      v0 = b.x;
      vp = b.y;
    } else {
      vm = a.x;
      v0 = a.y;
      vp = b.x;
    }
  };
  float am, a0, ap, aypm, ayp0, aypp, aymm, aym0, aymp, azmm, azm0, azmp;
  float sm, s0, sp;  // the shared row (j, k+1)
  float bm, b0, bp, bypm, byp0, bypp, bymm, bym0, bymp, bzpm, bzp0, bzpp;
  row(0, am, a0, ap);
  row(Y, aypm, ayp0, aypp);
  row(-Y, aymm, aym0, aymp);
  row(-Z, azmm, azm0, azmp);
  row(Z, sm, s0, sp);
  row(2 * Z, bm, b0, bp);
  row(2 * Z + Y, bypm, byp0, bypp);
  row(2 * Z - Y, bymm, bym0, bymp);
  row(3 * Z, bzpm, bzp0, bzpp);
  const float dyp = c0[Y + Z], dym = c0[-Y + Z];  // the shared yz cells (j±1, k+1)
  sa.sx = ap + am;
  sa.sy = ayp0 + aym0;
  sa.sz = s0 + azm0;
  sa.cxy = (aypp + aymm) - (aymp + aypm);
  sa.cxz = (sp + azmm) - (azmp + sm);
  sa.cyz = (dyp + c0[-Y - Z]) - (c0[Y - Z] + dym);
  sb.sx = bp + bm;
  sb.sy = byp0 + bym0;
  sb.sz = bzp0 + s0;
  sb.cxy = (bypp + bymm) - (bymp + bypm);
  sb.cxz = (bzpp + sm) - (sp + bzpm);
  sb.cyz = (c0[Y + 3 * Z] + dym) - (dyp + c0[-Y + 3 * Z]);
}

// cell_smooth32 for a side N known at compile time (N >= 64, so that a warp's 32
// cells share their row, and the y/z-boundary test below is uniform per warp).
// Rows on a y or z boundary take the general path; the others read their
// neighbours as pairs at immediate offsets (gather_n2).  The arithmetic is
// cell_smooth32's, so the bits are.
// With CO, q0 and g arrive in colour order (colour_index): q0 and g point at this
// colour's block, whose entry t is the cell the thread with index t updates, so a
// warp reads them contiguously; otherwise they are the natural n^3 arrays.
template <int N, bool CO>
__device__ __forceinline__ void cell_smooth32_n(float* __restrict__ e,
                                                const float* __restrict__ phi0,
                                                const float* __restrict__ q0,
                                                const float* __restrict__ g, float mu,
                                                const OpConst32& c, int colour, long long t) {
  static_assert(N >= 64 && (N & (N - 1)) == 0, "power of two, at least 64");
  constexpr int HN = N / 2;
  constexpr long long TOTAL = (long long)HN * HN * N;
  if (t >= TOTAL) return;
  const unsigned u = (unsigned)t;
  const int m = (int)(u % HN), jj = (int)((u / HN) % HN), k = (int)(u / (HN * HN));
  const int i = 2 * m + ((colour ^ k) & 1);
  const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
  const long long id = (long long)i + (long long)N * (j + (long long)N * k);
  const float q0v = CO ? q0[t] : q0[id], gv = CO ? g[t] : g[id];
  if (j == 0 || j == N - 1 || k == 0 || k == N - 1) {
    cell_smooth32_at(N, e, phi0, q0v, gv, mu, c, i, j, k, id);
    return;
  }
  // pair offsets (gather_n2); the x parity is uniform over the warp
  const int par = i & 1;
  const int lo = par ? -1 : (i == 0 ? N - 2 : -2);
  const int hi = par ? (i == N - 1 ? 1 - N : 1) : 0;
  const float *ce = e + id, *cp = phi0 + id;
  StencilT<float> se, sp;
  if (par) {
    se = gather_n2<N, 1>(ce, lo, hi);
    if (!c.linear) sp = gather_n2<N, 1>(cp, lo, hi);
  } else {
    se = gather_n2<N, 0>(ce, lo, hi);
    if (!c.linear) sp = gather_n2<N, 0>(cp, lo, hi);
  }
  const float dd = c.linear ? 0.f : dD32(se, sp, q0v, c);
  e[id] = gs_value32(se, dd, gv, mu, c);
}

// Two cells of one colour stage per thread (cell_smooth32_n on each, sharing the
// rows between them): tp < N^3/8 indexes pairs of planes, the plane pair kp holding
// the planes k = 4 (kp / 2) + kp % 2 and k + 2, so that every plane is covered once.
// A pair with a cell on a y or z boundary runs cell_smooth32_n on each cell.
template <int N, bool CO>
__device__ __forceinline__ void cell_smooth32_n_z2(float* __restrict__ e,
                                                   const float* __restrict__ phi0,
                                                   const float* __restrict__ q0,
                                                   const float* __restrict__ g, float mu,
                                                   const OpConst32& c, int colour, long long tp) {
  constexpr int HN = N / 2;
  constexpr long long HH = (long long)HN * HN;
  if (tp >= HH * (N / 2)) return;
  const unsigned u = (unsigned)tp;
  const int m = (int)(u % HN), jj = (int)((u / HN) % HN), kp = (int)(u / (HN * HN));
  const int k = 4 * (kp >> 1) + (kp & 1);
  const long long ta = ((long long)k * HN + jj) * HN + m, tb = ta + 2 * HH;
  const int i = 2 * m + ((colour ^ k) & 1);
  const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
  if (j == 0 || j == N - 1 || k == 0 || k + 2 == N - 1) {
    cell_smooth32_n<N, CO>(e, phi0, q0, g, mu, c, colour, ta);
    cell_smooth32_n<N, CO>(e, phi0, q0, g, mu, c, colour, tb);
    return;
  }
  const long long ida = (long long)i + (long long)N * (j + (long long)N * k);
  const long long idb = ida + 2LL * N * N;
  const float qa = CO ? q0[ta] : q0[ida], qb = CO ? q0[tb] : q0[idb];
  const float ga = CO ? g[ta] : g[ida], gb = CO ? g[tb] : g[idb];
  const int par = i & 1;
  const int lo = par ? -1 : (i == 0 ? N - 2 : -2);
  const int hi = par ? (i == N - 1 ? 1 - N : 1) : 0;
  StencilT<float> sea, seb, spa, spb;
  if (par) {
    gather_n2_z2<N, 1>(e + ida, lo, hi, sea, seb);
    if (!c.linear) gather_n2_z2<N, 1>(phi0 + ida, lo, hi, spa, spb);
  } else {
    gather_n2_z2<N, 0>(e + ida, lo, hi, sea, seb);
    if (!c.linear) gather_n2_z2<N, 0>(phi0 + ida, lo, hi, spa, spb);
  }
  const float dda = c.linear ? 0.f : dD32(sea, spa, qa, c);
  const float ddb = c.linear ? 0.f : dD32(seb, spb, qb, c);
  e[ida] = gs_value32(sea, dda, ga, mu, c);
  e[idb] = gs_value32(seb, ddb, gb, mu, c);
}

__device__ __forceinline__ void b_smooth_colour32(int n, float* __restrict__ e,
                                                         const float* __restrict__ phi0,
                                                         const float* __restrict__ q0,
                                                         const float* __restrict__ g,
                                                         const LevelScalars* __restrict__ sc,
                                                         OpConst32 c, int colour,
    long long blk) {
  __shared__ float s_mu;
  if (threadIdx.x == 0) s_mu = (float)sc->lambda;
  __syncthreads();
  cell_smooth32(n, e, phi0, q0, g, s_mu, c, colour, (long long)blk * blockDim.x + threadIdx.x);
}

// The colour stage of b_smooth_colour32 with two cells per thread: the cells
// x and x + 2 of one row and colour (n % 4 == 0).  They share the x + 1 column of
// their stencils, the second cell's loads sit 8 bytes past the first's, and the
// arithmetic runs on both in the two lanes of packed FP32x2 instructions, each
// lane doing exactly what b_smooth_colour32 does for its cell.
__device__ __forceinline__ void b_smooth_colour32_pair(int n, float* __restrict__ e,
                                                       const float* __restrict__ phi0,
                                                       const float* __restrict__ q0,
                                                       const float* __restrict__ g,
                                                       const LevelScalars* __restrict__ sc,
                                                       OpConst32 c, int colour, long long blk) {
  __shared__ float s_mu;
  if (threadIdx.x == 0) s_mu = (float)sc->lambda;
  __syncthreads();
  const int hn = n >> 1, qn = n >> 2;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  if (t >= (long long)qn * hn * n) return;
  // t -> (p, jj, k): p = t % qn, jj = (t / qn) % hn, k = t / (qn hn)
  const unsigned ut = (unsigned)t, uq = (unsigned)qn, uh = (unsigned)hn;
  int p, jj, k;
  if (((uq & (uq - 1u)) | (uh & (uh - 1u))) == 0u) {
    const unsigned rest = ut >> (__ffs(qn) - 1);
    p = (int)(ut & (uq - 1u));
    jj = (int)(rest & (uh - 1u));
    k = (int)(rest >> (__ffs(hn) - 1));
  } else {
    const unsigned rest = ut / uq;
    p = (int)(ut - rest * uq);
    jj = (int)(rest % uh);
    k = (int)(rest / uh);
  }
  const int i = 4 * p + ((colour ^ k) & 1);
  const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
  const long long id = lidx(i, j, k, n);
  const NbrOff o = nbr_offsets(i, j, k, n);
  const int xmA = o.xm;                        // -1, or n - 1 at i == 0
  const int xpB = (i + 3 == n) ? 3 - n : 3;   // x + 1 of the second cell, from the first
  // offsets (y, z part) of the 13 rows of the stencil
  const int y0 = 0, yp = o.yp, ym = o.ym, zp = o.zp, zm = o.zm;
  auto gather = [&](const float* __restrict__ b) {
    Stencil2 st;
    auto xrow = [&](int yz, float2& xpv, float2& xmv) {
      const float sh = b[yz + 1];  // x + 1 of the first cell = x - 1 of the second
      xpv = make_float2(sh, b[yz + xpB]);
      xmv = make_float2(b[yz + xmA], sh);
    };
    auto col = [&](int yz) { return make_float2(b[yz], b[yz + 2]); };
    float2 xp_, xm_, xpyp, xmyp, xpym, xmym, xpzp, xmzp, xpzm, xmzm;
    xrow(y0, xp_, xm_);
    xrow(yp, xpyp, xmyp);
    xrow(ym, xpym, xmym);
    xrow(zp, xpzp, xmzp);
    xrow(zm, xpzm, xmzm);
    const float2 ypv = col(yp), ymv = col(ym), zpv = col(zp), zmv = col(zm);
    const float2 ypzp = col(yp + zp), ymzm = col(ym + zm), ypzm = col(yp + zm), ymzp = col(ym + zp);
    st.sx = add2(xp_, xm_);
    st.sy = add2(ypv, ymv);
    st.sz = add2(zpv, zmv);
    st.cxy = sub2(add2(xpyp, xmym), add2(xpym, xmyp));
    st.cxz = sub2(add2(xpzp, xmzm), add2(xpzm, xmzp));
    st.cyz = sub2(add2(ypzp, ymzm), add2(ypzm, ymzp));
    return st;
  };
  float* const ea = e + id;
  const Stencil2 ee = gather(ea);
  float2 dd = make_float2(0.f, 0.f);
  if (!c.linear) dd = dD2(ee, gather(phi0 + id), make_float2(q0[id], q0[id + 2]), c);
  const float2 gv = make_float2(g[id], g[id + 2]);
  const float2 v = mul2(fma2(splat(-c.h2), add2(dd, add2(gv, splat(s_mu))),
                             add2(add2(ee.sx, ee.sy), ee.sz)),
                        splat(1.f / 6.f));
  ea[0] = v.x;
  ea[2] = v.y;
}

// The FP32 defect r = N(e) - g of fine cell (i,j,k) (linear index id); ctr
// returns e there.
__device__ __forceinline__ float fine_defect32(int nf, const float* __restrict__ e,
                                              const float* __restrict__ phi0,
                                              const float* __restrict__ q0,
                                              const float* __restrict__ g, const OpConst32& c,
                                              int i, int j, int k, long long id, float& ctr) {
  const StencilT<float> se = gather_periodic(e, i, j, k, nf);
  float dd = 0.f;
  if (!c.linear) {
    const StencilT<float> sp = gather_periodic(phi0, i, j, k, nf);
    dd = dD32(se, sp, q0[id], c);
  }
  ctr = e[id];
  const float lap = (se.sx + se.sy + se.sz) - 6.f * ctr;
  return fmaf(lap, c.inv_h2, -dd) - g[id];
}

__device__ __forceinline__ void b_residual_restrict32(
    int nf, const float* __restrict__ e, const float* __restrict__ phi0,
    const float* __restrict__ q0, const float* __restrict__ g, OpConst32 c,
    float* __restrict__ e_c, float* __restrict__ ehat_c, float* __restrict__ rg_c,
    Partial* __restrict__ partials,
    long long blk) {
  const int nc = nf >> 1;
  const long long ccells = (long long)nc * nc * nc;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < ccells) {
    int I, J, K;
    split3((unsigned)t, nc, I, J, K);
    // norms of the 8 children in FP32 (the inner problem's lambda needs FP32
    // accuracy only), merged into the FP64 block partial once per thread
    float se_sum = 0.f, sr = 0.f, fsum = 0.f, fmx = -INFINITY, fmn = INFINITY;
    int bad = 0;
#pragma unroll 2
    for (int ch = 0; ch < 8; ++ch) {
      const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
      const long long id = lidx(i, j, k, nf);
      float ctr;
      const float r = fine_defect32(nf, e, phi0, q0, g, c, i, j, k, id, ctr);
      if (isfinite(r)) {
        fsum += r;
        fmx = fmaxf(fmx, r);
        fmn = fminf(fmn, r);
      } else {
        ++bad;
      }
      se_sum += ctr;
      sr += r;
    }
    if (bad < 8) {
      p.sum = (double)fsum;
      p.dmax = (double)fmx;
      p.dmin = (double)fmn;
    }
    p.nonfinite = bad;
    e_c[t] = se_sum * 0.125f;
    ehat_c[t] = se_sum * 0.125f;
    rg_c[t] = sr * 0.125f;
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blk] = p;
}

// The FP32 residual restriction in two steps (as cell_defect64 and
// b_restrict_defects64): per fine cell r, then every coarse cell's 8 children in
// the order and block partition of b_residual_restrict32.
__device__ __forceinline__ void cell_defect32(int nf, const float* __restrict__ e,
                                              const float* __restrict__ phi0,
                                              const float* __restrict__ q0,
                                              const float* __restrict__ g, const OpConst32& c,
                                              float* __restrict__ rout, long long t) {
  const long long cells = (long long)nf * nf * nf;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nf, i, j, k);
  float ctr;
  rout[t] = fine_defect32(nf, e, phi0, q0, g, c, i, j, k, t, ctr);
}

__device__ __forceinline__ void b_restrict_defects32(
    int nf, const float* __restrict__ e, const float* __restrict__ rin, float* __restrict__ e_c,
    float* __restrict__ ehat_c, float* __restrict__ rg_c, Partial* __restrict__ partials,
    long long blk) {
  const int nc = nf >> 1;
  const long long ccells = (long long)nc * nc * nc;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < ccells) {
    int I, J, K;
    split3((unsigned)t, nc, I, J, K);
    float se_sum = 0.f, sr = 0.f, fsum = 0.f, fmx = -INFINITY, fmn = INFINITY;
    int bad = 0;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
      const long long id = lidx(i, j, k, nf);
      const float r = rin[id];
      if (isfinite(r)) {
        fsum += r;
        fmx = fmaxf(fmx, r);
        fmn = fminf(fmn, r);
      } else {
        ++bad;
      }
      se_sum += e[id];
      sr += r;
    }
    if (bad < 8) {
      p.sum = (double)fsum;
      p.dmax = (double)fmx;
      p.dmin = (double)fmn;
    }
    p.nonfinite = bad;
    e_c[t] = se_sum * 0.125f;
    ehat_c[t] = se_sum * 0.125f;
    rg_c[t] = sr * 0.125f;
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blk] = p;
}

// One coarse cell of the FP32 FAS right-hand side (t indexes the nc^3 cells; lam_f
// is the fine level's lambda; cell 0 also clears the coarse lambda).
__device__ __forceinline__ void cell_fas_rhs32(int nc, const float* __restrict__ e_c,
                                               const float* __restrict__ phi0_c,
                                               const float* __restrict__ q0_c,
                                               float* __restrict__ g_c, const OpConst32& c,
                                               double lam_f, LevelScalars* __restrict__ coarse_sc,
                                               long long t) {
  const long long cells = (long long)nc * nc * nc;
  if (t == 0) coarse_sc->lambda = 0.0;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nc, i, j, k);
  const StencilT<float> se = gather_periodic(e_c, i, j, k, nc);
  float dd = 0.f;
  if (!c.linear) {
    const StencilT<float> sp = gather_periodic(phi0_c, i, j, k, nc);
    dd = dD32(se, sp, q0_c[t], c);
  }
  const float lap = (se.sx + se.sy + se.sz) - 6.f * e_c[t];
  const float Nv = fmaf(lap, c.inv_h2, -dd);
  g_c[t] = Nv - g_c[t] + (float)lam_f;
}

__device__ __forceinline__ void b_fas_rhs32(int nc, const float* __restrict__ e_c,
                                                   const float* __restrict__ phi0_c,
                                                   const float* __restrict__ q0_c,
                                                   float* __restrict__ g_c, OpConst32 c,
                                                   const LevelScalars* __restrict__ fine_sc,
                                                   LevelScalars* __restrict__ coarse_sc,
    long long blk) {
  cell_fas_rhs32(nc, e_c, phi0_c, q0_c, g_c, c, fine_sc->lambda, coarse_sc,
                 (long long)blk * blockDim.x + threadIdx.x);
}

// One fine cell of the trilinear prolongation of e_c - ehat_c into e_f (t indexes
// the (2 nc)^3 fine cells).
__device__ __forceinline__ void cell_prolong32(int nc, const float* __restrict__ e_c,
                                               const float* __restrict__ ehat_c,
                                               float* __restrict__ e_f, long long t) {
  const int nf = nc << 1;
  const long long cells = (long long)nf * nf * nf;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nf, i, j, k);
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = (i & 1) ? wrap_up(I0, nc) : wrap_dn(I0, nc);
  const int J1 = (j & 1) ? wrap_up(J0, nc) : wrap_dn(J0, nc);
  const int K1 = (k & 1) ? wrap_up(K0, nc) : wrap_dn(K0, nc);
  auto v = [&](int a, int b, int cc) {
    const long long q = lidx(a, b, cc, nc);
    return e_c[q] - ehat_c[q];
  };
  const float s = 27.f * v(I0, J0, K0) + 9.f * (v(I1, J0, K0) + v(I0, J1, K0) + v(I0, J0, K1)) +
                  3.f * (v(I1, J1, K0) + v(I1, J0, K1) + v(I0, J1, K1)) + v(I1, J1, K1);
  e_f[t] += s * (1.f / 64.f);
}

// cell_prolong32 from the coarse correction corr_c = e_c - ehat_c formed beforehand
// (once per coarse cell instead of once per fine cell that reads it): the same
// values in the same sum.
__device__ __forceinline__ void cell_prolong_corr32(int nc, const float* __restrict__ corr_c,
                                                    float* __restrict__ e_f, long long t) {
  const int nf = nc << 1;
  const long long cells = (long long)nf * nf * nf;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nf, i, j, k);
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = (i & 1) ? wrap_up(I0, nc) : wrap_dn(I0, nc);
  const int J1 = (j & 1) ? wrap_up(J0, nc) : wrap_dn(J0, nc);
  const int K1 = (k & 1) ? wrap_up(K0, nc) : wrap_dn(K0, nc);
  auto v = [&](int a, int b, int cc) { return corr_c[lidx(a, b, cc, nc)]; };
  const float s = 27.f * v(I0, J0, K0) + 9.f * (v(I1, J0, K0) + v(I0, J1, K0) + v(I0, J0, K1)) +
                  3.f * (v(I1, J1, K0) + v(I1, J0, K1) + v(I0, J1, K1)) + v(I1, J1, K1);
  e_f[t] += s * (1.f / 64.f);
}

__device__ __forceinline__ void b_prolong_correct32(int nc, const float* __restrict__ e_c,
                                                           const float* __restrict__ ehat_c,
                                                           float* __restrict__ e_f,
    long long blk) {
  cell_prolong32(nc, e_c, ehat_c, e_f, (long long)blk * blockDim.x + threadIdx.x);
}

// The coarsest level of the inner correction cycle, in one CTA and in FP32 (the
// precision of the inner problem): four-colour sweeps of the FP32 smoother's own
// cell update until the residual falls by `drop`, stalls, reaches the FP32
// rounding floor or `max_sweeps` is spent, with the residual checked every two
// sweeps.  A single FP64 warp on 16 cells per colour (4^3) would take about 80
// microseconds per visit on GB300's FP64 pipe; in FP32 it is a few.
__device__ __forceinline__ void b_coarsest_corr32(int n, float* __restrict__ e,
                                                  const float* __restrict__ phi0,
                                                  const float* __restrict__ q0,
                                                  const float* __restrict__ g, OpConst32 c,
                                                  LevelScalars* __restrict__ sc, int max_sweeps,
                                                  double drop, long long blk) {
  extern __shared__ float smf[];
  __shared__ double s_mu, s_res;
  const int cells = n * n * n;
  float* se = smf;
  float* sp = smf + cells;
  float* sq = smf + 2 * cells;
  float* sg = smf + 3 * cells;
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    se[q] = e[q];
    sp[q] = phi0[q];
    sq[q] = q0[q];
    sg[q] = g[q];
  }
  if (threadIdx.x == 0) s_mu = sc->lambda;
  __syncthreads();
  double scale = 0.0;
  // residual of N(e) = g + mu: mu = mean(N(e) - g), res = max |N(e) - g - mu|
  auto residual = [&]() {
    Partial p;
    partial_init(p);
    float mag = 0.f;
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
      int i, j, k;
      split3((unsigned)q, n, i, j, k);
      const StencilT<float> a = gather_periodic(se, i, j, k, n);
      float dd = 0.f;
      if (!c.linear) dd = dD32(a, gather_periodic(sp, i, j, k, n), sq[q], c);
      const float lnb = (a.sx + a.sy) + a.sz;
      const float r = fmaf(lnb - 6.f * se[q], c.inv_h2, -dd) - sg[q];
      partial_add(p, (double)r, false);
      mag = fmaxf(mag, (fabsf(lnb) + 6.f * fabsf(se[q])) * c.inv_h2 + fabsf(dd) + fabsf(sg[q]));
    }
    scale = block_max((double)mag);
    p = block_reduce(p);
    if (threadIdx.x == 0) {
      const double mu = p.sum / (double)cells;
      s_mu = mu;
      s_res = (p.nonfinite > 0) ? NAN : fmax(p.dmax - mu, mu - p.dmin);
    }
    __syncthreads();
    return s_res;
  };
  // FP32 unit roundoff: the floor below which the residual is rounding noise
  auto done = [&](double r, double r0, double r_prev) {
    if (!(r > drop * r0)) return true;
    if (r <= 64.0 * 5.9604644775390625e-8 * scale) return true;
    return r >= 0.95 * r_prev;
  };
  const double r0 = residual();
  double r_prev = r0;
  const int per_colour = (n >> 1) * (n >> 1) * n;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    const float mu = (float)s_mu;
    for (int colour = 0; colour < 4; ++colour) {
      for (int t = threadIdx.x; t < per_colour; t += blockDim.x)
        cell_smooth32(n, se, sp, sq, sg, mu, c, colour, t);
      __syncthreads();
    }
    if ((sweep & 1) == 1 || sweep + 1 == max_sweeps) {
      const double r = residual();
      if (done(r, r0, r_prev)) break;
      r_prev = r;
    }
  }
  for (int q = threadIdx.x; q < cells; q += blockDim.x) e[q] = se[q];
  if (threadIdx.x == 0) {
    sc->lambda = s_mu;
    sc->res = s_res;
  }
}

}  // namespace mg
