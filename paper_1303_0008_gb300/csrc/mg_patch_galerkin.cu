// Linear coarse-grid correction of the refinement unions (the multigrid on the
// refinements of Sec. III.C of arXiv:1303.0008), with coarse operators built
// from the fine operator itself.
//
// The union FAS of mg_patch.cu rediscretises L^h on the coarse union levels.  In
// dense regions with alpha*kappa*delta >> 1 the linearised operator of Sec. III.B
// is strongly and irregularly anisotropic from cell to cell, the rediscretised
// coarse operator does not represent it, and the coarse-grid correction makes
// the error grow.  Here the correction solves instead the linear equation
//     J_H e_H = -R d,    J_H = R J P,
// where J is the Jacobian of L^h at the current union iterate (19 entries per
// row: the Newton linearisation of the root of Eq. two_branch through Sigma_ijk),
// R the mean of the 8 children and P the cell-centred trilinear prolongation
// with zero correction outside the union (the Dirichlet cells are fixed).  J_H
// is a 27-point operator; the next union level takes J_2H = R J_H P again.  The
// linear levels are relaxed by eight-colour Gauss-Seidel in FP32 (a 27-point
// stencil needs eight colours, (i&1) + 2(j&1) + 4(k&1)), and phi += P e_H.  The
// fixed point of the solve is untouched: the nonlinear Newton-Gauss-Seidel
// smoother and the FP64 residual of the union level decide it.
//
// Layout (per refinement level, union level m = 1, 2 with block side Bm = 8>>m):
// J[m] float [count][27][Bm^3] (entry o = (ox+1) + 3(oy+1) + 9(oz+1) of the row of
// cell t at J[(p*27 + o)*Bm^3 + t]), e[m], b[m] float [count][Bm^3].
#include <cstring>
#include <string>

#include "mg_internal.h"
#include "mg_patch_tile.cuh"
#include "mg_solver.h"

namespace mg {

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int gal_region1(int x, int B) { return x < 0 ? 0 : (x >= B ? 2 : 1); }

// index 0..26 of a neighbour block (the patch table's convention), of a local
// coordinate triple relative to a block of side B
__device__ __forceinline__ int gal_region(int x, int y, int z, int B) {
  return gal_region1(x, B) + 3 * (gal_region1(y, B) + 3 * gal_region1(z, B));
}

__device__ __forceinline__ int gal_wrap(int x, int B) { return x < 0 ? x + B : (x >= B ? x - B : x); }

// Value of a block-B field at local coordinates (x, y, z) in [-1, B] of patch p:
// the patch's own cell, the cell of the neighbouring patch, or 0 outside the union.
template <int B>
__device__ __forceinline__ float gal_fetch(const float* __restrict__ a, const int* __restrict__ nbr,
                                           int p, int x, int y, int z) {
  constexpr int BC = B * B * B;
  int q = p;
  if ((unsigned)x >= (unsigned)B || (unsigned)y >= (unsigned)B || (unsigned)z >= (unsigned)B) {
    q = nbr[p * 27 + gal_region(x, y, z, B)];
    if (q < 0) return 0.0f;
    x = gal_wrap(x, B);
    y = gal_wrap(y, B);
    z = gal_wrap(z, B);
  }
  return a[(long long)q * BC + x + B * (y + B * z)];
}

// The row of the Jacobian of L^h at one cell: face coefficients per axis and
// the magnitudes of the three cross-difference couplings.  The centre entry is
// -6/h^2 (with w = 1/3 Sigma_d does not involve the centre value).
//   L = (Sx + Sy + Sz - 6 phi)/h^2 - D(q),  q = src + e1h A2 + e2 B  (OP_SQRT),
//   A2 = a1 (a1 - a2) + a2^2,  a1 = Sx - Sy,  a2 = Sx - Sz,  B = Cxy^2 + Cxz^2 + Cyz^2,
// so dA2/dSx = a1 + a2, dA2/dSy = a2 - 2 a1, dA2/dSz = a1 - 2 a2, dB/dCxy = 2 Cxy,
// and dD/dq = sigma k2 / (2 sqrt q) (0 where the discriminant is clamped).  In
// the conjugate form (OP_CONJ) u = src + c1h A2 + c2 B and dD/du = 1/sqrt(q).
// Each coefficient is that of the (+,+) and (-,-) neighbours of a cross
// difference; the (+,-) and (-,+) neighbours take minus it.
// Evaluated in FP32 on an FP32 copy of the tile: the Galerkin operator only shapes
// the coarse-grid correction, so single precision suffices, and GB300's FP32 rate
// is many times its FP64 rate.
struct JacRow32 {
  float fx, fy, fz, exy, exz, eyz;
};

__device__ __forceinline__ JacRow32 jac_row32(const StencilT<float>& s, float src,
                                              const OpConst64& c) {
  JacRow32 r;
  const float inv_h2 = (float)c.inv_h2;
  r.fx = r.fy = r.fz = inv_h2;
  r.exy = r.exz = r.eyz = 0.f;
  if (c.mode == OP_LINEAR) return r;
  const float a1 = s.sx - s.sy, a2 = s.sx - s.sz;
  const float A2 = fmaf(a1, a1 - a2, a2 * a2);
  const float Bq = fmaf(s.cxy, s.cxy, fmaf(s.cxz, s.cxz, s.cyz * s.cyz));
  float kA = 0.f, kB = 0.f;
  if (c.mode == OP_SQRT) {
    const float q = fmaf((float)c.e1h, A2, fmaf((float)c.e2, Bq, src));
    if (q > 0.f) {
      const float dq = 0.5f * (float)c.k2s * rsqrtf(q);
      kA = dq * (float)c.e1h;
      kB = dq * (float)c.e2;
    }
  } else {
    const float u = fmaf((float)c.c1h, A2, fmaf((float)c.c2, Bq, src));
    const float q = fmaf((float)c.c3, u, 1.f);
    if (q > 0.f) {
      const float du = rsqrtf(q);
      kA = du * (float)c.c1h;
      kB = du * (float)c.c2;
    }
  }
  r.fx = fmaf(-kA, a1 + a2, inv_h2);
  r.fy = fmaf(-kA, a2 - 2.f * a1, inv_h2);
  r.fz = fmaf(-kA, a1 - 2.f * a2, inv_h2);
  r.exy = -2.f * kB * s.cxy;
  r.exz = -2.f * kB * s.cxz;
  r.eyz = -2.f * kB * s.cyz;
  return r;
}

// The 19 stencil offsets of the fine operator (entry e, axis 0..2): the centre,
// the six faces, then the edges in pairs (+,+), (-,-), (+,-), (-,+) of the xy, xz
// and yz planes.  Constant-folded once the loops over e are unrolled.
__host__ __device__ constexpr int s19(int e, int axis) {
  constexpr int tab[19][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                              {0, 0, 1},   {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
  return tab[e][axis];
}

__device__ __forceinline__ float row_entry(const JacRow32& r, float centre, int s) {
  switch (s) {
    case 0: return centre;
    case 1: case 2: return r.fx;
    case 3: case 4: return r.fy;
    case 5: case 6: return r.fz;
    case 7: case 8: return r.exy;
    case 9: case 10: return -r.exy;
    case 11: case 12: return r.exz;
    case 13: case 14: return -r.exz;
    case 15: case 16: return r.eyz;
    default: return -r.eyz;
  }
}

// Parents of a fine coordinate 2I + t (t in -1..2, relative to the coarse cell I)
// under cell-centred trilinear prolongation: offset of the near parent floor(t/2)
// (weight 3/4) and of the far one on the child's side (weight 1/4).
__host__ __device__ constexpr int gal_near(int t) { return t < 0 ? -1 : t / 2; }
__host__ __device__ constexpr int gal_far(int t) { return gal_near(t) + ((t & 1) ? 1 : -1); }

// Add (1/8) v P(fine cell 2I + t -> coarse) to the 27 accumulators of coarse cell I,
// keeping the coarse columns inside the union (bit o of cmask).
__device__ __forceinline__ void gal_scatter(float (&acc)[27], unsigned cmask, float v, int tx,
                                            int ty, int tz) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ox = (a & 1) ? gal_far(tx) : gal_near(tx);
    const int oy = (a & 2) ? gal_far(ty) : gal_near(ty);
    const int oz = (a & 4) ? gal_far(tz) : gal_near(tz);
    const float w = ((a & 1) ? 0.25f : 0.75f) * ((a & 2) ? 0.25f : 0.75f) *
                    ((a & 4) ? 0.25f : 0.75f) * 0.125f;
    const int o = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    if ((cmask >> o) & 1u) acc[o] = fmaf(w, v, acc[o]);
  }
}

// Face sums and cross differences of cell (i,j,k) of an FP32 copy of a ghosted
// 10^3 patch tile.
__device__ __forceinline__ StencilT<float> gather_tile32(const float* t, int i, int j, int k) {
  auto at = [&](int a, int b, int cc) { return t[(a + 1) + 10 * ((b + 1) + 10 * (cc + 1))]; };
  StencilT<float> s;
  s.sx = at(i + 1, j, k) + at(i - 1, j, k);
  s.sy = at(i, j + 1, k) + at(i, j - 1, k);
  s.sz = at(i, j, k + 1) + at(i, j, k - 1);
  s.cxy = (at(i + 1, j + 1, k) + at(i - 1, j - 1, k)) - (at(i + 1, j - 1, k) + at(i - 1, j + 1, k));
  s.cxz = (at(i + 1, j, k + 1) + at(i - 1, j, k - 1)) - (at(i + 1, j, k - 1) + at(i - 1, j, k + 1));
  s.cyz = (at(i, j + 1, k + 1) + at(i, j - 1, k - 1)) - (at(i, j + 1, k - 1) + at(i, j - 1, k + 1));
  return s;
}

// Bit r of the result is set when neighbour block r (0..26, the patch table's
// order; 13 is the patch itself) of patch p exists.
__device__ __forceinline__ unsigned exist_mask(const int* __restrict__ nbr, int p) {
  unsigned m = 0;
#pragma unroll
  for (int r = 0; r < 27; ++r)
    if (nbr[p * 27 + r] >= 0) m |= 1u << r;
  return m;
}

// Bit o (= (ox+1) + 3(oy+1) + 9(oz+1)) set when coarse cell (I, J, K) + O of a
// block of side H lies in the union (its own patch or an existing neighbour).
__device__ __forceinline__ unsigned coarse_mask(unsigned exm, int I, int J, int K, int H) {
  unsigned m = 0;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    if ((exm >> gal_region(I + ox, J + oy, K + oz, H)) & 1u) m |= 1u << o;
  }
  return m;
}

// ---------------------------------------------------------------------------
// Galerkin assembly
// ---------------------------------------------------------------------------
// J_1 = R J P from the nonlinear union level (8^3 per patch) to 4^3 per patch.
// One CTA of 64 threads per patch, one thread per coarse cell; each fine cell's
// Jacobian row is formed once, by the thread of its parent.
__global__ void __launch_bounds__(64) k_gal_assemble0(const double* __restrict__ phi,
                                                      const double* __restrict__ src,
                                                      const double* __restrict__ ghost,
                                                      const int* __restrict__ nbr, OpConst64 c,
                                                      float* __restrict__ J1) {
  __shared__ double tile[1000];
  __shared__ float tile32[1000];
  const int p = blockIdx.x;
  load_tile<8>(tile, p, phi, ghost, nbr);
  const unsigned exm = exist_mask(nbr, p);
  __syncthreads();
  for (int q = threadIdx.x; q < 1000; q += blockDim.x) tile32[q] = (float)tile[q];
  __syncthreads();
  const int t = threadIdx.x;
  const int I = t & 3, J = (t >> 2) & 3, K = t >> 4;
  const unsigned cmask = coarse_mask(exm, I, J, K, 4);
  float acc[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) acc[o] = 0.0f;
  const float centre = (float)(-6.0 * c.inv_h2);
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
    const int x = 2 * I + cx, y = 2 * J + cy, z = 2 * K + cz;
    const StencilT<float> s = gather_tile32(tile32, x, y, z);
    const JacRow32 r = jac_row32(s, (float)src[(long long)p * 512 + x + 8 * (y + 8 * z)], c);
#pragma unroll
    for (int e = 0; e < 19; ++e) {
      const int sx = s19(e, 0), sy = s19(e, 1), sz = s19(e, 2);
      // the fine column must be a union cell (the Dirichlet cells are fixed)
      if (!((exm >> gal_region(x + sx, y + sy, z + sz, 8)) & 1u)) continue;
      gal_scatter(acc, cmask, row_entry(r, centre, e), cx + sx, cy + sy, cz + sz);
    }
  }
#pragma unroll
  for (int o = 0; o < 27; ++o) J1[((long long)p * 27 + o) * 64 + t] = acc[o];
}

// J_c = R J_f P between two linear union levels (block BF -> BF/2); one thread
// per coarse cell.
template <int BF>
__global__ void __launch_bounds__(64) k_gal_assemble_lin(const float* __restrict__ Jf,
                                                         const int* __restrict__ nbr, int count,
                                                         float* __restrict__ Jc) {
  constexpr int H = BF / 2, HC = H * H * H, FC = BF * BF * BF;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)count * HC) return;
  const int p = (int)(g / HC), t = (int)(g % HC);
  const int I = t % H, J = (t / H) % H, K = t / (H * H);
  const unsigned exm = exist_mask(nbr, p);
  const unsigned cmask = coarse_mask(exm, I, J, K, H);
  float acc[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) acc[o] = 0.0f;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    const int cx = ch & 1, cy = (ch >> 1) & 1, cz = ch >> 2;
    const int x = 2 * I + cx, y = 2 * J + cy, z = 2 * K + cz;
    const int tf = x + BF * (y + BF * z);
#pragma unroll
    for (int e = 0; e < 27; ++e) {
      const int sx = e % 3 - 1, sy = (e / 3) % 3 - 1, sz = e / 9 - 1;
      if (!((exm >> gal_region(x + sx, y + sy, z + sz, BF)) & 1u)) continue;
      const float v = Jf[((long long)p * 27 + e) * FC + tf];
      gal_scatter(acc, cmask, v, cx + sx, cy + sy, cz + sz);
    }
  }
#pragma unroll
  for (int o = 0; o < 27; ++o) Jc[((long long)p * 27 + o) * HC + t] = acc[o];
}

// ---------------------------------------------------------------------------
// Linear union levels (27-point operator, FP32)
// ---------------------------------------------------------------------------
// b = -(R d) in FP32 and e = 0.
__global__ void __launch_bounds__(256) k_gal_rhs(long long n, const double* __restrict__ rd,
                                                 float* __restrict__ b, float* __restrict__ e) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    b[i] = (float)(-rd[i]);
    e[i] = 0.0f;
  }
}

// (J e)(cell t of patch p) without the centre term.
template <int B>
__device__ __forceinline__ float gal_offdiag(const float* __restrict__ J, const float* __restrict__ e,
                                             const int* __restrict__ nbr, int p, int i, int j,
                                             int k) {
  constexpr int BC = B * B * B;
  const int t = i + B * (j + B * k);
  float sum = 0.0f;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    if (o == 13) continue;
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    const float a = J[((long long)p * 27 + o) * BC + t];
    sum = fmaf(a, gal_fetch<B>(e, nbr, p, i + ox, j + oy, k + oz), sum);
  }
  return sum;
}

// One colour of eight-colour Gauss-Seidel on J e = b, block side B.
template <int B>
__global__ void __launch_bounds__(64) k_gal_smooth(const float* __restrict__ J,
                                                   const float* __restrict__ b,
                                                   float* __restrict__ e,
                                                   const int* __restrict__ nbr, int count,
                                                   int colour) {
  constexpr int H = B / 2, HC = H * H * H, BC = B * B * B;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)count * HC) return;
  const int p = (int)(g / HC), u = (int)(g % HC);
  const int i = 2 * (u % H) + (colour & 1);
  const int j = 2 * ((u / H) % H) + ((colour >> 1) & 1);
  const int k = 2 * (u / (H * H)) + (colour >> 2);
  const int t = i + B * (j + B * k);
  const float diag = J[((long long)p * 27 + 13) * BC + t];
  // a row whose assembled diagonal vanished (or is not finite) keeps its value
  if (!(fabsf(diag) > 0.f) || !isfinite(diag)) return;
  const float r = b[(long long)p * BC + t] - gal_offdiag<B>(J, e, nbr, p, i, j, k);
  e[(long long)p * BC + t] = r / diag;
}

// bc = R (b - J e) from block B to block B/2; one thread per coarse cell.
template <int B>
__global__ void __launch_bounds__(64) k_gal_resid_restrict(const float* __restrict__ J,
                                                           const float* __restrict__ b,
                                                           const float* __restrict__ e,
                                                           const int* __restrict__ nbr, int count,
                                                           float* __restrict__ bc,
                                                           float* __restrict__ ec) {
  constexpr int H = B / 2, HC = H * H * H, BC = B * B * B;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)count * HC) return;
  const int p = (int)(g / HC), u = (int)(g % HC);
  const int I = u % H, Jc = (u / H) % H, K = u / (H * H);
  float sum = 0.0f;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    const int i = 2 * I + (ch & 1), j = 2 * Jc + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
    const int t = i + B * (j + B * k);
    const float diag = J[((long long)p * 27 + 13) * BC + t];
    const float Je = fmaf(diag, e[(long long)p * BC + t], gal_offdiag<B>(J, e, nbr, p, i, j, k));
    sum += b[(long long)p * BC + t] - Je;
  }
  bc[g] = 0.125f * sum;
  ec[g] = 0.0f;
}

// out (block B) += theta P(ec) (block B/2), zero correction outside the union.
template <int B, typename T>
__global__ void __launch_bounds__(128) k_gal_prolong(const float* __restrict__ ec,
                                                     const int* __restrict__ nbr, int count,
                                                     T* __restrict__ out, float theta) {
  constexpr int H = B / 2, BC = B * B * B;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)count * BC) return;
  const int p = (int)(g / BC), t = (int)(g % BC);
  const int i = t % B, j = (t / B) % B, k = t / (B * B);
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = I0 + ((i & 1) ? 1 : -1), J1 = J0 + ((j & 1) ? 1 : -1), K1 = K0 + ((k & 1) ? 1 : -1);
  const float v = 27.0f * gal_fetch<H>(ec, nbr, p, I0, J0, K0) +
                  9.0f * (gal_fetch<H>(ec, nbr, p, I1, J0, K0) + gal_fetch<H>(ec, nbr, p, I0, J1, K0) +
                          gal_fetch<H>(ec, nbr, p, I0, J0, K1)) +
                  3.0f * (gal_fetch<H>(ec, nbr, p, I1, J1, K0) + gal_fetch<H>(ec, nbr, p, I1, J0, K1) +
                          gal_fetch<H>(ec, nbr, p, I0, J1, K1)) +
                  gal_fetch<H>(ec, nbr, p, I1, J1, K1);
  out[g] += (T)(v * (theta / 64.0f));
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static unsigned gal_blocks(long long items, int tpb) { return (unsigned)((items + tpb - 1) / tpb); }

mg_status galerkin_prepare(PatchLevel* pl) {
  if (pl->gJ[1]) return MG_OK;
  const size_t c = (size_t)(pl->count > 0 ? pl->count : 1);
  for (int m = 1; m < 3; ++m) {
    const size_t cells = c * (size_t)((8 >> m) * (8 >> m) * (8 >> m));
    if (cudaMalloc(&pl->gJ[m], sizeof(float) * 27 * cells) != cudaSuccess ||
        cudaMalloc(&pl->ge[m], sizeof(float) * cells) != cudaSuccess ||
        cudaMalloc(&pl->gb[m], sizeof(float) * cells) != cudaSuccess) {
      cudaGetLastError();
      set_error("refinement level: device allocation for the Galerkin correction failed");
      return MG_ENOMEM;
    }
  }
  return MG_OK;
}

void galerkin_release(PatchLevel* pl) {
  for (int m = 0; m < 3; ++m) {
    cudaFree(pl->gJ[m]);
    cudaFree(pl->ge[m]);
    cudaFree(pl->gb[m]);
    pl->gJ[m] = pl->ge[m] = pl->gb[m] = nullptr;
  }
}

static void gal_smooth(cudaStream_t st, PatchLevel* pl, int m, int sweeps) {
  const int P = pl->count;
  const long long per = (long long)P * ((8 >> m) * (8 >> m) * (8 >> m)) / 8;
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 8; ++colour) {
      if (m == 1)
        k_gal_smooth<4><<<gal_blocks(per, 64), 64, 0, st>>>(pl->gJ[1], pl->gb[1], pl->ge[1],
                                                            pl->d_nbr, P, colour);
      else
        k_gal_smooth<2><<<gal_blocks(per, 64), 64, 0, st>>>(pl->gJ[2], pl->gb[2], pl->ge[2],
                                                            pl->d_nbr, P, colour);
    }
  count_launches(8LL * sweeps);
}

static void gal_vcycle(cudaStream_t st, PatchLevel* pl, const mg_options& o, int m, int mlev) {
  const int P = pl->count;
  if (m == mlev - 1) {
    gal_smooth(st, pl, m, o.patch_coarse_sweeps);
    return;
  }
  gal_smooth(st, pl, m, o.nu_pre);
  // m == 1 here (the linear levels are 1 and 2)
  k_gal_resid_restrict<4><<<gal_blocks((long long)P * 8, 64), 64, 0, st>>>(
      pl->gJ[1], pl->gb[1], pl->ge[1], pl->d_nbr, P, pl->gb[2], pl->ge[2]);
  count_launches(1);
  gal_vcycle(st, pl, o, m + 1, mlev);
  k_gal_prolong<4, float><<<gal_blocks((long long)P * 64, 128), 128, 0, st>>>(
      pl->ge[2], pl->d_nbr, P, pl->ge[1], 1.0f);
  count_launches(1);
  gal_smooth(st, pl, m, o.nu_post);
}

// phi += theta P e_1 with e_1 the linear correction of the union's level 1: J_1
// assembled at the current iterate, right-hand side -R d (R d in rd, left by the
// residual restriction of the nonlinear union level), V-cycle over the linear
// union levels 1 .. mlev-1.
void galerkin_correction(cudaStream_t st, PatchLevel* pl, const mg_options& o,
                         const OpConst64& op0, const double* rd, int mlev) {
  const int P = pl->count;
  if (P == 0 || mlev < 2) return;
  k_gal_assemble0<<<P, 64, 0, st>>>(pl->phi, pl->src, pl->ghost, pl->d_nbr, op0, pl->gJ[1]);
  k_gal_rhs<<<gal_blocks((long long)P * 64, 256), 256, 0, st>>>((long long)P * 64, rd, pl->gb[1],
                                                                pl->ge[1]);
  count_launches(2);
  if (mlev > 2) {
    k_gal_assemble_lin<4><<<gal_blocks((long long)P * 8, 64), 64, 0, st>>>(pl->gJ[1], pl->d_nbr,
                                                                           P, pl->gJ[2]);
    count_launches(1);
  }
  gal_vcycle(st, pl, o, 1, mlev);
  k_gal_prolong<8, double><<<gal_blocks((long long)P * 512, 128), 128, 0, st>>>(
      pl->ge[1], pl->d_nbr, P, pl->phi, (float)o.patch_cgc);
  count_launches(1);
}

}  // namespace mg
