// Refinement levels: 8^3 patches solved with a coarse-to-fine Dirichlet fill
// (Sec. III.C first paragraph, Sec. IV.D of arXiv:1303.0008), by FAS multigrid on
// the union of the level's patches (Sec. III.C: multigrid on the refinements too).
//
// Layout: patch p of a level holds its 8^3 cells at phi[p*512 + i + 8(j + 8k)].
// A 27-entry table per patch gives the index of the patch in each neighbouring
// block (or -1).  Every kernel runs one CTA per patch and first loads the patch's
// ghosted tile, (b+2)^3 cells: the interior, neighbouring patches' cells, and
// for cells outside the union the fixed Dirichlet values.  The union coarsens
// per patch, 8^3 -> 4^3 -> 2^3 (union levels m = 0, 1, 2; cell size h_l 2^m).
//   m = 0 Dirichlet values: cell-centred trilinear interpolation of level l-1.
//   m >= 1 Dirichlet values: the cells of union level m sit exactly on cells of
//   level l-m (or, for m > l, of the domain restricted m-l times), whose values
//   are taken as they are.  The coarse levels only shape the correction, so any
//   fixed values keep the FAS scheme consistent; these are the closest to phi.
// The four-colour order uses level coordinates; origins are multiples of the
// block size, so local and global parities agree.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mg_internal.h"
#include "mg_patch_tile.cuh"
#include "mg_solver.h"

namespace mg {

#define PCK(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return MG_ECUDA;                                                       \
    }                                                                        \
  } while (0)

__device__ __forceinline__ int pwrap(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

// A field to take Dirichlet values from: a dense periodic n^3 array, or a patch
// set (8^3 blocks) with its block table.
struct FieldSrc {
  const double* dense;
  int n;                 // cells per side of the source's index space
  const double* pphi;    // patch set values
  const int* table;      // (n/8)^3 block -> patch or -1
  int* err;              // set to 1 when a needed cell is absent
};

__device__ __forceinline__ double fetch(const FieldSrc& s, int x, int y, int z) {
  x = pwrap(x, s.n);
  y = pwrap(y, s.n);
  z = pwrap(z, s.n);
  if (s.dense) return s.dense[lidx(x, y, z, s.n)];
  const int nb = s.n >> 3;
  const int q = s.table[(x >> 3) + nb * ((y >> 3) + nb * (z >> 3))];
  if (q < 0) {
    atomicExch(s.err, 1);
    return 0.0;
  }
  return s.pphi[(long long)q * 512 + (x & 7) + 8 * ((y & 7) + 8 * (z & 7))];
}

// ---------------------------------------------------------------------------
// Kernels (one CTA per patch)
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(128) k_patch_smooth(double* __restrict__ phi,
                                                      const double* __restrict__ src,
                                                      const double* __restrict__ f,
                                                      const double* __restrict__ ghost,
                                                      const int* __restrict__ nbr, OpConst64 c,
                                                      int colour) {
  constexpr int T = B + 2, BC = B * B * B;
  __shared__ double tile[T * T * T];
  const int p = blockIdx.x;
  load_tile<B>(tile, p, phi, ghost, nbr);
  __syncthreads();
  constexpr int H = B / 2;
  for (int t = threadIdx.x; t < H * H * B; t += blockDim.x) {
    const int m = t % H, jj = (t / H) % H, k = t / (H * H);
    const int i = 2 * m + ((colour ^ k) & 1);
    const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
    const long long id = (long long)p * BC + i + B * (j + B * k);
    const StencilT<double> s = gather_tile<B>(tile, i, j, k);
    bool g;
    const double D = root_D(s, src[id], c, g);
    const double rhs = f ? f[id] : 0.0;
    const double v = fma(-c.h2, D + rhs, s.sx + s.sy + s.sz) * (1.0 / 6.0);
    phi[id] = not_one(c.omega) ? fma(c.omega, v - tile_ctr<B>(tile, i, j, k),
                                     tile_ctr<B>(tile, i, j, k))
                               : v;
  }
}

// Residual d = L phi - f per cell of the union; with B > 2 also the restriction of
// phi and d to the union level below.  One partial per patch.
template <int B>
__global__ void __launch_bounds__(128) k_patch_residual_restrict(
    const double* __restrict__ phi, const double* __restrict__ src, const double* __restrict__ f,
    const double* __restrict__ ghost, const int* __restrict__ nbr, OpConst64 c,
    double* __restrict__ phi_c, double* __restrict__ phihat_c, double* __restrict__ rd_c,
    Partial* __restrict__ partials) {
  constexpr int T = B + 2, BC = B * B * B, H = B / 2, HC = H * H * H;
  __shared__ double tile[T * T * T];
  const int p = blockIdx.x;
  load_tile<B>(tile, p, phi, ghost, nbr);
  __syncthreads();
  Partial part;
  partial_init(part);
  if (phi_c) {
    for (int t = threadIdx.x; t < HC; t += blockDim.x) {
      const int I = t % H, J = (t / H) % H, K = t / (H * H);
      double sphi = 0.0, sd = 0.0;
#pragma unroll 1
      for (int ch = 0; ch < 8; ++ch) {
        const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
        const long long id = (long long)p * BC + i + B * (j + B * k);
        const StencilT<double> s = gather_tile<B>(tile, i, j, k);
        bool g;
        const double D = root_D(s, src[id], c, g);
        const double ctr = tile_ctr<B>(tile, i, j, k);
        double d = fma((s.sx + s.sy + s.sz) - 6.0 * ctr, c.inv_h2, -D);
        if (f) d -= f[id];
        partial_add(part, d, g);
        sphi += ctr;
        sd += d;
      }
      const long long cid = (long long)p * HC + t;
      phi_c[cid] = sphi * 0.125;
      phihat_c[cid] = sphi * 0.125;
      rd_c[cid] = sd * 0.125;
    }
  } else {
    for (int t = threadIdx.x; t < BC; t += blockDim.x) {
      const int i = t % B, j = (t / B) % B, k = t / (B * B);
      const long long id = (long long)p * BC + t;
      const StencilT<double> s = gather_tile<B>(tile, i, j, k);
      bool g;
      const double D = root_D(s, src[id], c, g);
      double d = fma((s.sx + s.sy + s.sz) - 6.0 * tile_ctr<B>(tile, i, j, k), c.inv_h2, -D);
      if (f) d -= f[id];
      partial_add(part, d, g);
    }
  }
  part = block_reduce(part);
  if (threadIdx.x == 0) partials[p] = part;
}

// f^H = L^H(R phi) - R d on union level with block B (no compatibility constant).
template <int B>
__global__ void __launch_bounds__(128) k_patch_fas_rhs(const double* __restrict__ phi,
                                                       const double* __restrict__ src,
                                                       double* __restrict__ f,
                                                       const double* __restrict__ ghost,
                                                       const int* __restrict__ nbr, OpConst64 c) {
  constexpr int T = B + 2, BC = B * B * B;
  __shared__ double tile[T * T * T];
  const int p = blockIdx.x;
  load_tile<B>(tile, p, phi, ghost, nbr);
  __syncthreads();
  for (int t = threadIdx.x; t < BC; t += blockDim.x) {
    const int i = t % B, j = (t / B) % B, k = t / (B * B);
    const long long id = (long long)p * BC + t;
    const StencilT<double> s = gather_tile<B>(tile, i, j, k);
    bool g;
    const double D = root_D(s, src[id], c, g);
    const double L = fma((s.sx + s.sy + s.sz) - 6.0 * tile_ctr<B>(tile, i, j, k), c.inv_h2, -D);
    f[id] = L - f[id];
  }
}

// phi (block B) += P(phi_c - phihat_c) (block B/2); the correction is zero at the
// fixed Dirichlet cells outside the union.
template <int B>
__global__ void __launch_bounds__(128) k_patch_prolong(const double* __restrict__ phi_c,
                                                       const double* __restrict__ phihat_c,
                                                       const int* __restrict__ nbr,
                                                       double* __restrict__ phi, double theta) {
  constexpr int H = B / 2, HT = H + 2, HC = H * H * H, BC = B * B * B;
  __shared__ double corr[HT * HT * HT];
  const int p = blockIdx.x;
  for (int q = threadIdx.x; q < HT * HT * HT; q += blockDim.x) {
    const int i = q % HT - 1, j = (q / HT) % HT - 1, k = q / (HT * HT) - 1;
    const int ox = i < 0 ? -1 : (i >= H ? 1 : 0);
    const int oy = j < 0 ? -1 : (j >= H ? 1 : 0);
    const int oz = k < 0 ? -1 : (k >= H ? 1 : 0);
    const int nb = ((ox | oy | oz) == 0) ? p : nbr[p * 27 + (ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1))];
    double v = 0.0;
    if (nb >= 0) {
      const long long id = (long long)nb * HC + (i - ox * H) + H * ((j - oy * H) + H * (k - oz * H));
      v = phi_c[id] - phihat_c[id];
    }
    corr[q] = v;
  }
  __syncthreads();
  auto e = [&](int a, int b, int cc) { return corr[(a + 1) + HT * ((b + 1) + HT * (cc + 1))]; };
  for (int t = threadIdx.x; t < BC; t += blockDim.x) {
    const int i = t % B, j = (t / B) % B, k = t / (B * B);
    const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
    const int I1 = I0 + ((i & 1) ? 1 : -1), J1 = J0 + ((j & 1) ? 1 : -1), K1 = K0 + ((k & 1) ? 1 : -1);
    const double v = 27.0 * e(I0, J0, K0) + 9.0 * (e(I1, J0, K0) + e(I0, J1, K0) + e(I0, J0, K1)) +
                     3.0 * (e(I1, J1, K0) + e(I1, J0, K1) + e(I0, J1, K1)) + e(I1, J1, K1);
    phi[(long long)p * BC + t] += v * (theta / 64.0);
  }
}

// Dirichlet values of the ghost shell of every patch at block B.  scale = 2^m
// (union level m of a level whose index space has side nside).  m == 0: trilinear
// interpolation of the parent level (side nside/2); m >= 1: the source cell
// (side nside >> m) as it is.  Cells inside a neighbouring patch and the corners
// are left as they are.
template <int B>
__global__ void __launch_bounds__(128) k_patch_ghosts(const int* __restrict__ origin,
                                                      const int* __restrict__ nbr, int m,
                                                      FieldSrc src, double* __restrict__ ghost) {
  constexpr int T = B + 2, TC = T * T * T;
  const int p = blockIdx.x;
  const int ox0 = origin[3 * p] >> m, oy0 = origin[3 * p + 1] >> m, oz0 = origin[3 * p + 2] >> m;
  for (int q = threadIdx.x; q < TC; q += blockDim.x) {
    const int i = q % T - 1, j = (q / T) % T - 1, k = q / (T * T) - 1;
    const int ox = i < 0 ? -1 : (i >= B ? 1 : 0);
    const int oy = j < 0 ? -1 : (j >= B ? 1 : 0);
    const int oz = k < 0 ? -1 : (k >= B ? 1 : 0);
    const int nout = (ox != 0) + (oy != 0) + (oz != 0);
    if (nout == 0 || nout == 3) continue;
    if (nbr[p * 27 + (ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1))] >= 0) continue;
    const int x = ox0 + i, y = oy0 + j, z = oz0 + k;
    double v;
    if (m == 0) {
      const int X = x >> 1, Y = y >> 1, Z = z >> 1;
      const int sX = (x & 1) ? 1 : -1, sY = (y & 1) ? 1 : -1, sZ = (z & 1) ? 1 : -1;
      v = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int cc = 0; cc < 2; ++cc) {
            const double wt = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (cc ? 0.25 : 0.75);
            v += wt * fetch(src, X + a * sX, Y + b * sY, Z + cc * sZ);
          }
    } else {
      v = fetch(src, x, y, z);
    }
    ghost[(long long)p * TC + q] = v;
  }
}

// Initial guess of a refinement level: every patch cell takes the cell-centred
// trilinear interpolation of the parent level (the values the coarse-to-fine
// fill gives its ghost cells), as a new refinement inherits the coarse solution.
__global__ void __launch_bounds__(128) k_patch_init(const int* __restrict__ origin, FieldSrc src,
                                                    double* __restrict__ phi) {
  const int p = blockIdx.x;
  const int ox0 = origin[3 * p], oy0 = origin[3 * p + 1], oz0 = origin[3 * p + 2];
  for (int t = threadIdx.x; t < 512; t += blockDim.x) {
    const int x = ox0 + (t & 7), y = oy0 + ((t >> 3) & 7), z = oz0 + (t >> 6);
    const int X = x >> 1, Y = y >> 1, Z = z >> 1;
    const int sX = (x & 1) ? 1 : -1, sY = (y & 1) ? 1 : -1, sZ = (z & 1) ? 1 : -1;
    double v = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int cc = 0; cc < 2; ++cc) {
          const double wt = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (cc ? 0.25 : 0.75);
          v += wt * fetch(src, X + a * sX, Y + b * sY, Z + cc * sZ);
        }
    phi[(long long)p * 512 + t] = v;
  }
}

// Mean of the 8 children within each patch (block B -> B/2).
template <int B>
__global__ void __launch_bounds__(128) k_patch_restrict(const double* __restrict__ fine,
                                                        double* __restrict__ coarse) {
  constexpr int H = B / 2, HC = H * H * H, BC = B * B * B;
  const int p = blockIdx.x;
  for (int t = threadIdx.x; t < HC; t += blockDim.x) {
    const int I = t % H, J = (t / H) % H, K = t / (H * H);
    double s = 0.0;
    for (int ch = 0; ch < 8; ++ch)
      s += fine[(long long)p * BC + (2 * I + (ch & 1)) + B * ((2 * J + ((ch >> 1) & 1)) + B * (2 * K + (ch >> 2)))];
    coarse[(long long)p * HC + t] = s * 0.125;
  }
}

// -(1/2) grad phi on the patches (8^3), SoA over count*512 cells.
__global__ void __launch_bounds__(128) k_patch_force(const double* __restrict__ phi,
                                                     const double* __restrict__ ghost,
                                                     const int* __restrict__ nbr, double inv2h,
                                                     long long total, double* __restrict__ out) {
  constexpr int B = 8, T = 10;
  __shared__ double tile[T * T * T];
  const int p = blockIdx.x;
  load_tile<B>(tile, p, phi, ghost, nbr);
  __syncthreads();
  auto at = [&](int a, int b, int c) { return tile[(a + 1) + T * ((b + 1) + T * (c + 1))]; };
  for (int t = threadIdx.x; t < 512; t += blockDim.x) {
    const int i = t % 8, j = (t / 8) % 8, k = t / 64;
    const long long id = (long long)p * 512 + t;
    out[id] = -0.5 * inv2h * (at(i + 1, j, k) - at(i - 1, j, k));
    out[total + id] = -0.5 * inv2h * (at(i, j + 1, k) - at(i, j - 1, k));
    out[2 * total + id] = -0.5 * inv2h * (at(i, j, k + 1) - at(i, j, k - 1));
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int block_of(int m) { return 8 >> m; }

template <typename K0, typename K1, typename K2>
static void dispatch(int m, K0 k0, K1 k1, K2 k2) {
  if (m == 0) k0();
  else if (m == 1) k1();
  else k2();
}

void patch_level_destroy(PatchLevel* pl) {
  if (!pl) return;
  cudaFree(pl->d_origin);
  cudaFree(pl->d_nbr);
  cudaFree(pl->phi);
  cudaFree(pl->delta);
  cudaFree(pl->src);
  cudaFree(pl->ghost);
  cudaFree(pl->d_table);
  for (int m = 0; m < 3; ++m) {
    cudaFree(pl->phi_c[m]);
    cudaFree(pl->phihat_c[m]);
    cudaFree(pl->f_c[m]);
    cudaFree(pl->src_c[m]);
    cudaFree(pl->delta_c[m]);
    cudaFree(pl->ghost_c[m]);
  }
  cudaFree(pl->d_sc);
  if (pl->h_sc) cudaFreeHost(pl->h_sc);
  cudaFree(pl->d_part);
  cudaFree(pl->d_err);
  cudaFree(pl->d_coarse_parent);
  galerkin_release(pl);
  delete pl;
}

mg_status patches_add(mg_grid* g, int level, int count, const int* origin) {
  if (level < 1 || level > 2) {
    set_error("mg_add_patches: level must be 1 or 2");
    return MG_EINVAL;
  }
  if (count < 0 || (count > 0 && !origin)) {
    set_error("mg_add_patches: bad count or NULL origins");
    return MG_EINVAL;
  }
  if (level == 2 && ((int)g->patch_levels.size() < 1 || !g->patch_levels[0] ||
                     g->patch_levels[0]->count == 0)) {
    set_error("mg_add_patches: level 2 needs level-1 patches first");
    return MG_ESTATE;
  }
  const int n0 = g->domains[0]->n;
  const int nside = n0 << level;
  const int nb = nside / 8;
  std::vector<int> table((size_t)nb * nb * nb, -1);
  for (int p = 0; p < count; ++p) {
    const int x = origin[3 * p], y = origin[3 * p + 1], z = origin[3 * p + 2];
    if (x < 0 || y < 0 || z < 0 || x >= nside || y >= nside || z >= nside || (x % 8) ||
        (y % 8) || (z % 8)) {
      set_error("mg_add_patches: origins must be multiples of 8 inside the level");
      return MG_EINVAL;
    }
    int& slot = table[(size_t)(x / 8) + nb * ((size_t)(y / 8) + nb * (size_t)(z / 8))];
    if (slot >= 0) {
      set_error("mg_add_patches: duplicate patch");
      return MG_EINVAL;
    }
    slot = p;
  }
  if ((int)g->patch_levels.size() < level) g->patch_levels.resize(level, nullptr);
  if (g->patch_levels[level - 1]) {
    cudaStreamSynchronize(g->stream);
    patch_level_destroy(g->patch_levels[level - 1]);
    g->patch_levels[level - 1] = nullptr;
  }
  // a level-1 change invalidates level 2 (its nesting and Dirichlet source)
  if (level == 1 && g->patch_levels.size() > 1 && g->patch_levels[1]) {
    patch_level_destroy(g->patch_levels[1]);
    g->patch_levels[1] = nullptr;
  }
  PatchLevel* pl = new (std::nothrow) PatchLevel();
  if (!pl) {
    set_error("host allocation");
    return MG_ENOMEM;
  }
  pl->level = level;
  pl->count = count;
  pl->nside = nside;
  pl->h_origin.assign(origin, origin + 3 * count);
  std::vector<int> nbr((size_t)27 * std::max(count, 1), -1);
  for (int p = 0; p < count; ++p) {
    const int bx = origin[3 * p] / 8, by = origin[3 * p + 1] / 8, bz = origin[3 * p + 2] / 8;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int X = (bx + dx + nb) % nb, Y = (by + dy + nb) % nb, Z = (bz + dz + nb) % nb;
          nbr[(size_t)p * 27 + (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1))] =
              table[(size_t)X + nb * ((size_t)Y + nb * (size_t)Z)];
        }
  }
  const size_t c = (size_t)std::max(count, 1);
  bool ok = true;
  ok = ok && cudaMalloc(&pl->d_origin, sizeof(int) * 3 * c) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->d_nbr, sizeof(int) * 27 * c) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->d_table, sizeof(int) * table.size()) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->phi, sizeof(double) * 512 * c) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->delta, sizeof(double) * 512 * c) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->src, sizeof(double) * 512 * c) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->ghost, sizeof(double) * 1000 * c) == cudaSuccess;
  for (int m = 1; m < 3; ++m) {
    const int b = block_of(m);
    const size_t cells = (size_t)b * b * b * c, tc = (size_t)(b + 2) * (b + 2) * (b + 2) * c;
    ok = ok && cudaMalloc(&pl->phi_c[m], sizeof(double) * cells) == cudaSuccess;
    ok = ok && cudaMalloc(&pl->phihat_c[m], sizeof(double) * cells) == cudaSuccess;
    ok = ok && cudaMalloc(&pl->f_c[m], sizeof(double) * cells) == cudaSuccess;
    ok = ok && cudaMalloc(&pl->src_c[m], sizeof(double) * cells) == cudaSuccess;
    ok = ok && cudaMalloc(&pl->delta_c[m], sizeof(double) * cells) == cudaSuccess;
    ok = ok && cudaMalloc(&pl->ghost_c[m], sizeof(double) * tc) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&pl->d_sc, sizeof(LevelScalars) * 4) == cudaSuccess;
  ok = ok && cudaMallocHost(&pl->h_sc, sizeof(LevelScalars)) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->d_part, sizeof(Partial) * c) == cudaSuccess;
  ok = ok && cudaMalloc(&pl->d_err, sizeof(int)) == cudaSuccess;
  if (level == 1) {
    const size_t half = (size_t)(n0 / 2) * (n0 / 2) * (n0 / 2);
    ok = ok && cudaMalloc(&pl->d_coarse_parent, sizeof(double) * half) == cudaSuccess;
  }
  if (!ok) {
    patch_level_destroy(pl);
    set_error("mg_add_patches: device allocation failed");
    return MG_ENOMEM;
  }
  cudaMemcpy(pl->d_origin, origin, sizeof(int) * 3 * count, cudaMemcpyHostToDevice);
  cudaMemcpy(pl->d_nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(pl->d_table, table.data(), sizeof(int) * table.size(), cudaMemcpyHostToDevice);
  cudaMemset(pl->phi, 0, sizeof(double) * 512 * c);
  cudaMemset(pl->delta, 0, sizeof(double) * 512 * c);
  cudaMemset(pl->ghost, 0, sizeof(double) * 1000 * c);
  for (int m = 1; m < 3; ++m) {
    const int b = block_of(m);
    cudaMemset(pl->ghost_c[m], 0, sizeof(double) * (b + 2) * (b + 2) * (b + 2) * c);
  }
  PCK(cudaDeviceSynchronize());
  g->patch_levels[level - 1] = pl;
  return MG_OK;
}

// Restrict the patch density to the union's coarse levels.
void patch_restrict_density(mg_grid* g, PatchLevel* pl) {
  if (pl->count == 0) return;
  k_patch_restrict<8><<<pl->count, 128, 0, g->stream>>>(pl->delta, pl->delta_c[1]);
  k_patch_restrict<4><<<pl->count, 128, 0, g->stream>>>(pl->delta_c[1], pl->delta_c[2]);
  count_launches(2);
}

struct PatchCycle {
  PatchLevel* pl;
  const mg_options* o;
  cudaStream_t st;
  OpConst64 ops[3];

  double* phi(int m) const { return m == 0 ? pl->phi : pl->phi_c[m]; }
  double* src(int m) const { return m == 0 ? pl->src : pl->src_c[m]; }
  double* f(int m) const { return m == 0 ? nullptr : pl->f_c[m]; }
  double* ghost(int m) const { return m == 0 ? pl->ghost : pl->ghost_c[m]; }

  void smooth(int m, int sweeps) const {
    const int P = pl->count;
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour) {
        dispatch(
            m,
            [&] { k_patch_smooth<8><<<P, 128, 0, st>>>(phi(0), src(0), f(0), ghost(0), pl->d_nbr, ops[0], colour); },
            [&] { k_patch_smooth<4><<<P, 128, 0, st>>>(phi(1), src(1), f(1), ghost(1), pl->d_nbr, ops[1], colour); },
            [&] { k_patch_smooth<2><<<P, 128, 0, st>>>(phi(2), src(2), f(2), ghost(2), pl->d_nbr, ops[2], colour); });
      }
    count_launches(4LL * sweeps);
  }

  // residual of union level m (restricted to m+1 when m < 2) and its scalars
  void residual(int m, bool restrict_down) const {
    const int P = pl->count;
    if (restrict_down) {
      dispatch(
          m,
          [&] { k_patch_residual_restrict<8><<<P, 128, 0, st>>>(phi(0), src(0), f(0), ghost(0), pl->d_nbr, ops[0], phi(1), pl->phihat_c[1], pl->f_c[1], pl->d_part); },
          [&] { k_patch_residual_restrict<4><<<P, 128, 0, st>>>(phi(1), src(1), f(1), ghost(1), pl->d_nbr, ops[1], phi(2), pl->phihat_c[2], pl->f_c[2], pl->d_part); },
          [&] {});
    } else {
      dispatch(
          m,
          [&] { k_patch_residual_restrict<8><<<P, 128, 0, st>>>(phi(0), src(0), f(0), ghost(0), pl->d_nbr, ops[0], nullptr, nullptr, nullptr, pl->d_part); },
          [&] { k_patch_residual_restrict<4><<<P, 128, 0, st>>>(phi(1), src(1), f(1), ghost(1), pl->d_nbr, ops[1], nullptr, nullptr, nullptr, pl->d_part); },
          [&] { k_patch_residual_restrict<2><<<P, 128, 0, st>>>(phi(2), src(2), f(2), ghost(2), pl->d_nbr, ops[2], nullptr, nullptr, nullptr, pl->d_part); });
    }
    count_launches(1);
    launch_finalize(st, pl->d_part, P, (double)P * 512.0, 0, pl->d_sc + m);
  }

  void fas_rhs(int m) const {
    const int P = pl->count;
    dispatch(
        m, [&] {},
        [&] { k_patch_fas_rhs<4><<<P, 128, 0, st>>>(phi(1), src(1), pl->f_c[1], ghost(1), pl->d_nbr, ops[1]); },
        [&] { k_patch_fas_rhs<2><<<P, 128, 0, st>>>(phi(2), src(2), pl->f_c[2], ghost(2), pl->d_nbr, ops[2]); });
    count_launches(1);
  }

  void prolong(int m) const {  // from m+1 to m
    const int P = pl->count;
    dispatch(
        m,
        [&] { k_patch_prolong<8><<<P, 128, 0, st>>>(phi(1), pl->phihat_c[1], pl->d_nbr, phi(0), o->patch_cgc); },
        [&] { k_patch_prolong<4><<<P, 128, 0, st>>>(phi(2), pl->phihat_c[2], pl->d_nbr, phi(1), o->patch_cgc); },
        [&] {});
    count_launches(1);
  }

  int mlev() const { return o->patch_mg_levels; }

  void descend(int m) const {
    if (m == mlev() - 1) {
      smooth(m, o->patch_coarse_sweeps);
      return;
    }
    smooth(m, o->nu_pre);
    residual(m, true);
    fas_rhs(m + 1);
    descend(m + 1);
    prolong(m);
    smooth(m, o->nu_post);
  }

  void part_a() const {
    smooth(0, o->nu_pre);
    residual(0, mlev() > 1);
    cudaMemcpyAsync(pl->h_sc, pl->d_sc, sizeof(LevelScalars), cudaMemcpyDeviceToHost, st);
  }

  void part_b() const {
    if (mlev() > 1 && o->patch_galerkin) {
      // linear correction with Galerkin coarse operators; f_c[1] holds R d
      galerkin_correction(st, pl, *o, ops[0], pl->f_c[1], mlev());
    } else if (mlev() > 1) {
      fas_rhs(1);
      descend(1);
      prolong(0);
    }
    smooth(0, o->nu_post);
  }
};

static FieldSrc dense_src(const double* a, int n, int* err) {
  return FieldSrc{a, n, nullptr, nullptr, err};
}

mg_status patch_level_solve(mg_grid* g, int level, int branch, double alpha, double kappa,
                            double tol, bool init_from_parent) {
  PatchLevel* pl = g->patch_levels[level - 1];
  cudaStream_t st = g->stream;
  const int P = pl->count;
  if (P == 0) return MG_OK;
  Domain* d0 = g->domains[0];
  const int n0 = d0->n;
  PatchCycle cyc{pl, &g->opt, st, {}};
  for (int m = 0; m < 3; ++m) {
    cyc.ops[m] = make_op64(pl->nside >> m, alpha, kappa, branch);
    cyc.ops[m].omega = g->opt.omega_patch;
    double a, b;
    src_coefficients(cyc.ops[m], kappa, &a, &b);
    const int bm = block_of(m);
    launch_affine64(st, (long long)P * bm * bm * bm, m == 0 ? pl->delta : pl->delta_c[m],
                    cyc.src(m), a, b, cyc.ops[m].c3,
                    g->opt.guard == MG_GUARD_FLOOR && cyc.ops[m].mode != OP_LINEAR, nullptr);
  }
  // Dirichlet values
  PCK(cudaMemsetAsync(pl->d_err, 0, sizeof(int), st));
  PatchLevel* parent = level == 2 ? g->patch_levels[0] : nullptr;
  const FieldSrc parent_src =
      level == 1 ? dense_src(d0->lv[0].phi, n0, pl->d_err)
                 : FieldSrc{nullptr, parent->nside, parent->phi, parent->d_table, pl->d_err};
  k_patch_ghosts<8><<<P, 128, 0, st>>>(pl->d_origin, pl->d_nbr, 0, parent_src, pl->ghost);
  if (init_from_parent) {
    k_patch_init<<<P, 128, 0, st>>>(pl->d_origin, parent_src, pl->phi);
    count_launches(1);
  }
  // union level m sits on level (level - m): level 0 dense, level 1 patches, or the
  // domain restricted once (m = 2 of level 1)
  for (int m = 1; m < 3; ++m) {
    FieldSrc s;
    const int on = level - m;
    if (on == 0) {
      s = dense_src(d0->lv[0].phi, n0, pl->d_err);
    } else if (on == 1) {
      s = FieldSrc{nullptr, parent->nside, parent->phi, parent->d_table, pl->d_err};
    } else {
      PatchLevel* l1 = g->patch_levels[0];
      launch_restrict64(st, n0 / 2, d0->lv[0].phi, l1->d_coarse_parent);
      s = dense_src(l1->d_coarse_parent, n0 / 2, pl->d_err);
    }
    if (m == 1)
      k_patch_ghosts<4><<<P, 128, 0, st>>>(pl->d_origin, pl->d_nbr, m, s, pl->ghost_c[1]);
    else
      k_patch_ghosts<2><<<P, 128, 0, st>>>(pl->d_origin, pl->d_nbr, m, s, pl->ghost_c[2]);
  }
  count_launches(3);
  int herr = 0;
  PCK(cudaMemcpyAsync(&herr, pl->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PCK(cudaStreamSynchronize(st));
  PCK(cudaGetLastError());
  if (herr) {
    set_error("refinement level " + std::to_string(level) +
              ": a Dirichlet value needs a parent cell that is not refined (proper nesting)");
    return MG_EINVAL;
  }
  if (g->opt.patch_galerkin && g->opt.patch_mg_levels > 1) {
    mg_status gs = galerkin_prepare(pl);
    if (gs != MG_OK) return gs;
  }
  cudaEvent_t w0 = nullptr, w1 = nullptr;
  PCK(cudaEventCreate(&w0));
  PCK(cudaEventCreate(&w1));
  PCK(cudaEventRecord(w0, st));
  // V-cycles on the union
  long long na = 0, nb = 0;
  cudaGraphExec_t ga = nullptr, gb = nullptr;
  if (g->opt.use_graphs) {
    ga = capture_graph(st, &na, [&] { cyc.part_a(); });
    gb = capture_graph(st, &nb, [&] { cyc.part_b(); });
  }
  const bool graphs = ga && gb;
  mg_status result = MG_OK;
  double first = -1.0;
  std::vector<double> hist;
  for (int cycle = 0;; ++cycle) {
    if (graphs) {
      PCK(cudaGraphLaunch(ga, st));
      tl_launches += na;
    } else {
      cyc.part_a();
    }
    PCK(cudaStreamSynchronize(st));
    PCK(cudaGetLastError());
    const double res = pl->h_sc[0].res;
    hist.push_back(res);
    if (first < 0) first = res;
    if (!(res == res)) {
      set_error("refinement level: residual is not finite");
      result = MG_ENAN;
      break;
    }
    if (res < tol) break;
    if (cycle >= g->opt.max_cycles || res > 1e3 * first ||
        (hist.size() > 8 && res > 0.9 * hist[hist.size() - 9])) {
      set_error("refinement level " + std::to_string(level) + ": no convergence");
      result = MG_ENOCONV;
      break;
    }
    if (graphs) {
      PCK(cudaGraphLaunch(gb, st));
      tl_launches += nb;
    } else {
      cyc.part_b();
    }
  }
  if (cudaEventRecord(w1, st) == cudaSuccess && cudaEventSynchronize(w1) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w0, w1);
    pl->last_wall_s = ms * 1e-3;
  }
  cudaEventDestroy(w0);
  cudaEventDestroy(w1);
  pl->last_cycles = (int)hist.size() - 1;
  pl->last_res = hist.empty() ? 0.0 : hist.back();
  pl->last_status = result;
  pl->last_hist = hist;
  if (result == MG_ENOCONV) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), " after %d cycles (residual %.3e -> %.3e)", (int)hist.size() - 1,
                  first, hist.empty() ? 0.0 : hist.back());
    set_error("refinement level " + std::to_string(level) + ": no convergence" + buf);
  }
  if (ga) cudaGraphExecDestroy(ga);
  if (gb) cudaGraphExecDestroy(gb);
  return result;
}

mg_status patch_force(mg_grid* g, int level, int patch, double* out) {
  PatchLevel* pl = g->patch_levels[level - 1];
  const long long total = (long long)pl->count * 512;
  if (patch < 0) {
    k_patch_force<<<pl->count, 128, 0, g->stream>>>(pl->phi, pl->ghost, pl->d_nbr,
                                                    0.5 * (double)pl->nside, total, out);
    count_launches(1);
    return MG_OK;
  }
  // one patch: compute all, then gather its 3 x 512 values
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(double) * 3 * total) != cudaSuccess) {
    set_error("mg_get_force: device allocation");
    return MG_ENOMEM;
  }
  k_patch_force<<<pl->count, 128, 0, g->stream>>>(pl->phi, pl->ghost, pl->d_nbr,
                                                  0.5 * (double)pl->nside, total, tmp);
  count_launches(1);
  for (int a = 0; a < 3; ++a)
    cudaMemcpyAsync(out + a * 512, tmp + a * total + (long long)patch * 512, sizeof(double) * 512,
                    cudaMemcpyDeviceToDevice, g->stream);
  cudaStreamSynchronize(g->stream);
  cudaFree(tmp);
  return MG_OK;
}

}  // namespace mg
