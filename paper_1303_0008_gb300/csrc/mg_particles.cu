// Particles to mesh (Sec. VI: the density on the mesh is obtained by assigning
// particles with the triangular-shaped-cloud scheme) and the refinement
// criterion on effective particle counts (Sec. III.B: a cell is refined when
// the effective number of particles in it exceeds N_pc).
//
// One thread per particle adds m W / h^3 to the 27 (TSC) or 8 (CIC) nearest
// cells of a periodic cell-centred grid with FP64 atomics; on a refinement
// level only the cells that belong to a patch receive mass.  The order of the
// atomic additions is not fixed, so the last bits of a cell's density can
// differ between runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

namespace {

// Where the mass goes: a dense nside^3 grid (table == nullptr) or the packed
// 8^3 patches of a level whose block table maps (x/8, y/8, z/8) to a patch.
struct MassGrid {
  double* rho;
  int nside;
  const int* table;
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// S = 1: cloud in cell, W(u) = 1 - |u|; S = 2: triangular-shaped cloud,
// W(u) = 3/4 - u^2 (|u| <= 1/2), (3/2 - |u|)^2 / 2 (1/2 < |u| < 3/2).
template <int S>
__global__ void __launch_bounds__(256) k_assign(long long count, const double* __restrict__ px,
                                                const double* __restrict__ py,
                                                const double* __restrict__ pz,
                                                const double* __restrict__ mass, double m_default,
                                                MassGrid G) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int n = G.nside;
  double pos[3] = {px[p], py[p], pz[p]};
  // periodic: fold into [0, 1); a particle with a non-finite coordinate adds nothing
  if (!(isfinite(pos[0]) && isfinite(pos[1]) && isfinite(pos[2]))) return;
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] -= floor(pos[a]);
  double w[3][3];
  int c0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double s = pos[a] * n - 0.5;  // position in units of cells from the first centre
    if (S == 2) {
      const double c = floor(s + 0.5);  // nearest centre, offset d in [-1/2, 1/2)
      const double d = s - c;
      c0[a] = (int)c - 1;
      w[a][0] = 0.5 * (0.5 - d) * (0.5 - d);
      w[a][1] = 0.75 - d * d;
      w[a][2] = 0.5 * (0.5 + d) * (0.5 + d);
    } else {
      const double c = floor(s);  // centre below, offset d in [0, 1)
      const double d = s - c;
      c0[a] = (int)c;
      w[a][0] = 1.0 - d;
      w[a][1] = d;
      w[a][2] = 0.0;
    }
    c0[a] = ((c0[a] % n) + n) % n;
  }
  const double m = (mass ? mass[p] : m_default) * (double)n * n * n;
  constexpr int NW = S == 2 ? 3 : 2;
#pragma unroll
  for (int dk = 0; dk < NW; ++dk)
#pragma unroll
    for (int dj = 0; dj < NW; ++dj)
#pragma unroll
      for (int di = 0; di < NW; ++di) {
        const int i = wrapi(c0[0] + di, n), j = wrapi(c0[1] + dj, n), k = wrapi(c0[2] + dk, n);
        const double v = m * (w[0][di] * w[1][dj] * w[2][dk]);
        long long idx;
        if (G.table) {
          const int nb = n >> 3;
          const int q = G.table[(i >> 3) + nb * ((j >> 3) + nb * (k >> 3))];
          if (q < 0) continue;
          idx = (long long)q * 512 + (i & 7) + 8 * ((j & 7) + 8 * (k & 7));
        } else {
          idx = (long long)i + (long long)n * (j + (long long)n * k);
        }
        atomicAdd(G.rho + idx, v);
      }
}

__global__ void __launch_bounds__(256) k_add_const(long long cells, double* __restrict__ x,
                                                   double c) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cells) x[t] += c;
}

// One flag per 4^3 block: 1 when a cell of the block has 1 + delta > limit.
// Dense level (table == nullptr): blocks of the nside^3 grid, x fastest.
// Patch level: 8 blocks per patch, patch-major, block (bx, by, bz) -> bx + 2(by + 2 bz).
__global__ void __launch_bounds__(64) k_flag_blocks(const double* __restrict__ delta, int n,
                                                    int patches, double limit,
                                                    int* __restrict__ flags) {
  const long long b = blockIdx.x;
  const int t = threadIdx.x;  // cell of the block: (t & 3, (t >> 2) & 3, t >> 4)
  long long idx;
  if (patches) {
    const long long q = b >> 3;
    const int lb = (int)(b & 7);
    const int x = 4 * (lb & 1) + (t & 3), y = 4 * ((lb >> 1) & 1) + ((t >> 2) & 3),
              z = 4 * (lb >> 2) + (t >> 4);
    idx = q * 512 + x + 8 * (y + 8 * z);
  } else {
    const int nb = n >> 2;
    const long long bx = b % nb, by = (b / nb) % nb, bz = b / ((long long)nb * nb);
    idx = (4 * bx + (t & 3)) + (long long)n * ((4 * by + ((t >> 2) & 3)) +
                                               (long long)n * (4 * bz + (t >> 4)));
  }
  const int hot = (1.0 + delta[idx]) > limit;
  const int any = __syncthreads_or(hot);
  if (t == 0) flags[b] = any;
}

unsigned blocks_of(long long work, int threads) {
  return (unsigned)((work + threads - 1) / threads);
}

}  // namespace

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_assign_density(mg_grid* g, int level, int scheme, long long count, const double* pos,
                            const double* mass, int on_device) {
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_assign_density: needs a domain handle");
  if (scheme != MG_CIC && scheme != MG_TSC) MG_FAIL(MG_EINVAL, "mg_assign_density: scheme");
  if (count <= 0 || !pos) MG_FAIL(MG_EINVAL, "mg_assign_density: no particles");
  MassGrid G{nullptr, 0, nullptr};
  size_t cells = 0;
  PatchLevel* pl = nullptr;
  if (level == 0) {
    Domain* d = g->domains[0];
    G = MassGrid{d->lv[0].delta, d->n, nullptr};
    cells = (size_t)d->lv[0].cells;
  } else {
    if (level < 1 || level > (int)g->patch_levels.size() || !g->patch_levels[level - 1] ||
        g->patch_levels[level - 1]->count == 0)
      MG_FAIL(MG_EINVAL, "mg_assign_density: no patches on that level");
    pl = g->patch_levels[level - 1];
    G = MassGrid{pl->delta, pl->nside, pl->d_table};
    cells = (size_t)pl->count * 512;
  }
  const double* dpos = pos;
  const double* dmass = mass;
  double* tmp = nullptr;
  if (!on_device) {
    const size_t np = (size_t)count * (mass ? 4 : 3);
    if (cudaMalloc(&tmp, sizeof(double) * np) != cudaSuccess)
      MG_FAIL(MG_ENOMEM, "mg_assign_density: device allocation");
    cudaMemcpyAsync(tmp, pos, sizeof(double) * 3 * count, cudaMemcpyHostToDevice, g->stream);
    if (mass)
      cudaMemcpyAsync(tmp + 3 * count, mass, sizeof(double) * count, cudaMemcpyHostToDevice,
                      g->stream);
    dpos = tmp;
    dmass = mass ? tmp + 3 * count : nullptr;
  }
  const cudaError_t ez = cudaMemsetAsync(G.rho, 0, sizeof(double) * cells, g->stream);
  if (ez != cudaSuccess) {
    if (tmp) cudaFree(tmp);
    MG_FAIL(MG_ECUDA, cudaGetErrorString(ez));
  }
  const unsigned nb = blocks_of(count, 256);
  if (scheme == MG_TSC)
    k_assign<2><<<nb, 256, 0, g->stream>>>(count, dpos, dpos + count, dpos + 2 * count, dmass,
                                           1.0 / (double)count, G);
  else
    k_assign<1><<<nb, 256, 0, g->stream>>>(count, dpos, dpos + count, dpos + 2 * count, dmass,
                                           1.0 / (double)count, G);
  k_add_const<<<blocks_of((long long)cells, 256), 256, 0, g->stream>>>((long long)cells, G.rho,
                                                                       -1.0);
  count_launches(2);
  const cudaError_t e = cudaGetLastError();
  if (tmp) {
    cudaStreamSynchronize(g->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) MG_FAIL(MG_ECUDA, cudaGetErrorString(e));
  if (level == 0) {
    domain_restrict_density(g->domains[0], g->stream);
    g->domains[0]->density_set = true;
  } else {
    patch_restrict_density(g, pl);
    pl->density_set = true;
  }
  MG_CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_refine_blocks(const mg_grid* g, int level, double npc, double particle_mass,
                           int32_t* origins, int max_count, int* found) {
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_refine_blocks: needs a domain handle");
  if (!found) MG_FAIL(MG_EINVAL, "mg_refine_blocks: found is NULL");
  if (!(npc >= 0.0) || !(particle_mass > 0.0)) MG_FAIL(MG_EINVAL, "mg_refine_blocks: npc/mass");
  if (max_count > 0 && !origins) MG_FAIL(MG_EINVAL, "mg_refine_blocks: origins is NULL");
  const double* delta;
  int n, patches = 0;
  long long nblocks;
  const PatchLevel* pl = nullptr;
  if (level == 0) {
    const Domain* d = g->domains[0];
    if (!d->density_set) MG_FAIL(MG_ESTATE, "mg_refine_blocks: density not set");
    if (d->n % 4) MG_FAIL(MG_EINVAL, "mg_refine_blocks: n must be a multiple of 4");
    delta = d->lv[0].delta;
    n = d->n;
    nblocks = (long long)(n / 4) * (n / 4) * (n / 4);
  } else {
    if (level < 1 || level > (int)g->patch_levels.size() || !g->patch_levels[level - 1] ||
        g->patch_levels[level - 1]->count == 0)
      MG_FAIL(MG_EINVAL, "mg_refine_blocks: no patches on that level");
    pl = g->patch_levels[level - 1];
    if (!pl->density_set) MG_FAIL(MG_ESTATE, "mg_refine_blocks: density not set");
    delta = pl->delta;
    n = pl->nside;
    patches = 1;
    nblocks = (long long)pl->count * 8;
  }
  // effective particles (1 + delta) h^3 / m_p > npc  <=>  1 + delta > npc m_p n^3
  const double limit = npc * particle_mass * (double)n * n * n;
  int* dflags = nullptr;
  if (cudaMalloc(&dflags, sizeof(int) * nblocks) != cudaSuccess)
    MG_FAIL(MG_ENOMEM, "mg_refine_blocks: device allocation");
  k_flag_blocks<<<(unsigned)nblocks, 64, 0, g->stream>>>(delta, n, patches, limit, dflags);
  count_launches(1);
  std::vector<int> flags((size_t)nblocks);
  cudaMemcpyAsync(flags.data(), dflags, sizeof(int) * nblocks, cudaMemcpyDeviceToHost, g->stream);
  const cudaError_t e = cudaStreamSynchronize(g->stream);
  cudaFree(dflags);
  if (e != cudaSuccess) MG_FAIL(MG_ECUDA, cudaGetErrorString(e));
  // origins of the next level's 8^3 patches: twice the 4^3 block origins, by z, y, x
  std::vector<std::array<int32_t, 3>> out;
  for (long long b = 0; b < nblocks; ++b) {
    if (!flags[(size_t)b]) continue;
    int x, y, z;
    if (!patches) {
      const int nb = n / 4;
      x = 4 * (int)(b % nb);
      y = 4 * (int)((b / nb) % nb);
      z = 4 * (int)(b / ((long long)nb * nb));
    } else {
      const long long q = b >> 3;
      const int lb = (int)(b & 7);
      x = pl->h_origin[3 * q] + 4 * (lb & 1);
      y = pl->h_origin[3 * q + 1] + 4 * ((lb >> 1) & 1);
      z = pl->h_origin[3 * q + 2] + 4 * (lb >> 2);
    }
    out.push_back({2 * x, 2 * y, 2 * z});
  }
  std::sort(out.begin(), out.end(), [](const std::array<int32_t, 3>& a,
                                        const std::array<int32_t, 3>& b) {
    return a[2] != b[2] ? a[2] < b[2] : (a[1] != b[1] ? a[1] < b[1] : a[0] < b[0]);
  });
  *found = (int)out.size();
  const int w = std::min<int>((int)out.size(), std::max(max_count, 0));
  for (int i = 0; i < w; ++i)
    for (int a = 0; a < 3; ++a) origins[3 * i + a] = out[(size_t)i][a];
  return MG_OK;
}

}  // extern "C"
