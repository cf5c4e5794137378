// Shared-memory tiles of refinement patches: the ghosted (B+2)^3 block of one
// patch with its neighbours' cells and the Dirichlet values outside the union.
// Used by the patch kernels (mg_patch.cu) and the union's linear coarse-grid
// correction (mg_patch_galerkin.cu).
#pragma once

#include "mg_common.cuh"

namespace mg {

// Load the ghosted tile of patch p at block size B into shared memory.
template <int B>
__device__ __forceinline__ void load_tile(double* __restrict__ tile, int p,
                                          const double* __restrict__ phi,
                                          const double* __restrict__ ghost,
                                          const int* __restrict__ nbr) {
  constexpr int T = B + 2, TC = T * T * T, BC = B * B * B;
  for (int q = threadIdx.x; q < TC; q += blockDim.x) {
    const int i = q % T - 1, j = (q / T) % T - 1, k = q / (T * T) - 1;
    const int ox = i < 0 ? -1 : (i >= B ? 1 : 0);
    const int oy = j < 0 ? -1 : (j >= B ? 1 : 0);
    const int oz = k < 0 ? -1 : (k >= B ? 1 : 0);
    double v;
    if ((ox | oy | oz) == 0) {
      v = phi[(long long)p * BC + i + B * (j + B * k)];
    } else {
      const int nb = nbr[p * 27 + (ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1))];
      if (nb >= 0)
        v = phi[(long long)nb * BC + (i - ox * B) + B * ((j - oy * B) + B * (k - oz * B))];
      else
        v = ghost[(long long)p * TC + q];
    }
    tile[q] = v;
  }
}

template <int B>
__device__ __forceinline__ StencilT<double> gather_tile(const double* tile, int i, int j, int k) {
  constexpr int T = B + 2;
  auto at = [&](int a, int b, int c) { return tile[(a + 1) + T * ((b + 1) + T * (c + 1))]; };
  StencilT<double> s;
  s.sx = at(i + 1, j, k) + at(i - 1, j, k);
  s.sy = at(i, j + 1, k) + at(i, j - 1, k);
  s.sz = at(i, j, k + 1) + at(i, j, k - 1);
  s.cxy = (at(i + 1, j + 1, k) + at(i - 1, j - 1, k)) - (at(i + 1, j - 1, k) + at(i - 1, j + 1, k));
  s.cxz = (at(i + 1, j, k + 1) + at(i - 1, j, k - 1)) - (at(i + 1, j, k - 1) + at(i - 1, j, k + 1));
  s.cyz = (at(i, j + 1, k + 1) + at(i, j - 1, k - 1)) - (at(i, j + 1, k - 1) + at(i, j - 1, k + 1));
  return s;
}

template <int B>
__device__ __forceinline__ double tile_ctr(const double* tile, int i, int j, int k) {
  constexpr int T = B + 2;
  return tile[(i + 1) + T * ((j + 1) + T * (k + 1))];
}

}  // namespace mg
