// The bottom of a V-cycle (every level with at most 16 cells per side, down to
// the coarsest) in ONE launch: a single cluster of CTAs runs the same per-thread
// bodies as the per-level kernels, block by block, with a cluster barrier between
// dependent phases.  The levels are tiny, so separate launches are bound by
// launch latency (a few microseconds each, about 60 per V-cycle); here the cost
// is one launch plus one cluster barrier per phase.  Every phase keeps the
// per-level kernels' block partition (256 threads per block), so the arithmetic,
// including the order of each reduction, is the same bit for bit.
//
// The cluster's CTAs are co-scheduled by the hardware, so the barrier always
// completes; it orders global memory at cluster scope (release/acquire).
#include <cooperative_groups.h>

#include <string>

#include "mg_bodies32.cuh"
#include "mg_bodies64.cuh"
#include "mg_internal.h"

namespace cg = cooperative_groups;

namespace mg {

__device__ __forceinline__ long long nblk256(long long work) { return (work + 255) / 256; }

__global__ void __launch_bounds__(256) k_subcycle64(const __grid_constant__ SubCycleArgs a) {
  PdlScope pdl_scope;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks();
  auto smooth = [&](const SubLevel64& L, int sweeps) {
    const long long blocks = nblk256((long long)L.n * L.n * L.n / 4);
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour) {
        for (long long b = rank; b < blocks; b += nb)
          b_smooth_colour64(L.n, L.phi, L.src, L.f, L.sc, L.op, colour, b);
        cl.sync();
      }
  };
  for (int l = 0; l + 1 < a.nlev; ++l) {
    const SubLevel64& L = a.lv[l];
    const SubLevel64& C = a.lv[l + 1];
    const long long cc = (long long)C.n * C.n * C.n;
    smooth(L, a.nu_pre);
    const long long rr = nblk256(cc);
    for (long long b = rank; b < rr; b += nb)
      b_residual_restrict64(L.n, L.phi, L.src, L.f, L.op, C.phi, C.phihat, C.f, a.part, b);
    cl.sync();
    if (rank == 0) b_finalize(a.part, (int)rr, (double)L.n * L.n * L.n, 1, L.sc, 0);
    cl.sync();
    for (long long b = rank; b < nblk256(cc); b += nb)
      b_fas_rhs64(C.n, C.phi, C.src, C.f, C.op, L.sc, C.sc, b);
    cl.sync();
  }
  {
    const SubLevel64& B = a.lv[a.nlev - 1];
    if (rank == 0) b_coarsest64(B.n, B.phi, B.src, B.f, B.op, B.sc, a.coarse_sweeps,
                                a.coarse_drop, 2, 0);
    cl.sync();
  }
  for (int l = a.nlev - 2; l >= 0; --l) {
    const SubLevel64& L = a.lv[l];
    const SubLevel64& C = a.lv[l + 1];
    const long long fine = (long long)L.n * L.n * L.n;
    for (long long b = rank; b < nblk256(fine); b += nb)
      b_prolong_correct64(C.n, C.phi, C.phihat, L.phi, b);
    cl.sync();
    smooth(L, a.nu_post);
  }
}

__global__ void __launch_bounds__(256) k_subcycle32(const __grid_constant__ SubCycleArgs a) {
  PdlScope pdl_scope;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks();
  auto smooth = [&](const SubLevel32& L, int sweeps) {
    const long long blocks = nblk256((long long)L.n * L.n * L.n / 4);
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour) {
        for (long long b = rank; b < blocks; b += nb)
          b_smooth_colour32(L.n, L.e, L.phi0, L.q0, L.rhs, L.sc32, L.op32, colour, b);
        cl.sync();
      }
  };
  for (int l = 0; l + 1 < a.nlev; ++l) {
    const SubLevel32& L = a.lv32[l];
    const SubLevel32& C = a.lv32[l + 1];
    const long long cc = (long long)C.n * C.n * C.n;
    smooth(L, a.nu_pre);
    const long long rr = nblk256(cc);
    for (long long b = rank; b < rr; b += nb)
      b_residual_restrict32(L.n, L.e, L.phi0, L.q0, L.rhs, L.op32, C.e, C.ehat, C.rhs, a.part, b);
    cl.sync();
    if (rank == 0) b_finalize(a.part, (int)rr, (double)L.n * L.n * L.n, 1, L.sc32, 0);
    cl.sync();
    for (long long b = rank; b < nblk256(cc); b += nb)
      b_fas_rhs32(C.n, C.e, C.phi0, C.q0, C.rhs, C.op32, L.sc32, C.sc32, b);
    cl.sync();
  }
  {
    const SubLevel32& B = a.lv32[a.nlev - 1];
    if (rank == 0) b_coarsest_corr64(B.n, B.e, B.phi0, B.q0, B.rhs, B.op32, B.sc32,
                                     a.coarse_sweeps, a.coarse_drop, 0);
    cl.sync();
  }
  for (int l = a.nlev - 2; l >= 0; --l) {
    const SubLevel32& L = a.lv32[l];
    const SubLevel32& C = a.lv32[l + 1];
    const long long fine = (long long)L.n * L.n * L.n;
    for (long long b = rank; b < nblk256(fine); b += nb)
      b_prolong_correct32(C.n, C.e, C.ehat, L.e, b);
    cl.sync();
    smooth(L, a.nu_post);
  }
}

// Cluster size: the portable 8 CTAs.  Measured on the six-solve 128^3 step, 8
// (and 4) CTAs beat 16 by 4 % (the cluster barriers between the many short
// phases cost more with more CTAs) and 1 CTA (the phases run serially) by 12 %.
constexpr int kClusterCtas = 8;

template <typename K>
static void launch_cluster(K kernel, cudaStream_t st, const SubCycleArgs& a, size_t smem,
                           int ctas) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kernel, a);
  count_launches(1);
}


// Kernel attributes, set once outside any stream capture.
void init_subcycle() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(k_subcycle64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       4 * sizeof(double) * 4096);
  cudaFuncSetAttribute(k_subcycle32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       4 * sizeof(double) * 4096);
  cudaGetLastError();
}

void launch_subcycle64(cudaStream_t st, const SubCycleArgs& a) {
  const int nc = a.lv[a.nlev - 1].n;
  launch_cluster(k_subcycle64, st, a, 3 * sizeof(double) * (size_t)nc * nc * nc, kClusterCtas);
}

void launch_subcycle32(cudaStream_t st, const SubCycleArgs& a) {
  const int nc = a.lv32[a.nlev - 1].n;
  launch_cluster(k_subcycle32, st, a, 4 * sizeof(double) * (size_t)nc * nc * nc, kClusterCtas);
}

}  // namespace mg
