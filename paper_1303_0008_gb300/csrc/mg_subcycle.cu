// The bottom of a V-cycle (every level with at most 16 cells per side, down to
// the coarsest) in ONE launch: a single cluster of CTAs runs the same per-cell
// code as the per-level kernels, phase by phase, with a cluster barrier between
// dependent phases.  The levels are tiny, so separate launches are bound by
// launch latency (a few microseconds each, about 60 per V-cycle); here the cost
// is one launch plus one cluster barrier per phase.
//
// Work that is independent per cell (colour stages, FAS right-hand sides,
// prolongation, the fine-cell defects) is spread in even, warp-aligned chunks
// over all CTAs: on GB300 an SM issues two FP64 lane-operations per clock, so a
// 16^3 level in 256-thread blocks would keep only a few SMs' FP64 pipes busy.
// The reductions (the coarse-cell walk over stored defects and the level norms)
// keep the per-level kernels' 256-thread block partition and order, so the
// results are the same bit for bit.
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

// The phase sequence of one sub-cycle over the CTAs of one cluster.
struct Phases {
  cg::cluster_group cl;
  int rank, nb;
  // items [0, count) in even chunks (whole warps) over the CTAs; cell(t) per item
  template <typename Cell>
  __device__ __forceinline__ void spread(long long count, Cell cell) {
    const long long chunk = (((count + nb - 1) / nb) + 31) & ~31LL;
    const long long lo = (long long)rank * chunk;
    const long long hi = lo + chunk < count ? lo + chunk : count;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) cell(t);
    cl.sync();
  }
  // 256-thread blocks [0, count) round-robin over the CTAs (the per-level
  // kernels' partition); body(b) per block, called by every thread of the CTA
  template <typename Body>
  __device__ __forceinline__ void blocks(long long count, Body body) {
    for (long long b = rank; b < count; b += nb) {
      body(b);
      __syncthreads();
    }
    cl.sync();
  }
};

__global__ void __launch_bounds__(256) k_subcycle64(const __grid_constant__ SubCycleArgs a) {
  PdlScope pdl_scope;
  __shared__ double s_c, s_lam;
  Phases ph{cg::this_cluster(), 0, 0};
  ph.rank = (int)ph.cl.block_rank();
  ph.nb = (int)ph.cl.num_blocks();
  auto smooth = [&](const SubLevel64& L, int sweeps) {
    if (threadIdx.x == 0) s_c = smooth_scalar64(L.sc, L.op);
    __syncthreads();
    const double sc = s_c;
    const long long per = (long long)L.n * L.n * L.n / 4;
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour)
        ph.spread(per, [&](long long t) {
          cell_smooth64(L.n, L.phi, L.src, L.f, sc, L.op, colour, t);
        });
  };
  for (int l = 0; l + 1 < a.nlev; ++l) {
    const SubLevel64& L = a.lv[l];
    const SubLevel64& C = a.lv[l + 1];
    const long long cc = (long long)C.n * C.n * C.n;
    smooth(L, a.nu_pre);
    ph.spread(8 * cc, [&](long long t) {
      cell_defect64(L.n, L.phi, L.src, L.f, L.op, a.def64, a.guard, t);
    });
    const long long rr = nblk256(cc);
    ph.blocks(rr, [&](long long b) {
      b_restrict_defects64(L.n, L.phi, a.def64, a.guard, C.phi, C.phihat, C.f, a.part, b);
    });
    // the level norms, merged by every CTA (as b_finalize does) so that the FAS
    // right-hand side needs no further barrier; rank 0 stores the scalars
    {
      const Partial p = merge_partials(a.part, (int)rr);
      if (threadIdx.x == 0) {
        s_lam = level_lambda(p, (double)L.n * L.n * L.n, 1);
        if (ph.rank == 0) store_scalars(p, s_lam, L.sc);
      }
      __syncthreads();
    }
    const double lam = s_lam;
    ph.spread(cc, [&](long long t) {
      cell_fas_rhs64(C.n, C.phi, C.src, C.f, C.op, lam, C.sc, t);
    });
  }
  {
    const SubLevel64& B = a.lv[a.nlev - 1];
    ph.blocks(1, [&](long long) {
      b_coarsest64(B.n, B.phi, B.src, B.f, B.op, B.sc, a.coarse_sweeps, a.coarse_drop, 2, 0);
    });
  }
  for (int l = a.nlev - 2; l >= 0; --l) {
    const SubLevel64& L = a.lv[l];
    const SubLevel64& C = a.lv[l + 1];
    ph.spread((long long)L.n * L.n * L.n, [&](long long t) {
      cell_prolong64(C.n, C.phi, C.phihat, L.phi, t);
    });
    smooth(L, a.nu_post);
  }
}

__global__ void __launch_bounds__(256) k_subcycle32(const __grid_constant__ SubCycleArgs a) {
  PdlScope pdl_scope;
  __shared__ float s_mu;
  __shared__ double s_lam;
  Phases ph{cg::this_cluster(), 0, 0};
  ph.rank = (int)ph.cl.block_rank();
  ph.nb = (int)ph.cl.num_blocks();
  auto smooth = [&](const SubLevel32& L, int sweeps) {
    if (threadIdx.x == 0) s_mu = (float)L.sc32->lambda;
    __syncthreads();
    const float mu = s_mu;
    const long long per = (long long)L.n * L.n * L.n / 4;
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour)
        ph.spread(per, [&](long long t) {
          cell_smooth32(L.n, L.e, L.phi0, L.q0, L.rhs, mu, L.op32, colour, t);
        });
  };
  for (int l = 0; l + 1 < a.nlev; ++l) {
    const SubLevel32& L = a.lv32[l];
    const SubLevel32& C = a.lv32[l + 1];
    const long long cc = (long long)C.n * C.n * C.n;
    smooth(L, a.nu_pre);
    ph.spread(8 * cc, [&](long long t) {
      cell_defect32(L.n, L.e, L.phi0, L.q0, L.rhs, L.op32, a.def32, t);
    });
    const long long rr = nblk256(cc);
    ph.blocks(rr, [&](long long b) {
      b_restrict_defects32(L.n, L.e, a.def32, C.e, C.ehat, C.rhs, a.part, b);
    });
    // the level norms, merged by every CTA (as b_finalize does) so that the FAS
    // right-hand side needs no further barrier; rank 0 stores the scalars
    {
      const Partial p = merge_partials(a.part, (int)rr);
      if (threadIdx.x == 0) {
        s_lam = level_lambda(p, (double)L.n * L.n * L.n, 1);
        if (ph.rank == 0) store_scalars(p, s_lam, L.sc32);
      }
      __syncthreads();
    }
    const double lam = s_lam;
    ph.spread(cc, [&](long long t) {
      cell_fas_rhs32(C.n, C.e, C.phi0, C.q0, C.rhs, C.op32, lam, C.sc32, t);
    });
  }
  {
    const SubLevel32& B = a.lv32[a.nlev - 1];
    ph.blocks(1, [&](long long) {
      b_coarsest_corr32(B.n, B.e, B.phi0, B.q0, B.rhs, B.op32, B.sc32, a.coarse_sweeps,
                        a.coarse_drop, 0);
    });
  }
  for (int l = a.nlev - 2; l >= 0; --l) {
    const SubLevel32& L = a.lv32[l];
    const SubLevel32& C = a.lv32[l + 1];
    ph.spread((long long)L.n * L.n * L.n, [&](long long t) {
      cell_prolong32(C.n, C.e, C.ehat, L.e, t);
    });
    smooth(L, a.nu_post);
  }
}

// Cluster size: 16 CTAs (the non-portable maximum) for the FP64 cycle, whose
// 16^3 level is bound by the FP64 pipes; the FP32 cycle is bound by latency.
constexpr int kClusterCtas64 = 16;
constexpr int kClusterCtas32 = 16;

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
  cudaFuncSetAttribute(k_subcycle64, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_subcycle32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaGetLastError();
}

void launch_subcycle64(cudaStream_t st, const SubCycleArgs& a) {
  const int nc = a.lv[a.nlev - 1].n;
  launch_cluster(k_subcycle64, st, a, 3 * sizeof(double) * (size_t)nc * nc * nc,
                 kClusterCtas64);
}

void launch_subcycle32(cudaStream_t st, const SubCycleArgs& a) {
  const int nc = a.lv32[a.nlev - 1].n;
  launch_cluster(k_subcycle32, st, a, 4 * sizeof(double) * (size_t)nc * nc * nc,
                 kClusterCtas32);
}

}  // namespace mg
