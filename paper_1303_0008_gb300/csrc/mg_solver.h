// Host-side state of libmg: the periodic level hierarchy of one domain, the
// refinement patch levels, and the batch work lists.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/mg.h"
#include "mg_common.cuh"

namespace mg {

// One multigrid level of a periodic domain (dense n^3 arrays, x fastest).
struct Level {
  int n = 0;
  long long cells = 0;
  double* phi = nullptr;     // field
  double* delta = nullptr;   // density contrast (restricted from the finest level)
  double* src = nullptr;     // per-solve source term of the operator
  double* f = nullptr;       // FAS right-hand side (coarse levels)
  double* phihat = nullptr;  // R phi^h kept for the correction (coarse levels)
  // mixed precision (FP32 correction operator), allocated on first use
  float* e = nullptr;        // correction
  float* ehat = nullptr;     // R e kept for the correction (coarse levels)
  float* phi0 = nullptr;     // FP32 copy of the expansion point
  float* q0 = nullptr;       // discriminant at the expansion point
  float* rhs = nullptr;      // right-hand side of N(e) = rhs (+ mu)
  float* src32 = nullptr;    // kappa * delta in FP32 (coarse levels)
  float* e2 = nullptr;       // second correction buffer of the one-launch sweep
  float* q0c = nullptr;      // finest level: q0 and rhs again, in colour order, for the
  float* rhsc = nullptr;     // colour stages (contiguous reads of a colour's own cells)
};

struct Domain {
  int n = 0;
  int nlev = 0;
  std::vector<Level> lv;
  LevelScalars* d_sc = nullptr;  // 2 * nlev + 2 entries (FP64 levels, FP32 levels, spare)
  LevelScalars* h_sc = nullptr;  // pinned mirror of d_sc[0] and d_sc[nlev]
  Partial* d_part = nullptr;
  int part_cap = 0;
  // per-fine-cell defects and guard flags of the two-step residual restriction
  // (kTwoStepMaxFine entries; the FP32 cycle stores floats in the same bytes)
  double* d_subdef = nullptr;
  unsigned char* d_subguard = nullptr;
  bool density_set = false;
  bool mixed_ready = false;
  // error flags of kernels that wait on asynchronous copies ([0]: a copy did not
  // arrive within barrier_timeout_s), and their pinned host mirror
  int* d_flags = nullptr;
  int* h_flags = nullptr;
  // CUDA graphs of the two halves of a V-cycle (captured per solve)
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
};

// One refinement level: 8^3 patches (Sec. III.C, first paragraph).
struct PatchLevel {
  int level = 0;       // 1 or 2
  int count = 0;
  int nside = 0;       // cells per side of this level's periodic index space
  bool density_set = false;
  bool phi_set = false;       // phi holds an initial guess (set by the caller or a solve)
  int* d_origin = nullptr;    // 3 * count
  int* d_nbr = nullptr;       // 27 * count: neighbour patch index or -1
  double* phi = nullptr;      // count * 512
  double* delta = nullptr;
  double* src = nullptr;
  double* ghost = nullptr;    // count * 1000 ghosted blocks: Dirichlet fill
  std::vector<int> h_origin;
  // union multigrid: coarse levels of the patch union (4^3 and 2^3 per patch)
  double* phi_c[3] = {nullptr, nullptr, nullptr};
  double* phihat_c[3] = {nullptr, nullptr, nullptr};
  double* f_c[3] = {nullptr, nullptr, nullptr};
  double* src_c[3] = {nullptr, nullptr, nullptr};
  double* delta_c[3] = {nullptr, nullptr, nullptr};
  double* ghost_c[3] = {nullptr, nullptr, nullptr};
  LevelScalars* d_sc = nullptr;
  LevelScalars* h_sc = nullptr;
  Partial* d_part = nullptr;
  int part_cap = 0;
  int* d_table = nullptr;           // (nside/8)^3 block -> patch index or -1
  int* d_err = nullptr;             // set when a Dirichlet value finds no parent cell
  double* d_coarse_parent = nullptr;  // level 1: the domain field restricted once
  // linear (Galerkin) coarse-grid correction of the union, union levels 1 and 2:
  // 27-point operator [count][27][cells per patch], correction and right-hand side
  float* gJ[3] = {nullptr, nullptr, nullptr};
  float* ge[3] = {nullptr, nullptr, nullptr};
  float* gb[3] = {nullptr, nullptr, nullptr};
  int last_cycles = 0;
  double last_wall_s = 0.0;  // device time of the last solve of this level (V-cycles)
  double last_res = 0.0;
  int last_status = 0;
  std::vector<double> last_hist;
};

struct BatchState;

}  // namespace mg

struct mg_grid {
  mg_options opt;
  std::vector<mg::Domain*> domains;
  bool batch = false;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  std::vector<mg::PatchLevel*> patch_levels;
  double* force_tmp = nullptr;
  size_t force_tmp_bytes = 0;
  // Newtonian potential: per level (0 = domain, l = refinement level l) phi_N, its
  // ghost shells, and scratch for phi + 2 phi_N; element counts per level
  std::vector<double*> nw_phi, nw_ghost, nw_psi, nw_psi_ghost;
  std::vector<size_t> nw_cells, nw_ghost_cells;
  bool newton_set = false;
  mg::BatchState* bs = nullptr;
};

namespace mg {

// mg_domain.cu
mg_status domain_create(Domain** out, int n, const mg_options& o);
void domain_destroy(Domain* d);
void domain_invalidate_graphs(Domain* d);
void domain_restrict_density(Domain* d, cudaStream_t st);
mg_status domain_solve(Domain* d, const mg_options& o, cudaStream_t st, int branch, double alpha,
                       double kappa, double tol, mg_solve_stats* stats);
int num_levels(int n, int coarsest);

// mg_patch.cu
mg_status patches_add(mg_grid* g, int level, int count, const int* origin);
void patch_level_destroy(PatchLevel* pl);
// init_from_parent: start from the trilinear interpolation of the level below
// instead of the field held by the level.
mg_status patch_level_solve(mg_grid* g, int level, int branch, double alpha, double kappa,
                            double tol, bool init_from_parent = false);
mg_status patch_force(mg_grid* g, int level, int patch, double* out);
void patch_restrict_density(mg_grid* g, PatchLevel* pl);

// mg_patch_galerkin.cu
mg_status galerkin_prepare(PatchLevel* pl);
void galerkin_release(PatchLevel* pl);
void galerkin_correction(cudaStream_t st, PatchLevel* pl, const mg_options& o,
                         const OpConst64& op0, const double* rd, int mlev);

// mg_batch.cu
mg_status batch_prepare(mg_grid* g);
void batch_release(mg_grid* g);
mg_status batch_solve(mg_grid* g, const int* branch, const double* alpha, const double* kappa,
                      double tol, mg_solve_stats* stats);

}  // namespace mg
