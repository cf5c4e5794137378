// Batched independent periodic solves: every stage of the V-cycle (a colour
// stage of the smoother on level l, a residual, a restriction, the coarsest
// solve, ...) is ONE launch over a work list holding that stage's work for all
// solves still running.  Solves of different sizes line up by level index from
// the finest; a solve takes part in the stages of the levels it has.  The two
// halves of a cycle are captured as CUDA graphs and replayed until the set of
// running solves changes (a solve converged or failed), when the lists are
// rebuilt and the graphs captured again.
//
// The per-thread code is the same as the single-grid kernels' (mg_bodies64.cuh,
// mg_bodies32.cuh); an item only tells a block which grid it works on.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mg_bodies32.cuh"
#include "mg_bodies64.cuh"
#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

#define BCK(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return MG_ECUDA;                                                       \
    }                                                                        \
  } while (0)

// One solve's view of level l (and of level l+1 when it exists) for one stage.
struct BItem {
  int block0;  // first block of this item in the launch
  int n;       // cells per side of level l
  double *phi, *src, *f, *phihat;
  const double* delta;
  float *e, *ehat, *phi0, *q0, *rhs;
  LevelScalars *sc, *sc32;
  double *cphi, *csrc, *cf, *cphihat;
  float *ce, *cehat, *cphi0, *cq0, *crhs;
  LevelScalars *csc, *csc32;
  Partial* part;
  LevelScalars* out;  // contiguous copy of the level-0 scalars (or null)
  OpConst64 op, cop;
  OpConst32 op32, cop32;
  float kappa;
  int floor;
};

__device__ __forceinline__ const BItem& find_item(const BItem* __restrict__ items, int count,
                                                  long long& local) {
  int lo = 0, hi = count - 1;
  const int b = (int)blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].block0 <= b) lo = mid;
    else hi = mid - 1;
  }
  local = b - items[lo].block0;
  return items[lo];
}

// ---- FP64 stages ----
__global__ void __launch_bounds__(256) kb_smooth64(const BItem* __restrict__ items, int count,
                                                   int colour) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_smooth_colour64(it.n, it.phi, it.src, it.f, it.sc, it.op, colour, blk);
}

__global__ void __launch_bounds__(256) kb_residual_restrict64(const BItem* __restrict__ items,
                                                              int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_residual_restrict64(it.n, it.phi, it.src, it.f, it.op, it.cphi, it.cphihat, it.cf, it.part,
                        blk);
}

// One block per item.  mode 0: partials of a residual-restriction (one per 256
// coarse cells); mode 1: partials of a per-cell kernel (one per 256 cells).
// use32: reduce into the FP32 inner scalars.  Level-0 scalars are copied to
// it.out, and with clear_mu the inner compatibility constant is reset.
__global__ void __launch_bounds__(256) kb_finalize(const BItem* __restrict__ items, int mode,
                                                   int use32, int clear_mu) {
  const BItem& it = items[blockIdx.x];
  const long long cells = (long long)it.n * it.n * it.n;
  // mode 0: restriction partials (one per 256 coarse cells); 1: one per 256
  // cells; 2: the hand-off's, one per 256 kHandoffCells cells
  const long long work = mode == 0 ? cells / 8 : cells;
  const int per = mode == 2 ? 256 * kHandoffCells : 256;
  const int nparts = (int)((work + per - 1) / per);
  LevelScalars* sc = use32 ? it.sc32 : it.sc;
  b_finalize(it.part, nparts, (double)cells, 1, sc, 0);
  if (threadIdx.x == 0) {
    if (it.out && !use32) *it.out = *sc;
    if (clear_mu && it.sc32) it.sc32->lambda = 0.0;
  }
}

__global__ void __launch_bounds__(256) kb_fas_rhs64(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_fas_rhs64(it.n / 2, it.cphi, it.csrc, it.cf, it.cop, it.sc, it.csc, blk);
}

__global__ void __launch_bounds__(256) kb_prolong64(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_prolong_correct64(it.n / 2, it.cphi, it.cphihat, it.phi, blk);
}

__global__ void __launch_bounds__(256) kb_coarsest64(const BItem* __restrict__ items, int sweeps,
                                                     double drop) {
  const BItem& it = items[blockIdx.x];
  b_coarsest64(it.n, it.phi, it.src, it.f, it.op, it.sc, sweeps, drop, 2, 0);
}

// ---- mixed-precision stages ----
__global__ void __launch_bounds__(256) kb_handoff64(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_residual_handoff64(it.n, it.phi, it.src, it.op, it.sc, it.rhs, it.q0, it.phi0, it.e, it.part,
                       blk);
}

__global__ void __launch_bounds__(256) kb_update64(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_update64((long long)it.n * it.n * it.n, it.phi, it.e, blk);
}

// phi0 of level l+1 = R phi0 of level l (blocks over the coarse cells)
__global__ void __launch_bounds__(256) kb_restrict_phi0(const BItem* __restrict__ items,
                                                        int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_restrict32(it.n / 2, it.phi0, it.cphi0, blk);
}

__global__ void __launch_bounds__(256) kb_q0_prep(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_q0_prep32(it.n, it.phi0, it.delta, it.op32, it.kappa, it.floor, it.q0, blk);
}

__global__ void __launch_bounds__(256) kb_smooth32(const BItem* __restrict__ items, int count,
                                                   int colour) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_smooth_colour32(it.n, it.e, it.phi0, it.q0, it.rhs, it.sc32, it.op32, colour, blk);
}

__global__ void __launch_bounds__(256) kb_residual_restrict32(const BItem* __restrict__ items,
                                                              int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_residual_restrict32(it.n, it.e, it.phi0, it.q0, it.rhs, it.op32, it.ce, it.cehat, it.crhs,
                        it.part, blk);
}

__global__ void __launch_bounds__(256) kb_fas_rhs32(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_fas_rhs32(it.n / 2, it.ce, it.cphi0, it.cq0, it.crhs, it.cop32, it.sc32, it.csc32, blk);
}

__global__ void __launch_bounds__(256) kb_prolong32(const BItem* __restrict__ items, int count) {
  long long blk;
  const BItem& it = find_item(items, count, blk);
  b_prolong_correct32(it.n / 2, it.ce, it.cehat, it.e, blk);
}

__global__ void __launch_bounds__(256) kb_coarsest_corr32(const BItem* __restrict__ items,
                                                          int sweeps, double drop) {
  const BItem& it = items[blockIdx.x];
  b_coarsest_corr32(it.n, it.e, it.phi0, it.q0, it.rhs, it.op32, it.sc32, sweeps, drop, 0);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// T_HAND: the outer residual hand-off, kHandoffCells cells per thread
enum ListType { T_SMOOTH = 0, T_RR, T_CELL, T_CCELL, T_ONE, T_HAND, T_NTYPES };

static long long blocks_of(ListType t, int n) {
  const long long cells = (long long)n * n * n;
  switch (t) {
    case T_SMOOTH: return (cells / 4 + 255) / 256;
    case T_RR: return (cells / 8 + 255) / 256;
    case T_CELL: return (cells + 255) / 256;
    case T_CCELL: return (cells / 8 + 255) / 256;
    case T_HAND: return (cells + 256 * kHandoffCells - 1) / (256 * kHandoffCells);
    default: return 1;
  }
}

struct StageList {
  BItem* d = nullptr;
  int count = 0;
  long long blocks = 0;
  int maxn = 0;
};

struct BatchState {
  std::vector<StageList> lists;  // [level][type][pred]
  StageList coarsest;
  int lmax = 0;
  LevelScalars* d_out = nullptr;
  LevelScalars* h_out = nullptr;
  std::vector<int> active;
  cudaGraphExec_t ga = nullptr, gb = nullptr;
  long long na = 0, nb = 0;
};

// which solves an item list holds: the level exists (P_HAS) or is above the
// solve's coarsest (P_DESC)
enum Pred { P_HAS = 0, P_DESC = 1 };

static StageList& list_at(BatchState* bs, int l, ListType t, Pred p) {
  return bs->lists[((size_t)l * T_NTYPES + t) * 2 + p];
}

static void free_lists(BatchState* bs) {
  for (auto& L : bs->lists) cudaFree(L.d);
  bs->lists.clear();
  cudaFree(bs->coarsest.d);
  bs->coarsest = StageList();
  if (bs->ga) cudaGraphExecDestroy(bs->ga);
  if (bs->gb) cudaGraphExecDestroy(bs->gb);
  bs->ga = bs->gb = nullptr;
}

mg_status batch_prepare(mg_grid* g) {
  BatchState* bs = new (std::nothrow) BatchState();
  if (!bs) {
    set_error("host allocation");
    return MG_ENOMEM;
  }
  g->bs = bs;
  const size_t S = g->domains.size();
  if (cudaMalloc(&bs->d_out, sizeof(LevelScalars) * S) != cudaSuccess ||
      cudaMallocHost(&bs->h_out, sizeof(LevelScalars) * S) != cudaSuccess) {
    set_error("mg_create_batch: allocation");
    return MG_ENOMEM;
  }
  for (Domain* d : g->domains) bs->lmax = std::max(bs->lmax, d->nlev);
  return MG_OK;
}

void batch_release(mg_grid* g) {
  BatchState* bs = g->bs;
  if (!bs) return;
  free_lists(bs);
  cudaFree(bs->d_out);
  if (bs->h_out) cudaFreeHost(bs->h_out);
  delete bs;
  g->bs = nullptr;
}

struct SolveParams {
  std::vector<std::vector<OpConst64>> ops;
  std::vector<std::vector<OpConst32>> ops32;
  std::vector<float> kappa;
  int floor;
};

static BItem make_item(mg_grid* g, const SolveParams& P, int s, int l) {
  Domain* d = g->domains[s];
  BItem it;
  std::memset(&it, 0, sizeof(it));
  const Level& L = d->lv[l];
  it.n = L.n;
  it.phi = L.phi;
  it.src = L.src;
  it.f = L.f;
  it.phihat = L.phihat;
  it.delta = L.delta;
  it.e = L.e;
  it.ehat = L.ehat;
  it.phi0 = L.phi0;
  it.q0 = L.q0;
  it.rhs = L.rhs;
  it.sc = d->d_sc + l;
  it.sc32 = d->d_sc + d->nlev + l;
  it.op = P.ops[s][l];
  if (!P.ops32.empty()) it.op32 = P.ops32[s][l];
  if (l + 1 < d->nlev) {
    const Level& C = d->lv[l + 1];
    it.cphi = C.phi;
    it.csrc = C.src;
    it.cf = C.f;
    it.cphihat = C.phihat;
    it.ce = C.e;
    it.cehat = C.ehat;
    it.cphi0 = C.phi0;
    it.cq0 = C.q0;
    it.crhs = C.rhs;
    it.csc = d->d_sc + l + 1;
    it.csc32 = d->d_sc + d->nlev + l + 1;
    it.cop = P.ops[s][l + 1];
    if (!P.ops32.empty()) it.cop32 = P.ops32[s][l + 1];
  }
  it.part = d->d_part;
  it.out = (l == 0) ? g->bs->d_out + s : nullptr;
  it.kappa = P.kappa[s];
  it.floor = P.floor;
  return it;
}

static mg_status upload(StageList& L, std::vector<BItem>& items) {
  cudaFree(L.d);
  L.d = nullptr;
  L.count = (int)items.size();
  if (items.empty()) return MG_OK;
  if (cudaMalloc(&L.d, sizeof(BItem) * items.size()) != cudaSuccess) {
    set_error("batch: work-list allocation");
    return MG_ENOMEM;
  }
  if (cudaMemcpy(L.d, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    set_error("batch: work-list upload");
    return MG_ECUDA;
  }
  return MG_OK;
}

static mg_status build_lists(mg_grid* g, const SolveParams& P) {
  BatchState* bs = g->bs;
  free_lists(bs);
  bs->lists.resize((size_t)bs->lmax * T_NTYPES * 2);
  for (int l = 0; l < bs->lmax; ++l)
    for (int t = 0; t < T_NTYPES; ++t)
      for (int p = 0; p < 2; ++p) {
        std::vector<BItem> items;
        long long blocks = 0;
        int maxn = 0;
        for (int s : bs->active) {
          const int nl = g->domains[s]->nlev;
          const bool ok = (p == P_HAS) ? (l < nl) : (l < nl - 1);
          if (!ok) continue;
          BItem it = make_item(g, P, s, l);
          it.block0 = (int)blocks;
          blocks += blocks_of((ListType)t, it.n);
          maxn = std::max(maxn, it.n);
          items.push_back(it);
        }
        StageList& L = list_at(bs, l, (ListType)t, (Pred)p);
        mg_status st = upload(L, items);
        if (st != MG_OK) return st;
        L.blocks = blocks;
        L.maxn = maxn;
      }
  std::vector<BItem> co;
  int maxn = 0;
  for (int s : bs->active) {
    BItem it = make_item(g, P, s, g->domains[s]->nlev - 1);
    it.block0 = (int)co.size();
    maxn = std::max(maxn, it.n);
    co.push_back(it);
  }
  mg_status st = upload(bs->coarsest, co);
  bs->coarsest.blocks = (long long)co.size();
  bs->coarsest.maxn = maxn;
  return st;
}

struct BatchCycle {
  mg_grid* g;
  BatchState* bs;
  const mg_options* o;
  cudaStream_t st;

  const StageList& L(int l, ListType t, Pred p) const { return list_at(bs, l, t, p); }

  template <typename K, typename... A>
  void launch(const StageList& sl, int threads, K kernel, A... args) const {
    if (sl.count == 0) return;
    kernel<<<(unsigned)sl.blocks, threads, 0, st>>>(sl.d, sl.count, args...);
    count_launches(1);
  }

  void finalize(int l, ListType src_type, int mode, int use32, int clear_mu) const {
    const StageList& one = L(l, T_ONE, src_type == T_RR ? P_DESC : P_HAS);
    if (one.count == 0) return;
    kb_finalize<<<one.count, 256, 0, st>>>(one.d, mode, use32, clear_mu);
    count_launches(1);
  }

  // ---- FP64 ----
  void smooth64(int l, int sweeps) const {
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 4; ++c) launch(L(l, T_SMOOTH, P_DESC), 256, kb_smooth64, c);
  }
  void part_a64() const {
    smooth64(0, o->nu_pre);
    launch(L(0, T_RR, P_DESC), 256, kb_residual_restrict64);
    finalize(0, T_RR, 0, 0, 0);
    cudaMemcpyAsync(bs->h_out, bs->d_out, sizeof(LevelScalars) * g->domains.size(),
                    cudaMemcpyDeviceToHost, st);
  }
  void part_b64() const {
    launch(L(0, T_CCELL, P_DESC), 256, kb_fas_rhs64);
    for (int l = 1; l < bs->lmax - 1; ++l) {
      smooth64(l, o->nu_pre);
      launch(L(l, T_RR, P_DESC), 256, kb_residual_restrict64);
      finalize(l, T_RR, 0, 0, 0);
      launch(L(l, T_CCELL, P_DESC), 256, kb_fas_rhs64);
    }
    const size_t smem = 3 * sizeof(double) * (size_t)bs->coarsest.maxn * bs->coarsest.maxn *
                        bs->coarsest.maxn;
    kb_coarsest64<<<bs->coarsest.count, 256, smem, st>>>(bs->coarsest.d, o->coarse_sweeps,
                                                         o->coarse_drop);
    count_launches(1);
    for (int l = bs->lmax - 2; l >= 0; --l) {
      launch(L(l, T_CELL, P_DESC), 256, kb_prolong64);
      smooth64(l, o->nu_post);
    }
  }

  // ---- mixed ----
  void smooth32(int l, int sweeps) const {
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 4; ++c) launch(L(l, T_SMOOTH, P_DESC), 256, kb_smooth32, c);
  }
  void part_a_mixed() const {
    launch(L(0, T_HAND, P_HAS), 256, kb_handoff64);
    finalize(0, T_HAND, 2, 0, 1);
    cudaMemcpyAsync(bs->h_out, bs->d_out, sizeof(LevelScalars) * g->domains.size(),
                    cudaMemcpyDeviceToHost, st);
  }
  void inner() const {
    for (int l = 0; l < bs->lmax - 1; ++l) {
      smooth32(l, o->nu_pre);
      launch(L(l, T_RR, P_DESC), 256, kb_residual_restrict32);
      finalize(l, T_RR, 0, 1, 0);
      launch(L(l, T_CCELL, P_DESC), 256, kb_fas_rhs32);
    }
    const size_t smem = 4 * sizeof(double) * (size_t)bs->coarsest.maxn * bs->coarsest.maxn *
                        bs->coarsest.maxn;
    kb_coarsest_corr32<<<bs->coarsest.count, 256, smem, st>>>(bs->coarsest.d, o->coarse_sweeps,
                                                              o->coarse_drop);
    count_launches(1);
    for (int l = bs->lmax - 2; l >= 0; --l) {
      launch(L(l, T_CELL, P_DESC), 256, kb_prolong32);
      smooth32(l, o->nu_post);
    }
  }
  void part_b_mixed() const {
    for (int l = 1; l < bs->lmax; ++l) {
      launch(L(l - 1, T_CCELL, P_DESC), 256, kb_restrict_phi0);
      launch(L(l, T_CELL, P_HAS), 256, kb_q0_prep);
    }
    for (int c = 0; c < o->inner_cycles; ++c) inner();
    launch(L(0, T_CELL, P_HAS), 256, kb_update64);
  }
};

mg_status mixed_prepare_domain(Domain* d);
void launch_gauge64(cudaStream_t st, long long cells, double* x, Partial* partials,
                    LevelScalars* sc);
mg_status domain_prepare_sources(Domain* d, cudaStream_t st, int branch, double alpha,
                                 double kappa, int guard, double omega,
                                 std::vector<OpConst64>& ops, double w);
OpConst32 make_op32(int n, double alpha, int branch);

mg_status batch_solve(mg_grid* g, const int* branch, const double* alpha, const double* kappa,
                      double tol, mg_solve_stats* stats) {
  BatchState* bs = g->bs;
  const mg_options& o = g->opt;
  cudaStream_t st = g->stream;
  const int S = (int)g->domains.size();
  const bool mixed = o.prec == MG_MIXED;
  std::vector<mg_solve_stats> local(S);
  mg_solve_stats* sv = stats ? stats : local.data();
  SolveParams P;
  P.ops.resize(S);
  P.kappa.resize(S);
  P.floor = o.guard == MG_GUARD_FLOOR;
  if (mixed) P.ops32.resize(S);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(kb_coarsest64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         3 * sizeof(double) * 4096);
    cudaFuncSetAttribute(kb_coarsest_corr32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         4 * sizeof(double) * 4096);
    attr = true;
  }
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  BCK(cudaEventRecord(e0, st));
  const long long launches0 = tl_launches;
  mg_status result = MG_OK;
  bs->active.clear();
  std::vector<double> first(S, -1.0);
  std::vector<std::vector<double>> hist(S);
  for (int s = 0; s < S; ++s) {
    Domain* d = g->domains[s];
    std::memset(&sv[s], 0, sizeof(mg_solve_stats));
    sv[s].levels = d->nlev;
    mg_status ps = domain_prepare_sources(d, st, branch[s], alpha[s], kappa[s], o.guard, o.omega,
                                          P.ops[s], 1.0 / 3.0);
    if (ps != MG_OK) return ps;
    P.kappa[s] = (float)kappa[s];
    if (mixed) {
      ps = mixed_prepare_domain(d);
      if (ps != MG_OK) return ps;
      P.ops32[s].resize(d->nlev);
      for (int l = 0; l < d->nlev; ++l) P.ops32[s][l] = make_op32(d->lv[l].n, alpha[s], branch[s]);
    }
    if (d->nlev == 1) {
      // a single-level grid has no V-cycle to batch: solve it on its own
      mg_status r = domain_solve(d, o, st, branch[s], alpha[s], kappa[s], tol, &sv[s]);
      if (r != MG_OK && result == MG_OK) result = r;
    } else {
      bs->active.push_back(s);
    }
  }
  BatchCycle cyc{g, bs, &o, st};
  bool rebuild = true;
  while (!bs->active.empty()) {
    if (rebuild) {
      mg_status r = build_lists(g, P);
      if (r != MG_OK) return r;
      if (o.use_graphs) {
        if (mixed) {
          bs->ga = capture_graph(st, &bs->na, [&] { cyc.part_a_mixed(); });
          bs->gb = capture_graph(st, &bs->nb, [&] { cyc.part_b_mixed(); });
        } else {
          bs->ga = capture_graph(st, &bs->na, [&] { cyc.part_a64(); });
          bs->gb = capture_graph(st, &bs->nb, [&] { cyc.part_b64(); });
        }
      }
      rebuild = false;
    }
    const bool graphs = bs->ga && bs->gb;
    if (graphs) {
      BCK(cudaGraphLaunch(bs->ga, st));
      tl_launches += bs->na;
    } else if (mixed) {
      cyc.part_a_mixed();
    } else {
      cyc.part_a64();
    }
    BCK(cudaStreamSynchronize(st));
    BCK(cudaGetLastError());
    std::vector<int> still;
    for (int s : bs->active) {
      const LevelScalars& h = bs->h_out[s];
      mg_solve_stats& x = sv[s];
      const double res = h.res;
      if (mixed) x.outer += 1;
      x.res = res;
      x.lambda = h.lambda;
      x.guard_hits = o.guard == MG_GUARD_FLOOR ? (long long)h.floored : h.guards;
      if (x.hist_len < 128) x.res_hist[x.hist_len++] = res;
      if (first[s] < 0) first[s] = res;
      hist[s].push_back(res);
      const size_t k = hist[s].size();
      mg_status sst = MG_OK;
      if (!(res == res)) sst = MG_ENAN;
      else if (res < tol) sst = MG_OK;
      else if ((int)k > o.max_cycles || res > 1e3 * first[s] ||
               (k > 8 && res > 0.9 * hist[s][k - 9]))
        sst = MG_ENOCONV;
      else {
        still.push_back(s);
        x.cycles += mixed ? o.inner_cycles : 1;
        continue;
      }
      x.status = sst;
      x.res0 = first[s];
      if (sst != MG_OK && result == MG_OK) {
        result = sst;
        set_error("batch: solve " + std::to_string(s) +
                  (sst == MG_ENAN ? ": residual is not finite" : ": no convergence"));
      }
    }
    if (still.size() != bs->active.size()) {
      bs->active = still;
      rebuild = true;
      if (bs->active.empty()) break;
      BCK(cudaStreamSynchronize(st));
      mg_status r = build_lists(g, P);  // the second half runs for the remaining solves
      if (r != MG_OK) return r;
      rebuild = false;
      if (o.use_graphs) {
        if (mixed) {
          bs->ga = capture_graph(st, &bs->na, [&] { cyc.part_a_mixed(); });
          bs->gb = capture_graph(st, &bs->nb, [&] { cyc.part_b_mixed(); });
        } else {
          bs->ga = capture_graph(st, &bs->na, [&] { cyc.part_a64(); });
          bs->gb = capture_graph(st, &bs->nb, [&] { cyc.part_b64(); });
        }
      }
    }
    if (bs->ga && bs->gb) {
      BCK(cudaGraphLaunch(bs->gb, st));
      tl_launches += bs->nb;
    } else if (mixed) {
      cyc.part_b_mixed();
    } else {
      cyc.part_b64();
    }
  }
  for (int s = 0; s < S; ++s) {
    Domain* d = g->domains[s];
    if (d->nlev > 1)
      launch_gauge64(st, d->lv[0].cells, d->lv[0].phi, d->d_part, d->d_sc + 2 * d->nlev + 1);
  }
  BCK(cudaEventRecord(e1, st));
  BCK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const long long launches = tl_launches - launches0;
  for (int s = 0; s < S; ++s) {
    if (g->domains[s]->nlev > 1) sv[s].wall_s = ms * 1e-3;
    sv[s].launches = launches;
  }
  BCK(cudaGetLastError());
  return result;
}

}  // namespace mg
