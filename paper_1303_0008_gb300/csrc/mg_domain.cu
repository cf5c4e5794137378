// Periodic domain grid: level hierarchy and the FP64 FAS V-cycle schedule
// (Sec. III.C of arXiv:1303.0008).
//
// One V-cycle, finest to coarsest and back:
//   pre-smooth (nu_pre four-colour Newton-Gauss-Seidel sweeps), residual fused
//   with the restriction of phi and d, the coarse right-hand side
//   f^H = L^H(R phi^h) - R(d^h - lambda^h), recursion, the coarsest solve,
//   phi^h += P(phi^H - R phi^h), post-smooth.
// The residual taken after the finest pre-smoothing doubles as the convergence
// test: when max|d - lambda| < tol the cycle stops there, so every cycle costs
// one finest-level residual.  The two halves of the cycle (up to that test,
// and after it) are captured once per solve as CUDA graphs and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

#define DCK(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return MG_ECUDA;                                                       \
    }                                                                        \
  } while (0)

int num_levels(int n, int coarsest) {
  int nl = 1;
  while (n > coarsest && (n % 2) == 0 && (n / 2) >= 4 && ((n / 2) % 2) == 0) {
    n /= 2;
    ++nl;
  }
  return nl;
}

static const int kMaxCoarsest = 16;  // the coarsest solve runs in one CTA's shared memory

mg_status domain_create(Domain** out, int n, const mg_options& o) {
  *out = nullptr;
  if (n < 4 || (n & 1) || n > 1024) {
    set_error("n must be even and in [4, 1024]");
    return MG_EINVAL;
  }
  const int nl = num_levels(n, o.coarsest);
  const int nc = n >> (nl - 1);
  if (nc > kMaxCoarsest) {
    set_error("n must be m * 2^k with the coarsest side m <= 16 (m even)");
    return MG_EINVAL;
  }
  Domain* d = new (std::nothrow) Domain();
  if (!d) {
    set_error("host allocation");
    return MG_ENOMEM;
  }
  init_subcycle();
  d->n = n;
  d->nlev = nl;
  d->lv.resize(nl);
  bool ok = true;
  for (int l = 0; l < nl; ++l) {
    Level& L = d->lv[l];
    L.n = n >> l;
    L.cells = (long long)L.n * L.n * L.n;
    const size_t b = (size_t)L.cells * sizeof(double);
    ok = ok && cudaMalloc(&L.phi, b) == cudaSuccess;
    ok = ok && cudaMalloc(&L.delta, b) == cudaSuccess;
    ok = ok && cudaMalloc(&L.src, b) == cudaSuccess;
    if (l > 0) {
      ok = ok && cudaMalloc(&L.f, b) == cudaSuccess;
      ok = ok && cudaMalloc(&L.phihat, b) == cudaSuccess;
    }
    if (ok) {
      cudaMemset(L.phi, 0, b);
      cudaMemset(L.delta, 0, b);
    }
  }
  d->part_cap = partials_needed(d->lv[0].cells);
  ok = ok && cudaMalloc(&d->d_part, sizeof(Partial) * d->part_cap) == cudaSuccess;
  {
    static_assert(kTwoStepMaxFine >= (long long)kSubcycleMaxN * kSubcycleMaxN * kSubcycleMaxN,
                  "the two-step scratch also serves the sub-cycle");
    const size_t sub = (size_t)kTwoStepMaxFine;
    ok = ok && cudaMalloc(&d->d_subdef, sizeof(double) * sub) == cudaSuccess;
    ok = ok && cudaMalloc(&d->d_subguard, sub) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&d->d_sc, sizeof(LevelScalars) * (2 * nl + 2)) == cudaSuccess;
  ok = ok && cudaMallocHost(&d->h_sc, sizeof(LevelScalars) * 2) == cudaSuccess;
  if (!ok) {
    domain_destroy(d);
    set_error("device allocation failed");
    return MG_ENOMEM;
  }
  cudaMemset(d->d_sc, 0, sizeof(LevelScalars) * (2 * nl + 2));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    domain_destroy(d);
    set_error("device initialisation failed");
    return MG_ECUDA;
  }
  *out = d;
  return MG_OK;
}

void domain_invalidate_graphs(Domain* d) {
  for (auto& g : d->gexec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void mixed_release(Domain* d);

void domain_destroy(Domain* d) {
  if (!d) return;
  domain_invalidate_graphs(d);
  for (Level& L : d->lv) {
    cudaFree(L.phi);
    cudaFree(L.delta);
    cudaFree(L.src);
    cudaFree(L.f);
    cudaFree(L.phihat);
  }
  mixed_release(d);
  cudaFree(d->d_part);
  cudaFree(d->d_subdef);
  cudaFree(d->d_subguard);
  cudaFree(d->d_sc);
  if (d->h_sc) cudaFreeHost(d->h_sc);
  delete d;
}

void domain_restrict_density(Domain* d, cudaStream_t st) {
  for (int l = 1; l < d->nlev; ++l)
    launch_restrict64(st, d->lv[l].n, d->lv[l - 1].delta, d->lv[l].delta);
}

// ---------------------------------------------------------------------------
// FP64 V-cycle
// ---------------------------------------------------------------------------
struct Cycle64 {
  Domain* d;
  const mg_options* o;
  cudaStream_t st;
  const OpConst64* ops;
  EventPairs* timer_a = nullptr;  // finest-level smoother launches of each half
  EventPairs* timer_b = nullptr;

  // The sub-V-cycle from level l down, in one cluster launch.
  void subcycle(int l) const {
    SubCycleArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nlev = d->nlev - l;
    for (int k = 0; k < a.nlev; ++k) {
      Level& L = d->lv[l + k];
      a.lv[k] = SubLevel64{L.n, L.phi, L.src, L.f, L.phihat, d->d_sc + l + k, ops[l + k]};
    }
    a.part = d->d_part;
    a.def64 = d->d_subdef;
    a.guard = d->d_subguard;
    a.nu_pre = o->nu_pre;
    a.nu_post = o->nu_post;
    a.coarse_sweeps = o->coarse_sweeps;
    a.coarse_drop = o->coarse_drop;
    launch_subcycle64(st, a);
  }

  void descend(int l) const {
    Level& L = d->lv[l];
    LevelScalars* sc = d->d_sc + l;
    if (o->fuse_coarse && l > 0 && L.n <= kSubcycleMaxN && d->nlev - l <= kSubcycleMaxLevels) {
      subcycle(l);
      return;
    }
    if (l == d->nlev - 1) {
      launch_coarsest64(st, L.n, L.phi, L.src, L.f, ops[l], sc, o->coarse_sweeps, o->coarse_drop);
      return;
    }
    Level& C = d->lv[l + 1];
    launch_smooth64(st, L.n, L.phi, L.src, L.f, sc, ops[l], o->nu_pre);
    launch_residual_restrict64(st, L.n, L.phi, L.src, L.f, ops[l], C.phi, C.phihat, C.f,
                               d->d_part, sc, d->d_subdef, d->d_subguard);
    launch_fas_rhs64(st, C.n, C.phi, C.src, C.f, ops[l + 1], sc, d->d_sc + l + 1);
    descend(l + 1);
    launch_prolong_correct64(st, C.n, C.phi, C.phihat, L.phi, true);
    launch_smooth64(st, L.n, L.phi, L.src, L.f, sc, ops[l], o->nu_post);
  }

  // Up to and including the convergence test (the residual after pre-smoothing).
  void part_a() const {
    Level& L = d->lv[0];
    Level& C = d->lv[1];
    launch_smooth64(st, L.n, L.phi, L.src, nullptr, d->d_sc, ops[0], o->nu_pre, timer_a);
    launch_residual_restrict64(st, L.n, L.phi, L.src, nullptr, ops[0], C.phi, C.phihat, C.f,
                               d->d_part, d->d_sc, d->d_subdef, d->d_subguard);
    cudaMemcpyAsync(d->h_sc, d->d_sc, sizeof(LevelScalars), cudaMemcpyDeviceToHost, st);
    if (o->tau_stop > 0.0) {
      // The first coarse FAS right-hand side is L^H(R phi) - R L^h(phi) + lambda^h, the
      // truncation-error estimate (finest f = 0); its spread goes to the host too.
      LevelScalars* tsc = d->d_sc + 2 * d->nlev;
      launch_fas_rhs64(st, C.n, C.phi, C.src, C.f, ops[1], d->d_sc, d->d_sc + 1);
      launch_spread64(st, C.cells, C.f, d->d_part, tsc);
      cudaMemcpyAsync(d->h_sc + 1, tsc, sizeof(LevelScalars), cudaMemcpyDeviceToHost, st);
    }
  }

  void part_b() const {
    Level& L = d->lv[0];
    Level& C = d->lv[1];
    if (!(o->tau_stop > 0.0))  // else part_a computed it
      launch_fas_rhs64(st, C.n, C.phi, C.src, C.f, ops[1], d->d_sc, d->d_sc + 1);
    descend(1);
    launch_prolong_correct64(st, C.n, C.phi, C.phihat, L.phi, true);
    launch_smooth64(st, L.n, L.phi, L.src, nullptr, d->d_sc, ops[0], o->nu_post, timer_b);
  }

  // Single-level grid: the coarsest solve is the whole cycle.
  void part_single() const {
    Level& L = d->lv[0];
    launch_coarsest64(st, L.n, L.phi, L.src, nullptr, ops[0], d->d_sc, o->coarse_sweeps,
                      o->coarse_drop);
    cudaMemcpyAsync(d->h_sc, d->d_sc, sizeof(LevelScalars), cudaMemcpyDeviceToHost, st);
  }
};

// Shared convergence bookkeeping of the domain solves.
struct ConvTracker {
  double tol;
  int max_checks;
  mg_solve_stats* s;
  double first = -1.0;
  std::vector<double> hist;

  // Returns MG_OK to continue, or the final status; sets *done when converged.
  mg_status step(double res, bool* done) {
    *done = false;
    hist.push_back(res);
    if (s->hist_len < 128) s->res_hist[s->hist_len++] = res;
    if (first < 0) first = res;
    s->res = res;
    if (!(res == res)) {
      set_error("residual is not finite");
      return MG_ENAN;
    }
    if (res < tol) {
      *done = true;
      return MG_OK;
    }
    if ((int)hist.size() > max_checks) {
      set_error("no convergence within max_cycles");
      return MG_ENOCONV;
    }
    if (res > 1e3 * first) {
      set_error("residual grew by more than 1e3");
      return MG_ENOCONV;
    }
    const size_t k = hist.size();
    if (k > 8 && res > 0.9 * hist[k - 9]) {
      set_error("residual stalled (less than 10% progress over 8 checks)");
      return MG_ENOCONV;
    }
    return MG_OK;
  }
};

mg_status mixed_solve(Domain* d, const mg_options& o, cudaStream_t st, const OpConst64* ops,
                      int branch, double alpha, double kappa, double tol, mg_solve_stats* s);

mg_status domain_prepare_sources(Domain* d, cudaStream_t st, int branch, double alpha,
                                 double kappa, int guard, double omega,
                                 std::vector<OpConst64>& ops, double w) {
  ops.resize(d->nlev);
  DCK(cudaMemsetAsync(d->d_sc, 0, sizeof(LevelScalars) * (2 * d->nlev + 2), st));
  for (int l = 0; l < d->nlev; ++l) {
    ops[l] = make_op64(d->lv[l].n, alpha, kappa, branch, w);
    ops[l].omega = omega;
    double a, b;
    src_coefficients(ops[l], kappa, &a, &b);
    launch_affine64(st, d->lv[l].cells, d->lv[l].delta, d->lv[l].src, a, b, ops[l].c3,
                    guard == MG_GUARD_FLOOR && ops[l].mode != OP_LINEAR,
                    l == 0 ? &d->d_sc[0].floored : nullptr);
  }
  DCK(cudaGetLastError());
  return MG_OK;
}

mg_status domain_solve(Domain* d, const mg_options& o, cudaStream_t st, int branch, double alpha,
                       double kappa, double tol, mg_solve_stats* s) {
  std::memset(s, 0, sizeof(*s));
  s->levels = d->nlev;
  const long long launches0 = tl_launches;
  std::vector<OpConst64> ops;
  mg_status rs = domain_prepare_sources(d, st, branch, alpha, kappa, o.guard, o.omega, ops, o.w);
  if (rs != MG_OK) return rs;
  cudaEvent_t e0, e1;
  DCK(cudaEventCreate(&e0));
  DCK(cudaEventCreate(&e1));
  DCK(cudaEventRecord(e0, st));
  mg_status result = MG_OK;
  if (o.prec == MG_MIXED && d->nlev > 1) {
    result = mixed_solve(d, o, st, ops.data(), branch, alpha, kappa, tol, s);
  } else {
    EventPairs ta, tb;
    ta.enabled = tb.enabled = o.time_kernels != 0;
    ta.first_only = tb.first_only = o.time_kernels == 2;
    Cycle64 cyc{d, &o, st, ops.data(), &ta, &tb};
    domain_invalidate_graphs(d);
    const bool single = d->nlev == 1;
    long long na = 0, nb = 0;
    if (o.use_graphs) {
      ta.capturing = tb.capturing = true;
      if (single) {
        d->gexec[0] = capture_graph(st, &na, [&] { cyc.part_single(); });
      } else {
        d->gexec[0] = capture_graph(st, &na, [&] { cyc.part_a(); });
        d->gexec[1] = capture_graph(st, &nb, [&] { cyc.part_b(); });
      }
      ta.capturing = tb.capturing = false;
    }
    const bool graphs = o.use_graphs && d->gexec[0] && (single || d->gexec[1]);
    const int pairs_a = ta.n, pairs_b = tb.n;
    const double cells_per_launch = (double)d->lv[0].cells / 4.0;
    bool b_pending = false;
    auto harvest = [&](EventPairs& t, int pairs) {
      if (!t.enabled) return;
      if (!graphs) pairs = t.n;
      const int keep = t.n;
      t.n = pairs;
      s->kernel_ms += t.read_ms();
      s->kernel_launches += pairs;
      s->kernel_cells += pairs * cells_per_launch;
      t.n = keep;
    };
    ConvTracker tr{tol, o.max_cycles, s};
    for (;;) {
      if (!graphs) ta.n = 0;
      if (graphs) {
        DCK(cudaGraphLaunch(d->gexec[0], st));
        tl_launches += na;
      } else if (single) {
        cyc.part_single();
      } else {
        cyc.part_a();
      }
      DCK(cudaStreamSynchronize(st));
      DCK(cudaGetLastError());
      if (!single) harvest(ta, pairs_a);
      if (b_pending) harvest(tb, pairs_b);
      b_pending = false;
      bool done;
      s->guard_hits = o.guard == MG_GUARD_FLOOR ? (long long)d->h_sc[0].floored
                                                : d->h_sc[0].guards;
      s->lambda = d->h_sc[0].lambda;
      if (o.tau_stop > 0.0 && !single) {
        // stop at a fraction of the truncation error as well (Sec. III.C)
        s->tau = d->h_sc[1].res;
        tr.tol = std::max(tol, o.tau_stop * s->tau);
      }
      result = tr.step(d->h_sc[0].res, &done);
      if (done || result != MG_OK) break;
      if (!single) {
        if (!graphs) tb.n = 0;
        if (graphs) {
          DCK(cudaGraphLaunch(d->gexec[1], st));
          tl_launches += nb;
        } else {
          cyc.part_b();
        }
        b_pending = true;
      }
      s->cycles += 1;
    }
    s->res0 = tr.first;
  }
  // gauge: mean(phi) = 0 on the finest level
  launch_gauge64(st, d->lv[0].cells, d->lv[0].phi, d->d_part, d->d_sc + 2 * d->nlev + 1);
  DCK(cudaEventRecord(e1, st));
  DCK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->wall_s = ms * 1e-3;
  s->status = result;
  s->launches = tl_launches - launches0;
  DCK(cudaGetLastError());
  return result;
}

}  // namespace mg
