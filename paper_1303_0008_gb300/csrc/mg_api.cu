// C-ABI of libmg and the host orchestration of the FAS V-cycle
// (Sec. III.C of arXiv:1303.0008).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace mg

using namespace mg;

extern "C" {

const char* mg_last_error(void) { return g_last_error.c_str(); }

void mg_default_options(mg_options* opt) {
  if (!opt) return;
  opt->prec = MG_FP64;
  opt->nu_pre = 2;
  opt->nu_post = 2;
  opt->coarsest = 4;
  opt->max_cycles = 100;
  opt->inner_cycles = 3;
  opt->use_graphs = 1;
  opt->coarse_sweeps = 4;
  opt->coarse_drop = 1e-2;
  opt->time_kernels = 0;
  opt->guard = MG_GUARD_FLOOR;
  opt->patch_coarse_sweeps = 8;
  opt->fuse_coarse = 1;
  opt->omega = 1.0;
  opt->omega_patch = 1.0;
  opt->patch_mg_levels = 3;
  opt->patch_cgc = 1.0;
  opt->sweep32 = 0;
  opt->pair32 = 0;
  opt->tau_stop = 0.0;
  opt->w = 1.0 / 3.0;
  opt->patch_galerkin = 1;
  opt->half32 = 0;
  opt->barrier_timeout_s = 1.0;
  opt->slab32 = 0;
  opt->tile32 = 4;
}

static mg_status check_options(const mg_options& o) {
  if (o.prec != MG_FP64 && o.prec != MG_MIXED) MG_FAIL(MG_EINVAL, "options: unknown precision");
  if (o.time_kernels < 0 || o.time_kernels > 2) MG_FAIL(MG_EINVAL, "options: time_kernels must be 0, 1 or 2");
  if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post < 1 || o.nu_pre > 16 ||
      o.nu_post > 16)
    MG_FAIL(MG_EINVAL, "options: nu_pre/nu_post must be in [0,16] with a positive sum");
  if (o.coarsest < 4) MG_FAIL(MG_EINVAL, "options: coarsest must be >= 4");
  if (o.max_cycles < 0 || o.max_cycles > 100000) MG_FAIL(MG_EINVAL, "options: max_cycles");
  if (o.inner_cycles < 1 || o.inner_cycles > 64) MG_FAIL(MG_EINVAL, "options: inner_cycles");
  if (o.coarse_sweeps < 1 || o.coarse_sweeps > 100000) MG_FAIL(MG_EINVAL, "options: coarse_sweeps");
  if (!(o.coarse_drop > 0.0 && o.coarse_drop < 1.0)) MG_FAIL(MG_EINVAL, "options: coarse_drop");
  if (o.guard != MG_GUARD_FLOOR && o.guard != MG_GUARD_ROOT) MG_FAIL(MG_EINVAL, "options: guard");
  if (o.patch_coarse_sweeps < 1 || o.patch_coarse_sweeps > 10000)
    MG_FAIL(MG_EINVAL, "options: patch_coarse_sweeps");
  if (o.fuse_coarse != 0 && o.fuse_coarse != 1) MG_FAIL(MG_EINVAL, "options: fuse_coarse");
  if (!(o.omega > 0.0 && o.omega <= 1.0) || !(o.omega_patch > 0.0 && o.omega_patch <= 1.0))
    MG_FAIL(MG_EINVAL, "options: omega and omega_patch must be in (0, 1]");
  if (o.patch_mg_levels < 1 || o.patch_mg_levels > 3) MG_FAIL(MG_EINVAL, "options: patch_mg_levels");
  if (!(o.patch_cgc > 0.0 && o.patch_cgc <= 1.0)) MG_FAIL(MG_EINVAL, "options: patch_cgc");
  if (o.sweep32 != 0 && o.sweep32 != 1) MG_FAIL(MG_EINVAL, "options: sweep32");
  if (o.pair32 != 0 && o.pair32 != 1) MG_FAIL(MG_EINVAL, "options: pair32");
  if (!(o.tau_stop >= 0.0 && o.tau_stop < 1e3)) MG_FAIL(MG_EINVAL, "options: tau_stop");
  if (!(o.w >= 0.0 && o.w < 1.0)) MG_FAIL(MG_EINVAL, "options: w");
  if (o.patch_galerkin != 0 && o.patch_galerkin != 1) MG_FAIL(MG_EINVAL, "options: patch_galerkin");
  if (o.half32 != 0 && o.half32 != 1) MG_FAIL(MG_EINVAL, "options: half32");
  if (!(o.barrier_timeout_s >= 0.0 && o.barrier_timeout_s <= 3600.0))
    MG_FAIL(MG_EINVAL, "options: barrier_timeout_s must be in [0, 3600]");
  if (o.slab32 != 0 && !(o.slab32 >= 8 && o.slab32 <= 256 && (o.slab32 & (o.slab32 - 1)) == 0))
    MG_FAIL(MG_EINVAL, "options: slab32 must be 0 or a power of two from 8 to 256");
  if (o.tile32 != 0 && o.tile32 != 1 && o.tile32 != 2 && o.tile32 != 4 && o.tile32 != 8)
    MG_FAIL(MG_EINVAL, "options: tile32 must be 0, 1, 2, 4 or 8");
  return MG_OK;
}

mg_status mg_create_grid(mg_grid** out, int n, const mg_options* opt) {
  if (!out) MG_FAIL(MG_EINVAL, "mg_create_grid: out is NULL");
  *out = nullptr;
  mg_options o;
  mg_default_options(&o);
  if (opt) o = *opt;
  mg_status st = check_options(o);
  if (st != MG_OK) return st;
  Domain* d = nullptr;
  st = domain_create(&d, n, o);
  if (st != MG_OK) return st;
  mg_grid* g = new (std::nothrow) mg_grid();
  if (!g) {
    domain_destroy(d);
    MG_FAIL(MG_ENOMEM, "mg_create_grid: host allocation");
  }
  g->opt = o;
  g->domains.push_back(d);
  g->batch = false;
  cudaGetDevice(&g->device);
  if (cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    domain_destroy(d);
    delete g;
    MG_FAIL(MG_ECUDA, "mg_create_grid: stream creation failed");
  }
  g->stream = g->own_stream;
  *out = g;
  return MG_OK;
}

mg_status mg_create_batch(mg_grid** out, int count, const int* n, const mg_options* opt) {
  if (!out || !n || count < 1 || count > 4096) MG_FAIL(MG_EINVAL, "mg_create_batch: bad arguments");
  *out = nullptr;
  mg_options o;
  mg_default_options(&o);
  if (opt) o = *opt;
  mg_status st = check_options(o);
  if (st != MG_OK) return st;
  mg_grid* g = new (std::nothrow) mg_grid();
  if (!g) MG_FAIL(MG_ENOMEM, "mg_create_batch: host allocation");
  g->opt = o;
  g->batch = true;
  cudaGetDevice(&g->device);
  for (int s = 0; s < count; ++s) {
    Domain* d = nullptr;
    st = domain_create(&d, n[s], o);
    if (st != MG_OK) {
      mg_destroy_grid(g);
      return st;
    }
    g->domains.push_back(d);
  }
  if (cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    mg_destroy_grid(g);
    MG_FAIL(MG_ECUDA, "mg_create_batch: stream creation failed");
  }
  g->stream = g->own_stream;
  st = batch_prepare(g);
  if (st != MG_OK) {
    mg_destroy_grid(g);
    return st;
  }
  *out = g;
  return MG_OK;
}

void mg_destroy_grid(mg_grid* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (Domain* d : g->domains) domain_destroy(d);
  for (auto& pl : g->patch_levels) patch_level_destroy(pl);
  batch_release(g);
  if (g->force_tmp) cudaFree(g->force_tmp);
  for (auto* v : {&g->nw_phi, &g->nw_ghost, &g->nw_psi, &g->nw_psi_ghost})
    for (double* p : *v) cudaFree(p);
  if (g->own_stream) cudaStreamDestroy(g->own_stream);
  delete g;
}

mg_status mg_get_level_stats(const mg_grid* g, int level, mg_solve_stats* out) {
  if (!g || !out || g->batch) MG_FAIL(MG_EINVAL, "mg_get_level_stats: arguments");
  if (level < 1 || level > (int)g->patch_levels.size() || !g->patch_levels[level - 1])
    MG_FAIL(MG_EINVAL, "mg_get_level_stats: no patches on that level");
  const PatchLevel* pl = g->patch_levels[level - 1];
  std::memset(out, 0, sizeof(*out));
  out->cycles = pl->last_cycles;
  out->status = pl->last_status;
  out->levels = 3;
  out->res = pl->last_res;
  out->wall_s = pl->last_wall_s;
  out->res0 = pl->last_hist.empty() ? 0.0 : pl->last_hist.front();
  for (double r : pl->last_hist)
    if (out->hist_len < 128) out->res_hist[out->hist_len++] = r;
  return MG_OK;
}

mg_status mg_get_options(const mg_grid* g, mg_options* out) {
  if (!g || !out) MG_FAIL(MG_EINVAL, "mg_get_options: NULL argument");
  *out = g->opt;
  return MG_OK;
}

mg_status mg_set_options(mg_grid* g, const mg_options* opt) {
  if (!g || !opt) MG_FAIL(MG_EINVAL, "mg_set_options: NULL argument");
  mg_options o = *opt;
  o.coarsest = g->opt.coarsest;
  mg_status st = check_options(o);
  if (st != MG_OK) return st;
  g->opt = o;
  for (Domain* d : g->domains) domain_invalidate_graphs(d);
  return MG_OK;
}

mg_status mg_set_stream(mg_grid* g, void* stream) {
  if (!g) MG_FAIL(MG_EINVAL, "mg_set_stream: NULL handle");
  MG_CK(cudaStreamSynchronize(g->stream));
  g->stream = stream ? (cudaStream_t)stream : g->own_stream;
  for (Domain* d : g->domains) domain_invalidate_graphs(d);
  return MG_OK;
}

static mg_status copy_in(mg_grid* g, double* dst, const double* src, size_t count, int on_device) {
  if (!src) MG_FAIL(MG_EINVAL, "input pointer is NULL");
  MG_CK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        g->stream));
  if (!on_device) MG_CK(cudaStreamSynchronize(g->stream));
  return MG_OK;
}

static mg_status copy_out(const mg_grid* g, double* dst, const double* src, size_t count,
                          int on_device) {
  if (!dst) MG_FAIL(MG_EINVAL, "output pointer is NULL");
  MG_CK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        g->stream));
  if (!on_device) MG_CK(cudaStreamSynchronize(g->stream));
  return MG_OK;
}

// Resolve (level, patch) to a device range.
static mg_status resolve(const mg_grid* g, int level, int patch, bool field, double** ptr,
                         size_t* count) {
  if (g->batch) {
    if (level != 0 || patch < 0 || patch >= (int)g->domains.size())
      MG_FAIL(MG_EINVAL, "batch handle: level must be 0 and patch a solve index");
    Domain* d = g->domains[patch];
    *ptr = field ? d->lv[0].phi : d->lv[0].delta;
    *count = (size_t)d->lv[0].cells;
    return MG_OK;
  }
  if (level == 0) {
    if (patch != -1) MG_FAIL(MG_EINVAL, "level 0 takes patch = -1");
    Domain* d = g->domains[0];
    *ptr = field ? d->lv[0].phi : d->lv[0].delta;
    *count = (size_t)d->lv[0].cells;
    return MG_OK;
  }
  if (level < 1 || level > (int)g->patch_levels.size() || !g->patch_levels[level - 1])
    MG_FAIL(MG_EINVAL, "no patches on that level");
  PatchLevel* pl = g->patch_levels[level - 1];
  if (patch < -1 || patch >= pl->count) MG_FAIL(MG_EINVAL, "patch index out of range");
  double* base = field ? pl->phi : pl->delta;
  if (patch == -1) {
    *ptr = base;
    *count = (size_t)pl->count * 512;
  } else {
    *ptr = base + (size_t)patch * 512;
    *count = 512;
  }
  return MG_OK;
}

mg_status mg_set_density(mg_grid* g, int level, int patch, const double* delta, int on_device) {
  if (!g) MG_FAIL(MG_EINVAL, "mg_set_density: NULL handle");
  double* dst;
  size_t cnt;
  mg_status st = resolve(g, level, patch, false, &dst, &cnt);
  if (st != MG_OK) return st;
  st = copy_in(g, dst, delta, cnt, on_device);
  if (st != MG_OK) return st;
  if (level == 0) {
    Domain* d = g->batch ? g->domains[patch] : g->domains[0];
    domain_restrict_density(d, g->stream);
    d->density_set = true;
    MG_CK(cudaGetLastError());
  } else {
    patch_restrict_density(g, g->patch_levels[level - 1]);
    MG_CK(cudaGetLastError());
    g->patch_levels[level - 1]->density_set = true;
  }
  return MG_OK;
}

mg_status mg_set_field(mg_grid* g, int level, int patch, const double* phi, int on_device) {
  if (!g) MG_FAIL(MG_EINVAL, "mg_set_field: NULL handle");
  double* dst;
  size_t cnt;
  mg_status st = resolve(g, level, patch, true, &dst, &cnt);
  if (st != MG_OK) return st;
  if (level > 0 && !g->batch) {
    PatchLevel* pl = g->patch_levels[level - 1];
    if (!phi) {
      // no values: the next solve starts the level from the level below
      if (patch != -1) MG_FAIL(MG_EINVAL, "mg_set_field: NULL phi resets a whole level (patch -1)");
      pl->phi_set = false;
      return MG_OK;
    }
    st = copy_in(g, dst, phi, cnt, on_device);
    if (st == MG_OK) pl->phi_set = true;
    return st;
  }
  return copy_in(g, dst, phi, cnt, on_device);
}

mg_status mg_get_field(const mg_grid* g, int level, int patch, double* out, int on_device) {
  if (!g) MG_FAIL(MG_EINVAL, "mg_get_field: NULL handle");
  double* src;
  size_t cnt;
  mg_status st = resolve(g, level, patch, true, &src, &cnt);
  if (st != MG_OK) return st;
  return copy_out(g, out, src, cnt, on_device);
}

mg_status mg_get_density(const mg_grid* g, int level, int patch, double* out, int on_device) {
  if (!g) MG_FAIL(MG_EINVAL, "mg_get_density: NULL handle");
  double* src;
  size_t cnt;
  mg_status st = resolve(g, level, patch, false, &src, &cnt);
  if (st != MG_OK) return st;
  return copy_out(g, out, src, cnt, on_device);
}

mg_status mg_get_force(const mg_grid* g_const, int level, int patch, double* out, int on_device) {
  mg_grid* g = const_cast<mg_grid*>(g_const);
  if (!g) MG_FAIL(MG_EINVAL, "mg_get_force: NULL handle");
  if (!out) MG_FAIL(MG_EINVAL, "mg_get_force: out is NULL");
  double* src;
  size_t cnt;
  mg_status st = resolve(g, level, patch, true, &src, &cnt);
  if (st != MG_OK) return st;
  const size_t bytes = 3 * cnt * sizeof(double);
  double* dst = out;
  if (!on_device) {
    if (g->force_tmp_bytes < bytes) {
      if (g->force_tmp) cudaFree(g->force_tmp);
      g->force_tmp = nullptr;
      g->force_tmp_bytes = 0;
      if (cudaMalloc(&g->force_tmp, bytes) != cudaSuccess)
        MG_FAIL(MG_ENOMEM, "mg_get_force: device allocation");
      g->force_tmp_bytes = bytes;
    }
    dst = g->force_tmp;
  }
  if (g->batch || level == 0) {
    Domain* d = g->batch ? g->domains[patch] : g->domains[0];
    launch_force64(g->stream, d->n, d->lv[0].phi, dst);
  } else {
    st = patch_force(g, level, patch, dst);
    if (st != MG_OK) return st;
  }
  MG_CK(cudaGetLastError());
  if (!on_device) {
    MG_CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, g->stream));
    MG_CK(cudaStreamSynchronize(g->stream));
  }
  return MG_OK;
}

mg_status mg_add_patches(mg_grid* g, int level, int count, const int32_t* origin) {
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_add_patches: needs a domain handle");
  return patches_add(g, level, count, origin);
}

static mg_status check_branch(int branch, double alpha) {
  if (branch < -1 || branch > 1) MG_FAIL(MG_EINVAL, "branch must be -1, 0 or +1");
  if (alpha == 0.0 && branch != 0) MG_FAIL(MG_EINVAL, "alpha = 0 is linear: branch must be 0");
  if (!std::isfinite(alpha)) MG_FAIL(MG_EINVAL, "alpha must be finite");
  return MG_OK;
}

mg_status mg_solve(mg_grid* g, int branch, double alpha, double kappa, double tol,
                   mg_solve_stats* stats) {
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_solve: needs a domain handle");
  mg_status st = check_branch(branch, alpha);
  if (st != MG_OK) return st;
  if (!std::isfinite(kappa) || !(tol > 0.0)) MG_FAIL(MG_EINVAL, "mg_solve: kappa/tol");
  Domain* d = g->domains[0];
  if (!d->density_set) MG_FAIL(MG_ESTATE, "mg_solve: density not set");
  if (g->opt.w != 1.0 / 3.0 && alpha != 0.0) {
    if (g->opt.prec != MG_FP64) MG_FAIL(MG_EINVAL, "mg_solve: w != 1/3 needs MG_FP64");
    for (PatchLevel* pl : g->patch_levels)
      if (pl && pl->count) MG_FAIL(MG_EINVAL, "mg_solve: w != 1/3 on refinement levels");
  }
  mg_solve_stats local;
  mg_solve_stats* s = stats ? stats : &local;
  st = domain_solve(d, g->opt, g->stream, branch, alpha, kappa, tol, s);
  if (st != MG_OK) return st;
  for (size_t l = 0; l < g->patch_levels.size(); ++l) {
    PatchLevel* pl = g->patch_levels[l];
    if (!pl || pl->count == 0) continue;
    if (!pl->density_set) MG_FAIL(MG_ESTATE, "mg_solve: patch density not set");
    mg_status ps = patch_level_solve(g, (int)l + 1, branch, alpha, kappa, tol, !pl->phi_set);
    pl->phi_set = true;  // the last iterate is the next solve's initial guess
    if (ps != MG_OK) return ps;
  }
  return MG_OK;
}

mg_status mg_solve_batch(mg_grid* g, const int* branch, const double* alpha, const double* kappa,
                         double tol, mg_solve_stats* stats) {
  if (!g || !g->batch) MG_FAIL(MG_EINVAL, "mg_solve_batch: needs a batch handle");
  if (!branch || !alpha || !kappa || !(tol > 0.0)) MG_FAIL(MG_EINVAL, "mg_solve_batch: arguments");
  if (g->opt.w != 1.0 / 3.0) MG_FAIL(MG_EINVAL, "mg_solve_batch: w must be 1/3");
  for (size_t s = 0; s < g->domains.size(); ++s) {
    mg_status st = check_branch(branch[s], alpha[s]);
    if (st != MG_OK) return st;
    if (!std::isfinite(kappa[s])) MG_FAIL(MG_EINVAL, "mg_solve_batch: kappa");
    if (!g->domains[s]->density_set) MG_FAIL(MG_ESTATE, "mg_solve_batch: density not set");
  }
  return batch_solve(g, branch, alpha, kappa, tol, stats);
}

// ---------------------------------------------------------------------------
// Single-kernel entry points
// ---------------------------------------------------------------------------
static mg_status check_n(int n) {
  if (n < 4 || (n & 1) || n > 1024) MG_FAIL(MG_EINVAL, "n must be even and in [4, 1024]");
  return MG_OK;
}

struct TmpBuf {
  void* p = nullptr;
  ~TmpBuf() {
    if (p) cudaFree(p);
  }
};

mg_status mg_op_residual(int n, const double* phi, const double* delta, const double* f,
                         int branch, double alpha, double kappa, double* d, double* norms,
                         void* stream) {
  mg_status st = check_n(n);
  if (st != MG_OK) return st;
  st = check_branch(branch, alpha);
  if (st != MG_OK) return st;
  if (!phi || !delta) MG_FAIL(MG_EINVAL, "mg_op_residual: NULL input");
  cudaStream_t s = (cudaStream_t)stream;
  const long long cells = (long long)n * n * n;
  const OpConst64 c = make_op64(n, alpha, kappa, branch);
  TmpBuf src, part, sc;
  if (cudaMalloc(&src.p, cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&part.p, partials_needed(cells) * sizeof(Partial)) != cudaSuccess ||
      cudaMalloc(&sc.p, sizeof(LevelScalars)) != cudaSuccess)
    MG_FAIL(MG_ENOMEM, "mg_op_residual: device allocation");
  double a, b;
  src_coefficients(c, kappa, &a, &b);
  launch_affine64(s, cells, delta, (double*)src.p, a, b);
  launch_residual64(s, n, phi, (double*)src.p, f, d, c, (Partial*)part.p, (LevelScalars*)sc.p, 1);
  MG_CK(cudaGetLastError());
  LevelScalars h;
  MG_CK(cudaMemcpyAsync(&h, sc.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  MG_CK(cudaStreamSynchronize(s));
  if (norms) {
    norms[0] = h.sum;
    norms[1] = h.dmax;
    norms[2] = h.dmin;
    norms[3] = (double)h.guards;
    norms[4] = (double)h.nonfinite;
  }
  return MG_OK;
}

mg_status mg_op_smooth(int n, double* phi, const double* delta, const double* f, int branch,
                       double alpha, double kappa, double lambda, int sweeps, void* stream) {
  mg_status st = check_n(n);
  if (st != MG_OK) return st;
  st = check_branch(branch, alpha);
  if (st != MG_OK) return st;
  if (!phi || !delta || sweeps < 0) MG_FAIL(MG_EINVAL, "mg_op_smooth: arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const long long cells = (long long)n * n * n;
  const OpConst64 c = make_op64(n, alpha, kappa, branch);
  TmpBuf src, sc;
  if (cudaMalloc(&src.p, cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sc.p, sizeof(LevelScalars)) != cudaSuccess)
    MG_FAIL(MG_ENOMEM, "mg_op_smooth: device allocation");
  LevelScalars h{};
  h.lambda = lambda;
  MG_CK(cudaMemcpyAsync(sc.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  double a, b;
  src_coefficients(c, kappa, &a, &b);
  launch_affine64(s, cells, delta, (double*)src.p, a, b);
  launch_smooth64(s, n, phi, (double*)src.p, f, (LevelScalars*)sc.p, c, sweeps);
  MG_CK(cudaGetLastError());
  MG_CK(cudaStreamSynchronize(s));
  return MG_OK;
}

mg_status mg_op_restrict(int n, const double* fine, double* coarse, void* stream) {
  mg_status st = check_n(n);
  if (st != MG_OK) return st;
  if (!fine || !coarse) MG_FAIL(MG_EINVAL, "mg_op_restrict: NULL pointer");
  launch_restrict64((cudaStream_t)stream, n / 2, fine, coarse);
  MG_CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_op_prolong_correct(int n, const double* coarse, const double* coarse_ref,
                                double* fine, void* stream) {
  mg_status st = check_n(n);
  if (st != MG_OK) return st;
  if (n / 2 < 2 || !coarse || !coarse_ref || !fine)
    MG_FAIL(MG_EINVAL, "mg_op_prolong_correct: arguments");
  launch_prolong_correct64((cudaStream_t)stream, n / 2, coarse, coarse_ref, fine);
  MG_CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_op_force(int n, const double* phi, double* out, void* stream) {
  mg_status st = check_n(n);
  if (st != MG_OK) return st;
  if (!phi || !out) MG_FAIL(MG_EINVAL, "mg_op_force: NULL pointer");
  launch_force64((cudaStream_t)stream, n, phi, out);
  MG_CK(cudaGetLastError());
  return MG_OK;
}

// ---------------------------------------------------------------------------
// Newtonian potential (Eq. newton) and total force -grad(phi_N + phi / 2)
// ---------------------------------------------------------------------------
namespace {

void free_vec(std::vector<double*>& v) {
  for (double* p : v) cudaFree(p);
  v.clear();
}

// phi_N buffers (zeroed when first made or when the patch layout changed) and
// the scratch of the total force, one entry per level.
mg_status ensure_newton(mg_grid* g) {
  const size_t nl = 1 + g->patch_levels.size();
  std::vector<size_t> cells(nl, 0), ghosts(nl, 0);
  cells[0] = (size_t)g->domains[0]->lv[0].cells;
  for (size_t l = 1; l < nl; ++l) {
    const PatchLevel* pl = g->patch_levels[l - 1];
    cells[l] = pl ? (size_t)pl->count * 512 : 0;
    ghosts[l] = pl ? (size_t)pl->count * 1000 : 0;
  }
  if (cells == g->nw_cells && ghosts == g->nw_ghost_cells) return MG_OK;
  for (auto* v : {&g->nw_phi, &g->nw_ghost, &g->nw_psi, &g->nw_psi_ghost}) free_vec(*v);
  g->newton_set = false;
  g->nw_cells.clear();
  g->nw_ghost_cells.clear();
  for (size_t l = 0; l < nl; ++l) {
    double *a = nullptr, *b = nullptr, *c = nullptr, *e = nullptr;
    bool ok = true;
    if (cells[l]) {
      ok = ok && cudaMalloc(&a, sizeof(double) * cells[l]) == cudaSuccess;
      ok = ok && cudaMalloc(&c, sizeof(double) * cells[l]) == cudaSuccess;
      if (ok) cudaMemsetAsync(a, 0, sizeof(double) * cells[l], g->stream);
    }
    if (ghosts[l]) {
      ok = ok && cudaMalloc(&b, sizeof(double) * ghosts[l]) == cudaSuccess;
      ok = ok && cudaMalloc(&e, sizeof(double) * ghosts[l]) == cudaSuccess;
      if (ok) cudaMemsetAsync(b, 0, sizeof(double) * ghosts[l], g->stream);
    }
    g->nw_phi.push_back(a);
    g->nw_psi.push_back(c);
    g->nw_ghost.push_back(b);
    g->nw_psi_ghost.push_back(e);
    if (!ok) {
      for (auto* v : {&g->nw_phi, &g->nw_ghost, &g->nw_psi, &g->nw_psi_ghost}) free_vec(*v);
      MG_FAIL(MG_ENOMEM, "mg_solve_newton: device allocation");
    }
  }
  g->nw_cells = cells;
  g->nw_ghost_cells = ghosts;
  return MG_OK;
}

// Exchange the solver's field (and ghost) buffers of every level with `phi`
// (and `ghost`); applying it twice restores the handle.
void swap_fields(mg_grid* g, std::vector<double*>& phi, std::vector<double*>& ghost) {
  std::swap(g->domains[0]->lv[0].phi, phi[0]);
  for (size_t l = 1; l < phi.size(); ++l) {
    PatchLevel* pl = g->patch_levels[l - 1];
    if (!pl || pl->count == 0) continue;
    std::swap(pl->phi, phi[l]);
    std::swap(pl->ghost, ghost[l]);
  }
}

}  // namespace

mg_status mg_solve_newton(mg_grid* g, double coef, double tol, mg_solve_stats* stats) {
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_solve_newton: needs a domain handle");
  if (!std::isfinite(coef) || !(tol > 0.0)) MG_FAIL(MG_EINVAL, "mg_solve_newton: coef/tol");
  Domain* d = g->domains[0];
  if (!d->density_set) MG_FAIL(MG_ESTATE, "mg_solve_newton: density not set");
  for (PatchLevel* pl : g->patch_levels)
    if (pl && pl->count && !pl->density_set)
      MG_FAIL(MG_ESTATE, "mg_solve_newton: patch density not set");
  mg_status st = ensure_newton(g);
  if (st != MG_OK) return st;
  mg_solve_stats local;
  mg_solve_stats* s = stats ? stats : &local;
  swap_fields(g, g->nw_phi, g->nw_ghost);
  st = domain_solve(d, g->opt, g->stream, 0, 0.0, coef, tol, s);
  for (size_t l = 0; st == MG_OK && l < g->patch_levels.size(); ++l) {
    PatchLevel* pl = g->patch_levels[l];
    if (!pl || pl->count == 0) continue;
    st = patch_level_solve(g, (int)l + 1, 0, 0.0, coef, tol);
  }
  swap_fields(g, g->nw_phi, g->nw_ghost);
  if (st == MG_OK) g->newton_set = true;
  return st;
}

mg_status mg_get_newton_field(const mg_grid* g_const, int level, int patch, double* out,
                              int on_device) {
  mg_grid* g = const_cast<mg_grid*>(g_const);
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_get_newton_field: needs a domain handle");
  if (!g->newton_set || ensure_newton(g) != MG_OK || !g->newton_set)
    MG_FAIL(MG_ESTATE, "mg_get_newton_field: no Newtonian solve yet");
  swap_fields(g, g->nw_phi, g->nw_ghost);
  const mg_status st = mg_get_field(g, level, patch, out, on_device);
  swap_fields(g, g->nw_phi, g->nw_ghost);
  return st;
}

mg_status mg_get_total_force(const mg_grid* g_const, int level, int patch, double* out,
                             int on_device) {
  mg_grid* g = const_cast<mg_grid*>(g_const);
  if (!g || g->batch) MG_FAIL(MG_EINVAL, "mg_get_total_force: needs a domain handle");
  if (!g->newton_set || ensure_newton(g) != MG_OK || !g->newton_set)
    MG_FAIL(MG_ESTATE, "mg_get_total_force: no Newtonian solve yet");
  if (level < 0 || level >= (int)g->nw_cells.size() || g->nw_cells[level] == 0)
    MG_FAIL(MG_EINVAL, "mg_get_total_force: no such level");
  // psi = phi + 2 phi_N (and the same for the ghost shells, which are linear in
  // the fields), then the fifth-force stencil -1/2 grad psi
  if (level == 0) {
    launch_axpy64(g->stream, (long long)g->nw_cells[0], g->domains[0]->lv[0].phi, g->nw_phi[0],
                  2.0, g->nw_psi[0]);
  } else {
    PatchLevel* pl = g->patch_levels[level - 1];
    launch_axpy64(g->stream, (long long)g->nw_cells[level], pl->phi, g->nw_phi[level], 2.0,
                  g->nw_psi[level]);
    launch_axpy64(g->stream, (long long)g->nw_ghost_cells[level], pl->ghost,
                  g->nw_ghost[level], 2.0, g->nw_psi_ghost[level]);
  }
  MG_CK(cudaGetLastError());
  swap_fields(g, g->nw_psi, g->nw_psi_ghost);
  const mg_status st = mg_get_force(g, level, patch, out, on_device);
  swap_fields(g, g->nw_psi, g->nw_psi_ghost);
  return st;
}

mg_status mg_slab_order(int n, int slab, int* colour, int* z0, int* nz, int cap, int* count) {
  if (!colour || !z0 || !nz || !count) MG_FAIL(MG_EINVAL, "mg_slab_order: NULL pointer");
  if (n < 16 || n > 1024 || slab < 8 || n % slab != 0 || n / slab < 2)
    MG_FAIL(MG_EINVAL, "mg_slab_order: needs slab >= 8, n % slab == 0 and n / slab >= 2");
  const int total = 4 * (n / slab);
  if (cap < total) MG_FAIL(MG_EINVAL, "mg_slab_order: cap smaller than 4 n / slab");
  int m = 0;
  for (int s = 0; s < n / slab; ++s)
    for (int c = 0; c < 4; ++c, ++m) {
      colour[m] = c;
      slab_range(n, slab, c, s, &z0[m], &nz[m]);
    }
  *count = total;
  return MG_OK;
}

}  // extern "C"
