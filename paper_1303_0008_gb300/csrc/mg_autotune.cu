// Autotuner: pick the sweep counts (and, for the mixed path, the inner V-cycles
// per FP64 correction and the shape of the FP32 sweep: four colour launches with
// their CTA tile, slabs of z planes in a staggered order, or two half sweeps over
// tiles of whole rows)
// that give the shortest time to the
// requested residual on the handle's own problem, and remember the choice in a
// small JSON file keyed by grid size, precision and device name.
//
// Each trial restores the field the caller left in the handle, solves with one
// candidate, and reads the device time of the solve (CUDA events).  Candidates
// that do not converge are discarded.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

static std::string cache_key(int n, int prec) {
  cudaDeviceProp p;
  int dev = 0;
  cudaGetDevice(&dev);
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
  for (char& c : name)
    if (c == '"' || c == '\\') c = '_';
  return "n=" + std::to_string(n) + ",prec=" + (prec == MG_MIXED ? "mixed" : "fp64") +
         ",device=" + name;
}

// The cache is one JSON object: {"<key>": {"nu_pre": a, "nu_post": b,
// "inner_cycles": c, "fuse_coarse": d, "seconds": t}, ...}.  This reader accepts
// exactly the layout the writer below produces.
static std::map<std::string, std::map<std::string, double>> read_cache(const std::string& path) {
  std::map<std::string, std::map<std::string, double>> out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  auto next_string = [&](std::string& v) -> bool {
    const size_t a = s.find('"', i);
    if (a == std::string::npos) return false;
    const size_t b = s.find('"', a + 1);
    if (b == std::string::npos) return false;
    v = s.substr(a + 1, b - a - 1);
    i = b + 1;
    return true;
  };
  while (true) {
    std::string key;
    if (!next_string(key)) break;
    const size_t open = s.find('{', i), close = s.find('}', i);
    if (open == std::string::npos || close == std::string::npos || close < open) break;
    i = open + 1;
    std::map<std::string, double> fields;
    while (true) {
      const size_t q = s.find('"', i);
      if (q == std::string::npos || q > close) break;
      std::string name;
      if (!next_string(name)) break;
      const size_t colon = s.find(':', i);
      if (colon == std::string::npos || colon > close) break;
      fields[name] = std::strtod(s.c_str() + colon + 1, nullptr);
      i = colon + 1;
    }
    out[key] = fields;
    i = close + 1;
  }
  return out;
}

static bool write_cache(const std::string& path,
                        const std::map<std::string, std::map<std::string, double>>& c) {
  std::ofstream f(path, std::ios::trunc);
  if (!f) return false;
  f << "{\n";
  size_t k = 0;
  for (const auto& e : c) {
    f << "  \"" << e.first << "\": {";
    size_t j = 0;
    for (const auto& v : e.second) {
      char buf[64];
      std::snprintf(buf, sizeof(buf), "%.9g", v.second);
      f << "\"" << v.first << "\": " << buf << (++j < e.second.size() ? ", " : "");
    }
    f << "}" << (++k < c.size() ? "," : "") << "\n";
  }
  f << "}\n";
  return (bool)f;
}

}  // namespace mg

using namespace mg;

extern "C" mg_status mg_autotune(mg_grid* g, int branch, double alpha, double kappa, double tol,
                                 const char* cache_path, int use_cache, mg_options* best,
                                 double* best_seconds) {
  if (!g || g->batch) {
    set_error("mg_autotune: needs a domain handle");
    return MG_EINVAL;
  }
  Domain* d = g->domains[0];
  if (!d->density_set) {
    set_error("mg_autotune: density not set");
    return MG_ESTATE;
  }
  const std::string key = cache_key(d->n, g->opt.prec);
  std::map<std::string, std::map<std::string, double>> cache;
  if (cache_path && *cache_path) cache = read_cache(cache_path);
  if (use_cache && cache.count(key)) {
    const auto& e = cache[key];
    mg_options o = g->opt;
    o.nu_pre = (int)e.at("nu_pre");
    o.nu_post = (int)e.at("nu_post");
    o.inner_cycles = (int)e.at("inner_cycles");
    o.fuse_coarse = (int)e.at("fuse_coarse");
    if (e.count("half32")) o.half32 = (int)e.at("half32");
    if (e.count("slab32")) o.slab32 = (int)e.at("slab32");
    if (e.count("tile32")) o.tile32 = (int)e.at("tile32");
    g->opt = o;
    if (best) *best = o;
    if (best_seconds) *best_seconds = e.count("seconds") ? e.at("seconds") : -1.0;
    return MG_OK;
  }
  // keep the caller's field to restart every trial from it
  double* saved = nullptr;
  const size_t bytes = sizeof(double) * (size_t)d->lv[0].cells;
  if (cudaMalloc(&saved, bytes) != cudaSuccess) {
    set_error("mg_autotune: device allocation");
    return MG_ENOMEM;
  }
  cudaMemcpyAsync(saved, d->lv[0].phi, bytes, cudaMemcpyDeviceToDevice, g->stream);
  const mg_options base = g->opt;
  // First stage: pre/post sweep pairs up to 5 that differ by at most one (the
  // strongly nonlinear workloads want more smoothing than the 2/2 default); for
  // the mixed path 3 or 4 inner V-cycles per FP64 correction; the coarse-level
  // fusion only where it matters (n <= 64).  The FP32 sweep shapes give the same
  // bits, so they change the cost of a sweep and not the cycle count: the second
  // stage tries them at the first stage's counts only.
  const int pairs[][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 2}, {2, 3}, {3, 3},
                          {4, 3}, {3, 4}, {4, 4}, {5, 4}, {4, 5}, {5, 5}};
  const bool mixed = base.prec == MG_MIXED;
  const int inner_set[] = {3, 4};
  const bool fuse_matters = d->n <= 64;
  std::vector<mg_options> cands;
  for (const auto& pp : pairs)
    for (int ic = 0; ic < (mixed ? 2 : 1); ++ic)
      for (int fuse = 0; fuse <= (fuse_matters ? 1 : 0); ++fuse) {
        mg_options o = base;
        o.nu_pre = pp[0];
        o.nu_post = pp[1];
        o.inner_cycles = mixed ? inner_set[ic] : base.inner_cycles;
        o.fuse_coarse = fuse_matters ? fuse : base.fuse_coarse;
        cands.push_back(o);
      }
  // small grids: two solves per candidate (the first also captures the graphs and
  // is noisier); from 128^3 on a solve is long enough to time once
  const int reps = d->n <= 64 ? 2 : 1;
  double t_best = 1e300;
  mg_options o_best = base;
  mg_status result = MG_ENOCONV;
  auto trial = [&](const mg_options& o) {
    double t = 0.0;
    bool ok = true;
    for (int rep = 0; rep < reps && ok; ++rep) {
      cudaMemcpyAsync(d->lv[0].phi, saved, bytes, cudaMemcpyDeviceToDevice, g->stream);
      mg_solve_stats st;
      const mg_status s = domain_solve(d, o, g->stream, branch, alpha, kappa, tol, &st);
      ok = (s == MG_OK);
      t = st.wall_s;
    }
    if (ok && t < t_best) {
      t_best = t;
      o_best = o;
      result = MG_OK;
    }
  };
  for (const mg_options& o : cands) trial(o);
  // Second stage (mixed, n >= 256): whole colour stages, slabs, half sweeps.
  if (mixed && result == MG_OK && d->n >= 256) {
    const mg_options first = o_best;
    std::vector<mg_options> shapes;
    mg_options o = first;
    o.half32 = 0;
    o.sweep32 = 0;
    o.pair32 = 0;
    o.slab32 = 0;
    for (int tz : {0, 1, 2, 4, 8}) {
      o.tile32 = tz;
      shapes.push_back(o);
    }
    o.tile32 = first.tile32;
    for (int S : {8, 16, 32, 64})
      if (slab_sweep_applies(d->n, S)) {
        o.slab32 = S;
        shapes.push_back(o);
      }
    if (half_sweep_supported(d->n)) {
      o.slab32 = 0;
      o.half32 = 1;
      shapes.push_back(o);
    }
    for (const mg_options& c : shapes)
      if (c.half32 != first.half32 || c.slab32 != first.slab32 || c.sweep32 != first.sweep32 ||
          c.pair32 != first.pair32 || c.tile32 != first.tile32)
        trial(c);
  }
  cudaMemcpyAsync(d->lv[0].phi, saved, bytes, cudaMemcpyDeviceToDevice, g->stream);
  cudaStreamSynchronize(g->stream);
  cudaFree(saved);
  if (result != MG_OK) {
    set_error("mg_autotune: no candidate converged");
    return result;
  }
  g->opt = o_best;
  if (best) *best = o_best;
  if (best_seconds) *best_seconds = t_best;
  if (cache_path && *cache_path) {
    cache[key] = {{"nu_pre", (double)o_best.nu_pre},
                  {"nu_post", (double)o_best.nu_post},
                  {"inner_cycles", (double)o_best.inner_cycles},
                  {"fuse_coarse", (double)o_best.fuse_coarse},
                  {"half32", (double)o_best.half32},
                  {"slab32", (double)o_best.slab32},
                  {"tile32", (double)o_best.tile32},
                  {"seconds", t_best}};
    if (!write_cache(cache_path, cache)) {
      set_error("mg_autotune: cannot write the cache file");
      return MG_EINVAL;
    }
  }
  return MG_OK;
}
