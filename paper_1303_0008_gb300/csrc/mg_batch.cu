// Batched independent periodic solves.
#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

mg_status batch_prepare(mg_grid* g) { return MG_OK; }
void batch_release(mg_grid* g) {}
mg_status batch_solve(mg_grid* g, const int* branch, const double* alpha, const double* kappa,
                      double tol, mg_solve_stats* stats) {
  mg_status result = MG_OK;
  for (size_t s = 0; s < g->domains.size(); ++s) {
    mg_solve_stats local;
    mg_status st = domain_solve(g->domains[s], g->opt, g->stream, branch[s], alpha[s], kappa[s],
                                tol, stats ? &stats[s] : &local);
    if (st != MG_OK && result == MG_OK) result = st;
  }
  return result;
}

}  // namespace mg
