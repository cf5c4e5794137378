/*
 * CPU baseline of the oracle: the periodic FAS solve of mg_oracle.c with the
 * Newton-Gauss-Seidel sweeps taken in four-colour order and every loop split
 * over the host cores with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY, like mg_oracle.c: only the test suite and the
 * benchmark's CPU-baseline leg load it, and it shares nothing with the CUDA
 * library.  It includes mg_oracle.c for the cell operator of Sec. III.B
 * (orc_cell_operator), the restriction of Sec. III.C and the projection onto
 * the bordered periodic system, so that both orders apply the same per-cell
 * arithmetic; what differs is only the order of the updates.
 *
 * Order (a reading of Sec. III.B, which sweeps the cells in no stated order):
 * colour c = ((i + k) & 1) + 2 ((j + k) & 1).  No face or edge neighbour of a
 * cell has its colour, so the cells of one colour are independent given the
 * other three and may be updated in parallel; each update is the same Newton
 * step phi -= (L - f - lambda) / (dL/dphi) as the lexicographic sweep.  Both
 * orders converge to the same discrete solution (the pin of this file).
 */
#include "mg_oracle.c"

#include <omp.h>

/* d = L^h phi - f, periodic, in parallel over planes.  Returns guarded cells. */
static long orcc_residual(int n, double h, const double* phi, const double* delta,
                          const double* f, const orc_params* p, double* d) {
  long guards = 0;
#pragma omp parallel for schedule(static) reduction(+ : guards)
  for (int k = 0; k < n; ++k) {
    double v[3][3][3];
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = orc_idx(i, j, k, n);
        double L, dL;
        int g;
        orc_gather_periodic(phi, n, i, j, k, v);
        orc_cell_operator(v, delta[c], h, p, &L, &dL, &g);
        guards += g;
        d[c] = L - (f ? f[c] : 0.0);
      }
  }
  return guards;
}

/* One four-colour Newton-Gauss-Seidel sweep of L^h phi = f + lambda. */
static void orcc_sweep(int n, double h, double* phi, const double* delta,
                       const double* f, double lambda, const orc_params* p) {
  for (int colour = 0; colour < 4; ++colour) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
      double v[3][3][3];
      for (int j = 0; j < n; ++j) {
        /* cells of this colour in row (j, k): i with (i + k) & 1 == colour & 1 */
        if ((((j + k) & 1) << 1) != (colour & 2)) continue;
        for (int i = ((colour & 1) ^ (k & 1)); i < n; i += 2) {
          long c = orc_idx(i, j, k, n);
          double L, dL;
          int g;
          orc_gather_periodic(phi, n, i, j, k, v);
          orc_cell_operator(v, delta[c], h, p, &L, &dL, &g);
          phi[c] -= (L - (f ? f[c] : 0.0) - lambda) / dL;
        }
      }
    }
  }
}

static void orcc_restrict(int nc, const double* fine, double* coarse) {
  int nf = 2 * nc;
#pragma omp parallel for schedule(static)
  for (int K = 0; K < nc; ++K)
    for (int J = 0; J < nc; ++J)
      for (int I = 0; I < nc; ++I) {
        double s = 0.0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
              s += fine[orc_idx(2 * I + dx, 2 * J + dy, 2 * K + dz, nf)];
        coarse[orc_idx(I, J, K, nc)] = s / 8.0;
      }
}

static void orcc_prolong_add(int nc, const double* corr, double* fine) {
  int nf = 2 * nc;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nf; ++k)
    for (int j = 0; j < nf; ++j)
      for (int i = 0; i < nf; ++i)
        fine[orc_idx(i, j, k, nf)] += orc_trilinear_periodic(corr, nc, i, j, k);
}

/* lambda = mean(d); returns max|d - lambda| (parallel form of orc_project). */
static double orcc_project(long cells, const double* d, double* lambda_out) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (long c = 0; c < cells; ++c) s += d[c];
  double lam = s / (double)cells;
  double m = 0.0;
  int nan = 0;
#pragma omp parallel for schedule(static) reduction(max : m) reduction(| : nan)
  for (long c = 0; c < cells; ++c) {
    double a = fabs(d[c] - lam);
    if (a != a) nan = 1;
    else if (a > m) m = a;
  }
  *lambda_out = lam;
  return nan ? NAN : m;
}

static double orcc_level_residual(orc_level* lv, const orc_params* p, long* guards) {
  long g = orcc_residual(lv->n, lv->h, lv->phi, lv->delta, lv->f, p, lv->d);
  if (guards) *guards = g;
  return orcc_project(orc_cells(lv->n), lv->d, &lv->lambda);
}

static void orcc_coarsest_solve(orc_level* lv, const orc_params* p) {
  double r0 = orcc_level_residual(lv, p, NULL);
  for (int s = 0; s < 200; ++s) {
    orcc_sweep(lv->n, lv->h, lv->phi, lv->delta, lv->f, lv->lambda, p);
    double r = orcc_level_residual(lv, p, NULL);
    if (!(r > 1e-6 * r0)) break;
  }
}

/* The V-cycle of Sec. III.C in the order of orc_vcycle. */
static void orcc_vcycle(orc_level* lv, int l, int nlev, const orc_params* p,
                        int nu_pre, int nu_post, double* rd) {
  orc_level* L0 = &lv[l];
  if (l == nlev - 1) {
    orcc_coarsest_solve(L0, p);
    return;
  }
  orc_level* L1 = &lv[l + 1];
  long cf = orc_cells(L0->n), cc = orc_cells(L1->n);
  for (int s = 0; s < nu_pre; ++s)
    orcc_sweep(L0->n, L0->h, L0->phi, L0->delta, L0->f, L0->lambda, p);
  orcc_level_residual(L0, p, NULL);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < cf; ++c) L0->d[c] -= L0->lambda;
  orcc_restrict(L1->n, L0->phi, L1->phi);
  memcpy(L1->phihat, L1->phi, sizeof(double) * cc);
  orcc_restrict(L1->n, L0->d, rd);
  orcc_residual(L1->n, L1->h, L1->phi, L1->delta, NULL, p, L1->f);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < cc; ++c) L1->f[c] -= rd[c];
  L1->lambda = 0.0;
  orcc_vcycle(lv, l + 1, nlev, p, nu_pre, nu_post, rd);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < cc; ++c) L1->phihat[c] = L1->phi[c] - L1->phihat[c];
  orcc_prolong_add(L1->n, L1->phihat, L0->phi);
  for (int s = 0; s < nu_post; ++s)
    orcc_sweep(L0->n, L0->h, L0->phi, L0->delta, L0->f, L0->lambda, p);
}

/*
 * orc_fas_solve with four-colour sweeps on `threads` OpenMP threads (0: the
 * OpenMP default, all cores).  Same arguments and stats layout as
 * orc_fas_solve, plus stats[6 + max_cycles] = the thread count used.
 */
int orc_fas_solve_colour(int n, const double* delta, double* phi, double alpha_B,
                         double kappa, int branch, double w, double tol,
                         int max_cycles, int nu_pre, int nu_post, int coarsest,
                         int threads, double* stats) {
  if (n < 4 || (n % 2) != 0 || max_cycles < 0 || nu_pre < 0 || nu_post < 0 || threads < 0)
    return ORC_EINVAL;
  if (alpha_B == 0.0 && branch < 0) return ORC_EINVAL;
  if (threads > 0) omp_set_num_threads(threads);
  orc_params p = {alpha_B, kappa, w, branch};
  int nlev = orc_num_levels(n, coarsest);
  orc_level* lv = (orc_level*)calloc((size_t)nlev, sizeof(orc_level));
  if (!lv) return ORC_ENOMEM;
  int m = n;
  int oom = 0;
  for (int l = 0; l < nlev; ++l, m /= 2) {
    long cells = orc_cells(m);
    lv[l].n = m;
    lv[l].h = 1.0 / (double)m;
    lv[l].phi = (l == 0) ? phi : (double*)calloc((size_t)cells, sizeof(double));
    lv[l].delta = (double*)calloc((size_t)cells, sizeof(double));
    lv[l].f = (l == 0) ? NULL : (double*)calloc((size_t)cells, sizeof(double));
    lv[l].d = (double*)calloc((size_t)cells, sizeof(double));
    lv[l].phihat = (double*)calloc((size_t)cells, sizeof(double));
    if (!lv[l].phi || !lv[l].delta || (l > 0 && !lv[l].f) || !lv[l].d || !lv[l].phihat)
      oom = 1;
  }
  double* rd = nlev > 1 ? (double*)malloc(sizeof(double) * (size_t)orc_cells(n / 2)) : NULL;
  if (nlev > 1 && !rd) oom = 1;
  if (oom) {
    for (int l = 0; l < nlev; ++l) {
      if (l > 0) { free(lv[l].phi); free(lv[l].f); }
      free(lv[l].delta); free(lv[l].d); free(lv[l].phihat);
    }
    free(lv);
    free(rd);
    return ORC_ENOMEM;
  }
  memcpy(lv[0].delta, delta, sizeof(double) * (size_t)orc_cells(n));
  for (int l = 1; l < nlev; ++l) orcc_restrict(lv[l].n, lv[l - 1].delta, lv[l].delta);

  long guards = 0;
  double res = orcc_level_residual(&lv[0], &p, &guards);
  double res0 = res;
  int status = ORC_OK, cycles = 0;
  if (stats) stats[5] = res0;
  while (!(res < tol)) {
    if (res != res) { status = ORC_ENAN; break; }
    if (cycles >= max_cycles) { status = ORC_ENOCONV; break; }
    orcc_vcycle(lv, 0, nlev, &p, nu_pre, nu_post, rd);
    res = orcc_level_residual(&lv[0], &p, &guards);
    if (stats) stats[6 + cycles] = res;
    ++cycles;
    if (res > 1e3 * res0) { status = ORC_ENOCONV; break; }
  }
  long cells = orc_cells(n);
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (long c = 0; c < cells; ++c) s += phi[c];
  s /= (double)cells;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < cells; ++c) phi[c] -= s;
  if (stats) {
    stats[0] = cycles;
    stats[1] = res;
    stats[2] = lv[0].lambda;
    stats[3] = (double)guards;
    stats[4] = status;
    stats[6 + max_cycles] = (double)omp_get_max_threads();
  }
  for (int l = 0; l < nlev; ++l) {
    if (l > 0) { free(lv[l].phi); free(lv[l].f); }
    free(lv[l].delta);
    free(lv[l].d);
    free(lv[l].phihat);
  }
  free(lv);
  free(rd);
  return status;
}

/* `sweeps` four-colour sweeps of L^h phi = f + lambda on `threads` threads (0:
 * all); returns the thread count used.  For timing the sweep on its own. */
int orc_colour_sweeps(int n, double* phi, const double* delta, const double* f,
                      double lambda, double alpha_B, double kappa, int branch, double w,
                      int sweeps, int threads) {
  if (threads > 0) omp_set_num_threads(threads);
  orc_params p = {alpha_B, kappa, w, branch};
  for (int s = 0; s < sweeps; ++s)
    orcc_sweep(n, 1.0 / (double)n, phi, delta, f, lambda, &p);
  return omp_get_max_threads();
}
