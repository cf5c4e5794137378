/*
 * CPU oracle for the DGP brane-bending scalar field solver (arXiv:1303.0008).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library; the two meet only through seeded inputs.
 *
 * Plain, slow, obviously correct FP64 C.  Every function cites the passage of the
 * paper it follows.  The solve is the paper's algorithm in the paper's order:
 *   - the discrete operator L^h and its Sigma_ijk (Sec. III.B, the expanded
 *     Sigma_ijk equation and the L^h equation), with w = 1/3 (Sec. III.A, after
 *     Eq. two_branch) unless the caller passes another w;
 *   - the root of Eq. two_branch with the sign chosen by the caller, the
 *     physical one being sgn(alpha) (Eq. one_branch);
 *   - one Newton-Raphson step per cell, phi_new = phi_old - L/(dL/dphi), in
 *     lexicographic Gauss-Seidel order (Sec. III.B, the Newton-Gauss-Seidel
 *     update and its Jacobian diagonal);
 *   - FAS V-cycles: residual, restriction, coarse equation
 *     L^H(phi^H) = L^H(R phi^h) - R d^h, prolongation of the correction
 *     (Sec. III.C, Eqs. fine_grid_eqn onward), repeated until |d^h| < eps.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   - parameters: the caller gives alpha_B = R_c^2/(3 beta a^4) (the coefficient
 *     of the nonlinear term of Eq. code_eqn) and kappa = Omega_m a / beta (its
 *     source coefficient).  The paper's alpha is 1/alpha_B and its
 *     source term inside Sigma is alpha * kappa * delta.  alpha_B = 0 is the
 *     linearised limit, L^h phi = lap(phi)/h^2 - kappa delta.
 *   - guard: when alpha^2 + 4(1-w) Sigma < 0 the square root is taken of 0 (the
 *     real part of the complex root), the cell is counted, and the
 *     1/sqrt term of the Jacobian is dropped.
 *   - periodic compatibility: on a periodic grid the discrete nonlinear term
 *     does not sum to zero, so the solved system is L^h phi = f + lambda with
 *     lambda = mean(L^h phi - f) and mean(phi) = 0; the reported residual is
 *     max|d - lambda|.  Refinement levels (Dirichlet) have lambda = 0.
 *   - transfers: R = mean of the 8 children; P = cell-centred trilinear
 *     (weights 3/4 and 1/4 per axis).
 *   - refinements: a level-l cell outside every level-l patch but inside the
 *     stencil of a patch cell takes the trilinear interpolation of level l-1
 *     (Sec. III.C, first paragraph, and Sec. IV.D); the patch union is solved
 *     with those values fixed, by plain lexicographic Newton-Gauss-Seidel until
 *     |d| < eps (the fixed point does not depend on the iteration).
 *   - force: g = -(1/2) grad(phi) with the central difference of Sec. III.B
 *     (the fifth force is half the gradient of phi, Sec. II.B).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 4
#define ORC_ENAN 5

static long orc_idx(int i, int j, int k, int n) {
  return (long)i + (long)n * ((long)j + (long)n * (long)k);
}

static int orc_wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

/* Parameters of the equation in the caller's convention (see the header). */
typedef struct {
  double alpha_B; /* coefficient of [(lap phi)^2 - (grad grad phi)^2] */
  double kappa;   /* source coefficient, rhs = kappa * delta           */
  double w;       /* operator-splitting constant, 1/3 in the paper     */
  int branch;     /* sign in front of the square root; 0 = sgn(alpha) */
} orc_params;

/*
 * The paper's L^h and dL^h/dphi_ijk at one cell from its 3x3x3 neighbourhood
 * v[dz+1][dy+1][dx+1] (only the 6 faces, 12 edges and the centre are read).
 *   Sec. III.B: second differences, cross differences with the 1/(4h^2)
 *   factor, Sigma_ijk expanded term by term, L^h, and dL^h/dphi.
 */
static void orc_cell_operator(const double v[3][3][3], double delta, double h,
                              const orc_params* p, double* L, double* dL,
                              int* guard) {
  const double c = v[1][1][1];
  const double dxx = v[1][1][2] + v[1][1][0] - 2.0 * c;
  const double dyy = v[1][2][1] + v[1][0][1] - 2.0 * c;
  const double dzz = v[2][1][1] + v[0][1][1] - 2.0 * c;
  /* phi(i+1,j+1)+phi(i-1,j-1)-phi(i+1,j-1)-phi(i-1,j+1), and the xz, yz ones */
  const double cxy = v[1][2][2] + v[1][0][0] - v[1][0][2] - v[1][2][0];
  const double cxz = v[2][1][2] + v[0][1][0] - v[0][1][2] - v[2][1][0];
  const double cyz = v[2][2][1] + v[0][0][1] - v[0][2][1] - v[2][0][1];
  const double lapraw = dxx + dyy + dzz;
  const double h2 = h * h;
  const double h4 = h2 * h2;
  const double w = p->w;
  *guard = 0;
  if (p->alpha_B == 0.0) {
    /* linearised limit: the root tends to kappa*delta as alpha -> infinity */
    *L = lapraw / h2 - p->kappa * delta;
    *dL = -6.0 / h2;
    return;
  }
  const double alpha = 1.0 / p->alpha_B; /* the paper's alpha */
  double sigma = (1.0 - w) / h4 * (dxx * dxx + dyy * dyy + dzz * dzz);
  sigma -= 2.0 / h4 * w * dxx * dyy;
  sigma -= 2.0 / h4 * w * dxx * dzz;
  sigma -= 2.0 / h4 * w * dyy * dzz;
  sigma += 1.0 / (8.0 * h4) * cxy * cxy;
  sigma += 1.0 / (8.0 * h4) * cxz * cxz;
  sigma += 1.0 / (8.0 * h4) * cyz * cyz;
  sigma += alpha * p->kappa * delta;
  double disc = alpha * alpha + 4.0 * (1.0 - w) * sigma;
  if (disc < 0.0) {
    disc = 0.0;
    *guard = 1;
  }
  const double sgn = (p->branch == 0) ? (alpha > 0.0 ? 1.0 : -1.0)
                                      : (p->branch > 0 ? 1.0 : -1.0);
  const double root = sqrt(disc);
  const double lap_phi = (-alpha + sgn * root) / (2.0 * (1.0 - w));
  *L = lapraw / h2 - lap_phi;
  *dL = -6.0 / h2;
  if (root > 0.0) *dL += sgn * 4.0 * (1.0 - 3.0 * w) / (h4 * root) * lapraw;
}

/* Gather the 3x3x3 neighbourhood of (i,j,k) on a periodic n^3 grid. */
static void orc_gather_periodic(const double* phi, int n, int i, int j, int k,
                                double v[3][3][3]) {
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        v[dz + 1][dy + 1][dx + 1] =
            phi[orc_idx(orc_wrap(i + dx, n), orc_wrap(j + dy, n),
                        orc_wrap(k + dz, n), n)];
}

/* d = L^h phi - f on a periodic grid (Sec. III.C, residual equation).
 * f may be NULL (f = 0, the finest level).  Returns the number of guarded cells. */
long orc_residual(int n, double h, const double* phi, const double* delta,
                  const double* f, double alpha_B, double kappa, int branch,
                  double w, double* d) {
  orc_params p = {alpha_B, kappa, w, branch};
  long guards = 0;
  double v[3][3][3];
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = orc_idx(i, j, k, n);
        double L, dL;
        int g;
        orc_gather_periodic(phi, n, i, j, k, v);
        orc_cell_operator(v, delta[c], h, &p, &L, &dL, &g);
        guards += g;
        d[c] = L - (f ? f[c] : 0.0);
      }
  return guards;
}

/* One lexicographic Newton-Gauss-Seidel sweep of L^h phi = f + lambda
 * (Sec. III.B, Newton-Gauss-Seidel update), periodic grid, in place. */
static void orc_sweep_periodic(int n, double h, double* phi, const double* delta,
                               const double* f, double lambda,
                               const orc_params* p) {
  double v[3][3][3];
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = orc_idx(i, j, k, n);
        double L, dL;
        int g;
        orc_gather_periodic(phi, n, i, j, k, v);
        orc_cell_operator(v, delta[c], h, p, &L, &dL, &g);
        phi[c] -= (L - (f ? f[c] : 0.0) - lambda) / dL;
      }
}

/*
 * Source floor (a reading of Sec. III.A): the operator splitting keeps the
 * discriminant alpha^2 + 4(1-w) Sigma of Eq. two_branch non-negative for any field
 * as long as its source part alpha^2 + 4(1-w) alpha kappa delta is, i.e.
 * 1 + 4(1-w) alpha_B kappa delta >= 0.  Cells below that bound get the delta that
 * meets it with equality.  out may alias delta.  Returns the cells changed.
 */
long orc_density_floor(long cells, const double* delta, double alpha_B, double kappa,
                       double w, double* out) {
  const double t = 4.0 * (1.0 - w) * alpha_B * kappa;
  long hits = 0;
  for (long c = 0; c < cells; ++c) {
    double v = delta[c];
    if (t != 0.0 && 1.0 + t * v < 0.0) {
      v = -1.0 / t;
      ++hits;
    }
    out[c] = v;
  }
  return hits;
}

/* Cell-centred full weighting: the mean of the 8 children (reading of the
 * restriction operator R of Sec. III.C).  nc = coarse cells per side. */
void orc_restrict(int nc, const double* fine, double* coarse) {
  int nf = 2 * nc;
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

/* Cell-centred trilinear value of a periodic coarse field at the centre of fine
 * cell (i,j,k): per axis weight 3/4 on the parent and 1/4 on the parent's
 * neighbour on the child's side (reading of the prolongation P of Sec. III.C). */
static double orc_trilinear_periodic(const double* coarse, int nc, int i, int j,
                                     int k) {
  int I = i >> 1, J = j >> 1, K = k >> 1;
  int sI = (i & 1) ? 1 : -1, sJ = (j & 1) ? 1 : -1, sK = (k & 1) ? 1 : -1;
  double val = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        double wt = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (c ? 0.25 : 0.75);
        val += wt * coarse[orc_idx(orc_wrap(I + a * sI, nc),
                                   orc_wrap(J + b * sJ, nc),
                                   orc_wrap(K + c * sK, nc), nc)];
      }
  return val;
}

/* fine += P(corr), corr on the nc^3 coarse grid (Sec. III.C, correction). */
void orc_prolong_add(int nc, const double* corr, double* fine) {
  int nf = 2 * nc;
  for (int k = 0; k < nf; ++k)
    for (int j = 0; j < nf; ++j)
      for (int i = 0; i < nf; ++i)
        fine[orc_idx(i, j, k, nf)] += orc_trilinear_periodic(corr, nc, i, j, k);
}

/* Force output: g = -(1/2) grad phi, central differences (Sec. III.B gradient;
 * the fifth force is half the gradient of phi, Sec. II.B).  out: 3 x n^3 SoA. */
void orc_force(int n, double h, const double* phi, double* out) {
  long cells = (long)n * n * n;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        long c = orc_idx(i, j, k, n);
        double gx = (phi[orc_idx(orc_wrap(i + 1, n), j, k, n)] -
                     phi[orc_idx(orc_wrap(i - 1, n), j, k, n)]) / (2.0 * h);
        double gy = (phi[orc_idx(i, orc_wrap(j + 1, n), k, n)] -
                     phi[orc_idx(i, orc_wrap(j - 1, n), k, n)]) / (2.0 * h);
        double gz = (phi[orc_idx(i, j, orc_wrap(k + 1, n), n)] -
                     phi[orc_idx(i, j, orc_wrap(k - 1, n), n)]) / (2.0 * h);
        out[c] = -0.5 * gx;
        out[cells + c] = -0.5 * gy;
        out[2 * cells + c] = -0.5 * gz;
      }
}

/* ---------------------------------------------------------------------------
 * Periodic FAS V-cycle (Sec. III.C).
 * ------------------------------------------------------------------------- */
typedef struct {
  int n;
  double h;
  double *phi, *delta, *f, *d, *phihat;
  double lambda;
} orc_level;

/* lambda = mean(d), returns max|d - lambda| (the residual of the bordered
 * periodic system; see the header). */
static double orc_project(long cells, const double* d, double* lambda_out) {
  double s = 0.0;
  for (long c = 0; c < cells; ++c) s += d[c];
  double lam = s / (double)cells;
  double m = 0.0;
  for (long c = 0; c < cells; ++c) {
    double a = fabs(d[c] - lam);
    if (!(a <= m)) m = a; /* propagates NaN */
  }
  *lambda_out = lam;
  return m;
}

static long orc_cells(int n) { return (long)n * n * n; }

static double orc_level_residual(orc_level* lv, const orc_params* p,
                                 long* guards) {
  long g = orc_residual(lv->n, lv->h, lv->phi, lv->delta, lv->f, p->alpha_B,
                        p->kappa, p->branch, p->w, lv->d);
  if (guards) *guards = g;
  return orc_project(orc_cells(lv->n), lv->d, &lv->lambda);
}

/* Coarsest level: sweeps until the residual falls by 1e-6 or 200 sweeps. */
static void orc_coarsest_solve(orc_level* lv, const orc_params* p) {
  double r0 = orc_level_residual(lv, p, NULL);
  for (int s = 0; s < 200; ++s) {
    orc_sweep_periodic(lv->n, lv->h, lv->phi, lv->delta, lv->f, lv->lambda, p);
    double r = orc_level_residual(lv, p, NULL);
    if (!(r > 1e-6 * r0)) break;
  }
}

static void orc_vcycle(orc_level* lv, int l, int nlev, const orc_params* p,
                       int nu_pre, int nu_post) {
  orc_level* L0 = &lv[l];
  if (l == nlev - 1) {
    orc_coarsest_solve(L0, p);
    return;
  }
  orc_level* L1 = &lv[l + 1];
  long cf = orc_cells(L0->n), cc = orc_cells(L1->n);
  for (int s = 0; s < nu_pre; ++s)
    orc_sweep_periodic(L0->n, L0->h, L0->phi, L0->delta, L0->f, L0->lambda, p);
  /* d^h = L^h(phi^h) - f^h, lambda^h = mean(d^h), r = d - lambda */
  orc_level_residual(L0, p, NULL);
  for (long c = 0; c < cf; ++c) L0->d[c] -= L0->lambda;
  /* coarse equation: L^H(phi^H) = L^H(R phi^h) - R d^h */
  orc_restrict(L1->n, L0->phi, L1->phi);
  memcpy(L1->phihat, L1->phi, sizeof(double) * cc);
  double* rd = (double*)malloc(sizeof(double) * cc);
  orc_restrict(L1->n, L0->d, rd);
  orc_residual(L1->n, L1->h, L1->phi, L1->delta, NULL, p->alpha_B, p->kappa,
               p->branch, p->w, L1->f);
  for (long c = 0; c < cc; ++c) L1->f[c] -= rd[c];
  free(rd);
  L1->lambda = 0.0;
  orc_vcycle(lv, l + 1, nlev, p, nu_pre, nu_post);
  /* phi^h += P(phi^H - R phi^h) */
  for (long c = 0; c < cc; ++c) L1->phihat[c] = L1->phi[c] - L1->phihat[c];
  orc_prolong_add(L1->n, L1->phihat, L0->phi);
  for (int s = 0; s < nu_post; ++s)
    orc_sweep_periodic(L0->n, L0->h, L0->phi, L0->delta, L0->f, L0->lambda, p);
}

/* Number of multigrid levels: halve while the coarse size stays even, >= 4
 * and the current size is above `coarsest`. */
int orc_num_levels(int n, int coarsest) {
  int nl = 1;
  while (n > coarsest && (n % 2) == 0 && (n / 2) >= 4 && ((n / 2) % 2) == 0) {
    n /= 2;
    ++nl;
  }
  return nl;
}

/*
 * Solve L^h phi = lambda (f = 0 on the finest level, Sec. III.C) on a periodic
 * n^3 grid by FAS V-cycles until max|d - lambda| < tol.  phi is the initial
 * guess on entry and the gauge-fixed (zero-mean) solution on exit.
 * stats (may be NULL), 6 + max_cycles entries:
 *   [0] cycles  [1] final residual  [2] lambda  [3] guarded cells (last residual)
 *   [4] status  [5] initial residual  [6..] residual after each cycle
 */
int orc_fas_solve(int n, const double* delta, double* phi, double alpha_B,
                  double kappa, int branch, double w, double tol,
                  int max_cycles, int nu_pre, int nu_post, int coarsest,
                  double* stats) {
  if (n < 4 || (n % 2) != 0 || max_cycles < 0 || nu_pre < 0 || nu_post < 0)
    return ORC_EINVAL;
  if (alpha_B == 0.0 && branch < 0) return ORC_EINVAL;
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
  if (oom) {
    for (int l = 0; l < nlev; ++l) {
      if (l > 0) { free(lv[l].phi); free(lv[l].f); }
      free(lv[l].delta); free(lv[l].d); free(lv[l].phihat);
    }
    free(lv);
    return ORC_ENOMEM;
  }
  memcpy(lv[0].delta, delta, sizeof(double) * (size_t)orc_cells(n));
  for (int l = 1; l < nlev; ++l) orc_restrict(lv[l].n, lv[l - 1].delta, lv[l].delta);

  long guards = 0;
  double res = orc_level_residual(&lv[0], &p, &guards);
  double res0 = res;
  int status = ORC_OK, cycles = 0;
  if (stats) stats[5] = res0;
  while (!(res < tol)) {
    if (res != res) { status = ORC_ENAN; break; }
    if (cycles >= max_cycles) { status = ORC_ENOCONV; break; }
    orc_vcycle(lv, 0, nlev, &p, nu_pre, nu_post);
    res = orc_level_residual(&lv[0], &p, &guards);
    if (stats) stats[6 + cycles] = res;
    ++cycles;
    if (res > 1e3 * res0) { status = ORC_ENOCONV; break; }
  }
  /* gauge: mean(phi) = 0 */
  long cells = orc_cells(n);
  double s = 0.0;
  for (long c = 0; c < cells; ++c) s += phi[c];
  s /= (double)cells;
  for (long c = 0; c < cells; ++c) phi[c] -= s;
  if (stats) {
    stats[0] = cycles;
    stats[1] = res;
    stats[2] = lv[0].lambda;
    stats[3] = (double)guards;
    stats[4] = status;
  }
  for (int l = 0; l < nlev; ++l) {
    if (l > 0) { free(lv[l].phi); free(lv[l].f); }
    free(lv[l].delta);
    free(lv[l].d);
    free(lv[l].phihat);
  }
  free(lv);
  return status;
}

/* Plain lexicographic Newton-Gauss-Seidel sweeps on a periodic grid with a given
 * f and lambda (used by the tests to check the smoother's fixed point). */
void orc_gs_sweeps(int n, double* phi, const double* delta, const double* f,
                   double lambda, double alpha_B, double kappa, int branch,
                   double w, int sweeps) {
  orc_params p = {alpha_B, kappa, w, branch};
  for (int s = 0; s < sweeps; ++s)
    orc_sweep_periodic(n, 1.0 / (double)n, phi, delta, f, lambda, &p);
}

/* ---------------------------------------------------------------------------
 * Refinement levels (Sec. III.C first paragraph; Sec. IV.D).
 *
 * Level l has cells of size h_l = 1/(n0 * 2^l) on a periodic index space of
 * side n_l = n0 * 2^l.  A patch is an 8^3 block of level-l cells whose origin is
 * a multiple of 8.  Patch p stores its cells at phi[p*512 + i + 8(j + 8k)].
 * The parent level (l-1) is either the periodic domain grid (l = 1, a dense
 * n0^3 array) or another patch set.
 * ------------------------------------------------------------------------- */
#define ORC_PS 8
#define ORC_PC 512

typedef struct {
  int n;               /* cells per side of this level's index space */
  int count;           /* patches */
  const int32_t* org;  /* 3*count origins (level cells) */
  int* table;          /* (n/8)^3 block -> patch index or -1 */
} orc_patchset;

static int orc_patchset_init(orc_patchset* ps, int n, int count,
                             const int32_t* org) {
  int nb = n / ORC_PS;
  ps->n = n;
  ps->count = count;
  ps->org = org;
  ps->table = (int*)malloc(sizeof(int) * (size_t)nb * nb * nb);
  if (!ps->table) return ORC_ENOMEM;
  for (long b = 0; b < (long)nb * nb * nb; ++b) ps->table[b] = -1;
  for (int q = 0; q < count; ++q) {
    int x = org[3 * q], y = org[3 * q + 1], z = org[3 * q + 2];
    if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n ||
        (x % ORC_PS) || (y % ORC_PS) || (z % ORC_PS))
      return ORC_EINVAL;
    long b = orc_idx(x / ORC_PS, y / ORC_PS, z / ORC_PS, nb);
    if (ps->table[b] >= 0) return ORC_EINVAL; /* duplicate */
    ps->table[b] = q;
  }
  return ORC_OK;
}

/* Location of level cell (x,y,z) (periodic): patch index and offset, or -1. */
static int orc_patch_find(const orc_patchset* ps, int x, int y, int z,
                          long* off) {
  x = orc_wrap(x, ps->n);
  y = orc_wrap(y, ps->n);
  z = orc_wrap(z, ps->n);
  int nb = ps->n / ORC_PS;
  int q = ps->table[orc_idx(x / ORC_PS, y / ORC_PS, z / ORC_PS, nb)];
  if (q < 0) return -1;
  *off = (long)q * ORC_PC +
         orc_idx(x % ORC_PS, y % ORC_PS, z % ORC_PS, ORC_PS);
  return q;
}

/* Value of the parent level at parent cell (X,Y,Z); sets *missing if absent. */
static double orc_parent_value(int parent_is_domain, int n_parent,
                               const double* parent_dense,
                               const orc_patchset* parent_ps,
                               const double* parent_phi, int X, int Y, int Z,
                               int* missing) {
  if (parent_is_domain)
    return parent_dense[orc_idx(orc_wrap(X, n_parent), orc_wrap(Y, n_parent),
                                orc_wrap(Z, n_parent), n_parent)];
  long off;
  if (orc_patch_find(parent_ps, X, Y, Z, &off) < 0) {
    *missing = 1;
    return 0.0;
  }
  return parent_phi[off];
}

/* Trilinear interpolation of the parent level at the centre of level cell
 * (x,y,z): the same cell-centred weights as the prolongation. */
static double orc_ghost_value(int parent_is_domain, int n_parent,
                              const double* parent_dense,
                              const orc_patchset* parent_ps,
                              const double* parent_phi, int x, int y, int z,
                              int* missing) {
  int X = x >> 1, Y = y >> 1, Z = z >> 1;
  int sX = (x & 1) ? 1 : -1, sY = (y & 1) ? 1 : -1, sZ = (z & 1) ? 1 : -1;
  double val = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        double wt = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (c ? 0.25 : 0.75);
        val += wt * orc_parent_value(parent_is_domain, n_parent, parent_dense,
                                     parent_ps, parent_phi, X + a * sX,
                                     Y + b * sY, Z + c * sZ, missing);
      }
  return val;
}

typedef struct {
  orc_patchset ps;
  int parent_is_domain;
  int n_parent;
  const double* parent_dense;
  orc_patchset parent_ps;
  const double* parent_phi;
} orc_reflevel;

/* Neighbourhood of a patch cell: union cells from their patch, other cells
 * from the coarse-to-fine fill. */
static int orc_gather_patch(const orc_reflevel* rl, const double* phi, int q,
                            int i, int j, int k, double v[3][3][3]) {
  int missing = 0;
  int x0 = rl->ps.org[3 * q] + i, y0 = rl->ps.org[3 * q + 1] + j,
      z0 = rl->ps.org[3 * q + 2] + k;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz == 3) { v[dz + 1][dy + 1][dx + 1] = 0.0; continue; } /* unused corner */
        long off;
        if (orc_patch_find(&rl->ps, x0 + dx, y0 + dy, z0 + dz, &off) >= 0)
          v[dz + 1][dy + 1][dx + 1] = phi[off];
        else
          v[dz + 1][dy + 1][dx + 1] = orc_ghost_value(
              rl->parent_is_domain, rl->n_parent, rl->parent_dense,
              &rl->parent_ps, rl->parent_phi, x0 + dx, y0 + dy, z0 + dz,
              &missing);
      }
  return missing;
}

static int orc_reflevel_init(orc_reflevel* rl, int n0, int level, int count,
                             const int32_t* org, const double* parent,
                             int parent_count, const int32_t* parent_org) {
  memset(rl, 0, sizeof(*rl));
  if (level < 1 || n0 < 4) return ORC_EINVAL;
  int n = n0 << level;
  int st = orc_patchset_init(&rl->ps, n, count, org);
  if (st) return st;
  rl->parent_is_domain = (level == 1);
  rl->n_parent = n / 2;
  if (rl->parent_is_domain) {
    rl->parent_dense = parent;
  } else {
    st = orc_patchset_init(&rl->parent_ps, n / 2, parent_count, parent_org);
    if (st) return st;
    rl->parent_phi = parent;
  }
  return ORC_OK;
}

static void orc_reflevel_free(orc_reflevel* rl) {
  free(rl->ps.table);
  free(rl->parent_ps.table);
}

/*
 * Residual d = L^h phi on the union of the level's patches (Dirichlet fill
 * from the parent, f = 0, lambda = 0).  parent = the dense n0^3 domain field
 * when level == 1, else the packed parent patch field with its origins.
 * Returns the number of guarded cells, or -1 when a ghost needs a parent cell
 * that does not exist (nesting violated).
 */
long orc_patch_residual(int n0, int level, int count, const int32_t* org,
                        const double* phi, const double* delta,
                        const double* parent, int parent_count,
                        const int32_t* parent_org, double alpha_B,
                        double kappa, int branch, double w, double* d) {
  orc_reflevel rl;
  if (orc_reflevel_init(&rl, n0, level, count, org, parent, parent_count,
                        parent_org)) {
    orc_reflevel_free(&rl);
    return -1;
  }
  orc_params p = {alpha_B, kappa, w, branch};
  double h = 1.0 / (double)(n0 << level);
  long guards = 0;
  int missing = 0;
  double v[3][3][3];
  for (int q = 0; q < count; ++q)
    for (int k = 0; k < ORC_PS; ++k)
      for (int j = 0; j < ORC_PS; ++j)
        for (int i = 0; i < ORC_PS; ++i) {
          long c = (long)q * ORC_PC + orc_idx(i, j, k, ORC_PS);
          double L, dL;
          int g;
          missing |= orc_gather_patch(&rl, phi, q, i, j, k, v);
          orc_cell_operator(v, delta[c], h, &p, &L, &dL, &g);
          guards += g;
          d[c] = L;
        }
  orc_reflevel_free(&rl);
  return missing ? -1 : guards;
}

/*
 * Solve a refinement level: lexicographic Newton-Gauss-Seidel over the patches
 * (in list order, cells in lexicographic order) until max|d| < tol (tested every
 * 10 sweeps) or max_sweeps.  phi holds the initial guess on entry.
 * stats (may be NULL): [0] sweeps [1] residual [2] guarded cells [3] status.
 */
int orc_patch_solve(int n0, int level, int count, const int32_t* org,
                    double* phi, const double* delta, const double* parent,
                    int parent_count, const int32_t* parent_org,
                    double alpha_B, double kappa, int branch, double w,
                    double tol, int max_sweeps, double* stats) {
  orc_reflevel rl;
  int st = orc_reflevel_init(&rl, n0, level, count, org, parent, parent_count,
                             parent_org);
  if (st) { orc_reflevel_free(&rl); return st; }
  orc_params p = {alpha_B, kappa, w, branch};
  double h = 1.0 / (double)(n0 << level);
  double v[3][3][3];
  int sweeps = 0, status = ORC_OK;
  double res = 0.0;
  long guards = 0;
  for (;;) {
    /* max |d| over the union (every 10 sweeps) */
    int missing = 0;
    res = 0.0;
    guards = 0;
    for (int q = 0; q < count; ++q)
      for (int k = 0; k < ORC_PS; ++k)
        for (int j = 0; j < ORC_PS; ++j)
          for (int i = 0; i < ORC_PS; ++i) {
            long c = (long)q * ORC_PC + orc_idx(i, j, k, ORC_PS);
            double L, dL;
            int g;
            missing |= orc_gather_patch(&rl, phi, q, i, j, k, v);
            orc_cell_operator(v, delta[c], h, &p, &L, &dL, &g);
            guards += g;
            double a = fabs(L);
            if (!(a <= res)) res = a;
          }
    if (missing) { status = ORC_EINVAL; break; }
    if (res != res) { status = ORC_ENAN; break; }
    if (res < tol) break;
    if (sweeps >= max_sweeps) { status = ORC_ENOCONV; break; }
    for (int s = 0; s < 10; ++s, ++sweeps)
      for (int q = 0; q < count; ++q)
        for (int k = 0; k < ORC_PS; ++k)
          for (int j = 0; j < ORC_PS; ++j)
            for (int i = 0; i < ORC_PS; ++i) {
              long c = (long)q * ORC_PC + orc_idx(i, j, k, ORC_PS);
              double L, dL;
              int g;
              orc_gather_patch(&rl, phi, q, i, j, k, v);
              orc_cell_operator(v, delta[c], h, &p, &L, &dL, &g);
              phi[c] -= L / dL;
            }
  }
  if (stats) {
    stats[0] = sweeps;
    stats[1] = res;
    stats[2] = (double)guards;
    stats[3] = status;
  }
  orc_reflevel_free(&rl);
  return status;
}

/* Coarse-to-fine fill values for every stencil cell of a patch that lies
 * outside the union: out[q*1000 + (i+1) + 10((j+1) + 10(k+1))] for the 10^3
 * ghosted block of patch q; entries inside the union, the corners and the
 * interior are left untouched.  Returns -1 if nesting is violated. */
int orc_patch_ghosts(int n0, int level, int count, const int32_t* org,
                     const double* parent, int parent_count,
                     const int32_t* parent_org, double* out) {
  orc_reflevel rl;
  if (orc_reflevel_init(&rl, n0, level, count, org, parent, parent_count,
                        parent_org)) {
    orc_reflevel_free(&rl);
    return -1;
  }
  int missing = 0;
  for (int q = 0; q < count; ++q)
    for (int k = -1; k <= ORC_PS; ++k)
      for (int j = -1; j <= ORC_PS; ++j)
        for (int i = -1; i <= ORC_PS; ++i) {
          int out_i = (i < 0 || i >= ORC_PS), out_j = (j < 0 || j >= ORC_PS),
              out_k = (k < 0 || k >= ORC_PS);
          int nout = out_i + out_j + out_k;
          if (nout == 0 || nout == 3) continue;
          int x = org[3 * q] + i, y = org[3 * q + 1] + j, z = org[3 * q + 2] + k;
          long off;
          if (orc_patch_find(&rl.ps, x, y, z, &off) >= 0) continue;
          out[(long)q * 1000 + orc_idx(i + 1, j + 1, k + 1, 10)] =
              orc_ghost_value(rl.parent_is_domain, rl.n_parent,
                              rl.parent_dense, &rl.parent_ps, rl.parent_phi, x,
                              y, z, &missing);
        }
  orc_reflevel_free(&rl);
  return missing ? -1 : 0;
}

/* ------------------------------------------------------------------------
 * Mass assignment of particles to a periodic cell-centred grid (Sec. VI: the
 * density on the mesh comes from the triangular-shaped-cloud scheme; the
 * cloud-in-cell scheme is the lower-order member of the same family).
 *
 * Grid of side `nside`, h = 1/nside; cell i has centre (i + 1/2) h.  A particle
 * at x puts the fraction W(u) of its mass into every cell whose centre lies u
 * cells away (per axis, product over axes), with
 *   CIC: W(u) = 1 - |u|                 for |u| < 1
 *   TSC: W(u) = 3/4 - u^2               for |u| <= 1/2
 *        W(u) = (3/2 - |u|)^2 / 2       for 1/2 < |u| < 3/2
 * and 0 beyond.  Masses are in units of the total mass of the box (mean
 * density 1); NULL means 1/count each.  Adds m W / h^3 to rho (x fastest).
 * ---------------------------------------------------------------------- */
static double orc_cloud_weight(int scheme, double u) {
  double a = fabs(u);
  if (scheme == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a <= 0.5) return 0.75 - u * u;
  if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
  return 0.0;
}

int orc_assign(int nside, int scheme, long count, const double* x, const double* y,
               const double* z, const double* mass, double* rho) {
  if (scheme != 1 && scheme != 2) return 1;
  const double inv_h3 = (double)nside * nside * nside;
  for (long p = 0; p < count; ++p) {
    const double m = mass ? mass[p] : 1.0 / (double)count;
    const double s[3] = {x[p] * nside - 0.5, y[p] * nside - 0.5, z[p] * nside - 0.5};
    long base[3];
    for (int a = 0; a < 3; ++a) base[a] = (long)floor(s[a]);
    /* every cell within two cells of the particle, weight from the definition */
    for (int dk = -1; dk <= 2; ++dk)
      for (int dj = -1; dj <= 2; ++dj)
        for (int di = -1; di <= 2; ++di) {
          const long ci = base[0] + di, cj = base[1] + dj, ck = base[2] + dk;
          const double w = orc_cloud_weight(scheme, s[0] - (double)ci) *
                           orc_cloud_weight(scheme, s[1] - (double)cj) *
                           orc_cloud_weight(scheme, s[2] - (double)ck);
          if (w == 0.0) continue;
          const long i = ((ci % nside) + nside) % nside, j = ((cj % nside) + nside) % nside,
                     k = ((ck % nside) + nside) % nside;
          rho[i + (long)nside * (j + (long)nside * k)] += m * w * inv_h3;
        }
  }
  return 0;
}
