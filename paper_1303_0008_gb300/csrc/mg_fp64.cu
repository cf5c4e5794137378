// FP64 kernels of the periodic FAS V-cycle (Sec. III.B and III.C of
// arXiv:1303.0008): four-colour Newton-Gauss-Seidel sweep, residual with its
// norms, residual evaluation fused with full-weighting restriction, the coarse
// FAS right-hand side, trilinear prolongation of the correction, the coarsest
// solve in one CTA, density restriction, gauge fix and the force output.
//
// Every kernel works on dense n^3 arrays, x fastest (idx = i + n(j + n k)), with
// periodic wrap.  They are FP64-ALU bound on GB300 (about 35-45 FP64 operations
// per cell against 24 bytes of traffic), so they favour a low FP64 instruction
// count over memory tiling.
#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_bodies64.cuh"

namespace mg {

// ---------------------------------------------------------------------------
// Four-colour Gauss-Seidel: colour c = ((i+k)&1) + 2((j+k)&1).  No face or edge
// neighbour of a cell shares its colour (only the corners do, and they are not
// in the 19-point stencil), so the cells of one colour update independently
// and each update is the exact Newton step of Sec. III.B.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_smooth_colour64(int n, double* __restrict__ phi,
                                                         const double* __restrict__ src,
                                                         const double* __restrict__ f,
                                                         const LevelScalars* __restrict__ sc,
                                                         OpConst64 c, int colour) {
  PdlScope pdl_scope;
  b_smooth_colour64(n, phi, src, f, sc, c, colour, blockIdx.x);
}

// d = L^h phi - f with block partial norms.
__global__ void __launch_bounds__(256) k_residual64(int n, const double* __restrict__ phi,
                                                    const double* __restrict__ src,
                                                    const double* __restrict__ f,
                                                    double* __restrict__ dout, OpConst64 c,
                                                    Partial* __restrict__ partials) {
  PdlScope pdl_scope;
  const long long cells = (long long)n * n * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < cells) {
    const int i = (int)(t % n);
    const int j = (int)((t / n) % n);
    const int k = (int)(t / ((long long)n * n));
    const StencilT<double> s = gather_periodic(phi, i, j, k, n);
    bool g;
    const double D = root_Dc(s, phi[t], src[t], c, g);
    const double lap = (s.sx + s.sy + s.sz) - 6.0 * phi[t];
    double d = fma(lap, c.inv_h2, -D);
    if (f) d -= f[t];
    if (dout) dout[t] = d;
    partial_add(p, d, g);
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blockIdx.x] = p;
}

// Residual of the 8 children of each coarse cell, averaged (full weighting),
// together with R phi; the partial norms cover every fine cell.
__global__ void __launch_bounds__(256) k_residual_restrict64(
    int nf, const double* __restrict__ phi, const double* __restrict__ src,
    const double* __restrict__ f, OpConst64 c, double* __restrict__ phi_c,
    double* __restrict__ phihat_c, double* __restrict__ rd_c, Partial* __restrict__ partials) {
  PdlScope pdl_scope;
  b_residual_restrict64(nf, phi, src, f, c, phi_c, phihat_c, rd_c, partials, blockIdx.x);
}

// The same residual restriction in two launches, for levels whose coarse cells
// fill only a few 256-thread blocks: per fine cell the defect and guard flag
// (blocks of any size), then the walk over each coarse cell's children in the
// order and 256-thread partition of k_residual_restrict64 (the same bits).
__global__ void __launch_bounds__(256) k_defect64(int nf, const double* __restrict__ phi,
                                                  const double* __restrict__ src,
                                                  const double* __restrict__ f, OpConst64 c,
                                                  double* __restrict__ dout,
                                                  unsigned char* __restrict__ gout) {
  PdlScope pdl_scope;
  cell_defect64(nf, phi, src, f, c, dout, gout, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_restrict_defects64(
    int nf, const double* __restrict__ phi, const double* __restrict__ din,
    const unsigned char* __restrict__ gin, double* __restrict__ phi_c,
    double* __restrict__ phihat_c, double* __restrict__ rd_c, Partial* __restrict__ partials) {
  PdlScope pdl_scope;
  b_restrict_defects64(nf, phi, din, gin, phi_c, phihat_c, rd_c, partials, blockIdx.x);
}

// The coarse correction phihat_c <- phi_c - phihat_c (R phi is not needed after
// the prolongation), then the prolongation from it: the subtraction is done once
// per coarse cell instead of once per fine cell that reads it.
__global__ void __launch_bounds__(256) k_correction64(long long cells,
                                                      const double* __restrict__ phi_c,
                                                      double* __restrict__ phihat_c) {
  PdlScope pdl_scope;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cells) phihat_c[t] = phi_c[t] - phihat_c[t];
}

__global__ void __launch_bounds__(256) k_prolong_corr64(int nc, const double* __restrict__ corr_c,
                                                        double* __restrict__ phi_f) {
  PdlScope pdl_scope;
  cell_prolong_corr64(nc, corr_c, phi_f, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// One block: reduce the partials in a fixed order and publish the scalars.
__global__ void __launch_bounds__(256) k_finalize(const Partial* __restrict__ partials, int nparts,
                                                  double cells, int periodic,
                                                  LevelScalars* __restrict__ sc) {
  PdlScope pdl_scope;
  b_finalize(partials, nparts, cells, periodic, sc, blockIdx.x);
}

// f^H = L^H(R phi) - (R d - lambda^h); lambda^H starts at 0.
__global__ void __launch_bounds__(256) k_fas_rhs64(int nc, const double* __restrict__ phi_c,
                                                   const double* __restrict__ src_c,
                                                   double* __restrict__ f_c, OpConst64 c,
                                                   const LevelScalars* __restrict__ fine_sc,
                                                   LevelScalars* __restrict__ coarse_sc) {
  PdlScope pdl_scope;
  b_fas_rhs64(nc, phi_c, src_c, f_c, c, fine_sc, coarse_sc, blockIdx.x);
}

// phi^h += P(phi^H - R phi^h): cell-centred trilinear, per axis 3/4 on the parent
// and 1/4 on the parent's neighbour on the child's side.
__global__ void __launch_bounds__(256) k_prolong_correct64(int nc, const double* __restrict__ phi_c,
                                                           const double* __restrict__ phihat_c,
                                                           double* __restrict__ phi_f) {
  PdlScope pdl_scope;
  b_prolong_correct64(nc, phi_c, phihat_c, phi_f, blockIdx.x);
}

// Coarsest level in one CTA (n^3 <= 4096 cells in shared memory): four-colour
// sweeps until max|d - lambda| has fallen by `drop` or `max_sweeps` sweeps.
__global__ void __launch_bounds__(256) k_coarsest64(int n, double* __restrict__ phi,
                                                    const double* __restrict__ src,
                                                    const double* __restrict__ f, OpConst64 c,
                                                    LevelScalars* __restrict__ sc, int max_sweeps,
                                                    double drop, int check_every) {
  PdlScope pdl_scope;
  b_coarsest64(n, phi, src, f, c, sc, max_sweeps, drop, check_every, blockIdx.x);
}

// coarse = mean of the 8 children.
__global__ void __launch_bounds__(256) k_restrict64(int nc, const double* __restrict__ fine,
                                                    double* __restrict__ coarse) {
  PdlScope pdl_scope;
  const int nf = nc << 1;
  const long long cells = (long long)nc * nc * nc;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const int I = (int)(t % nc);
  const int J = (int)((t / nc) % nc);
  const int K = (int)(t / ((long long)nc * nc));
  double s = 0.0;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    s += fine[lidx(2 * I + (ch & 1), 2 * J + ((ch >> 1) & 1), 2 * K + (ch >> 2), nf)];
  coarse[t] = s * 0.125;
}

// src = a * delta + b, optionally held where 1 + c3 kappa delta < 0 (the bound under
// which the root of Eq. two_branch stays real for any field): in the sqrt form
// (b = 1) src >= 0, in the kappa*delta form c3 * src >= -1.  Floored cells are
// counted into *floored.
__global__ void __launch_bounds__(256) k_affine64(long long cells, const double* __restrict__ delta,
                                                  double* __restrict__ out, double a, double b,
                                                  double c3, int floor,
                                                  unsigned long long* __restrict__ floored) {
  PdlScope pdl_scope;
  b_affine64(cells, delta, out, a, b, c3, floor, floored, blockIdx.x);
}

// Partial sums of x (for the gauge fix).
__global__ void __launch_bounds__(256) k_sum_partials(long long cells, const double* __restrict__ x,
                                                      Partial* __restrict__ partials) {
  PdlScope pdl_scope;
  b_sum_partials(cells, x, partials, blockIdx.x);
}

// x -= mean (the mean sits in sc->lambda, computed by k_finalize).
__global__ void __launch_bounds__(256) k_sub_mean(long long cells, double* __restrict__ x,
                                                  const LevelScalars* __restrict__ sc) {
  PdlScope pdl_scope;
  b_sub_mean(cells, x, sc, blockIdx.x);
}

// g = -(1/2) grad phi, central differences; out is 3 x n^3 (x, y, z).
__global__ void __launch_bounds__(256) k_force64(int n, const double* __restrict__ phi,
                                                 double* __restrict__ out) {
  PdlScope pdl_scope;
  const long long cells = (long long)n * n * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const int i = (int)(t % n);
  const int j = (int)((t / n) % n);
  const int k = (int)(t / ((long long)n * n));
  const double sc = -0.25 * (double)n;  // -(1/2) / (2h)
  out[t] = sc * (phi[lidx(wrap_up(i, n), j, k, n)] - phi[lidx(wrap_dn(i, n), j, k, n)]);
  out[cells + t] = sc * (phi[lidx(i, wrap_up(j, n), k, n)] - phi[lidx(i, wrap_dn(j, n), k, n)]);
  out[2 * cells + t] = sc * (phi[lidx(i, j, wrap_up(k, n), n)] - phi[lidx(i, j, wrap_dn(k, n), n)]);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long work, int threads) {
  return (unsigned)((work + threads - 1) / threads);
}

OpConst64 make_op64(int n, double alpha, double kappa, int branch, double w) {
  OpConst64 c{};
  const double h = 1.0 / (double)n;
  c.h2 = h * h;
  c.inv_h2 = (double)n * (double)n;
  c.h2_6 = c.h2 / 6.0;
  c.omega = 1.0;
  const double h4 = c.h2 * c.h2;
  c.c3 = 4.0 * (1.0 - w) * alpha;
  if (alpha == 0.0) {
    c.mode = OP_LINEAR;
    return c;
  }
  const double sigma = (branch == 0) ? 1.0 : ((branch > 0) == (alpha > 0) ? 1.0 : -1.0);
  c.k2 = 2.0 / c.c3;
  c.k2s = sigma * c.k2;
  c.c1 = alpha / (3.0 * h4);
  c.c2 = alpha / (8.0 * h4);
  c.e1 = c.c3 * c.c1;
  c.e2 = c.c3 * c.c2;
  c.e1h = 2.0 * c.e1;
  c.c1h = 2.0 * c.c1;
  c.upd_s = -c.h2 * c.k2s / 6.0;
  // k2 (sigma sqrt(q) - 1) loses about |k2| * eps to cancellation on the physical
  // root; below |alpha| = 1e-4 the conjugate form 2u/(1+sqrt q) is used instead.
  c.mode = (sigma > 0 && fabs(alpha) < 1e-4) ? OP_CONJ : OP_SQRT;
  if (w != 1.0 / 3.0) {
    // Sec. III.B with a general splitting constant: q = src + c3 alpha Sigma_ijk
    c.mode = OP_GENW;
    c.gA = c.c3 * alpha * (1.0 - w) / h4;
    c.gB = -2.0 * c.c3 * alpha * w / h4;
    c.gC = c.c3 * alpha / (8.0 * h4);
    c.gAB = c.gA + c.gB;
  }
  return c;
}

void src_coefficients(const OpConst64& c, double kappa, double* a, double* b) {
  if (c.mode == OP_SQRT || c.mode == OP_GENW) {
    *a = c.c3 * kappa;
    *b = 1.0;
  } else {
    *a = kappa;
    *b = 0.0;
  }
}

thread_local long long tl_launches = 0;

// Threads per block of a per-cell FP64 launch: 256, or 64 where 256-thread
// blocks would not give every SM two blocks.  An SM retires only two FP64
// lane-operations per clock, so on small levels the launch time is set by how
// many SMs the cells reach.  Per-cell results do not depend on the partition.
int tpb_for(long long items) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 1;
  }
  return (long long)blocks_for(items, 256) < 2LL * sms ? 64 : 256;
}

void launch_smooth64(cudaStream_t st, int n, double* phi, const double* src, const double* f,
                     const LevelScalars* sc, const OpConst64& c, int sweeps, EventPairs* timer) {
  const long long per = (long long)(n / 2) * (n / 2) * n;
  const int tpb = tpb_for(per);
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 4; ++colour) {
      // an event between two launches removes their programmatic overlap, so the
      // sampled mode brackets one colour stage per call
      const bool timed = timer && (!timer->first_only || (s == 0 && colour == 0));
      if (timed) timer->begin(st);
      launch_k(k_smooth_colour64, blocks_for(per, tpb), tpb, 0, st, n, phi, src, f, sc, c, colour);
      if (timed) timer->end(st);
    }
  count_launches(4LL * sweeps);
}

int partials_needed(long long cells) { return (int)blocks_for(cells, 128) + 1; }

void launch_residual64(cudaStream_t st, int n, const double* phi, const double* src,
                       const double* f, double* dout, const OpConst64& c, Partial* partials,
                       LevelScalars* sc, int periodic) {
  const long long cells = (long long)n * n * n;
  const unsigned nb = blocks_for(cells, 256);
  launch_k(k_residual64, nb, 256, 0, st, n, phi, src, f, dout, c, partials);
  launch_k(k_finalize, 1, 256, 0, st, partials, (int)nb, (double)cells, periodic, sc);
  count_launches(2);
}

void launch_residual_restrict64(cudaStream_t st, int nf, const double* phi, const double* src,
                                const double* f, const OpConst64& c, double* phi_c,
                                double* phihat_c, double* rd_c, Partial* partials,
                                LevelScalars* sc, double* def, unsigned char* guard) {
  const long long fcells = (long long)nf * nf * nf;
  const long long ccells = fcells / 8;
  const unsigned nb = blocks_for(ccells, 256);
  if (def && guard && fcells <= kTwoStepMaxFine) {
    const int tpb = tpb_for(fcells);
    launch_k(k_defect64, blocks_for(fcells, tpb), tpb, 0, st, nf, phi, src, f, c, def, guard);
    launch_k(k_restrict_defects64, nb, 256, 0, st, nf, phi, (const double*)def,
             (const unsigned char*)guard, phi_c, phihat_c, rd_c, partials);
    count_launches(1);
  } else {
    launch_k(k_residual_restrict64, nb, 256, 0, st, nf, phi, src, f, c, phi_c, phihat_c, rd_c,
             partials);
  }
  launch_k(k_finalize, 1, 256, 0, st, partials, (int)nb, (double)fcells, 1, sc);
  count_launches(2);
}

void launch_fas_rhs64(cudaStream_t st, int nc, const double* phi_c, const double* src_c,
                      double* f_c, const OpConst64& c, const LevelScalars* fine_sc,
                      LevelScalars* coarse_sc) {
  const long long cells = (long long)nc * nc * nc;
  const int tpb = tpb_for(cells);
  launch_k(k_fas_rhs64, blocks_for(cells, tpb), tpb, 0, st, nc, phi_c, src_c, f_c, c, fine_sc,
           coarse_sc);
  count_launches(1);
}

void launch_prolong_correct64(cudaStream_t st, int nc, const double* phi_c,
                              const double* phihat_c, double* phi_f, bool clobber_hat) {
  const long long cells = 8LL * nc * nc * nc;
  if (clobber_hat && cells >= kCorrectionMinFine) {
    const long long cc = cells / 8;
    double* corr = const_cast<double*>(phihat_c);
    launch_k(k_correction64, blocks_for(cc, 256), 256, 0, st, cc, phi_c, corr);
    launch_k(k_prolong_corr64, blocks_for(cells, 256), 256, 0, st, nc, (const double*)corr, phi_f);
    count_launches(1);
    return;
  }
  const int tpb = tpb_for(cells);
  launch_k(k_prolong_correct64, blocks_for(cells, tpb), tpb, 0, st, nc, phi_c, phihat_c, phi_f);
  count_launches(1);
}

void launch_coarsest64(cudaStream_t st, int n, double* phi, const double* src, const double* f,
                       const OpConst64& c, LevelScalars* sc, int max_sweeps, double drop) {
  const size_t smem = 3 * sizeof(double) * (size_t)n * n * n;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_coarsest64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         3 * sizeof(double) * 4096);
    attr_set = true;
  }
  launch_k(k_coarsest64, 1, 256, smem, st, n, phi, src, f, c, sc, max_sweeps, drop, 2);
  count_launches(1);
}

void launch_restrict64(cudaStream_t st, int nc, const double* fine, double* coarse) {
  const long long cells = (long long)nc * nc * nc;
  launch_k(k_restrict64, blocks_for(cells, 256), 256, 0, st, nc, fine, coarse);
  count_launches(1);
}

void launch_affine64(cudaStream_t st, long long cells, const double* x, double* out, double a,
                     double b, double c3, int floor, unsigned long long* floored) {
  launch_k(k_affine64, blocks_for(cells, 256), 256, 0, st, cells, x, out, a, b, c3, floor, floored);
  count_launches(1);
}

void launch_gauge64(cudaStream_t st, long long cells, double* x, Partial* partials,
                    LevelScalars* sc) {
  const unsigned nb = blocks_for(cells, 256);
  launch_k(k_sum_partials, nb, 256, 0, st, cells, x, partials);
  launch_k(k_finalize, 1, 256, 0, st, partials, (int)nb, (double)cells, 1, sc);
  launch_k(k_sub_mean, nb, 256, 0, st, cells, x, sc);
  count_launches(3);
}

// max |x - mean x| into sc->res (sc->lambda = mean x)
void launch_spread64(cudaStream_t st, long long cells, const double* x, Partial* partials,
                     LevelScalars* sc) {
  const unsigned nb = blocks_for(cells, 256);
  launch_k(k_sum_partials, nb, 256, 0, st, cells, x, partials);
  launch_k(k_finalize, 1, 256, 0, st, partials, (int)nb, (double)cells, 1, sc);
  count_launches(2);
}

// out = x + a y
__global__ void __launch_bounds__(256) k_axpy64(long long cells, const double* __restrict__ x,
                                                const double* __restrict__ y, double a,
                                                double* __restrict__ out) {
  PdlScope pdl_scope;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cells) out[t] = fma(a, y[t], x[t]);
}

void launch_axpy64(cudaStream_t st, long long cells, const double* x, const double* y, double a,
                   double* out) {
  if (cells <= 0) return;
  launch_k(k_axpy64, blocks_for(cells, 256), 256, 0, st, cells, x, y, a, out);
  count_launches(1);
}

void launch_force64(cudaStream_t st, int n, const double* phi, double* out) {
  const long long cells = (long long)n * n * n;
  launch_k(k_force64, blocks_for(cells, 256), 256, 0, st, n, phi, out);
  count_launches(1);
}

}  // namespace mg

namespace mg {
void launch_finalize(cudaStream_t st, const Partial* partials, int nparts, double cells,
                     int periodic, LevelScalars* sc) {
  launch_k(k_finalize, 1, 256, 0, st, partials, nparts, cells, periodic, sc);
  count_launches(1);
}
}  // namespace mg
