// Per-thread bodies of the FP64 kernels of mg_fp64.cu.  Each b_* body takes the
// block index as an argument so that the single-grid kernels (blk = blockIdx.x)
// and the batched work-list kernels of mg_batch.cu (blk = block within its item)
// run the same code; the cell_* functions take the item index itself, so that
// the cluster sub-cycle (mg_subcycle.cu) can spread items over its CTAs freely.
#pragma once

#include "mg_common.cuh"

namespace mg {

// The block-wide constant of a colour stage (thread 0 computes it into shared
// memory): -h^2 (lambda - k2)/6 in the sqrt form, -h^2 lambda/6 in the root form,
// lambda itself for OP_GENW.
__device__ __forceinline__ double smooth_scalar64(const LevelScalars* __restrict__ sc,
                                                  const OpConst64& c) {
  return c.mode == OP_GENW ? sc->lambda
                           : -c.h2_6 * (c.mode == OP_SQRT ? sc->lambda - c.k2 : sc->lambda);
}

// One cell of a colour stage: t indexes the colour's n^3/4 cells; t >= n^3/4 does
// nothing.
__device__ __forceinline__ void cell_smooth64(int n, double* __restrict__ phi,
                                              const double* __restrict__ src,
                                              const double* __restrict__ f, double s_c,
                                              const OpConst64& c, int colour, long long t) {
  // phi_new = (Sx + Sy + Sz - h^2 (D + f + lambda)) / 6.  In the sqrt form,
  // D = k2s sqrt(q) - k2, so phi_new = upd_s sqrt(q) + (Sx+Sy+Sz)/6 - h^2 f/6 + C with
  // the block-wide C = -h^2 (lambda - k2)/6 (s_c).
  const int hn = n >> 1;
  const long long total = (long long)hn * hn * n;
  if (t >= total) return;
  int m, jj, k;
  split3((unsigned)t, hn, m, jj, k);
  const int i = 2 * m + ((colour ^ k) & 1);
  const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
  const long long id = lidx(i, j, k, n);
  const StencilT<double> s = gather_periodic(phi, i, j, k, n);
  if (c.mode == OP_GENW) {
    const double old = phi[id];
    const double v = genw_newton(s, old, src[id], (f ? f[id] : 0.0) + s_c, c);
    phi[id] = not_one(c.omega) ? fma(c.omega, v - old, old) : v;
    return;
  }
  const double lapnb = s.sx + s.sy + s.sz;
  double acc = fma(lapnb, 1.0 / 6.0, s_c);
  if (f) acc = fma(f[id], -c.h2_6, acc);
  double v;
  if (c.mode == OP_SQRT) {
    const double B = fma(s.cxy, s.cxy, fma(s.cxz, s.cxz, s.cyz * s.cyz));
    const double q = fma(c.e1h, half_A(s), fma(c.e2, B, src[id]));
    v = fma(c.upd_s, sqrt_clamped(q), acc);
  } else {
    bool g;
    v = fma(-c.h2_6, root_D(s, src[id], c, g), acc);
  }
  if (not_one(c.omega)) {
    const double old = phi[id];
    v = fma(c.omega, v - old, old);
  }
  phi[id] = v;
}

__device__ __forceinline__ void b_smooth_colour64(int n, double* __restrict__ phi,
                                                         const double* __restrict__ src,
                                                         const double* __restrict__ f,
                                                         const LevelScalars* __restrict__ sc,
                                                         OpConst64 c, int colour,
    long long blk) {
  __shared__ double s_c;
  if (threadIdx.x == 0) s_c = smooth_scalar64(sc, c);
  __syncthreads();
  cell_smooth64(n, phi, src, f, s_c, c, colour, (long long)blk * blockDim.x + threadIdx.x);
}

// The defect d = L(phi) - f of fine cell (i,j,k) (linear index id) and its guard
// flag; ctr returns phi there.
__device__ __forceinline__ double fine_defect64(int nf, const double* __restrict__ phi,
                                               const double* __restrict__ src,
                                               const double* __restrict__ f,
                                               const OpConst64& c, int i, int j, int k,
                                               long long id, double& ctr, bool& g) {
  const StencilT<double> s = gather_periodic(phi, i, j, k, nf);
  ctr = phi[id];
  const double D = root_Dc(s, ctr, src[id], c, g);
  const double lap = (s.sx + s.sy + s.sz) - 6.0 * ctr;
  double d = fma(lap, c.inv_h2, -D);
  if (f) d -= f[id];
  return d;
}

__device__ __forceinline__ void b_residual_restrict64(
    int nf, const double* __restrict__ phi, const double* __restrict__ src,
    const double* __restrict__ f, OpConst64 c, double* __restrict__ phi_c,
    double* __restrict__ phihat_c, double* __restrict__ rd_c, Partial* __restrict__ partials,
    long long blk) {
  const int nc = nf >> 1;
  const long long ccells = (long long)nc * nc * nc;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < ccells) {
    int I, J, K;
    split3((unsigned)t, nc, I, J, K);
    // The partial norms of the 8 children.  With every child finite, the sum is sd
    // itself (the same additions in the same order) and the extremes are kept as
    // integer order keys, so that the FP64 pipe, GB300's limit here, does only the
    // two sums per child.  A non-finite child sends the coarse cell through the
    // element-wise partial_add again (same values).
    double sphi = 0.0, sd = 0.0;
    long long kmax = order_key(-INFINITY), kmin = order_key(INFINITY), guards = 0;
    int bad = 0;
#pragma unroll 1
    for (int ch = 0; ch < 8; ++ch) {
      const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
      const long long id = lidx(i, j, k, nf);
      bool g;
      double ctr;
      const double d = fine_defect64(nf, phi, src, f, c, i, j, k, id, ctr, g);
      const bool fin = finite_bits(d);
      const long long key = order_key(d);
      kmax = (fin && key > kmax) ? key : kmax;
      kmin = (fin && key < kmin) ? key : kmin;
      bad += fin ? 0 : 1;
      guards += g ? 1 : 0;
      sphi += ctr;
      sd += d;
    }
    if (bad == 0) {
      p.sum = sd;
      p.dmax = from_order_key(kmax);
      p.dmin = from_order_key(kmin);
      p.guards = guards;
    } else {
#pragma unroll 1
      for (int ch = 0; ch < 8; ++ch) {
        const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
        bool g;
        double ctr;
        partial_add(p, fine_defect64(nf, phi, src, f, c, i, j, k, lidx(i, j, k, nf), ctr, g), g);
      }
    }
    phi_c[t] = sphi * 0.125;
    phihat_c[t] = sphi * 0.125;
    rd_c[t] = sd * 0.125;
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blk] = p;
}

// The residual restriction in two steps, for launches whose per-coarse-cell
// loop would leave most SMs idle: cell_defect64 stores each fine cell's defect
// and guard flag (t indexes the nf^3 fine cells), then b_restrict_defects64
// walks every coarse cell's 8 children in the order of b_residual_restrict64,
// with its block partition, so both give the same bits.
__device__ __forceinline__ void cell_defect64(int nf, const double* __restrict__ phi,
                                              const double* __restrict__ src,
                                              const double* __restrict__ f, const OpConst64& c,
                                              double* __restrict__ dout,
                                              unsigned char* __restrict__ gout, long long t) {
  const long long cells = (long long)nf * nf * nf;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nf, i, j, k);
  bool g;
  double ctr;
  dout[t] = fine_defect64(nf, phi, src, f, c, i, j, k, t, ctr, g);
  gout[t] = g ? 1 : 0;
}

__device__ __forceinline__ void b_restrict_defects64(
    int nf, const double* __restrict__ phi, const double* __restrict__ din,
    const unsigned char* __restrict__ gin, double* __restrict__ phi_c,
    double* __restrict__ phihat_c, double* __restrict__ rd_c, Partial* __restrict__ partials,
    long long blk) {
  const int nc = nf >> 1;
  const long long ccells = (long long)nc * nc * nc;
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < ccells) {
    int I, J, K;
    split3((unsigned)t, nc, I, J, K);
    double sphi = 0.0, sd = 0.0;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
      const long long id = lidx(i, j, k, nf);
      const double d = din[id];
      partial_add(p, d, gin[id] != 0);
      sphi += phi[id];
      sd += d;
    }
    phi_c[t] = sphi * 0.125;
    phihat_c[t] = sphi * 0.125;
    rd_c[t] = sd * 0.125;
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blk] = p;
}

// The level norms from the per-block partials: the block-wide merge of b_finalize
// (thread 0 holds the result), and the scalars it stores.
__device__ __forceinline__ Partial merge_partials(const Partial* __restrict__ partials,
                                                  int nparts) {
  Partial p;
  partial_init(p);
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) partial_merge(p, partials[b]);
  return block_reduce(p);
}

__device__ __forceinline__ double level_lambda(const Partial& p, double cells, int periodic) {
  return periodic ? p.sum / cells : 0.0;
}

__device__ __forceinline__ void store_scalars(const Partial& p, double lam,
                                              LevelScalars* __restrict__ sc) {
  sc->lambda = lam;
  sc->sum = p.sum;
  sc->dmax = p.dmax;
  sc->dmin = p.dmin;
  sc->res = (p.nonfinite > 0) ? NAN : fmax(p.dmax - lam, lam - p.dmin);
  sc->guards = p.guards;
  sc->nonfinite = p.nonfinite;
}

__device__ __forceinline__ void b_finalize(const Partial* __restrict__ partials, int nparts,
                                                  double cells, int periodic,
                                                  LevelScalars* __restrict__ sc,
    long long blk) {
  const Partial p = merge_partials(partials, nparts);
  if (threadIdx.x == 0) store_scalars(p, level_lambda(p, cells, periodic), sc);
}

// One coarse cell of the FAS right-hand side f_c = L_c(phi_c) - f_c + lambda_f
// (t indexes the nc^3 cells; lam_f is the fine level's lambda; cell 0 also clears
// the coarse lambda).
__device__ __forceinline__ void cell_fas_rhs64(int nc, const double* __restrict__ phi_c,
                                               const double* __restrict__ src_c,
                                               double* __restrict__ f_c, const OpConst64& c,
                                               double lam_f, LevelScalars* __restrict__ coarse_sc,
                                               long long t) {
  const long long cells = (long long)nc * nc * nc;
  if (t == 0) coarse_sc->lambda = 0.0;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nc, i, j, k);
  const StencilT<double> s = gather_periodic(phi_c, i, j, k, nc);
  bool g;
  const double D = root_Dc(s, phi_c[t], src_c[t], c, g);
  const double lap = (s.sx + s.sy + s.sz) - 6.0 * phi_c[t];
  const double L = fma(lap, c.inv_h2, -D);
  f_c[t] = L - f_c[t] + lam_f;
}

__device__ __forceinline__ void b_fas_rhs64(int nc, const double* __restrict__ phi_c,
                                                   const double* __restrict__ src_c,
                                                   double* __restrict__ f_c, OpConst64 c,
                                                   const LevelScalars* __restrict__ fine_sc,
                                                   LevelScalars* __restrict__ coarse_sc,
    long long blk) {
  cell_fas_rhs64(nc, phi_c, src_c, f_c, c, fine_sc->lambda, coarse_sc,
                 (long long)blk * blockDim.x + threadIdx.x);
}

// One fine cell of the trilinear prolongation of the coarse correction
// phi_c - phihat_c, added to phi_f (t indexes the (2 nc)^3 fine cells).
__device__ __forceinline__ void cell_prolong64(int nc, const double* __restrict__ phi_c,
                                               const double* __restrict__ phihat_c,
                                               double* __restrict__ phi_f, long long t) {
  const int nf = nc << 1;
  const long long cells = (long long)nf * nf * nf;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nf, i, j, k);
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = (i & 1) ? wrap_up(I0, nc) : wrap_dn(I0, nc);
  const int J1 = (j & 1) ? wrap_up(J0, nc) : wrap_dn(J0, nc);
  const int K1 = (k & 1) ? wrap_up(K0, nc) : wrap_dn(K0, nc);
  auto e = [&](int a, int b, int cc) {
    const long long q = lidx(a, b, cc, nc);
    return phi_c[q] - phihat_c[q];
  };
  const double v = 27.0 * e(I0, J0, K0) + 9.0 * (e(I1, J0, K0) + e(I0, J1, K0) + e(I0, J0, K1)) +
                   3.0 * (e(I1, J1, K0) + e(I1, J0, K1) + e(I0, J1, K1)) + e(I1, J1, K1);
  phi_f[t] += v * (1.0 / 64.0);
}

// cell_prolong64 with the coarse correction phi_c - phihat_c already formed in
// corr_c (the same subtractions, so the same bits).
__device__ __forceinline__ void cell_prolong_corr64(int nc, const double* __restrict__ corr_c,
                                                    double* __restrict__ phi_f, long long t) {
  const int nf = nc << 1;
  const long long cells = (long long)nf * nf * nf;
  if (t >= cells) return;
  int i, j, k;
  split3((unsigned)t, nf, i, j, k);
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = (i & 1) ? wrap_up(I0, nc) : wrap_dn(I0, nc);
  const int J1 = (j & 1) ? wrap_up(J0, nc) : wrap_dn(J0, nc);
  const int K1 = (k & 1) ? wrap_up(K0, nc) : wrap_dn(K0, nc);
  auto e = [&](int a, int b, int cc) { return corr_c[lidx(a, b, cc, nc)]; };
  const double v = 27.0 * e(I0, J0, K0) + 9.0 * (e(I1, J0, K0) + e(I0, J1, K0) + e(I0, J0, K1)) +
                   3.0 * (e(I1, J1, K0) + e(I1, J0, K1) + e(I0, J1, K1)) + e(I1, J1, K1);
  phi_f[t] += v * (1.0 / 64.0);
}

__device__ __forceinline__ void b_prolong_correct64(int nc, const double* __restrict__ phi_c,
                                                           const double* __restrict__ phihat_c,
                                                           double* __restrict__ phi_f,
    long long blk) {
  cell_prolong64(nc, phi_c, phihat_c, phi_f, (long long)blk * blockDim.x + threadIdx.x);
}

__device__ __forceinline__ void b_coarsest64(int n, double* __restrict__ phi,
                                                    const double* __restrict__ src,
                                                    const double* __restrict__ f, OpConst64 c,
                                                    LevelScalars* __restrict__ sc, int max_sweeps,
                                                    double drop, int check_every,
    long long blk) {
  extern __shared__ double smem64[];
  __shared__ double s_lam, s_res0, s_res;
  const int cells = n * n * n;
  double* sphi = smem64;
  double* ssrc = smem64 + cells;
  double* sf = smem64 + 2 * cells;
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    sphi[q] = phi[q];
    ssrc[q] = src[q];
    sf[q] = f ? f[q] : 0.0;
  }
  if (threadIdx.x == 0) s_lam = sc->lambda;
  __syncthreads();
  double scale = 0.0;
  auto residual = [&](double& res_out) {
    Partial p;
    partial_init(p);
    double mag = 0.0;
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
      const int i = q % n, j = (q / n) % n, k = q / (n * n);
      const StencilT<double> s = gather_periodic<double>(sphi, i, j, k, n);
      bool g;
      const double D = root_Dc(s, sphi[q], ssrc[q], c, g);
      const double lnb = s.sx + s.sy + s.sz;
      const double lap = lnb - 6.0 * sphi[q];
      partial_add(p, fma(lap, c.inv_h2, -D) - sf[q], g);
      mag = fmax(mag, (fabs(lnb) + 6.0 * fabs(sphi[q])) * c.inv_h2 + fabs(D) + fabs(sf[q]));
    }
    scale = block_max(mag);
    p = block_reduce(p);
    if (threadIdx.x == 0) {
      const double lam = p.sum / (double)cells;
      s_lam = lam;
      s_res = (p.nonfinite > 0) ? NAN : fmax(p.dmax - lam, lam - p.dmin);
      sc->guards = p.guards;
      sc->nonfinite = p.nonfinite;
    }
    __syncthreads();
    res_out = s_res;
  };
  double r;
  residual(r);
  if (threadIdx.x == 0) s_res0 = r;
  __syncthreads();
  const double r0 = s_res0;
  double r_prev = r0;
  const int hn = n >> 1;
  const int per_colour = hn * hn * n;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int colour = 0; colour < 4; ++colour) {
      for (int t = threadIdx.x; t < per_colour; t += blockDim.x) {
        const int m = t % hn, jj = (t / hn) % hn, k = t / (hn * hn);
        const int i = 2 * m + ((colour ^ k) & 1);
        const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
        const int id = i + n * (j + n * k);
        const StencilT<double> s = gather_periodic<double>(sphi, i, j, k, n);
        double v;
        if (c.mode == OP_GENW) {
          v = genw_newton(s, sphi[id], ssrc[id], sf[id] + s_lam, c);
        } else {
          bool g;
          const double D = root_D(s, ssrc[id], c, g);
          v = fma(-c.h2, D + sf[id] + s_lam, s.sx + s.sy + s.sz) * (1.0 / 6.0);
        }
        sphi[id] = not_one(c.omega) ? fma(c.omega, v - sphi[id], sphi[id]) : v;
      }
      __syncthreads();
    }
    if ((sweep + 1) % check_every == 0 || sweep + 1 == max_sweeps) {
      residual(r);
      if (coarsest_done(r, r0, r_prev, scale, drop)) break;
      r_prev = r;
    }
  }
  for (int q = threadIdx.x; q < cells; q += blockDim.x) phi[q] = sphi[q];
  if (threadIdx.x == 0) {
    sc->lambda = s_lam;
    sc->res = s_res;
  }
}

__device__ __forceinline__ void b_affine64(long long cells, const double* __restrict__ delta,
                                                  double* __restrict__ out, double a, double b,
                                                  double c3, int floor,
                                                  unsigned long long* __restrict__ floored,
    long long blk) {
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  bool hit = false;
  if (t < cells) {
    double v = fma(a, delta[t], b);
    if (floor) {
      const double lhs = (b != 0.0) ? v : fma(c3, v, 1.0);  // 1 + c3 kappa delta
      if (lhs < 0.0) {
        hit = true;
        v = (b != 0.0) ? 0.0 : -1.0 / c3;
      }
    }
    out[t] = v;
  }
  if (floored) {
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(floored, (unsigned long long)__popc(ballot));
  }
}

__device__ __forceinline__ void b_sum_partials(long long cells, const double* __restrict__ x,
                                                      Partial* __restrict__ partials,
    long long blk) {
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < cells) partial_add(p, x[t], false);
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blk] = p;
}

__device__ __forceinline__ void b_sub_mean(long long cells, double* __restrict__ x,
                                                  const LevelScalars* __restrict__ sc,
    long long blk) {
  const long long t = (long long)blk * blockDim.x + threadIdx.x;
  if (t < cells) x[t] -= sc->lambda;
}

}  // namespace mg
