// Mixed precision: FP32 correction V-cycles inside an FP64 defect-correction
// loop, for the FAS solve of Sec. III.C of arXiv:1303.0008.
//
// Outer step (FP64): d = L^h phi, lambda = mean(d), res = max|d - lambda|.  The
// same kernel leaves, in FP32, the right-hand side g = lambda_prev - d, the
// discriminant q0 = 1 + 4(1-w) alpha u(phi) of the root of Eq. two_branch and a
// copy phi0 of the expansion point.
// Inner problem (FP32): find e with N(e) = L^h(phi0 + e) - L^h(phi0) = g + mu (mu
// a compatibility constant, as lambda for phi), by FAS V-cycles whose smoother
// is the exact pointwise Newton step of Sec. III.B applied to N.  N is evaluated
// without cancellation:
//     Delta Sigma_d = sum_t w_t a_t(e) (2 a_t(phi0) + a_t(e))
// over the six linear forms a_t of Sigma_d (w = 1/3), Delta u = alpha Delta Sigma_d,
// q1 = q0 + 4(1-w) alpha Delta u, and the change of the root
//     Delta D = sigma 2 Delta u / (sqrt q0 + sqrt q1)      (q0, q1 >= 0)
//     Delta D = sigma k2 (sqrt max(q1,0) - sqrt max(q0,0)) (otherwise).
// The coarsest inner level is solved in FP64.  Then phi += e in FP64.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mg_internal.h"
#include "mg_solver.h"

namespace mg {

#define MCK(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return MG_ECUDA;                                                       \
    }                                                                        \
  } while (0)

// The change of the root D when phi0 moves by e, from the stencils of e and phi0.
template <typename T>
__device__ __forceinline__ T delta_D(const StencilT<T>& se, const StencilT<T>& sp, T q0, T g1,
                                     T g2, T c3, T k2, T sigma, T& du_out) {
  const T a1e = se.sx - se.sy, a2e = se.sx - se.sz, a3e = se.sy - se.sz;
  const T a1p = sp.sx - sp.sy, a2p = sp.sx - sp.sz, a3p = sp.sy - sp.sz;
  const T two = T(2);
  const T dA = a1e * (two * a1p + a1e) + a2e * (two * a2p + a2e) + a3e * (two * a3p + a3e);
  const T dB = se.cxy * (two * sp.cxy + se.cxy) + se.cxz * (two * sp.cxz + se.cxz) +
               se.cyz * (two * sp.cyz + se.cyz);
  const T du = g1 * dA + g2 * dB;
  du_out = du;
  const T q1 = q0 + c3 * du;
  const T s0 = sqrt(q0 > T(0) ? q0 : T(0));
  const T s1 = sqrt(q1 > T(0) ? q1 : T(0));
  if (q0 >= T(0) && q1 >= T(0)) {
    const T den = s0 + s1;
    return den > T(0) ? sigma * two * du / den : T(0);
  }
  return sigma * k2 * (s1 - s0);
}

__device__ __forceinline__ float dD32(const StencilT<float>& se, const StencilT<float>& sp,
                                      float q0, const OpConst32& c) {
  if (c.linear) return 0.f;
  float du;
  return delta_D<float>(se, sp, q0, c.g1, c.g2, c.c3, c.k2, c.sigma, du);
}

// ---------------------------------------------------------------------------
// FP64 outer residual with the FP32 hand-off.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_residual_handoff64(
    int n, const double* __restrict__ phi, const double* __restrict__ src, OpConst64 c,
    const LevelScalars* __restrict__ sc, float* __restrict__ g, float* __restrict__ q0,
    float* __restrict__ phi0, float* __restrict__ e, Partial* __restrict__ partials) {
  const long long cells = (long long)n * n * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < cells) {
    const int i = (int)(t % n);
    const int j = (int)((t / n) % n);
    const int k = (int)(t / ((long long)n * n));
    const StencilT<double> s = gather_periodic(phi, i, j, k, n);
    double q = 1.0, D;
    bool guard = false;
    if (c.mode == OP_LINEAR) {
      D = src[t];
    } else {
      const double a1 = s.sx - s.sy, a2 = s.sx - s.sz, a3 = s.sy - s.sz;
      const double A = fma(a1, a1, fma(a2, a2, a3 * a3));
      const double B = fma(s.cxy, s.cxy, fma(s.cxz, s.cxz, s.cyz * s.cyz));
      if (c.mode == OP_SQRT) {
        q = fma(c.e1, A, fma(c.e2, B, src[t]));
        D = fma(c.k2s, sqrt(q < 0.0 ? 0.0 : q), -c.k2);
      } else {
        const double u = fma(c.c1, A, fma(c.c2, B, src[t]));
        q = fma(c.c3, u, 1.0);
        D = (q < 0.0) ? -c.k2 : (2.0 * u) / (1.0 + sqrt(q));
      }
      guard = q < 0.0;
    }
    const double ctr = phi[t];
    const double lap = (s.sx + s.sy + s.sz) - 6.0 * ctr;
    const double d = fma(lap, c.inv_h2, -D);
    partial_add(p, d, guard);
    g[t] = (float)(sc->lambda - d);
    q0[t] = (float)q;
    phi0[t] = (float)ctr;
    e[t] = 0.f;
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blockIdx.x] = p;
}

// phi += e (FP64).
__global__ void __launch_bounds__(256) k_update64(long long cells, double* __restrict__ phi,
                                                  const float* __restrict__ e) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cells) phi[t] += (double)e[t];
}

// ---------------------------------------------------------------------------
// FP32 inner kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_restrict32(int nc, const float* __restrict__ fine,
                                                    float* __restrict__ coarse) {
  const int nf = nc << 1;
  const long long cells = (long long)nc * nc * nc;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const int I = (int)(t % nc);
  const int J = (int)((t / nc) % nc);
  const int K = (int)(t / ((long long)nc * nc));
  float s = 0.f;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    s += fine[lidx(2 * I + (ch & 1), 2 * J + ((ch >> 1) & 1), 2 * K + (ch >> 2), nf)];
  coarse[t] = s * 0.125f;
}

// q0 = 1 + 4(1-w) alpha (kappa delta + alpha Sigma_d(phi0)) on a coarse level; with
// the source floor, 1 + 4(1-w) alpha kappa delta is held at >= 0 first.
__global__ void __launch_bounds__(256) k_q0_prep32(int n, const float* __restrict__ phi0,
                                                   const double* __restrict__ delta,
                                                   OpConst32 c, float kappa, int floor,
                                                   float* __restrict__ q0) {
  const long long cells = (long long)n * n * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  if (c.linear) {
    q0[t] = 1.f;
    return;
  }
  const int i = (int)(t % n);
  const int j = (int)((t / n) % n);
  const int k = (int)(t / ((long long)n * n));
  const StencilT<float> s = gather_periodic(phi0, i, j, k, n);
  const float a1 = s.sx - s.sy, a2 = s.sx - s.sz, a3 = s.sy - s.sz;
  const float A = a1 * a1 + a2 * a2 + a3 * a3;
  const float B = s.cxy * s.cxy + s.cxz * s.cxz + s.cyz * s.cyz;
  float qs = fmaf(c.c3 * kappa, (float)delta[t], 1.f);
  if (floor && qs < 0.f) qs = 0.f;
  q0[t] = fmaf(c.c3, c.g1 * A + c.g2 * B, qs);
}

__global__ void __launch_bounds__(256) k_smooth_colour32(int n, float* __restrict__ e,
                                                         const float* __restrict__ phi0,
                                                         const float* __restrict__ q0,
                                                         const float* __restrict__ g,
                                                         const LevelScalars* __restrict__ sc,
                                                         OpConst32 c, int colour) {
  const int hn = n >> 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)hn * hn * n;
  if (t >= total) return;
  const int m = (int)(t % hn);
  const long long rest = t / hn;
  const int jj = (int)(rest % hn);
  const int k = (int)(rest / hn);
  const int i = 2 * m + ((colour ^ k) & 1);
  const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
  const long long id = lidx(i, j, k, n);
  const StencilT<float> se = gather_periodic(e, i, j, k, n);
  float dd = 0.f;
  if (!c.linear) {
    const StencilT<float> sp = gather_periodic(phi0, i, j, k, n);
    dd = dD32(se, sp, q0[id], c);
  }
  const float rhs = g[id] + (float)sc->lambda;
  e[id] = fmaf(-c.h2, dd + rhs, se.sx + se.sy + se.sz) * (1.f / 6.f);
}

// rho = N(e) - g on the 8 children of each coarse cell; R e and R rho.
__global__ void __launch_bounds__(128) k_residual_restrict32(
    int nf, const float* __restrict__ e, const float* __restrict__ phi0,
    const float* __restrict__ q0, const float* __restrict__ g, OpConst32 c,
    float* __restrict__ e_c, float* __restrict__ ehat_c, float* __restrict__ rg_c,
    Partial* __restrict__ partials) {
  const int nc = nf >> 1;
  const long long ccells = (long long)nc * nc * nc;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Partial p;
  partial_init(p);
  if (t < ccells) {
    const int I = (int)(t % nc);
    const int J = (int)((t / nc) % nc);
    const int K = (int)(t / ((long long)nc * nc));
    float se_sum = 0.f, sr = 0.f;
#pragma unroll 1
    for (int ch = 0; ch < 8; ++ch) {
      const int i = 2 * I + (ch & 1), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch >> 2);
      const long long id = lidx(i, j, k, nf);
      const StencilT<float> se = gather_periodic(e, i, j, k, nf);
      float dd = 0.f;
      if (!c.linear) {
        const StencilT<float> sp = gather_periodic(phi0, i, j, k, nf);
        dd = dD32(se, sp, q0[id], c);
      }
      const float ctr = e[id];
      const float lap = (se.sx + se.sy + se.sz) - 6.f * ctr;
      const float r = fmaf(lap, c.inv_h2, -dd) - g[id];
      partial_add(p, (double)r, false);
      se_sum += ctr;
      sr += r;
    }
    e_c[t] = se_sum * 0.125f;
    ehat_c[t] = se_sum * 0.125f;
    rg_c[t] = sr * 0.125f;
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) partials[blockIdx.x] = p;
}

// g^H = N^H(R e) - (R rho - mu^h); mu^H starts at 0.
__global__ void __launch_bounds__(256) k_fas_rhs32(int nc, const float* __restrict__ e_c,
                                                   const float* __restrict__ phi0_c,
                                                   const float* __restrict__ q0_c,
                                                   float* __restrict__ g_c, OpConst32 c,
                                                   const LevelScalars* __restrict__ fine_sc,
                                                   LevelScalars* __restrict__ coarse_sc) {
  const long long cells = (long long)nc * nc * nc;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) coarse_sc->lambda = 0.0;
  if (t >= cells) return;
  const int i = (int)(t % nc);
  const int j = (int)((t / nc) % nc);
  const int k = (int)(t / ((long long)nc * nc));
  const StencilT<float> se = gather_periodic(e_c, i, j, k, nc);
  float dd = 0.f;
  if (!c.linear) {
    const StencilT<float> sp = gather_periodic(phi0_c, i, j, k, nc);
    dd = dD32(se, sp, q0_c[t], c);
  }
  const float lap = (se.sx + se.sy + se.sz) - 6.f * e_c[t];
  const float Nv = fmaf(lap, c.inv_h2, -dd);
  g_c[t] = Nv - g_c[t] + (float)fine_sc->lambda;
}

__global__ void __launch_bounds__(256) k_prolong_correct32(int nc, const float* __restrict__ e_c,
                                                           const float* __restrict__ ehat_c,
                                                           float* __restrict__ e_f) {
  const int nf = nc << 1;
  const long long cells = (long long)nf * nf * nf;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  const int i = (int)(t % nf);
  const int j = (int)((t / nf) % nf);
  const int k = (int)(t / ((long long)nf * nf));
  const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
  const int I1 = (i & 1) ? wrap_up(I0, nc) : wrap_dn(I0, nc);
  const int J1 = (j & 1) ? wrap_up(J0, nc) : wrap_dn(J0, nc);
  const int K1 = (k & 1) ? wrap_up(K0, nc) : wrap_dn(K0, nc);
  auto v = [&](int a, int b, int cc) {
    const long long q = lidx(a, b, cc, nc);
    return e_c[q] - ehat_c[q];
  };
  const float s = 27.f * v(I0, J0, K0) + 9.f * (v(I1, J0, K0) + v(I0, J1, K0) + v(I0, J0, K1)) +
                  3.f * (v(I1, J1, K0) + v(I1, J0, K1) + v(I0, J1, K1)) + v(I1, J1, K1);
  e_f[t] += s * (1.f / 64.f);
}

// Coarsest inner level in one CTA, in FP64: sweeps of N(e) = g + mu until the
// residual fell by `drop` or `max_sweeps`.
__global__ void __launch_bounds__(256) k_coarsest_corr64(int n, float* __restrict__ e,
                                                         const float* __restrict__ phi0,
                                                         const float* __restrict__ q0,
                                                         const float* __restrict__ g, OpConst32 c,
                                                         LevelScalars* __restrict__ sc,
                                                         int max_sweeps, double drop) {
  extern __shared__ double smc[];
  __shared__ double s_mu, s_res0, s_res;
  const int cells = n * n * n;
  double* se = smc;
  double* sp = smc + cells;
  double* sq = smc + 2 * cells;
  double* sg = smc + 3 * cells;
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    se[q] = e[q];
    sp[q] = phi0[q];
    sq[q] = q0[q];
    sg[q] = g[q];
  }
  if (threadIdx.x == 0) s_mu = sc->lambda;
  __syncthreads();
  const double h2 = (double)c.h2, inv_h2 = (double)c.inv_h2;
  const double g1 = (double)c.g1, g2 = (double)c.g2, c3 = (double)c.c3, k2 = (double)c.k2,
               sigma = (double)c.sigma;
  auto ddv = [&](const StencilT<double>& a, const StencilT<double>& b, double qq) {
    if (c.linear) return 0.0;
    double du;
    return delta_D<double>(a, b, qq, g1, g2, c3, k2, sigma, du);
  };
  auto residual = [&]() {
    Partial p;
    partial_init(p);
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
      const int i = q % n, j = (q / n) % n, k = q / (n * n);
      const StencilT<double> a = gather_periodic<double>(se, i, j, k, n);
      const StencilT<double> b = gather_periodic<double>(sp, i, j, k, n);
      const double lap = (a.sx + a.sy + a.sz) - 6.0 * se[q];
      partial_add(p, fma(lap, inv_h2, -ddv(a, b, sq[q])) - sg[q], false);
    }
    p = block_reduce(p);
    if (threadIdx.x == 0) {
      const double mu = p.sum / (double)cells;
      s_mu = mu;
      s_res = (p.nonfinite > 0) ? NAN : fmax(p.dmax - mu, mu - p.dmin);
    }
    __syncthreads();
    return s_res;
  };
  const double r0 = residual();
  const int hn = n >> 1;
  const int per_colour = hn * hn * n;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int colour = 0; colour < 4; ++colour) {
      for (int t = threadIdx.x; t < per_colour; t += blockDim.x) {
        const int m = t % hn, jj = (t / hn) % hn, k = t / (hn * hn);
        const int i = 2 * m + ((colour ^ k) & 1);
        const int j = 2 * jj + (((colour >> 1) ^ k) & 1);
        const int id = i + n * (j + n * k);
        const StencilT<double> a = gather_periodic<double>(se, i, j, k, n);
        const StencilT<double> b = gather_periodic<double>(sp, i, j, k, n);
        se[id] = fma(-h2, ddv(a, b, sq[id]) + sg[id] + s_mu, a.sx + a.sy + a.sz) * (1.0 / 6.0);
      }
      __syncthreads();
    }
    if ((sweep & 1) == 1 || sweep + 1 == max_sweeps) {
      const double r = residual();
      if (!(r > drop * r0)) break;
    }
  }
  for (int q = threadIdx.x; q < cells; q += blockDim.x) e[q] = (float)se[q];
  if (threadIdx.x == 0) {
    sc->lambda = s_mu;
    sc->res = s_res;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static inline unsigned nblk(long long work, int threads) {
  return (unsigned)((work + threads - 1) / threads);
}

void launch_finalize(cudaStream_t st, const Partial* partials, int nparts, double cells,
                     int periodic, LevelScalars* sc);

OpConst32 make_op32(int n, double alpha, int branch) {
  OpConst32 c{};
  const double h = 1.0 / (double)n;
  const double h2 = h * h, h4 = h2 * h2;
  c.h2 = (float)h2;
  c.inv_h2 = (float)((double)n * (double)n);
  c.linear = alpha == 0.0;
  const double c3 = 4.0 * (2.0 / 3.0) * alpha;
  c.c3 = (float)c3;
  c.g1 = (float)(alpha / (3.0 * h4));
  c.g2 = (float)(alpha / (8.0 * h4));
  c.k2 = c.linear ? 0.f : (float)(2.0 / c3);
  const bool physical = (branch == 0) || ((branch > 0) == (alpha > 0));
  c.sigma = physical ? 1.f : -1.f;
  return c;
}

void mixed_release(Domain* d) {
  for (Level& L : d->lv) {
    cudaFree(L.e);
    cudaFree(L.ehat);
    cudaFree(L.phi0);
    cudaFree(L.q0);
    cudaFree(L.rhs);
    cudaFree(L.src32);
    L.e = L.ehat = L.phi0 = L.q0 = L.rhs = L.src32 = nullptr;
  }
  d->mixed_ready = false;
}

static mg_status mixed_prepare(Domain* d) {
  if (d->mixed_ready) return MG_OK;
  bool ok = true;
  for (int l = 0; l < d->nlev; ++l) {
    Level& L = d->lv[l];
    const size_t b = (size_t)L.cells * sizeof(float);
    ok = ok && cudaMalloc(&L.e, b) == cudaSuccess;
    ok = ok && cudaMalloc(&L.phi0, b) == cudaSuccess;
    ok = ok && cudaMalloc(&L.q0, b) == cudaSuccess;
    ok = ok && cudaMalloc(&L.rhs, b) == cudaSuccess;
    if (l > 0) ok = ok && cudaMalloc(&L.ehat, b) == cudaSuccess;
  }
  if (!ok) {
    mixed_release(d);
    set_error("device allocation failed (mixed precision arrays)");
    return MG_ENOMEM;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_coarsest_corr64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         4 * sizeof(double) * 4096);
    attr = true;
  }
  d->mixed_ready = true;
  return MG_OK;
}

struct CycleMixed {
  Domain* d;
  const mg_options* o;
  cudaStream_t st;
  const OpConst64* ops;
  const OpConst32* ops32;
  float kappa;
  int floor;

  LevelScalars* sc32(int l) const { return d->d_sc + d->nlev + l; }

  void smooth(int l, int sweeps) const {
    Level& L = d->lv[l];
    const long long per = (long long)(L.n / 2) * (L.n / 2) * L.n;
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour)
        k_smooth_colour32<<<nblk(per, 256), 256, 0, st>>>(L.n, L.e, L.phi0, L.q0, L.rhs, sc32(l),
                                                         ops32[l], colour);
    count_launches(4LL * sweeps);
  }

  void inner(int l) const {
    Level& L = d->lv[l];
    if (l == d->nlev - 1) {
      const size_t smem = 4 * sizeof(double) * (size_t)L.cells;
      k_coarsest_corr64<<<1, 256, smem, st>>>(L.n, L.e, L.phi0, L.q0, L.rhs, ops32[l], sc32(l),
                                              o->coarse_sweeps, o->coarse_drop);
      count_launches(1);
      return;
    }
    Level& C = d->lv[l + 1];
    smooth(l, o->nu_pre);
    const unsigned nb = nblk(C.cells, 128);
    k_residual_restrict32<<<nb, 128, 0, st>>>(L.n, L.e, L.phi0, L.q0, L.rhs, ops32[l], C.e,
                                               C.ehat, C.rhs, d->d_part);
    launch_finalize(st, d->d_part, (int)nb, (double)L.cells, 1, sc32(l));
    k_fas_rhs32<<<nblk(C.cells, 256), 256, 0, st>>>(C.n, C.e, C.phi0, C.q0, C.rhs, ops32[l + 1],
                                                     sc32(l), sc32(l + 1));
    inner(l + 1);
    k_prolong_correct32<<<nblk(L.cells, 256), 256, 0, st>>>(C.n, C.e, C.ehat, L.e);
    count_launches(3);  // residual-restrict, FAS right-hand side, prolongation
    smooth(l, o->nu_post);
  }

  // FP64 residual, FP32 hand-off, convergence scalars to the host.
  void part_a() const {
    Level& L = d->lv[0];
    const unsigned nb = nblk(L.cells, 256);
    k_residual_handoff64<<<nb, 256, 0, st>>>(L.n, L.phi, L.src, ops[0], d->d_sc, L.rhs, L.q0,
                                              L.phi0, L.e, d->d_part);
    count_launches(1);
    launch_finalize(st, d->d_part, (int)nb, (double)L.cells, 1, d->d_sc);
    cudaMemcpyAsync(d->h_sc, d->d_sc, sizeof(LevelScalars), cudaMemcpyDeviceToHost, st);
  }

  // Coarse copies of the expansion point, the inner V-cycles, phi += e.
  void part_b() const {
    for (int l = 1; l < d->nlev; ++l) {
      Level& L = d->lv[l];
      k_restrict32<<<nblk(L.cells, 256), 256, 0, st>>>(L.n, d->lv[l - 1].phi0, L.phi0);
      k_q0_prep32<<<nblk(L.cells, 256), 256, 0, st>>>(L.n, L.phi0, L.delta, ops32[l], kappa, floor,
                                                      L.q0);
      count_launches(2);
    }
    cudaMemsetAsync(sc32(0), 0, sizeof(LevelScalars), st);
    for (int c = 0; c < o->inner_cycles; ++c) inner(0);
    Level& L = d->lv[0];
    k_update64<<<nblk(L.cells, 256), 256, 0, st>>>(L.cells, L.phi, L.e);
    count_launches(1);
  }
};


mg_status mixed_solve(Domain* d, const mg_options& o, cudaStream_t st, const OpConst64* ops,
                      int branch, double alpha, double kappa, double tol, mg_solve_stats* s) {
  mg_status ps = mixed_prepare(d);
  if (ps != MG_OK) return ps;
  std::vector<OpConst32> ops32(d->nlev);
  for (int l = 0; l < d->nlev; ++l) ops32[l] = make_op32(d->lv[l].n, alpha, branch);
  CycleMixed cyc{d, &o, st, ops, ops32.data(), (float)kappa, o.guard == MG_GUARD_FLOOR};
  domain_invalidate_graphs(d);
  long long na = 0, nb = 0;
  if (o.use_graphs) {
    d->gexec[2] = capture_graph(st, &na, [&] { cyc.part_a(); });
    d->gexec[3] = capture_graph(st, &nb, [&] { cyc.part_b(); });
  }
  const bool graphs = o.use_graphs && d->gexec[2] && d->gexec[3];
  double first = -1.0;
  std::vector<double> hist;
  mg_status result = MG_OK;
  for (;;) {
    if (graphs) {
      MCK(cudaGraphLaunch(d->gexec[2], st));
      tl_launches += na;
    } else {
      cyc.part_a();
    }
    MCK(cudaStreamSynchronize(st));
    MCK(cudaGetLastError());
    const double res = d->h_sc[0].res;
    s->outer += 1;
    s->guard_hits = o.guard == MG_GUARD_FLOOR ? (long long)d->h_sc[0].floored
                                              : d->h_sc[0].guards;
    s->lambda = d->h_sc[0].lambda;
    s->res = res;
    if (s->hist_len < 128) s->res_hist[s->hist_len++] = res;
    if (first < 0) first = res;
    hist.push_back(res);
    if (!(res == res)) {
      set_error("residual is not finite");
      result = MG_ENAN;
      break;
    }
    if (res < tol) break;
    if (s->outer > o.max_cycles) {
      set_error("no convergence within max_cycles outer corrections");
      result = MG_ENOCONV;
      break;
    }
    if (res > 1e3 * first) {
      set_error("residual grew by more than 1e3");
      result = MG_ENOCONV;
      break;
    }
    const size_t k = hist.size();
    if (k > 6 && res > 0.9 * hist[k - 7]) {
      set_error("residual stalled (less than 10% progress over 6 corrections)");
      result = MG_ENOCONV;
      break;
    }
    if (graphs) {
      MCK(cudaGraphLaunch(d->gexec[3], st));
      tl_launches += nb;
    } else {
      cyc.part_b();
    }
    s->cycles += o.inner_cycles;
  }
  s->res0 = first;
  return result;
}

}  // namespace mg
