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
#include <utility>
#include <vector>

#include "mg_internal.h"
#include "mg_bodies32.cuh"
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

// ---------------------------------------------------------------------------
// FP64 outer residual with the FP32 hand-off.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_residual_handoff64(
    int n, const double* __restrict__ phi, const double* __restrict__ src, OpConst64 c,
    const LevelScalars* __restrict__ sc, float* __restrict__ g, float* __restrict__ q0,
    float* __restrict__ phi0, float* __restrict__ e, Partial* __restrict__ partials,
    float* __restrict__ gc, float* __restrict__ q0c) {
  PdlScope pdl_scope;
  b_residual_handoff64(n, phi, src, c, sc, g, q0, phi0, e, partials, blockIdx.x, gc, q0c);
}

// phi += e (FP64).
__global__ void __launch_bounds__(256) k_update64(long long cells, double* __restrict__ phi,
                                                  const float* __restrict__ e) {
  PdlScope pdl_scope;
  b_update64(cells, phi, e, blockIdx.x);
}

// ---------------------------------------------------------------------------
// FP32 inner kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_restrict32(int nc, const float* __restrict__ fine,
                                                    float* __restrict__ coarse) {
  PdlScope pdl_scope;
  b_restrict32(nc, fine, coarse, blockIdx.x);
}

// q0 = 1 + 4(1-w) alpha (kappa delta + alpha Sigma_d(phi0)) on a coarse level; with
// the source floor, 1 + 4(1-w) alpha kappa delta is held at >= 0 first.
__global__ void __launch_bounds__(256) k_q0_prep32(int n, const float* __restrict__ phi0,
                                                   const double* __restrict__ delta,
                                                   OpConst32 c, float kappa, int floor,
                                                   float* __restrict__ q0) {
  PdlScope pdl_scope;
  b_q0_prep32(n, phi0, delta, c, kappa, floor, q0, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_smooth_colour32(int n, float* __restrict__ e,
                                                         const float* __restrict__ phi0,
                                                         const float* __restrict__ q0,
                                                         const float* __restrict__ g,
                                                         const LevelScalars* __restrict__ sc,
                                                         OpConst32 c, int colour) {
  PdlScope pdl_scope;
  b_smooth_colour32(n, e, phi0, q0, g, sc, c, colour, blockIdx.x);
}

constexpr int ilog2(unsigned v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Which of a colour's N^3/4 cells thread tid of a 256-thread CTA blk updates.
// tzl < 0: consecutive cells (a CTA covers 256 cells of one or a few rows of the
// colour).  tzl = 0..3: a CTA covers a tile of 32 cells in x by 8 / 2^tzl rows of the
// colour by 2^tzl planes, so that the rows its warps read around their cells
// overlap inside the CTA and its L1.  Each warp holds 32 consecutive cells of one
// row either way, and every cell is updated once.
template <int N, int TZL>
__device__ __forceinline__ long long colour_cell(unsigned blk, unsigned tid) {
  if (TZL < 0) return (long long)blk * 256 + tid;
  constexpr unsigned HN = N / 2, BX = HN / 32;
  constexpr unsigned tzl = TZL < 0 ? 0 : TZL, tyl = 3 - tzl, byl = ilog2(HN) - tyl;
  const unsigned w = tid >> 5, r = blk / BX;
  const unsigned m = (blk % BX) * 32 + (tid & 31);
  const unsigned jj = ((r & ((1u << byl) - 1)) << tyl) + (w & ((1u << tyl) - 1));
  const unsigned k = ((r >> byl) << tzl) + (w >> tyl);
  return ((long long)k * HN + jj) * HN + m;
}

// The same colour stage for a power-of-two side N >= 64 known at compile time
// (immediate neighbour offsets; cell_smooth32_n).
// CO: q0 and g in colour order (the finest level, where the hand-off writes them
// so), the pointers already at this colour's block.  TZL: the CTA tile (colour_cell).
// From N = 256 on each thread updates two cells, on planes k and k + 2, that share
// rows (cell_smooth32_n_z2: 24 loads per array for two cells instead of 28; the
// 512^3 stage 339 -> 325 us, the 256^3 stage 53.3 -> 50.1 us, the same bits); at
// 64 and 128 one cell per thread is as fast or faster.
template <int N>
constexpr bool colour32_two_cells() { return N >= 256; }

template <int N, bool CO, int TZL>
__global__ void __launch_bounds__(256) k_smooth_colour32_n(float* __restrict__ e,
                                                           const float* __restrict__ phi0,
                                                           const float* __restrict__ q0,
                                                           const float* __restrict__ g,
                                                           const LevelScalars* __restrict__ sc,
                                                           OpConst32 c, int colour) {
  PdlScope pdl_scope;
  __shared__ float s_mu;
  if (threadIdx.x == 0) s_mu = (float)sc->lambda;
  __syncthreads();
  if (colour32_two_cells<N>())
    cell_smooth32_n_z2<N, CO>(e, phi0, q0, g, s_mu, c, colour,
                              colour_cell<N, TZL>(blockIdx.x, threadIdx.x));
  else
    cell_smooth32_n<N, CO>(e, phi0, q0, g, s_mu, c, colour,
                           colour_cell<N, TZL>(blockIdx.x, threadIdx.x));
}

// One colour stage of k_smooth_colour32_n with the CTA tile tzl (-1 .. 3).
template <int N, bool CO>
static void launch_colour32_n(cudaStream_t st, int tzl, float* e, const float* phi0,
                              const float* q0, const float* g, const LevelScalars* sc,
                              const OpConst32& c, int colour) {
  const unsigned nb = (unsigned)((long long)(N / 2) * (N / 2) * N /
                                 (colour32_two_cells<N>() ? 2 : 1) / 256);
  switch (tzl) {
    case 0: launch_k(k_smooth_colour32_n<N, CO, 0>, nb, 256, 0, st, e, phi0, q0, g, sc, c, colour); break;
    case 1: launch_k(k_smooth_colour32_n<N, CO, 1>, nb, 256, 0, st, e, phi0, q0, g, sc, c, colour); break;
    case 2: launch_k(k_smooth_colour32_n<N, CO, 2>, nb, 256, 0, st, e, phi0, q0, g, sc, c, colour); break;
    case 3: launch_k(k_smooth_colour32_n<N, CO, 3>, nb, 256, 0, st, e, phi0, q0, g, sc, c, colour); break;
    default: launch_k(k_smooth_colour32_n<N, CO, -1>, nb, 256, 0, st, e, phi0, q0, g, sc, c, colour);
  }
}

// The colour stage of k_smooth_colour32_n on the planes z0, ..., z0 + nz - 1 (mod
// N) only: one launch of a sweep run slab by slab (slab_range).
template <int N, bool CO>
__global__ void __launch_bounds__(256) k_smooth_slab32(float* __restrict__ e,
                                                       const float* __restrict__ phi0,
                                                       const float* __restrict__ q0,
                                                       const float* __restrict__ g,
                                                       const LevelScalars* __restrict__ sc,
                                                       OpConst32 c, int colour, int z0, int nz) {
  PdlScope pdl_scope;
  __shared__ float s_mu;
  if (threadIdx.x == 0) s_mu = (float)sc->lambda;
  __syncthreads();
  constexpr long long HH = (long long)(N / 2) * (N / 2);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= HH * nz) return;
  const int k = (z0 + (int)(t / HH)) & (N - 1);
  cell_smooth32_n<N, CO>(e, phi0, q0, g, s_mu, c, colour, (long long)k * HH + t % HH);
}

// The same colour stage with two cells of a row per thread (n % 4 == 0).
__global__ void __launch_bounds__(256) k_smooth_colour32_pair(int n, float* __restrict__ e,
                                                              const float* __restrict__ phi0,
                                                              const float* __restrict__ q0,
                                                              const float* __restrict__ g,
                                                              const LevelScalars* __restrict__ sc,
                                                              OpConst32 c, int colour) {
  PdlScope pdl_scope;
  b_smooth_colour32_pair(n, e, phi0, q0, g, sc, c, colour, blockIdx.x);
}

// rho = N(e) - g on the 8 children of each coarse cell; R e and R rho.
__global__ void __launch_bounds__(256) k_residual_restrict32(
    int nf, const float* __restrict__ e, const float* __restrict__ phi0,
    const float* __restrict__ q0, const float* __restrict__ g, OpConst32 c,
    float* __restrict__ e_c, float* __restrict__ ehat_c, float* __restrict__ rg_c,
    Partial* __restrict__ partials) {
  PdlScope pdl_scope;
  b_residual_restrict32(nf, e, phi0, q0, g, c, e_c, ehat_c, rg_c, partials, blockIdx.x);
}

// The same in two launches for small levels (as k_defect64 and
// k_restrict_defects64): per fine cell rho, then the walk over the children.
__global__ void __launch_bounds__(256) k_defect32(int nf, const float* __restrict__ e,
                                                  const float* __restrict__ phi0,
                                                  const float* __restrict__ q0,
                                                  const float* __restrict__ g, OpConst32 c,
                                                  float* __restrict__ rout) {
  PdlScope pdl_scope;
  cell_defect32(nf, e, phi0, q0, g, c, rout, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_restrict_defects32(
    int nf, const float* __restrict__ e, const float* __restrict__ rin, float* __restrict__ e_c,
    float* __restrict__ ehat_c, float* __restrict__ rg_c, Partial* __restrict__ partials) {
  PdlScope pdl_scope;
  b_restrict_defects32(nf, e, rin, e_c, ehat_c, rg_c, partials, blockIdx.x);
}

// g^H = N^H(R e) - (R rho - mu^h); mu^H starts at 0.
__global__ void __launch_bounds__(256) k_fas_rhs32(int nc, const float* __restrict__ e_c,
                                                   const float* __restrict__ phi0_c,
                                                   const float* __restrict__ q0_c,
                                                   float* __restrict__ g_c, OpConst32 c,
                                                   const LevelScalars* __restrict__ fine_sc,
                                                   LevelScalars* __restrict__ coarse_sc) {
  PdlScope pdl_scope;
  b_fas_rhs32(nc, e_c, phi0_c, q0_c, g_c, c, fine_sc, coarse_sc, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_prolong_correct32(int nc, const float* __restrict__ e_c,
                                                           const float* __restrict__ ehat_c,
                                                           float* __restrict__ e_f) {
  PdlScope pdl_scope;
  b_prolong_correct32(nc, e_c, ehat_c, e_f, blockIdx.x);
}

// ehat_c <- e_c - ehat_c (R e is not needed after the prolongation), then the
// prolongation from it (as k_correction64 and k_prolong_corr64).
__global__ void __launch_bounds__(256) k_correction32(long long cells, const float* __restrict__ e_c,
                                                      float* __restrict__ ehat_c) {
  PdlScope pdl_scope;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cells) ehat_c[t] = e_c[t] - ehat_c[t];
}

__global__ void __launch_bounds__(256) k_prolong_corr32(int nc, const float* __restrict__ corr_c,
                                                        float* __restrict__ e_f) {
  PdlScope pdl_scope;
  cell_prolong_corr32(nc, corr_c, e_f, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Coarsest inner level in one CTA, in FP32: sweeps of N(e) = g + mu until the
// residual fell by `drop` or `max_sweeps`.
__global__ void __launch_bounds__(256) k_coarsest_corr32(int n, float* __restrict__ e,
                                                         const float* __restrict__ phi0,
                                                         const float* __restrict__ q0,
                                                         const float* __restrict__ g, OpConst32 c,
                                                         LevelScalars* __restrict__ sc,
                                                         int max_sweeps, double drop) {
  PdlScope pdl_scope;
  b_coarsest_corr32(n, e, phi0, q0, g, c, sc, max_sweeps, drop, blockIdx.x);
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
  c.sigma2 = 2.f * c.sigma;
  c.sk2 = c.sigma * c.k2;
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
    cudaFree(L.e2);
    cudaFree(L.q0c);
    cudaFree(L.rhsc);
    L.e = L.ehat = L.phi0 = L.q0 = L.rhs = L.src32 = L.e2 = L.q0c = L.rhsc = nullptr;
  }
  cudaFree(d->d_flags);
  if (d->h_flags) cudaFreeHost(d->h_flags);
  d->d_flags = d->h_flags = nullptr;
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
    if (sweep32_eligible(L.n)) ok = ok && cudaMalloc(&L.e2, b) == cudaSuccess;
    if (l == 0 && L.n >= 64 && L.n <= 1024 && (L.n & (L.n - 1)) == 0) {
      ok = ok && cudaMalloc(&L.q0c, b) == cudaSuccess;
      ok = ok && cudaMalloc(&L.rhsc, b) == cudaSuccess;
    }
  }
  ok = ok && cudaMalloc(&d->d_flags, 4 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&d->h_flags, 4 * sizeof(int)) == cudaSuccess;
  if (ok) ok = cudaMemset(d->d_flags, 0, 4 * sizeof(int)) == cudaSuccess;
  if (!ok) {
    mixed_release(d);
    set_error("device allocation failed (mixed precision arrays)");
    return MG_ENOMEM;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_coarsest_corr32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         4 * sizeof(double) * 4096);
    attr = true;
  }
  init_sweep32();
  init_half32();
  d->mixed_ready = true;
  return MG_OK;
}

mg_status mixed_prepare_domain(Domain* d) { return mixed_prepare(d); }

struct CycleMixed {
  Domain* d;
  const mg_options* o;
  cudaStream_t st;
  const OpConst64* ops;
  const OpConst32* ops32;
  float kappa;
  int floor;
  EventPairs* timer;  // finest-level colour stages (time_kernels), or null

  LevelScalars* sc32(int l) const { return d->d_sc + d->nlev + l; }

  void smooth(int l, int sweeps) const {
    Level& L = d->lv[l];
    if (o->half32 && L.e2 && half_sweep_supported(L.n)) {
      // each sweep as two half sweeps e -> e2 (or back); an odd count ends in e2
      // and is copied back
      EventPairs* t = (l == 0 && timer && timer->enabled) ? timer : nullptr;
      float* cur = L.e;
      float* nxt = L.e2;
      for (int s = 0; s < sweeps; ++s) {
        const bool timed = t && (!t->first_only || s == 0);
        launch_half_sweep32(st, L.n, cur, nxt, L.phi0, L.q0, L.rhs, sc32(l), ops32[l],
                            d->d_flags, o->barrier_timeout_s, timed ? t : nullptr);
        std::swap(cur, nxt);
      }
      if (cur != L.e)
        cudaMemcpyAsync(L.e, cur, sizeof(float) * (size_t)L.cells, cudaMemcpyDeviceToDevice, st);
      return;
    }
    if (o->sweep32 && L.e2) {
      // pairs of one-launch sweeps e -> e2 -> e; an odd last sweep goes e -> e2
      // and is copied back
      for (int s = 0; s < sweeps; s += 2) {
        launch_sweep32(st, L.n, L.e, L.e2, L.phi0, L.q0, L.rhs, sc32(l), ops32[l]);
        if (s + 1 < sweeps)
          launch_sweep32(st, L.n, L.e2, L.e, L.phi0, L.q0, L.rhs, sc32(l), ops32[l]);
        else
          cudaMemcpyAsync(L.e, L.e2, sizeof(float) * (size_t)L.cells, cudaMemcpyDeviceToDevice,
                          st);
      }
      return;
    }
    if (o->pair32 && L.n % 4 == 0) {
      const long long pairs = (long long)(L.n / 4) * (L.n / 2) * L.n;
      for (int s = 0; s < sweeps; ++s)
        for (int colour = 0; colour < 4; ++colour)
          launch_k(k_smooth_colour32_pair, nblk(pairs, 256), 256, 0, st, L.n, L.e, L.phi0, L.q0,
                   L.rhs, sc32(l), ops32[l], colour);
      count_launches(4LL * sweeps);
      return;
    }
    const long long per = (long long)(L.n / 2) * (L.n / 2) * L.n;
    EventPairs* t = (l == 0 && timer && timer->enabled) ? timer : nullptr;
    // the finest level reads q0 and g in colour order (written so by the hand-off)
    const bool co = L.q0c != nullptr;
    if (slab_sweep_applies(L.n, o->slab32)) {
      slab_sweeps(l, sweeps, co, t);
      return;
    }
    // CTA tiles of tile32 planes (log2; -1: consecutive cells)
    const int tzl = o->tile32 > 0 ? ilog2((unsigned)o->tile32) : -1;
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour) {
        const unsigned nb = nblk(per, 256);
        // an event between two launches removes their programmatic overlap, so the
        // sampled mode brackets one colour stage per call
        const bool timed = t && (!t->first_only || (s == 0 && colour == 0));
        if (timed) t->begin(st);
        const float* qv = co ? L.q0c + colour * per : L.q0;
        const float* gv = co ? L.rhsc + colour * per : L.rhs;
        auto stage = [&](auto launch_co, auto launch_nat) {
          (co ? launch_co : launch_nat)(st, tzl, L.e, L.phi0, qv, gv, sc32(l), ops32[l], colour);
        };
        switch (L.n) {
          case 64: stage(launch_colour32_n<64, true>, launch_colour32_n<64, false>); break;
          case 128: stage(launch_colour32_n<128, true>, launch_colour32_n<128, false>); break;
          case 256: stage(launch_colour32_n<256, true>, launch_colour32_n<256, false>); break;
          case 512: stage(launch_colour32_n<512, true>, launch_colour32_n<512, false>); break;
          case 1024: stage(launch_colour32_n<1024, true>, launch_colour32_n<1024, false>); break;
          default:
            launch_k(k_smooth_colour32, nb, 256, 0, st, L.n, L.e, L.phi0, L.q0, L.rhs, sc32(l),
                     ops32[l], colour);
        }
        if (timed) t->end(st);
      }
    count_launches(4LL * sweeps);
  }

  // Sweeps in the staggered slab order (slab_range); a timed unit is one whole sweep.
  void slab_sweeps(int l, int sweeps, bool co, EventPairs* t) const {
    Level& L = d->lv[l];
    const int S = o->slab32, ns = L.n / S;
    const long long hh = (long long)(L.n / 2) * (L.n / 2);
    for (int sw = 0; sw < sweeps; ++sw) {
      const bool timed = t && (!t->first_only || sw == 0);
      if (timed) t->begin(st);
      for (int s = 0; s < ns; ++s)
        for (int colour = 0; colour < 4; ++colour) {
          int z0 = 0, nz = 0;
          slab_range(L.n, S, colour, s, &z0, &nz);
          const unsigned nb = nblk(hh * nz, 256);
          const float* qv = co ? L.q0c + colour * hh * L.n : L.q0;
          const float* gv = co ? L.rhsc + colour * hh * L.n : L.rhs;
          auto stage = [&](auto kern) {
            launch_k(kern, nb, 256, 0, st, L.e, L.phi0, qv, gv, sc32(l), ops32[l], colour, z0, nz);
          };
          switch (L.n) {
            case 256:
              co ? stage(k_smooth_slab32<256, true>) : stage(k_smooth_slab32<256, false>);
              break;
            case 512:
              co ? stage(k_smooth_slab32<512, true>) : stage(k_smooth_slab32<512, false>);
              break;
            default:
              co ? stage(k_smooth_slab32<1024, true>) : stage(k_smooth_slab32<1024, false>);
          }
        }
      if (timed) t->end(st);
    }
    count_launches(4LL * ns * sweeps);
  }

  void subcycle(int l) const {
    SubCycleArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nlev = d->nlev - l;
    for (int k = 0; k < a.nlev; ++k) {
      Level& L = d->lv[l + k];
      a.lv32[k] = SubLevel32{L.n, L.e, L.ehat, L.phi0, L.q0, L.rhs, sc32(l + k), ops32[l + k]};
    }
    a.part = d->d_part;
    a.def32 = reinterpret_cast<float*>(d->d_subdef);
    a.nu_pre = o->nu_pre;
    a.nu_post = o->nu_post;
    a.coarse_sweeps = o->coarse_sweeps;
    a.coarse_drop = o->coarse_drop;
    launch_subcycle32(st, a);
  }

  void inner(int l) const {
    Level& L = d->lv[l];
    if (o->fuse_coarse && l > 0 && L.n <= kSubcycleMaxN && d->nlev - l <= kSubcycleMaxLevels) {
      subcycle(l);
      return;
    }
    if (l == d->nlev - 1) {
      const size_t smem = 4 * sizeof(double) * (size_t)L.cells;
      launch_k(k_coarsest_corr32, 1, 256, smem, st, L.n, L.e, L.phi0, L.q0, L.rhs, ops32[l], sc32(l),
                                              o->coarse_sweeps, o->coarse_drop);
      count_launches(1);
      return;
    }
    Level& C = d->lv[l + 1];
    smooth(l, o->nu_pre);
    const unsigned nb = nblk(C.cells, 256);
    if (L.cells <= kTwoStepMaxFine) {
      // small level: per-fine-cell defects spread over the GPU, then the walk over
      // each coarse cell's children (the same bits as the fused kernel)
      float* def = reinterpret_cast<float*>(d->d_subdef);
      launch_k(k_defect32, nblk(L.cells, 64), 64, 0, st, L.n, L.e, L.phi0, L.q0, L.rhs, ops32[l],
               def);
      launch_k(k_restrict_defects32, nb, 256, 0, st, L.n, L.e, (const float*)def, C.e, C.ehat,
               C.rhs, d->d_part);
      count_launches(1);
    } else {
      launch_k(k_residual_restrict32, nb, 256, 0, st, L.n, L.e, L.phi0, L.q0, L.rhs, ops32[l], C.e,
               C.ehat, C.rhs, d->d_part);
    }
    launch_finalize(st, d->d_part, (int)nb, (double)L.cells, 1, sc32(l));
    launch_k(k_fas_rhs32, nblk(C.cells, 256), 256, 0, st, C.n, C.e, C.phi0, C.q0, C.rhs, ops32[l + 1],
                                                     sc32(l), sc32(l + 1));
    inner(l + 1);
    if (L.cells >= kCorrectionMinFine) {
      launch_k(k_correction32, nblk(C.cells, 256), 256, 0, st, C.cells, C.e, C.ehat);
      launch_k(k_prolong_corr32, nblk(L.cells, 256), 256, 0, st, C.n, (const float*)C.ehat, L.e);
      count_launches(1);
    } else {
      launch_k(k_prolong_correct32, nblk(L.cells, 256), 256, 0, st, C.n, C.e, C.ehat, L.e);
    }
    count_launches(3);  // residual-restrict, FAS right-hand side, prolongation
    smooth(l, o->nu_post);
  }

  // FP64 residual, FP32 hand-off, convergence scalars to the host.
  void part_a() const {
    Level& L = d->lv[0];
    const unsigned nb = nblk(L.cells, 256 * kHandoffCells);
    launch_k(k_residual_handoff64, nb, 256, 0, st, L.n, L.phi, L.src, ops[0], d->d_sc, L.rhs, L.q0,
             L.phi0, L.e, d->d_part, L.rhsc, L.q0c);
    count_launches(1);
    launch_finalize(st, d->d_part, (int)nb, (double)L.cells, 1, d->d_sc);
    cudaMemcpyAsync(d->h_sc, d->d_sc, sizeof(LevelScalars), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(d->h_flags, d->d_flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  }

  // Coarse copies of the expansion point, the inner V-cycles, phi += e.
  void part_b() const {
    for (int l = 1; l < d->nlev; ++l) {
      Level& L = d->lv[l];
      launch_k(k_restrict32, nblk(L.cells, 256), 256, 0, st, L.n, d->lv[l - 1].phi0, L.phi0);
      launch_k(k_q0_prep32, nblk(L.cells, 256), 256, 0, st, L.n, L.phi0, L.delta, ops32[l], kappa, floor,
                                                      L.q0);
      count_launches(2);
    }
    cudaMemsetAsync(sc32(0), 0, sizeof(LevelScalars), st);
    for (int c = 0; c < o->inner_cycles; ++c) inner(0);
    Level& L = d->lv[0];
    launch_k(k_update64, nblk(L.cells, 256), 256, 0, st, L.cells, L.phi, L.e);
    count_launches(1);
  }
};


mg_status mixed_solve(Domain* d, const mg_options& o, cudaStream_t st, const OpConst64* ops,
                      int branch, double alpha, double kappa, double tol, mg_solve_stats* s) {
  mg_status ps = mixed_prepare(d);
  if (ps != MG_OK) return ps;
  std::vector<OpConst32> ops32(d->nlev);
  for (int l = 0; l < d->nlev; ++l) ops32[l] = make_op32(d->lv[l].n, alpha, branch);
  // the finest FP32 colour stages are timed when they run as per-colour launches
  EventPairs tb;
  const bool half = o.half32 && half_sweep_supported(d->lv[0].n);
  const bool slab = !half && !o.sweep32 && !o.pair32 && slab_sweep_applies(d->lv[0].n, o.slab32);
  tb.enabled = o.time_kernels != 0 && (half || (!o.sweep32 && !o.pair32));
  tb.first_only = o.time_kernels == 2;
  MCK(cudaMemsetAsync(d->d_flags, 0, sizeof(int), st));
  CycleMixed cyc{d, &o, st, ops, ops32.data(), (float)kappa, o.guard == MG_GUARD_FLOOR, &tb};
  domain_invalidate_graphs(d);
  long long na = 0, nb = 0;
  if (o.use_graphs) {
    tb.capturing = true;
    d->gexec[2] = capture_graph(st, &na, [&] { cyc.part_a(); });
    d->gexec[3] = capture_graph(st, &nb, [&] { cyc.part_b(); });
    tb.capturing = false;
  }
  const bool graphs = o.use_graphs && d->gexec[2] && d->gexec[3];
  const int pairs_b = tb.n;
  // a timed unit is one colour stage, one half sweep, or one whole sweep of slabs
  const double cells_per_launch = (double)d->lv[0].cells / (half ? 2.0 : slab ? 1.0 : 4.0);
  bool b_pending = false;
  auto harvest = [&]() {
    if (!tb.enabled || !b_pending) return;
    const int pairs = graphs ? pairs_b : tb.n;
    const int keep = tb.n;
    tb.n = pairs;
    s->kernel_ms += tb.read_ms();
    s->kernel_launches += pairs;
    s->kernel_cells += pairs * cells_per_launch;
    tb.n = keep;
    b_pending = false;
  };
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
    harvest();
    if (d->h_flags[0]) {
      set_error("an FP32 half sweep waited longer than barrier_timeout_s for its data");
      result = MG_ETIMEOUT;
      break;
    }
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
    if (!graphs) tb.n = 0;
    if (graphs) {
      MCK(cudaGraphLaunch(d->gexec[3], st));
      tl_launches += nb;
    } else {
      cyc.part_b();
    }
    b_pending = true;
    s->cycles += o.inner_cycles;
  }
  s->res0 = first;
  return result;
}

}  // namespace mg
