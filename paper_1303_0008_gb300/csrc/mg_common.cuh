// Device-side building blocks shared by the CUDA kernels of libmg.
//
// The discrete operator is the one of Sec. III.B of arXiv:1303.0008 (the L^h
// equation with its Sigma_ijk), written for the operator-splitting constant
// w = 1/3 (Sec. III.A).  With w = 1/3 the non-source part of Sigma,
//     Sigma_d h^4 = [(Sx-Sy)^2 + (Sx-Sz)^2 + (Sy-Sz)^2]/3 + (Cxy^2 + Cxz^2 + Cyz^2)/8,
// (Sx = phi_{i+1} + phi_{i-1}, Cxy the four-point cross difference), does not
// involve the centre value, so the Newton step of Sec. III.B is the exact
// pointwise solve of L^h phi = rhs for the centre cell.
//
// Parameters follow the library convention: alpha is the coefficient of the
// nonlinear term of Eq. code_eqn (the paper's alpha is 1/alpha), kappa the source
// coefficient.  With u = kappa*delta + alpha*Sigma_d and q = 1 + 4(1-w) alpha u,
// the root of Eq. two_branch is D = (sigma sqrt(q) - 1) / (2(1-w) alpha) where
// sigma = +1 picks the physical root of Eq. one_branch.  When q < 0 the square
// root is taken of 0 (the real part of the complex root) and the cell counts as
// guarded.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mg {

// How the root D is evaluated.
enum OpMode : int {
  OP_LINEAR = 0,  // alpha == 0: D = kappa*delta
  OP_SQRT = 1,    // D = k2 (sigma sqrt(q) - 1); src = 1 + c3 kappa delta
  OP_CONJ = 2,    // physical root as 2u/(1+sqrt(q)) for small |alpha|; src = kappa delta
  OP_GENW = 3     // splitting w != 1/3: Sigma involves the centre value (full Newton step)
};

// Per-level constants of the FP64 operator.
struct OpConst64 {
  double h2;      // h^2
  double inv_h2;  // 1/h^2
  double e1, e2;  // OP_SQRT: q = src + e1*A + e2*B
  double c1, c2;  // OP_CONJ: u = src + c1*A + c2*B
  double c3;      // 4(1-w) alpha
  double k2s;     // sigma * k2, k2 = 2/c3
  double k2;
  double e1h, c1h;  // 2*e1, 2*c1: the same terms written with A/2
  double h2_6;      // h^2/6
  double upd_s;     // -h^2 k2s / 6: the smoother's coefficient of sqrt(q)
  double omega;     // relaxation of the pointwise Newton step (1 = the plain step)
  // OP_GENW: q = src + gA (Dxx^2 + Dyy^2 + Dzz^2) + gB (Dxx Dyy + Dxx Dzz + Dyy Dzz)
  //            + gC (Cxy^2 + Cxz^2 + Cyz^2), the D's including the centre value;
  //          gAB = gA + gB, so dq/dphi_centre = -4 gAB (Sx + Sy + Sz - 6 phi)
  double gA, gB, gC, gAB;
  int mode;
};

// Per-level constants of the FP32 correction operator (mixed precision).
struct OpConst32 {
  float h2, inv_h2;
  float g1, g2;   // alpha/(3h^4), alpha/(8h^4): Delta u = g1*dA + g2*dB
  float c3;       // 4(1-w) alpha
  float k2;       // 2/c3 (0 when alpha == 0)
  float sigma;    // +1 physical root, -1 the other one
  float sigma2;   // 2 sigma
  float sk2;      // sigma k2
  int linear;     // alpha == 0
};

// Scalars that a residual evaluation leaves for one level.
struct LevelScalars {
  double lambda;     // compatibility constant mean(d) (periodic), 0 (Dirichlet)
  double res;        // max |d - lambda|
  double sum;        // sum of d
  double dmax, dmin;
  long long guards;  // cells with q < 0
  long long nonfinite;
  unsigned long long floored;  // cells whose source was held at the real-root bound
};

// Programmatic dependent launch.  Kernels launched with launch_k() may start
// while the grid before them in the stream is still finishing; each such kernel
// opens a PdlScope first, which waits until that grid has completed and its
// writes are visible (griddepcontrol.wait), and on exit lets the next grid
// begin launching (griddepcontrol.launch_dependents).  What overlaps is launch
// latency and the scheduling of CTAs, never a kernel's memory accesses.
struct PdlScope {
  __device__ __forceinline__ PdlScope() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
  __device__ __forceinline__ ~PdlScope() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  }
};

// Split a cell index t (< 2^31; grids have n <= 1024) into (t % d, (t / d) % d,
// t / d^2) with 32-bit arithmetic; shifts and masks when d is a power of two.
__device__ __forceinline__ void split3(unsigned t, int d, int& i, int& j, int& k) {
  const unsigned ud = (unsigned)d;
  if ((ud & (ud - 1u)) == 0u) {
    const int s = __ffs(d) - 1;
    const unsigned r = t >> s;
    i = (int)(t & (ud - 1u));
    j = (int)(r & (ud - 1u));
    k = (int)(r >> s);
  } else {
    const unsigned r = t / ud, r2 = r / ud;
    i = (int)(t - r * ud);
    j = (int)(r - r2 * ud);
    k = (int)r2;
  }
}

__device__ __forceinline__ int wrap_up(int i, int n) { return (i + 1 == n) ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return (i == 0) ? n - 1 : i - 1; }

__device__ __forceinline__ long long lidx(int i, int j, int k, int n) {
  return (long long)i + (long long)n * ((long long)j + (long long)n * (long long)k);
}

// Cells per thread of the outer FP64 residual with its FP32 hand-off.
constexpr int kHandoffCells = 4;


// The 18 stencil neighbours of one cell in the form the operator uses: face pair
// sums and cross differences (without the 1/4).
template <typename T>
struct StencilT {
  T sx, sy, sz, cxy, cxz, cyz;
};

// Offsets from cell (i,j,k) to its six face neighbours in a periodic n^3 array,
// x fastest, with the wrap folded in (n <= 1024, so every offset fits in 32 bits).
struct NbrOff {
  int xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ NbrOff nbr_offsets(int i, int j, int k, int n) {
  const int n2 = n * n, n3 = n2 * n;
  NbrOff o;
  o.xp = (i + 1 == n) ? 1 - n : 1;
  o.xm = (i == 0) ? n - 1 : -1;
  o.yp = (j + 1 == n) ? n - n2 : n;
  o.ym = (j == 0) ? n2 - n : -n;
  o.zp = (k + 1 == n) ? n2 - n3 : n2;
  o.zm = (k == 0) ? n3 - n2 : -n2;
  return o;
}

// Face sums and cross differences around the cell at c (a pointer to it).
template <typename T>
__device__ __forceinline__ StencilT<T> gather_at(const T* __restrict__ c, const NbrOff& o) {
  StencilT<T> s;
  s.sx = c[o.xp] + c[o.xm];
  s.sy = c[o.yp] + c[o.ym];
  s.sz = c[o.zp] + c[o.zm];
  s.cxy = (c[o.xp + o.yp] + c[o.xm + o.ym]) - (c[o.xp + o.ym] + c[o.xm + o.yp]);
  s.cxz = (c[o.xp + o.zp] + c[o.xm + o.zm]) - (c[o.xp + o.zm] + c[o.xm + o.zp]);
  s.cyz = (c[o.yp + o.zp] + c[o.ym + o.zm]) - (c[o.yp + o.zm] + c[o.ym + o.zp]);
  return s;
}

// Gather the face sums and cross differences of cell (i,j,k) of a periodic n^3
// array.
template <typename T>
__device__ __forceinline__ StencilT<T> gather_periodic(const T* __restrict__ p, int i, int j,
                                                       int k, int n) {
  return gather_at(p + lidx(i, j, k, n), nbr_offsets(i, j, k, n));
}

// A/2 with A = (Sx-Sy)^2 + (Sx-Sz)^2 + (Sy-Sz)^2 = 2[a1(a1-a2) + a2^2], a1 = Sx-Sy,
// a2 = Sx-Sz (the form is positive definite, so no cancellation).
__device__ __forceinline__ double half_A(const StencilT<double>& s) {
  const double a1 = s.sx - s.sy, a2 = s.sx - s.sz;
  return fma(a1, a1 - a2, a2 * a2);
}

// sqrt(q) for q >= 0 as q * rsqrt(q) (rsqrt is within 1 ulp); 0 stays 0 and a NaN
// stays NaN.
__device__ __forceinline__ double sqrt_nonneg(double q) {
  return (q == 0.0) ? 0.0 : q * rsqrt(q);
}

// sqrt_nonneg(q < 0 ? 0 : q) with both tests on the bit pattern (integer ALU
// instructions instead of FP64 compares, which share GB300's narrow FP64 pipe).
// As a signed 64-bit integer, +0 is 0 and the negative non-NaN doubles (-0 to
// -inf) are exactly the values <= the pattern of -inf; negative NaNs lie above it
// and, like every other input, take q * rsqrt(q).  Same result for every q.
__device__ __forceinline__ double sqrt_clamped(double q) {
  const long long b = __double_as_longlong(q);
  return (b == 0 || b <= (long long)0xFFF0000000000000ULL) ? 0.0 : q * rsqrt(q);
}

// q < 0 on the bit pattern: the negative non-NaN doubles other than -0.
__device__ __forceinline__ bool neg_guard(double q) {
  const long long b = __double_as_longlong(q);
  return b <= (long long)0xFFF0000000000000ULL && b != (long long)0x8000000000000000ULL;
}

// x != 1.0 on the bit pattern (for the relaxation factor, validated in (0, 1]).
__device__ __forceinline__ bool not_one(double x) {
  return __double_as_longlong(x) != 0x3FF0000000000000LL;
}

// An integer key of a double whose order is the numeric order (-0 below +0): the
// bit pattern with the magnitude bits flipped for negative values.  The map is
// its own inverse.
__device__ __forceinline__ long long order_key(double d) {
  const long long b = __double_as_longlong(d);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double from_order_key(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

// isfinite(d) on the bit pattern: the exponent field is not all ones.
__device__ __forceinline__ bool finite_bits(double d) {
  return ((__double_as_longlong(d) >> 52) & 0x7ff) != 0x7ff;
}

// D (the root of Eq. two_branch) from the stencil and the per-cell source term.
// `guard` is set when the discriminant is negative.
__device__ __forceinline__ double root_D(const StencilT<double>& s, double src,
                                         const OpConst64& c, bool& guard) {
  if (c.mode == OP_LINEAR) {
    guard = false;
    return src;
  }
  const double A2 = half_A(s);
  const double B = fma(s.cxy, s.cxy, fma(s.cxz, s.cxz, s.cyz * s.cyz));
  if (c.mode == OP_SQRT) {
    const double q = fma(c.e1h, A2, fma(c.e2, B, src));
    guard = neg_guard(q);
    return fma(c.k2s, sqrt_clamped(q), -c.k2);
  }
  const double u = fma(c.c1h, A2, fma(c.c2, B, src));
  const double q = fma(c.c3, u, 1.0);
  guard = q < 0.0;
  if (guard) return -c.k2;
  return (2.0 * u) / (1.0 + sqrt(q));
}

// Discriminant of a cell for a general splitting constant w (Sec. III.B,
// Sigma_ijk with every second difference taken through the centre value).
__device__ __forceinline__ double genw_q(const StencilT<double>& s, double ctr, double src,
                                         const OpConst64& c) {
  const double dxx = fma(-2.0, ctr, s.sx), dyy = fma(-2.0, ctr, s.sy), dzz = fma(-2.0, ctr, s.sz);
  const double sq = fma(dxx, dxx, fma(dyy, dyy, dzz * dzz));
  const double cr = fma(dxx, dyy, fma(dxx, dzz, dyy * dzz));
  const double cc = fma(s.cxy, s.cxy, fma(s.cxz, s.cxz, s.cyz * s.cyz));
  return fma(c.gA, sq, fma(c.gB, cr, fma(c.gC, cc, src)));
}

// D of any mode; ctr (the cell's own value) enters only for OP_GENW.
__device__ __forceinline__ double root_Dc(const StencilT<double>& s, double ctr, double src,
                                          const OpConst64& c, bool& guard) {
  if (c.mode != OP_GENW) return root_D(s, src, c, guard);
  const double q = genw_q(s, ctr, src, c);
  guard = neg_guard(q);
  return fma(c.k2s, sqrt_clamped(q), -c.k2);
}

// Newton step of one cell for OP_GENW: phi - L/(dL/dphi) with
// L = (Sx + Sy + Sz - 6 phi)/h^2 - D - rhs and dL/dphi = -6/h^2 - dD/dphi, where
// dD/dphi = -2 k2s gAB (Sx + Sy + Sz - 6 phi) / sqrt(q) (taken as 0 for q <= 1e-12).
__device__ __forceinline__ double genw_newton(const StencilT<double>& s, double ctr, double src,
                                              double rhs, const OpConst64& c) {
  const double q = genw_q(s, ctr, src, c);
  const double sq = sqrt_nonneg(q < 0.0 ? 0.0 : q);
  const double D = fma(c.k2s, sq, -c.k2);
  const double lap6 = fma(-6.0, ctr, s.sx + s.sy + s.sz);
  const double L = fma(lap6, c.inv_h2, -D) - rhs;
  const double dD = q > 1e-12 ? -2.0 * c.k2s * c.gAB * lap6 / sq : 0.0;
  const double J = fma(-6.0, c.inv_h2, -dD);
  return ctr - L / J;
}

// Deterministic block reduction of (sum, max, min, guards, nonfinite).
struct Partial {
  double sum, dmax, dmin;
  long long guards, nonfinite;
};

__device__ __forceinline__ void partial_init(Partial& p) {
  p.sum = 0.0;
  p.dmax = -INFINITY;
  p.dmin = INFINITY;
  p.guards = 0;
  p.nonfinite = 0;
}

// The extremes compare integer order keys (order_key) rather than FP64 values:
// the FP64 pipe is the limit of the kernels that call this per cell.
__device__ __forceinline__ void partial_add(Partial& p, double d, bool guard) {
  if (finite_bits(d)) {
    p.sum += d;
    const long long k = order_key(d);
    if (k > order_key(p.dmax)) p.dmax = d;
    if (k < order_key(p.dmin)) p.dmin = d;
  } else {
    p.nonfinite += 1;
  }
  p.guards += guard ? 1 : 0;
}

__device__ __forceinline__ void partial_merge(Partial& a, const Partial& b) {
  a.sum += b.sum;
  a.dmax = fmax(a.dmax, b.dmax);
  a.dmin = fmin(a.dmin, b.dmin);
  a.guards += b.guards;
  a.nonfinite += b.nonfinite;
}

__device__ __forceinline__ Partial warp_reduce(Partial p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Partial q;
    q.sum = __shfl_down_sync(0xffffffffu, p.sum, o);
    q.dmax = __shfl_down_sync(0xffffffffu, p.dmax, o);
    q.dmin = __shfl_down_sync(0xffffffffu, p.dmin, o);
    q.guards = __shfl_down_sync(0xffffffffu, p.guards, o);
    q.nonfinite = __shfl_down_sync(0xffffffffu, p.nonfinite, o);
    partial_merge(p, q);
  }
  return p;
}

// Reduce over the block; thread 0 returns the block's value.  blockDim.x must
// be a multiple of 32 and at most 1024.
__device__ __forceinline__ Partial block_reduce(Partial p) {
  __shared__ Partial sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  p = warp_reduce(p);
  if (lane == 0) sh[wid] = p;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    Partial q;
    if (lane < nw) q = sh[lane];
    else partial_init(q);
    q = warp_reduce(q);
    p = q;
  }
  __syncthreads();
  return p;
}

// Maximum over the block; every thread returns it.
__device__ __forceinline__ double block_max(double v) {
  __shared__ double shm[32];
  __shared__ double result;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) shm[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double w = lane < nw ? shm[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_down_sync(0xffffffffu, w, o));
    if (lane == 0) result = w;
  }
  __syncthreads();
  return result;
}

// Stopping rule of the one-CTA coarsest solves: the residual fell by `drop`, or
// it reached the rounding level of the operator's terms (`scale` is the largest
// term), or it stopped falling.
__device__ __forceinline__ bool coarsest_done(double r, double r0, double r_prev, double scale,
                                              double drop) {
  if (!(r > drop * r0)) return true;
  if (r <= 64.0 * 1.1102230246251565e-16 * scale) return true;
  return r >= 0.95 * r_prev;
}

}  // namespace mg
