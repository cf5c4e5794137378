// One full four-colour Newton-Gauss-Seidel sweep of the FP32 correction
// operator N(e) = g + mu in ONE launch (the smoother of Sec. III.B applied to the
// correction equation of the mixed-precision solve).
//
// The per-colour kernels stream the whole e and phi0 arrays four times per sweep,
// because every colour stage reads the 18 neighbours of its cells.  Here a CTA
// owns a 64 x 16 column of the grid over a run of z planes and marches up that
// run, keeping a ring of planes of e and phi0 in shared memory.  The colour
// stages form a wavefront in two phases per step t: phase A updates colour 0 on
// plane t and colour 2 on plane t-3, phase B colour 1 on plane t-1 and colour 3
// on plane t-4.  Colour c on plane p needs colours < c already updated on planes
// p-1..p+1 and colours > c not yet updated there; these lags give exactly that,
// and the two stages of a phase touch disjoint cells and read nothing the other
// writes.  The sweep is therefore the same sequence of cell updates as the
// per-colour kernels, with the same bits.
//
// Each CTA loads its tile with a 4-cell halo in x and y (a 72 x 24 window) and
// recomputes the halo cells' earlier colour stages itself, the valid region
// shrinking by one cell per stage.  Neighbouring CTAs therefore never exchange
// data: every CTA reads the previous sweep's values from `e_in` and writes only
// its own tile to `e_out` (two buffers, swapped by the caller between sweeps).
// Along z the run starts 3 planes early for the same reason.
//
// Shared memory holds each plane row split by x parity ([even x | odd x]), so
// the cells of one colour in a row are contiguous: a thread updates two cells of
// one colour (x and x+2) with 64-bit shared loads of neighbour pairs and packed
// FP32x2 arithmetic (the cell pair rides in the two lanes of each instruction).
// Per cell and sweep the kernel moves the algorithmic 20 bytes of HBM traffic
// (read e, phi0, q0, g; write e) plus the halo re-reads, which hit L2.
#include <cuda_runtime.h>

#include "mg_bodies32.cuh"
#include "mg_internal.h"

namespace mg {

namespace sw {
constexpr int TX = 64, TY = 16, H = 4;
constexpr int WX = TX + 2 * H;          // 72: window width
constexpr int WY = TY + 2 * H;          // 24: window rows
constexpr int HALF = WX / 2;            // 36: cells of one x parity in a window row
constexpr int ROW = WX;                 // floats per row: even half, then odd half
constexpr int PLANE = WY * ROW;         // 1728
constexpr int PAD = 4;                  // guard floats around each plane (16 B aligned)
constexpr int SLOT = PLANE + 2 * PAD;   // 1736 floats = 6944 B per ring slot
constexpr int RING = 8;                 // planes t-5 .. t+2
constexpr int THREADS = 224;
constexpr int PAIRS = HALF / 2;         // 18 cell pairs per half row
constexpr int GROUPS = WX / 4;          // 18 float4 per window row
constexpr int LOADS = WY * GROUPS;      // 432 float4 per plane and array
constexpr int NLOAD = (2 * LOADS + THREADS - 1) / THREADS;  // 4 float4 per thread and plane
constexpr int STAGE_ROWS0 = 11;         // rows of one colour that stage 0 updates
constexpr size_t SMEM = (size_t)2 * RING * SLOT * sizeof(float) + (WX + WY) * sizeof(int);
}  // namespace sw

struct Sweep32Args {
  int n, zc, tiles_x, tiles_y, chunks;
  const float* e_in;
  float* e_out;
  const float* phi0;
  const float* q0;
  const float* g;
  const LevelScalars* sc;
  OpConst32 c;
};

namespace {

__device__ __forceinline__ int pmod(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}
// k within one period of [0, n)
__device__ __forceinline__ int wrap1(int k, int n) { return k < 0 ? k + n : (k >= n ? k - n : k); }
__device__ __forceinline__ int slot_of(int k) { return (k + 8 * sw::RING) & (sw::RING - 1); }

// x neighbours of a cell pair from the other-parity half row at p (the pair at
// the same index) and its aligned neighbour pair on the side the pair needs.
template <int A>
__device__ __forceinline__ void xpair(const float* p, float2& xp, float2& xm) {
  const float2 o = ld2(p);
  const float2 s = ld2(p + (A ? 2 : -2));
  if (A) {
    xm = o;
    xp = make_float2(o.y, s.x);
  } else {
    xp = o;
    xm = make_float2(s.y, o.x);
  }
}

// Face sums and cross differences of a cell pair (same order of operations as
// gather_at): cen / oth are the offsets of the pair's own-parity and
// other-parity half rows inside a plane.
template <int A>
__device__ __forceinline__ Stencil2 gather2(const float* Xm, const float* X0, const float* Xp,
                                            int cen, int oth) {
  using namespace sw;
  float2 xp, xm, xpyp, xmyp, xpym, xmym, xpzp, xmzp, xpzm, xmzm;
  xpair<A>(X0 + oth, xp, xm);
  xpair<A>(X0 + oth + ROW, xpyp, xmyp);
  xpair<A>(X0 + oth - ROW, xpym, xmym);
  xpair<A>(Xp + oth, xpzp, xmzp);
  xpair<A>(Xm + oth, xpzm, xmzm);
  const float2 yp = ld2(X0 + cen + ROW), ym = ld2(X0 + cen - ROW);
  const float2 zp = ld2(Xp + cen), zm = ld2(Xm + cen);
  const float2 ypzp = ld2(Xp + cen + ROW), ymzp = ld2(Xp + cen - ROW);
  const float2 ypzm = ld2(Xm + cen + ROW), ymzm = ld2(Xm + cen - ROW);
  Stencil2 s;
  s.sx = add2(xp, xm);
  s.sy = add2(yp, ym);
  s.sz = add2(zp, zm);
  s.cxy = sub2(add2(xpyp, xmym), add2(xpym, xmyp));
  s.cxz = sub2(add2(xpzp, xmzm), add2(xpzm, xmzp));
  s.cyz = sub2(add2(ypzp, ymzm), add2(ypzm, ymzp));
  return s;
}

// Window row of this thread's cell pair for colour stage S on a plane whose
// colour-S cells sit on rows of parity b.
template <int S>
__device__ __forceinline__ int stage_row(int b, int qrow) {
  return (1 + S) + (((1 + S) ^ b) & 1) + 2 * qrow;
}

template <int S>
__device__ __forceinline__ bool stage_lane() {
  return threadIdx.x < sw::PAIRS * (sw::STAGE_ROWS0 - S);
}

template <int A, bool LIN>
__device__ __forceinline__ void stage_pair(float* se, const float* sp, int k, int row, int m,
                                           float2 q0, float2 g, float mu, const OpConst32& c) {
  using namespace sw;
  const int om = slot_of(k - 1) * SLOT + PAD, o0 = slot_of(k) * SLOT + PAD,
            op = slot_of(k + 1) * SLOT + PAD;
  const int cen = row * ROW + A * HALF + m;
  const int oth = row * ROW + (1 - A) * HALF + m;
  const Stencil2 ee = gather2<A>(se + om, se + o0, se + op, cen, oth);
  float2 dd = make_float2(0.f, 0.f);
  if (!LIN) {
    const Stencil2 pp = gather2<A>(sp + om, sp + o0, sp + op, cen, oth);
    dd = dD2(ee, pp, q0, c);
  }
  const float2 v = mul2(fma2(splat(-c.h2), add2(dd, add2(g, splat(mu))),
                             add2(add2(ee.sx, ee.sy), ee.sz)),
                        splat(1.f / 6.f));
  *reinterpret_cast<float2*>(se + o0 + cen) = v;
}

// Colour stage S on window plane k (global plane k mod n).
template <int S, bool LIN>
__device__ __forceinline__ void stage(float* se, const float* sp, int k, int qrow, int m,
                                      float2 q0, float2 g, float mu, const OpConst32& c) {
  if (!stage_lane<S>()) return;
  const int a = (S ^ k) & 1, b = ((S >> 1) ^ k) & 1;
  const int row = stage_row<S>(b, qrow);
  if (a)
    stage_pair<1, LIN>(se, sp, k, row, m, q0, g, mu, c);
  else
    stage_pair<0, LIN>(se, sp, k, row, m, q0, g, mu, c);
}

// q0 and g of this thread's cell pair for stage S on plane k (xw: wrapped x,
// yw: wrapped y times n).
template <int S>
__device__ __forceinline__ void fetch_qg(const float* __restrict__ q0a,
                                         const float* __restrict__ ga, int n, const int* xw,
                                         const int* yw, int k, int qrow, int m, float2& q,
                                         float2& g) {
  if (!stage_lane<S>()) return;
  const int a = (S ^ k) & 1, b = ((S >> 1) ^ k) & 1;
  const int base = wrap1(k, n) * n * n + yw[stage_row<S>(b, qrow)];
  const int ia = base + xw[2 * m + a], ib = base + xw[2 * m + 2 + a];
  q = make_float2(__ldg(q0a + ia), __ldg(q0a + ib));
  g = make_float2(__ldg(ga + ia), __ldg(ga + ib));
}

// This thread's share of a window plane of e_in and phi0: its float4 loads
// (global offsets within a plane, per item) and where they go in a ring slot.
struct LoadPlan {
  int goff[sw::NLOAD];
  int soff[sw::NLOAD];  // ring-relative, includes the array (e or phi0) base
  int arr;              // bit r: load r reads phi0
  int live;             // bit r: load r exists
};

template <bool LIN>
__device__ __forceinline__ void plan_loads(LoadPlan& L, const int* xw, const int* yw) {
  using namespace sw;
  L.arr = 0;
  L.live = 0;
#pragma unroll
  for (int r = 0; r < NLOAD; ++r) {
    const int l = threadIdx.x + r * THREADS;
    const int arr = l >= LOADS;
    const int rem = l - arr * LOADS;
    const int row = rem / GROUPS, q = rem - row * GROUPS;
    const bool live = l < (LIN ? LOADS : 2 * LOADS);
    L.goff[r] = live ? yw[row] + xw[4 * q] : 0;
    L.soff[r] = arr * RING * SLOT + PAD + row * ROW + 2 * q;
    L.arr |= arr << r;
    L.live |= (int)live << r;
  }
}

__device__ __forceinline__ void plane_issue(const Sweep32Args& A, const LoadPlan& L, int k,
                                            float4 (&st)[sw::NLOAD]) {
  const int pb = wrap1(k, A.n) * A.n * A.n;
#pragma unroll
  for (int r = 0; r < sw::NLOAD; ++r)
    if ((L.live >> r) & 1)
      st[r] = __ldg(reinterpret_cast<const float4*>(((L.arr >> r) & 1 ? A.phi0 : A.e_in) + pb +
                                                    L.goff[r]));
}

// Store a staged plane into its ring slot, split by x parity.
__device__ __forceinline__ void plane_commit(float* ring, const LoadPlan& L, int k,
                                             const float4 (&st)[sw::NLOAD]) {
  float* base = ring + slot_of(k) * sw::SLOT;
#pragma unroll
  for (int r = 0; r < sw::NLOAD; ++r)
    if ((L.live >> r) & 1) {
      float* dst = base + L.soff[r];
      *reinterpret_cast<float2*>(dst) = make_float2(st[r].x, st[r].z);
      *reinterpret_cast<float2*>(dst + sw::HALF) = make_float2(st[r].y, st[r].w);
    }
}

// The finished tile of plane k (x0 + [0, w), y0 + [0, h)) to e_out.
__device__ __forceinline__ void plane_write(const Sweep32Args& A, const float* se, int k, int x0,
                                            int y0, int w, int h) {
  using namespace sw;
  const int n = A.n;
  const float* P = se + slot_of(k) * SLOT + PAD;
  const int pb = wrap1(k, n) * n * n;
  for (int v = threadIdx.x; v < TY * (TX / 4); v += THREADS) {
    const int row = v / (TX / 4), q = v - row * (TX / 4);
    if (row >= h || 4 * q >= w) continue;
    const float* src = P + (row + H) * ROW + 2 + 2 * q;
    const float2 ev = ld2(src), od = ld2(src + HALF);
    *reinterpret_cast<float4*>(A.e_out + pb + (y0 + row) * n + x0 + 4 * q) =
        make_float4(ev.x, od.x, ev.y, od.y);
  }
}

template <bool LIN>
__device__ __forceinline__ void sweep_item(const Sweep32Args& A, float* ring, int* xw, int* yw,
                                           int item, float mu) {
  using namespace sw;
  const int n = A.n;
  float* const se = ring;
  const float* const sp = ring + RING * SLOT;
  const int ntile = A.tiles_x * A.tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
  const int z0 = chunk * A.zc, zend = min(z0 + A.zc, n);
  const int w = min(TX, n - x0), h = min(TY, n - y0);
  const int qrow = threadIdx.x / PAIRS, m = 2 * (threadIdx.x % PAIRS);
  const OpConst32& c = A.c;

  __syncthreads();  // the previous item is done with the tables and the ring
  for (int v = threadIdx.x; v < WX + WY; v += THREADS) {
    if (v < WX)
      xw[v] = pmod(x0 - H + v, n);
    else
      yw[v - WX] = pmod(y0 - H + (v - WX), n) * n;
  }
  __syncthreads();

  LoadPlan L;
  plan_loads<LIN>(L, xw, yw);
  float4 st[NLOAD];
  for (int k = z0 - 4; k <= z0 - 2; ++k) {
    plane_issue(A, L, k, st);
    plane_commit(ring, L, k, st);
  }
  plane_issue(A, L, z0 - 1, st);
  const int t0 = z0 - 3;
  float2 q0s0{}, q0s1{}, q0s2{}, q0s3{}, gs0{}, gs1{}, gs2{}, gs3{};
  fetch_qg<0>(A.q0, A.g, n, xw, yw, t0, qrow, m, q0s0, gs0);
  fetch_qg<1>(A.q0, A.g, n, xw, yw, t0 - 1, qrow, m, q0s1, gs1);
  fetch_qg<2>(A.q0, A.g, n, xw, yw, t0 - 3, qrow, m, q0s2, gs2);
  fetch_qg<3>(A.q0, A.g, n, xw, yw, t0 - 4, qrow, m, q0s3, gs3);
  __syncthreads();

  const int tend = zend + 3;  // the last plane read (by colour 0 on plane zend + 2)
  for (int t = t0; t < zend + 4; ++t) {
    // phase A: colour 0 on plane t, colour 2 on plane t - 3
    if (t < zend + 3) stage<0, LIN>(se, sp, t, qrow, m, q0s0, gs0, mu, c);
    if (t - 3 >= z0 - 1 && t - 3 < zend + 1) stage<2, LIN>(se, sp, t - 3, qrow, m, q0s2, gs2, mu, c);
    fetch_qg<0>(A.q0, A.g, n, xw, yw, t + 1, qrow, m, q0s0, gs0);
    fetch_qg<2>(A.q0, A.g, n, xw, yw, t - 2, qrow, m, q0s2, gs2);
    __syncthreads();
    // phase B: colour 1 on plane t - 1, colour 3 on plane t - 4
    if (t - 1 >= z0 - 2 && t - 1 < zend + 2) stage<1, LIN>(se, sp, t - 1, qrow, m, q0s1, gs1, mu, c);
    const bool out = t - 4 >= z0;
    if (out) stage<3, LIN>(se, sp, t - 4, qrow, m, q0s3, gs3, mu, c);
    fetch_qg<1>(A.q0, A.g, n, xw, yw, t, qrow, m, q0s1, gs1);
    fetch_qg<3>(A.q0, A.g, n, xw, yw, t - 3, qrow, m, q0s3, gs3);
    if (t + 2 <= tend) {
      plane_commit(ring, L, t + 2, st);
      if (t + 3 <= tend) plane_issue(A, L, t + 3, st);
    }
    __syncthreads();
    if (out) plane_write(A, se, t - 4, x0, y0, w, h);
  }
}

__global__ void __launch_bounds__(sw::THREADS, 2) k_sweep32(const __grid_constant__ Sweep32Args A) {
  PdlScope pdl_scope;
  extern __shared__ __align__(16) float sm[];
  int* const xw = reinterpret_cast<int*>(sm + 2 * sw::RING * sw::SLOT);
  int* const yw = xw + sw::WX;
  const float mu = (float)A.sc->lambda;
  const int nitems = A.tiles_x * A.tiles_y * A.chunks;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    if (A.c.linear)
      sweep_item<true>(A, sm, xw, yw, item, mu);
    else
      sweep_item<false>(A, sm, xw, yw, item, mu);
  }
}

int g_sweep_sms = 0;

}  // namespace

bool sweep32_eligible(int n) { return n >= 32 && n % 4 == 0; }

void init_sweep32() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(k_sweep32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw::SMEM);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_sweep_sms, cudaDevAttrMultiProcessorCount, dev);
  if (g_sweep_sms <= 0) g_sweep_sms = 1;
  cudaGetLastError();
}

// Plane-run length: the candidate with the smallest estimated time, counting
// whole waves of resident CTAs (two per SM) times the steps of one run.
static int sweep_chunk(int n, int tiles, int sms) {
  int best = n;
  long long best_cost = -1;
  for (int zc : {8, 16, 32, 64, 128}) {
    if (zc > n) break;
    const int chunks = (n + zc - 1) / zc;
    const long long items = (long long)tiles * chunks;
    const long long slots = 2LL * sms;
    const long long waves = (items + slots - 1) / slots;
    const long long cost = waves * (zc + 7);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

void launch_sweep32(cudaStream_t st, int n, const float* e_in, float* e_out, const float* phi0,
                    const float* q0, const float* g, const LevelScalars* sc, const OpConst32& c) {
  Sweep32Args a;
  a.n = n;
  a.tiles_x = (n + sw::TX - 1) / sw::TX;
  a.tiles_y = (n + sw::TY - 1) / sw::TY;
  a.zc = sweep_chunk(n, a.tiles_x * a.tiles_y, g_sweep_sms);
  a.chunks = (n + a.zc - 1) / a.zc;
  a.e_in = e_in;
  a.e_out = e_out;
  a.phi0 = phi0;
  a.q0 = q0;
  a.g = g;
  a.sc = sc;
  a.c = c;
  const long long items = (long long)a.tiles_x * a.tiles_y * a.chunks;
  const int grid = (int)(items < 2LL * g_sweep_sms ? items : 2LL * g_sweep_sms);
  launch_k(k_sweep32, grid, sw::THREADS, sw::SMEM, st, a);
  count_launches(1);
}

}  // namespace mg
