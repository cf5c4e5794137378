// Half sweeps of the FP32 correction smoother (the four-colour Newton-Gauss-Seidel
// sweep of Sec. III.B applied to the correction equation of the mixed-precision
// solve), two colours per launch.
//
// Colour c = ((i+k)&1) + 2((j+k)&1).  Colours 2hb and 2hb+1 (hb = 0 or 1) live on
// the x rows (j, k) with (j+k)&1 == hb and alternate along them.  A colour-2hb
// cell ("A") reads only cells of other colours; a colour-2hb+1 cell ("B") reads
// A cells at x+-1 and at (0, +-1, +-1), and the other half's colours elsewhere.
// One launch updates A then B for every row of its parity:
//   - a CTA owns TY whole rows (x = 0 .. N-1, so the x wrap is an index mask)
//     and a run of z planes, and marches up the run: step t updates A on plane t
//     and B on plane t-2; B then finds every A value it needs (planes t-3 .. t-1)
//     already updated, and A reads only B values, which are never updated in
//     shared memory, so both run in one phase per step;
//   - B on rows j0 .. j0+TY-1 needs A on rows j0-1 and j0+TY too, which belong to
//     the neighbouring CTAs: the CTA recomputes A on those halo rows itself (and
//     on plane z0-1 below its run) from values that are not updated in this
//     launch, and writes back only its own rows and planes;
//   - planes of e and phi0, TY+4 rows each, arrive two planes ahead in a raw ring
//     of two shared-memory slots by bulk asynchronous copies (cp.async.bulk,
//     completing on an mbarrier); the threads then split each row by x parity
//     into a ring of five compute slots, so that the cells of one colour, which
//     alternate along x, sit side by side: each thread updates two neighbouring
//     cells of one colour with packed FP32x2 arithmetic and 64-bit shared loads.
// The update of every cell is the per-colour kernels' arithmetic (gs_value32,
// dD32) on the same neighbour values in the same order, so a sweep gives the
// same bits as four per-colour launches.
//
// Buffers: the first half sweep (hb = 0) reads every cell from e_in and writes
// colours 0 and 1 to e_out; the second reads rows of colours 0 and 1 from e_out
// and the others from e_in, and writes colours 2 and 3 to e_out.  e_out then
// holds the whole sweep; e_in is untouched (other CTAs read it while this one
// writes).
//
// Each wait on a copy is bounded by a wall-clock limit (%globaltimer); a CTA
// whose copy does not arrive in time sets *err, waits (bounded) for its copies
// still in flight, and returns.
#include <cuda_runtime.h>

#include "mg_bodies32.cuh"
#include "mg_internal.h"

namespace mg {

namespace hsw {
constexpr int SPLIT = 5;  // compute slots: planes t-3 .. t+1
constexpr int RAW = 2;    // landing slots: plane t+1 (being split) and plane t+2 (arriving)
constexpr int TY = 4;     // rows per tile: A on TY+2 rows, loads of TY+4 rows per plane
constexpr int ROWS = TY + 4;
// threads: one cell pair of A (TY/2 + 1 rows) or of B (TY/2 rows) each
template <int N>
constexpr int threads() {
  return (TY + 1) * (N / 4);
}
template <int N>
constexpr size_t smem_bytes() {
  return (size_t)2 * (SPLIT + RAW) * ROWS * N * sizeof(float);
}
}  // namespace hsw

struct HalfArgs {
  const float* e_in;
  float* e_out;
  const float* phi0;
  const float* q0;
  const float* g;
  const LevelScalars* sc;
  OpConst32 c;
  int hb;        // 0: colours 0 and 1; 1: colours 2 and 3
  int zch;       // z runs per column of tiles
  int* err;      // set to 1 by a CTA whose copy did not arrive in time
  unsigned long long limit_ns;
};

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait until phase `parity` of the barrier has completed, at most limit_ns (a
// limit of 0 accepts only a phase that has completed already).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (global_ns() - t0 >= limit_ns) return false;
    if (mbar_try(bar, parity)) return true;
  }
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

}  // namespace

// Face sums and cross differences of two neighbouring cells of one colour (x and
// x+2), from rows split by x parity: own / oth point at the pair's own-parity and
// other-parity halves of the centre row (index m, the pair's first cell), M and P
// offsets of the planes below and above, R the row pitch.  A = 1 for odd x.  The
// sums of gather_at in the same order, lane by lane.
template <int HN, int A>
__device__ __forceinline__ Stencil2 gather_split(const float* own, const float* oth, int m,
                                                 int M, int P, int R) {
  auto xpair = [&](const float* h, float2& xp, float2& xm) {
    const float2 o = ld2(h + m);
    const float2 s2 = ld2(h + ((m + (A ? 2 : -2)) & (HN - 1)));
    if (A) {
      xm = o;
      xp = make_float2(o.y, s2.x);
    } else {
      xp = o;
      xm = make_float2(s2.y, o.x);
    }
  };
  float2 xp, xm, xpyp, xmyp, xpym, xmym, xpzp, xmzp, xpzm, xmzm;
  xpair(oth, xp, xm);
  xpair(oth + R, xpyp, xmyp);
  xpair(oth - R, xpym, xmym);
  xpair(oth + P, xpzp, xmzp);
  xpair(oth + M, xpzm, xmzm);
  const float* c = own + m;
  const float2 yp = ld2(c + R), ym = ld2(c - R), zp = ld2(c + P), zm = ld2(c + M);
  const float2 ypzp = ld2(c + P + R), ymzm = ld2(c + M - R), ypzm = ld2(c + M + R),
               ymzp = ld2(c + P - R);
  Stencil2 s;
  s.sx = add2(xp, xm);
  s.sy = add2(yp, ym);
  s.sz = add2(zp, zm);
  s.cxy = sub2(add2(xpyp, xmym), add2(xpym, xmyp));
  s.cxz = sub2(add2(xpzp, xmzm), add2(xpzm, xmzp));
  s.cyz = sub2(add2(ypzp, ymzm), add2(ypzm, ymzp));
  return s;
}

template <int N, int A>
__device__ __forceinline__ float2 pair_update(const float* se, const float* sp, int base_c,
                                              int M, int P, int m, float2 q0, float2 g, float mu,
                                              const OpConst32& c) {
  constexpr int HN = N / 2;
  const Stencil2 ee = gather_split<HN, A>(se + base_c + A * HN, se + base_c + (1 - A) * HN, m, M,
                                          P, N);
  float2 dd = make_float2(0.f, 0.f);
  if (!c.linear) {
    const Stencil2 pp = gather_split<HN, A>(sp + base_c + A * HN, sp + base_c + (1 - A) * HN, m,
                                            M, P, N);
    dd = dD2(ee, pp, q0, c);
  }
  return mul2(fma2(splat(-c.h2), add2(dd, add2(g, splat(mu))), add2(add2(ee.sx, ee.sy), ee.sz)),
              splat(1.f / 6.f));
}

template <int N>
__global__ void __launch_bounds__(hsw::threads<N>()) k_half32(HalfArgs a) {
  using namespace hsw;
  constexpr int SLOT = ROWS * N;  // floats per slot and array
  constexpr int HN = N / 2, QN = N / 4;
  constexpr int NT = threads<N>();
  constexpr int APAIRS = (TY / 2 + 1) * QN;
  extern __shared__ __align__(128) float smem[];
  float* se = smem;                        // split e:    [SPLIT][ROWS][even | odd]
  float* sp = se + SPLIT * SLOT;           // split phi0
  float* re = sp + SPLIT * SLOT;           // raw e:      [RAW][ROWS][N]
  float* rp = re + RAW * SLOT;             // raw phi0
  __shared__ __align__(8) unsigned long long bar[RAW];
  __shared__ float s_mu;

  const int tiles = N / TY;
  const int tile = (int)(blockIdx.x % tiles), run = (int)(blockIdx.x / tiles);
  const int j0 = tile * TY;
  const int z0 = (int)((long long)run * N / a.zch), z1 = (int)((long long)(run + 1) * N / a.zch);
  const int qmax = z1 - z0 + 3;  // local plane q = plane - (z0 - 2), 0 .. qmax
  const int hb = a.hb;
  const int tid = threadIdx.x;

  if (tid == 0) {
    for (int s = 0; s < RAW; ++s) mbar_init(smem_u32(&bar[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_mu = (float)a.sc->lambda;
  }
  __syncthreads();

  // Plane q into raw slot q % RAW: TY+4 rows of e (per row from e_out or e_in in
  // the second half sweep) and of phi0 (one copy, two where the rows wrap in y).
  // Lane 0 of warp 0 arms the barrier, then each lane issues one row.
  auto issue = [&](int q) {
    const int slot = q % RAW;
    const int k = (z0 - 2 + q + N) & (N - 1);
    const unsigned b = smem_u32(&bar[slot]);
    const int lane = tid;  // warp 0 only
    if (lane == 0) mbar_expect(b, (unsigned)(2 * SLOT * sizeof(float)));
    __syncwarp();
    if (lane < ROWS) {
      const int j = (j0 - 2 + lane) & (N - 1);
      const float* src = (hb == 1 && ((j + k) & 1) == 0) ? a.e_out : a.e_in;
      bulk_g2s(smem_u32(re + slot * SLOT + lane * N), src + ((long long)k * N + j) * N,
               N * sizeof(float), b);
    } else if (lane == ROWS) {
      const int jstart = (j0 - 2) & (N - 1);
      const int first = jstart + ROWS <= N ? ROWS : N - jstart;  // rows before the y wrap
      float* dp = rp + slot * SLOT;
      bulk_g2s(smem_u32(dp), a.phi0 + ((long long)k * N + jstart) * N,
               (unsigned)(first * N * sizeof(float)), b);
      if (first < ROWS)
        bulk_g2s(smem_u32(dp + first * N), a.phi0 + (long long)k * N * N,
                 (unsigned)((ROWS - first) * N * sizeof(float)), b);
    }
  };
  int issued = 0;  // valid in warp 0
  // Wait for raw plane q, split its rows by x parity into compute slot q % SPLIT,
  // and send raw plane q + RAW into the freed raw slot.  false: the wait ran out.
  auto advance = [&](int q) -> bool {
    // one warp polls the barrier; the others wait at the block barrier, which
    // costs them no issue slots
    const bool arrived =
        tid >= 32 || mbar_wait(smem_u32(&bar[q % RAW]), (unsigned)((q / RAW) & 1), a.limit_ns);
    if (!__syncthreads_and(arrived)) return false;
    constexpr int V = SLOT / 4;  // float4 per array
    for (int v = tid; v < 2 * V; v += NT) {
      const bool arr = v >= V;
      const int w = arr ? v - V : v;
      const float4 x = reinterpret_cast<const float4*>((arr ? rp : re) + (q % RAW) * SLOT)[w];
      const int row = w / (N / 4), g4 = w - row * (N / 4);
      float* d = (arr ? sp : se) + (q % SPLIT) * SLOT + row * N;
      *reinterpret_cast<float2*>(d + 2 * g4) = make_float2(x.x, x.z);        // even x
      *reinterpret_cast<float2*>(d + HN + 2 * g4) = make_float2(x.y, x.w);   // odd x
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid < 32 && q + RAW <= qmax) {
      issue(q + RAW);
      issued = q + RAW + 1;
    }
    return true;
  };

  if (tid < 32) {
    for (int q = 0; q < RAW && q <= qmax; ++q) issue(q);
    issued = RAW < qmax + 1 ? RAW : qmax + 1;
  }
  bool ok = advance(0) && advance(1);

  // this thread's cell pair: A pairs first (rows of A), then B pairs
  const bool isA = tid < APAIRS;
  const int w = isA ? tid : tid - APAIRS;
  const int prow = w / QN;            // which of the stage's rows of parity hb
  const int m = 2 * (w - prow * QN);  // first cell of the pair in the half row

  for (int qa = 1; ok && qa <= qmax; ++qa) {
    if (qa + 1 <= qmax && !(ok = advance(qa + 1))) break;
    const int t = z0 - 2 + qa;  // plane of A in this step; B works on plane t - 2
    if (isA) {
      if (t <= z1) {
        const int k = (t + N) & (N - 1);
        // rows of parity hb among window rows 1 .. TY+2 (j0-1 .. j0+TY)
        const int r = 1 + ((((j0 - 1) + k) & 1) != hb) + 2 * prow;
        const int j = (j0 - 2 + r) & (N - 1);
        const int par = k & 1;  // (x + k) even: colour 2hb
        const int x = 2 * m + par;
        const long long id = ((long long)k * N + j) * N + x;
        const float2 q0 = make_float2(__ldg(a.q0 + id), __ldg(a.q0 + id + 2));
        const float2 gg = make_float2(__ldg(a.g + id), __ldg(a.g + id + 2));
        const int base = (qa % SPLIT) * SLOT + r * N;
        const int M = ((qa - 1) % SPLIT - qa % SPLIT) * SLOT;
        const int P = ((qa + 1) % SPLIT - qa % SPLIT) * SLOT;
        const float2 v = par ? pair_update<N, 1>(se, sp, base, M, P, m, q0, gg, s_mu, a.c)
                             : pair_update<N, 0>(se, sp, base, M, P, m, q0, gg, s_mu, a.c);
        *reinterpret_cast<float2*>(se + base + par * HN + m) = v;
        if (t >= z0 && t < z1 && r >= 2 && r < TY + 2) {
          a.e_out[id] = v.x;
          a.e_out[id + 2] = v.y;
        }
      }
    } else if (t - 2 >= z0 && t - 2 < z1) {
      const int qb = qa - 2;
      const int k = (t - 2 + N) & (N - 1);
      const int r = 2 + (((j0 + k) & 1) != hb) + 2 * prow;  // window rows 2 .. TY+1
      const int j = (j0 - 2 + r) & (N - 1);
      const int par = (k & 1) ^ 1;  // (x + k) odd: colour 2hb+1
      const int x = 2 * m + par;
      const long long id = ((long long)k * N + j) * N + x;
      const float2 q0 = make_float2(__ldg(a.q0 + id), __ldg(a.q0 + id + 2));
      const float2 gg = make_float2(__ldg(a.g + id), __ldg(a.g + id + 2));
      const int base = (qb % SPLIT) * SLOT + r * N;
      const int M = ((qb - 1) % SPLIT - qb % SPLIT) * SLOT;
      const int P = ((qb + 1) % SPLIT - qb % SPLIT) * SLOT;
      const float2 v = par ? pair_update<N, 1>(se, sp, base, M, P, m, q0, gg, s_mu, a.c)
                           : pair_update<N, 0>(se, sp, base, M, P, m, q0, gg, s_mu, a.c);
      a.e_out[id] = v.x;
      a.e_out[id + 2] = v.y;
    }
    __syncthreads();
  }
  if (!ok && tid == 0) {
    atomicExch(a.err, 1);
    // copies still in flight land in this CTA's shared memory: wait for them
    // (bounded by the larger of the limit and one second) before the CTA exits
    const unsigned long long drain = a.limit_ns > 1000000000ull ? a.limit_ns : 1000000000ull;
    const int start = issued > RAW ? issued - RAW : 0;
    for (int q = start; q < issued; ++q)
      mbar_wait(smem_u32(&bar[q % RAW]), (unsigned)((q / RAW) & 1), drain);
  }
}

template <int N>
static void launch_half_n(cudaStream_t st, const HalfArgs& a) {
  const unsigned grid = (unsigned)((N / hsw::TY) * a.zch);
  k_half32<N><<<grid, hsw::threads<N>(), hsw::smem_bytes<N>(), st>>>(a);
}

bool half_sweep_supported(int n) { return n == 256 || n == 512; }

void init_half32() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_half32<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)hsw::smem_bytes<512>());
  cudaFuncSetAttribute(k_half32<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)hsw::smem_bytes<256>());
  done = true;
}

// One four-colour sweep as two half sweeps: e_in -> e_out.  With a timer, the
// first half sweep is bracketed by an event pair.
void launch_half_sweep32(cudaStream_t st, int n, const float* e_in, float* e_out,
                         const float* phi0, const float* q0, const float* g,
                         const LevelScalars* sc, const OpConst32& c, int* err, double limit_s,
                         EventPairs* timer) {
  HalfArgs a;
  a.e_in = e_in;
  a.e_out = e_out;
  a.phi0 = phi0;
  a.q0 = q0;
  a.g = g;
  a.sc = sc;
  a.c = c;
  a.err = err;
  a.limit_ns = (unsigned long long)(limit_s * 1e9);
  // z runs per column of tiles: (n / TY) * zch CTAs is a multiple of the 152 SMs
  a.zch = 19;
  for (int hb = 0; hb < 2; ++hb) {
    a.hb = hb;
    if (timer && hb == 0) timer->begin(st);
    if (n == 512) launch_half_n<512>(st, a);
    else launch_half_n<256>(st, a);
    if (timer && hb == 0) timer->end(st);
  }
  count_launches(2);
}

}  // namespace mg
