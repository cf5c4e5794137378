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
//     and B on plane t-1, so B finds every A value it needs already updated;
//   - B on rows j0 .. j0+TY-1 needs A on rows j0-1 and j0+TY too, which belong to
//     the neighbouring CTAs: the CTA recomputes A on those halo rows itself (and
//     on plane z0-1 below its run) from values that are not updated in this
//     launch, and writes back only its own rows and planes;
//   - planes of e and phi0, TY+4 rows each, stream into a ring of five shared
//     memory slots with bulk asynchronous copies (cp.async.bulk, completing on an
//     mbarrier), one plane ahead of the compute.
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
constexpr int SLOTS = 5;     // planes t-2 .. t+1 in use, plane t+2 arriving
constexpr int THREADS = 512;
template <int N>
struct Tile;
template <>
struct Tile<512> {
  static constexpr int TY = 4;
};
template <>
struct Tile<256> {
  static constexpr int TY = 4;
};
template <int N>
constexpr size_t smem_bytes() {
  return (size_t)2 * SLOTS * (Tile<N>::TY + 4) * N * sizeof(float);
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

// Face sums and cross differences of the cell at x of window row r of plane
// slots C (centre), M (z-1), P (z+1); the sums of gather_at in the same order.
template <int N>
__device__ __forceinline__ StencilT<float> gather_win(const float* C, const float* M,
                                                     const float* P, int x) {
  const int xp = (x + 1) & (N - 1), xm = (x - 1) & (N - 1);
  StencilT<float> s;
  s.sx = C[xp] + C[xm];
  s.sy = C[N + x] + C[-N + x];
  s.sz = P[x] + M[x];
  s.cxy = (C[N + xp] + C[-N + xm]) - (C[-N + xp] + C[N + xm]);
  s.cxz = (P[xp] + M[xm]) - (M[xp] + P[xm]);
  s.cyz = (P[N + x] + M[-N + x]) - (M[N + x] + P[-N + x]);
  return s;
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(hsw::THREADS, 1) k_half32(HalfArgs a) {
  using namespace hsw;
  constexpr int TY = Tile<N>::TY;
  constexpr int ROWS = TY + 4;
  constexpr int SLOT = ROWS * N;  // floats per slot and array
  constexpr int HN = N / 2;
  extern __shared__ __align__(128) float smem[];
  float* se = smem;               // e:    [SLOTS][ROWS][N]
  float* sp = smem + SLOTS * SLOT;  // phi0: [SLOTS][ROWS][N]
  __shared__ __align__(8) unsigned long long bar[SLOTS];
  __shared__ float s_mu;

  const int tiles = N / TY;
  const int tile = (int)(blockIdx.x % tiles), run = (int)(blockIdx.x / tiles);
  const int j0 = tile * TY;
  const int z0 = (int)((long long)run * N / a.zch), z1 = (int)((long long)(run + 1) * N / a.zch);
  const int qmax = z1 - z0 + 3;  // local plane q = plane - (z0 - 2), 0 .. qmax
  const int hb = a.hb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) mbar_init(smem_u32(&bar[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_mu = (float)a.sc->lambda;
  }
  __syncthreads();

  // Plane q into its slot: TY+4 rows of e (per row from e_out or e_in in the
  // second half sweep) and of phi0 (one or two copies: the rows wrap in y).
  auto issue = [&](int q) {
    const int slot = q % SLOTS;
    const int k = (z0 - 2 + q + N) & (N - 1);
    const unsigned b = smem_u32(&bar[slot]);
    mbar_expect(b, (unsigned)(2 * SLOT * sizeof(float)));
    float* de = se + slot * SLOT;
    float* dp = sp + slot * SLOT;
    for (int r = 0; r < ROWS; ++r) {
      const int j = (j0 - 2 + r) & (N - 1);
      const long long off = ((long long)k * N + j) * N;
      const float* src = (hb == 1 && ((j + k) & 1) == 0) ? a.e_out : a.e_in;
      bulk_g2s(smem_u32(de + r * N), src + off, N * sizeof(float), b);
    }
    const int jstart = (j0 - 2) & (N - 1);
    const int first = jstart + ROWS <= N ? ROWS : N - jstart;  // rows before the y wrap
    bulk_g2s(smem_u32(dp), a.phi0 + ((long long)k * N + jstart) * N,
             (unsigned)(first * N * sizeof(float)), b);
    if (first < ROWS)
      bulk_g2s(smem_u32(dp + first * N), a.phi0 + (long long)k * N * N,
               (unsigned)((ROWS - first) * N * sizeof(float)), b);
  };
  auto wait_plane = [&](int q) -> bool {
    return mbar_wait(smem_u32(&bar[q % SLOTS]), (unsigned)((q / SLOTS) & 1), a.limit_ns);
  };

  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) issue(q);
  int issued = 3;
  // every decision to stop is taken by the whole CTA (the vote is a barrier too)
  bool ok = __syncthreads_and(wait_plane(0) && wait_plane(1));

  for (int q = 1; ok && q < qmax; ++q) {
    const int t = z0 - 2 + q;  // plane of A in this step
    if (threadIdx.x == 0 && q + 2 <= qmax) {
      // the slot of plane q+2 held plane q-3, which nobody reads any more (the
      // threads' writes to it were ordered before the copy engine's by the fence
      // and barrier that ended the previous step)
      issue(q + 2);
      issued = q + 3;
    }
    ok = __syncthreads_and(wait_plane(q + 1));
    if (!ok) break;
    // ---- A on plane t: window rows 1 .. TY+2 (j0-1 .. j0+TY) of parity hb ----
    {
      const int kA = (t + N) & (N - 1);
      float* C = se + (q % SLOTS) * SLOT;
      const float* M = se + ((q - 1) % SLOTS) * SLOT;
      const float* P = se + ((q + 1) % SLOTS) * SLOT;
      const float* Cp = sp + (q % SLOTS) * SLOT;
      const float* Mp = sp + ((q - 1) % SLOTS) * SLOT;
      const float* Pp = sp + ((q + 1) % SLOTS) * SLOT;
      // rows of parity hb among 1 .. TY+2: the first is 1 or 2
      const int rfirst = 1 + ((((j0 - 1) + kA) & 1) != hb);
      constexpr int NRA = TY / 2 + 1;
      const bool own_plane = t >= z0 && t < z1;
      for (int w = threadIdx.x; w < NRA * HN; w += THREADS) {
        const int r = rfirst + 2 * (w / HN);
        const int x = 2 * (w % HN) + (kA & 1);  // (x + k) even: colour 2hb
        const int o = r * N;
        const StencilT<float> s = gather_win<N>(C + o, M + o, P + o, x);
        const int j = (j0 - 2 + r) & (N - 1);
        const long long id = ((long long)kA * N + j) * N + x;
        float dd = 0.f;
        if (!a.c.linear)
          dd = dD32(s, gather_win<N>(Cp + o, Mp + o, Pp + o, x), a.q0[id], a.c);
        const float v = gs_value32(s, dd, a.g[id], s_mu, a.c);
        C[o + x] = v;
        if (own_plane && r >= 2 && r < TY + 2) a.e_out[id] = v;
      }
    }
    __syncthreads();
    // ---- B on plane t-1: window rows 2 .. TY+1 (j0 .. j0+TY-1) of parity hb ----
    if (t - 1 >= z0 && t - 1 < z1) {
      const int kB = (t - 1 + N) & (N - 1);
      const float* C = se + ((q - 1) % SLOTS) * SLOT;
      const float* M = se + ((q - 2) % SLOTS) * SLOT;
      const float* P = se + (q % SLOTS) * SLOT;
      const float* Cp = sp + ((q - 1) % SLOTS) * SLOT;
      const float* Mp = sp + ((q - 2) % SLOTS) * SLOT;
      const float* Pp = sp + (q % SLOTS) * SLOT;
      const int rfirst = 2 + (((j0 + kB) & 1) != hb);
      constexpr int NRB = TY / 2;
      for (int w = threadIdx.x; w < NRB * HN; w += THREADS) {
        const int r = rfirst + 2 * (w / HN);
        const int x = 2 * (w % HN) + ((kB & 1) ^ 1);  // (x + k) odd: colour 2hb+1
        const int o = r * N;
        const StencilT<float> s = gather_win<N>(C + o, M + o, P + o, x);
        const int j = (j0 - 2 + r) & (N - 1);
        const long long id = ((long long)kB * N + j) * N + x;
        float dd = 0.f;
        if (!a.c.linear)
          dd = dD32(s, gather_win<N>(Cp + o, Mp + o, Pp + o, x), a.q0[id], a.c);
        a.e_out[id] = gs_value32(s, dd, a.g[id], s_mu, a.c);
      }
    }
    // shared-memory writes of this step before the copies the next step issues
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(a.err, 1);
    // copies still in flight land in this CTA's shared memory: wait for them
    // (bounded by the larger of the limit and one second) before the CTA exits
    const unsigned long long drain = a.limit_ns > 1000000000ull ? a.limit_ns : 1000000000ull;
    const int start = issued > SLOTS ? issued - SLOTS : 0;
    for (int q = start; q < issued; ++q)
      mbar_wait(smem_u32(&bar[q % SLOTS]), (unsigned)((q / SLOTS) & 1), drain);
  }
}

template <int N>
static void launch_half_n(cudaStream_t st, const HalfArgs& a) {
  const unsigned grid = (unsigned)((N / hsw::Tile<N>::TY) * a.zch);
  k_half32<N><<<grid, hsw::THREADS, hsw::smem_bytes<N>(), st>>>(a);
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
