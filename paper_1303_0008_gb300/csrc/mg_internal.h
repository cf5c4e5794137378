// Host-side declarations shared by the translation units of libmg.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "mg_common.cuh"

namespace mg {

void set_error(const std::string& msg);

// Status returns of the C-ABI entry points.
#define MG_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
      return MG_ECUDA;                                                                \
    }                                                                                 \
  } while (0)

#define MG_FAIL(code, msg)  \
  do {                      \
    set_error(msg);         \
    return code;            \
  } while (0)

// Launch `k` on `st` with programmatic stream serialisation allowed: the kernel
// may be scheduled while its predecessor in the stream finishes.  Every kernel
// launched this way opens a PdlScope before touching memory.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                            cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(block, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Kernel launches issued by this thread (graph captures included).
extern thread_local long long tl_launches;
inline void count_launches(long long k) { tl_launches += k; }

// CUDA event pairs around individual kernel launches on one stream; while the
// stream is being captured the records become external event nodes of the graph.
struct EventPairs {
  std::vector<cudaEvent_t> start, stop;
  int n = 0;
  bool capturing = false;
  bool enabled = false;
  bool first_only = false;  // time only the first colour stage of each smoothing call
  ~EventPairs() {
    for (auto e : start) cudaEventDestroy(e);
    for (auto e : stop) cudaEventDestroy(e);
  }
  void begin(cudaStream_t st) {
    if (!enabled) return;
    if ((int)start.size() <= n) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      start.push_back(a);
      stop.push_back(b);
    }
    if (capturing) cudaEventRecordWithFlags(start[n], st, cudaEventRecordExternal);
    else cudaEventRecord(start[n], st);
  }
  void end(cudaStream_t st) {
    if (!enabled) return;
    if (capturing) cudaEventRecordWithFlags(stop[n], st, cudaEventRecordExternal);
    else cudaEventRecord(stop[n], st);
    ++n;
  }
  // Summed milliseconds of the recorded pairs (their work must have completed).
  double read_ms() const {
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, start[i], stop[i]) == cudaSuccess) total += ms;
    }
    return total;
  }
};

// Capture `body` as a graph; *launches receives the kernels it holds (they are
// not counted as issued until the graph is launched).
template <typename F>
inline cudaGraphExec_t capture_graph(cudaStream_t st, long long* launches, const F& body) {
  cudaGraph_t graph = nullptr;
  const long long before = tl_launches;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  body();
  *launches = tl_launches - before;
  tl_launches = before;
  if (cudaStreamEndCapture(st, &graph) != cudaSuccess || !graph) {
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    exec = nullptr;
  }
  cudaGraphDestroy(graph);
  return exec;
}

// ---- FP64 periodic kernels (mg_fp64.cu) ----
OpConst64 make_op64(int n, double alpha, double kappa, int branch, double w = 1.0 / 3.0);
void src_coefficients(const OpConst64& c, double kappa, double* a, double* b);
int partials_needed(long long cells);
void launch_smooth64(cudaStream_t st, int n, double* phi, const double* src, const double* f,
                     const LevelScalars* sc, const OpConst64& c, int sweeps,
                     EventPairs* timer = nullptr);
void launch_finalize(cudaStream_t st, const Partial* partials, int nparts, double cells,
                     int periodic, LevelScalars* sc);
void launch_residual64(cudaStream_t st, int n, const double* phi, const double* src,
                       const double* f, double* dout, const OpConst64& c, Partial* partials,
                       LevelScalars* sc, int periodic);
// With def/guard (kTwoStepMaxFine entries) and nf^3 <= kTwoStepMaxFine, the
// restriction runs as a per-fine-cell defect launch plus the coarse walk, so that
// the FP64 work of a small level spreads over the GPU (same bits as the fused form).
void launch_residual_restrict64(cudaStream_t st, int nf, const double* phi, const double* src,
                                const double* f, const OpConst64& c, double* phi_c,
                                double* phihat_c, double* rd_c, Partial* partials,
                                LevelScalars* sc, double* def = nullptr,
                                unsigned char* guard = nullptr);
// Threads per block of a per-cell FP64 launch over `items` cells (256, or 64 on
// small levels).
int tpb_for(long long items);
void launch_fas_rhs64(cudaStream_t st, int nc, const double* phi_c, const double* src_c,
                      double* f_c, const OpConst64& c, const LevelScalars* fine_sc,
                      LevelScalars* coarse_sc);
// clobber_hat: phihat_c may be overwritten (with phi_c - phihat_c); from
// kCorrectionMinFine fine cells on, the correction is then formed once per coarse
// cell before the prolongation (same bits).
constexpr long long kCorrectionMinFine = 128LL * 128 * 128;
void launch_prolong_correct64(cudaStream_t st, int nc, const double* phi_c,
                              const double* phihat_c, double* phi_f, bool clobber_hat = false);
void launch_coarsest64(cudaStream_t st, int n, double* phi, const double* src, const double* f,
                       const OpConst64& c, LevelScalars* sc, int max_sweeps, double drop);
void launch_restrict64(cudaStream_t st, int nc, const double* fine, double* coarse);
void launch_affine64(cudaStream_t st, long long cells, const double* x, double* out, double a,
                     double b, double c3 = 0.0, int floor = 0,
                     unsigned long long* floored = nullptr);
void launch_gauge64(cudaStream_t st, long long cells, double* x, Partial* partials,
                    LevelScalars* sc);
void launch_force64(cudaStream_t st, int n, const double* phi, double* out);
void launch_spread64(cudaStream_t st, long long cells, const double* x, Partial* partials,
                     LevelScalars* sc);
void launch_axpy64(cudaStream_t st, long long cells, const double* x, const double* y, double a,
                   double* out);

}  // namespace mg

namespace mg {

// Levels at or below this side run their whole sub-V-cycle in one launch of a
// single thread-block cluster (see mg_subcycle.cu).
// levels with more cells per side run faster as per-level launches (entering the
// sub-cycle at 32 slowed the six-solve 128^3 step by 3.5 % (FP64) and left the
// mixed step unchanged)
constexpr int kSubcycleMaxN = 16;
// Fine levels up to this many cells restrict their residual in two launches
// (32^3: the fused launch would put 16 blocks on 16 SMs).  The scratch of the
// sub-cycle's residual step (kSubcycleMaxN^3 cells) shares the same buffer.
constexpr long long kTwoStepMaxFine = 32768;
constexpr int kSubcycleMaxLevels = 8;

struct SubLevel64 {
  int n;
  double *phi, *src, *f, *phihat;
  LevelScalars* sc;
  OpConst64 op;
};

struct SubLevel32 {
  int n;
  float *e, *ehat, *phi0, *q0, *rhs;
  LevelScalars* sc32;
  OpConst32 op32;
};

struct SubCycleArgs {
  int nlev;  // levels handled, the entry level first
  SubLevel64 lv[kSubcycleMaxLevels];
  SubLevel32 lv32[kSubcycleMaxLevels];
  Partial* part;
  double* def64;          // kSubcycleMaxN^3 fine-cell defects (FP64 cycle)
  float* def32;           // the same for the FP32 cycle
  unsigned char* guard;   // kSubcycleMaxN^3 guard flags (FP64 cycle)
  int nu_pre, nu_post, coarse_sweeps;
  double coarse_drop;
};

// Enqueue the FP64 (or FP32-correction) sub-V-cycle described by `a` on `st`.
void launch_subcycle64(cudaStream_t st, const SubCycleArgs& a);
void launch_subcycle32(cudaStream_t st, const SubCycleArgs& a);
void init_subcycle();

// Two-launch four-colour sweep of the FP32 correction operator (mg_halfsweep32.cu):
// colours 0 and 1, then 2 and 3, each launch streaming planes of whole rows
// through shared memory with bulk asynchronous copies; e_in -> e_out, n = 256 or
// 512.  *err is set when a copy does not arrive within limit_s seconds.
bool half_sweep_supported(int n);
void init_half32();
void launch_half_sweep32(cudaStream_t st, int n, const float* e_in, float* e_out,
                         const float* phi0, const float* q0, const float* g,
                         const LevelScalars* sc, const OpConst32& c, int* err, double limit_s,
                         EventPairs* timer = nullptr);

// Staggered slab order of one four-colour sweep (option slab32, mg_mixed.cu).
// The n planes are cut into n / S slabs of S planes; slab s of colour c covers
// planes [a, b) (mod n) with
//   a = c (s = 0), S s - c (s > 0);   b = S (s + 1) - c (s < n/S - 1), n + c (last).
// The launches run slab by slab and, within a slab, colour by colour.  A cell of
// colour c reads only cells of the other colours, on its own plane and the two
// beside it.  When slab s of colour c runs, colour c - 1 has updated every plane up
// to b (its own slab s ends one plane later) and down to a - 1, and colour c + 1 has
// updated nothing that colour c still reads (its slabs end one plane earlier);
// colour c's first c planes wait for the last slab, after colour c - 1 has wrapped
// around.  So every cell sees the values of the whole-stage order, and the planes a
// launch reads were read or written by the launch before it.
inline bool slab_sweep_applies(int n, int S) {
  return S >= 8 && n >= 256 && (n & (n - 1)) == 0 && n % S == 0 && n / S >= 2;
}
inline void slab_range(int n, int S, int colour, int s, int* z0, int* nz) {
  const int ns = n / S;
  const int a = s == 0 ? colour : S * s - colour;
  const int b = s == ns - 1 ? n + colour : S * (s + 1) - colour;
  *z0 = a;
  *nz = b - a;
}

// One-launch four-colour sweep of the FP32 correction operator (mg_sweep32.cu):
// reads e_in, writes every cell of e_out; n >= 32 and n % 4 == 0.
bool sweep32_eligible(int n);
void init_sweep32();
void launch_sweep32(cudaStream_t st, int n, const float* e_in, float* e_out, const float* phi0,
                    const float* q0, const float* g, const LevelScalars* sc, const OpConst32& c);

}  // namespace mg
