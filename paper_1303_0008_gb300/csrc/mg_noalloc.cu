// mg_op_residual_noalloc: the residual-and-norms entry point for callers that
// cannot allocate device memory.
//
// mg_op_residual allocates three temporaries per call (the per-cell source term,
// the per-block partial norms and the scalar record) with cudaMalloc and frees
// them with cudaFree.  Some callers cannot afford that: cudaMalloc and cudaFree
// synchronise the whole device, which stalls every other stream of a program
// that overlaps work, and a program whose device memory is already handed out
// by its own pool (a framework's caching allocator holding the card) can see
// cudaMalloc fail.  This variant allocates nothing: the partial norms and the
// scalar record live in one file-scope __device__ array of fixed size, and the
// source term is formed inside the kernel instead of in a temporary.
//
// The array is NOT per call: every call on a device uses the same storage and
// leaves its contents behind.  Calls that overlap on the GPU (two streams, or two
// host threads) race on it; the caller must order them.  Each call overwrites
// every entry it reads, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <string>

#include "../../include/mg.h"
#include "mg_internal.h"

namespace mg {

// Largest grid the fixed storage covers: one partial per 256-cell block.
static constexpr long long kNoAllocMaxCells = 256LL * 256 * 256;
static constexpr int kNoAllocThreads = 256;
static constexpr int kNoAllocMaxBlocks = (int)(kNoAllocMaxCells / kNoAllocThreads);

struct NoAllocScratch {
  Partial partials[kNoAllocMaxBlocks];
  LevelScalars scalars;
};

// About 2.6 MB, held by every device that loads the library until the process ends.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// d = L^h phi - f with the source term a*delta + b formed per cell (the same
// fma as the source-preparation kernel, so the values match bit for bit).
__global__ void __launch_bounds__(kNoAllocThreads) k_residual64_noalloc(
    int n, const double* __restrict__ phi, const double* __restrict__ delta, double a, double b,
    const double* __restrict__ f, double* __restrict__ dout, OpConst64 c,
    NoAllocScratch* __restrict__ scratch) {
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
    const double D = root_D(s, fma(a, delta[t], b), c, g);
    const double lap = (s.sx + s.sy + s.sz) - 6.0 * phi[t];
    double d = fma(lap, c.inv_h2, -D);
    if (f) d -= f[t];
    if (dout) dout[t] = d;
    partial_add(p, d, g);
  }
  p = block_reduce(p);
  if (threadIdx.x == 0) scratch->partials[blockIdx.x] = p;
}

// Device address of the scratch array, looked up once per device.  Host threads
// may race to fill an entry; they all store the same address.  The address
// belongs to the device's primary context: after cudaDeviceReset it is stale,
// and this entry point must not be used again in that process.
static constexpr int kMaxDevices = 64;
static std::atomic<NoAllocScratch*> g_scratch_ptr[kMaxDevices] = {};

static mg_status scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("mg_op_residual_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return MG_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("mg_op_residual_noalloc: device index out of range");
    return MG_EINVAL;
  }
  NoAllocScratch* cached = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!cached) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error(std::string("mg_op_residual_noalloc: cudaGetSymbolAddress: ") +
                cudaGetErrorString(e));
      return MG_ECUDA;
    }
    cached = (NoAllocScratch*)ptr;
    g_scratch_ptr[dev].store(cached, std::memory_order_release);
  }
  *out = cached;
  return MG_OK;
}

}  // namespace mg

using namespace mg;

extern "C" mg_status mg_op_residual_noalloc(int n, const double* phi, const double* delta,
                                            const double* f, int branch, double alpha,
                                            double kappa, double* d, double* norms,
                                            void* stream) {
  if (n < 4 || (n & 1)) {
    set_error("mg_op_residual_noalloc: n must be even and at least 4");
    return MG_EINVAL;
  }
  if ((long long)n * n * n > kNoAllocMaxCells) {
    set_error("mg_op_residual_noalloc: n = " + std::to_string(n) +
              " exceeds the maximum of 256 (its fixed scratch covers 256^3 cells)");
    return MG_EINVAL;
  }
  if (branch < -1 || branch > 1 || (alpha == 0.0 && branch != 0) || !std::isfinite(alpha) ||
      !phi || !delta) {
    set_error("mg_op_residual_noalloc: bad branch, non-finite alpha or NULL input");
    return MG_EINVAL;
  }
  NoAllocScratch* scratch = nullptr;
  mg_status st = scratch_for_current_device(&scratch);
  if (st != MG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const long long cells = (long long)n * n * n;
  const OpConst64 c = make_op64(n, alpha, kappa, branch);
  double a, b;
  src_coefficients(c, kappa, &a, &b);
  const unsigned nb = (unsigned)((cells + kNoAllocThreads - 1) / kNoAllocThreads);
  k_residual64_noalloc<<<nb, kNoAllocThreads, 0, s>>>(n, phi, delta, a, b, f, d, c, scratch);
  count_launches(1);
  launch_finalize(s, scratch->partials, (int)nb, (double)cells, 1, &scratch->scalars);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("mg_op_residual_noalloc: launch: ") + cudaGetErrorString(e));
    return MG_ECUDA;
  }
  // like mg_op_residual, the call returns once the kernels have finished, so that
  // an execution error is reported here whether or not the norms are wanted
  LevelScalars h;
  e = cudaMemcpyAsync(&h, &scratch->scalars, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("mg_op_residual_noalloc: ") + cudaGetErrorString(e));
    return MG_ECUDA;
  }
  if (norms) {
    norms[0] = h.sum;
    norms[1] = h.dmax;
    norms[2] = h.dmin;
    norms[3] = (double)h.guards;
    norms[4] = (double)h.nonfinite;
  }
  return MG_OK;
}
