// Allocation-free batched banded solve: pent_gbsv_batch_noalloc.
//
// Some callers cannot call cudaMalloc at all: code running inside a framework
// whose caching allocator owns the device, plug-ins that are handed buffers but
// no allocator, or a stream that is about to be captured into a CUDA graph
// (allocation would break or serialise the capture).  For them this entry point
// factors and solves a batch of equal-length systems in one kernel, using only
// the caller's inputs and outputs plus a fixed scratch area that the library
// itself owns: a file-scope __device__ array, created when a device loads the
// library and held until the process exits.
//
// The kernel is the one-thread-per-system FP64 solve with the factorisation
// folded into its forward sweep (the pivots and the forward substitution both
// walk the rows upwards), so the only scratch is, per row, gamma, delta and g
// for the back substitution.  Nothing in the scratch has to start at zero: each
// thread writes its own rows on the way up before it reads them on the way down.
// All calls share the one array, so calls whose kernels overlap on the GPU
// (different streams without ordering) race on it.
#include <cstdint>
#include <mutex>

#include "../../include/pentbatch.h"
#include "internal.cuh"

namespace pent {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
struct ScratchAddr {
  void* ctx = nullptr;  // the context the address belongs to
  void* ptr = nullptr;
};
ScratchAddr g_noalloc_addr[kMaxDevices];

// The current context (driver entry point through the runtime: the library links no
// driver library), or nullptr if the query is unavailable.
void* current_context() {
  using GetCtx = int (*)(void**);
  static const GetCtx get = []() -> GetCtx {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<GetCtx>(fn);
  }();
  void* ctx = nullptr;
  if (!get || get(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of the scratch array in the current context.  In host code
// g_noalloc_scratch names a host-side shadow, not device memory, so the address
// comes from cudaGetSymbolAddress.  It is looked up again on every call whose
// stream is not being captured (a context that was torn down and created again
// loads the module afresh, possibly elsewhere); during a capture the address
// found by an earlier call in the same context is used, and a capture with no
// such call fails with an error instead of using a stale address.
cudaError_t noalloc_scratch(cudaStream_t st, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  void* ctx = current_context();
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  ScratchAddr& c = g_noalloc_addr[dev];
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    c.ctx = ctx;
    c.ptr = p;
  } else if (!c.ptr || !ctx || c.ctx != ctx) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = c.ptr;
  return cudaSuccess;
}

// One thread per system; warp k owns systems 32k..32k+31 and their record rows
// k*n .. k*n+n-1, each record row holding (gamma, delta, g) for the 32 lanes.
// Factorisation: Sec. 2.4, factorisation steps 1-14 (generic row step with
// out-of-range quantities zero); substitutions: Sec. 2.4, the steps for g and x.
__global__ void __launch_bounds__(128) k_gbsv64_noalloc(int64_t batch, int64_t n, const double* __restrict__ a,
                                                        const double* __restrict__ b, const double* __restrict__ c,
                                                        const double* __restrict__ d, const double* __restrict__ e,
                                                        const double* f, double* x, double* __restrict__ rec,
                                                        unsigned long long* info) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= batch) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t k = q / kWarp;
  const int64_t o = q * n;
  auto at = [&](int64_t r, int p) -> double& { return rec[((k * n + r) * 3 + p) * kWarp + lane]; };
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;  // gamma, delta of rows r-2, r-1
  double g2 = 0.0, g1 = 0.0;                              // g of rows r-2, r-1
  bool failed = false;
  for (int64_t r = 0; r < n; ++r) {
    const double ar = (r >= 2) ? a[o + r] : 0.0;
    const double br = (r >= 1) ? b[o + r] : 0.0;
    const double cr = c[o + r];
    const double dr = (r + 1 < n) ? d[o + r] : 0.0;
    const double er = (r + 2 < n) ? e[o + r] : 0.0;
    double gamma = 0.0, delta = 0.0, g = 0.0;
    if (!failed) {
      const double beta = br - ar * gam2;
      const double alpha = cr - ar * del2 - beta * gam1;
      if (!(alpha != 0.0) || !isfinite(alpha)) {
        if (info) atomicMin(info, ((unsigned long long)q << 32) | (unsigned long long)(uint32_t)r);
        failed = true;
      } else {
        gamma = (dr - beta * del1) / alpha;
        delta = er / alpha;
        g = (f[o + r] - ar * g2 - beta * g1) / alpha;
      }
    }
    at(r, 0) = gamma;
    at(r, 1) = delta;
    at(r, 2) = g;
    gam2 = gam1;
    del2 = del1;
    gam1 = gamma;
    del1 = delta;
    g2 = g1;
    g1 = g;
  }
  double x1 = 0.0, x2 = 0.0;
  for (int64_t r = n - 1; r >= 0; --r) {
    const double xv = at(r, 2) - at(r, 0) * x1 - at(r, 1) * x2;
    x[o + r] = xv;
    x2 = x1;
    x1 = xv;
  }
}

}  // namespace
}  // namespace pent

using namespace pent;

extern "C" pent_status pent_gbsv_batch_noalloc(int64_t batch, int64_t n, const double* a, const double* b,
                                               const double* c, const double* d, const double* e, const double* f,
                                               double* x, unsigned long long* d_info, void* cuda_stream) {
  if (batch < 1 || n < 1 || !a || !b || !c || !d || !e || !f || !x) return PENT_EINVAL;
  const uintptr_t all = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d | (uintptr_t)e | (uintptr_t)f |
                        (uintptr_t)x | (uintptr_t)d_info;
  if (all % sizeof(double)) return PENT_EINVAL;
  // records: ceil(batch/32) warps x n rows x 3 doubles x 32 lanes
  const int64_t groups = (batch + kWarp - 1) / kWarp;
  if (n > (int64_t)(kNoAllocScratchBytes / (3 * kWarp * sizeof(double))) ||
      groups > (int64_t)(kNoAllocScratchBytes / (3 * kWarp * sizeof(double))) / n)
    return PENT_EINVAL;  // beyond the fixed scratch: ceil(batch/32) * 32 * n * 24 bytes must fit in 32 MiB
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* scratch = nullptr;
  if (noalloc_scratch(st, &scratch) != cudaSuccess) return PENT_ECUDA;
  if (d_info && cudaMemsetAsync(d_info, 0x7f, sizeof(unsigned long long), st) != cudaSuccess) return PENT_ECUDA;
  const int block = 128;
  const int64_t grid = (batch + block - 1) / block;
  k_gbsv64_noalloc<<<(unsigned)grid, block, 0, st>>>(batch, n, a, b, c, d, e, f, x, static_cast<double*>(scratch),
                                                     d_info);
  return cudaGetLastError() == cudaSuccess ? PENT_OK : PENT_ECUDA;
}
