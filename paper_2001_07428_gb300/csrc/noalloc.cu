// noalloc.cu -- residual norms without any device allocation.
//
// Some callers cannot call cudaMalloc: an application whose caching allocator already owns the
// device memory it may use, code that must not trigger cudaMalloc's implicit device-wide
// synchronisation while other streams are running, or a plug-in that is given no allocation
// rights.  jtrlan_residual_norms_noalloc serves them: it runs the same residual kernel as the
// solver's convergence check, with its scratch (per-block partial sums, column indices,
// eigenvalues, results) in one file-scope device array instead of context-owned buffers.
//
// The array is a module global: every GPU that loads the library holds it until the process
// exits, and all calls on a device share it.  Its device address is looked up once per device
// (cudaGetSymbolAddress with that device current) on the first call there and cached; a
// cudaDeviceReset (or any other reset of the primary context) leaves that cached address stale, so
// the entry point must not be used on a device after such a reset in the same process.
#include <cstdio>
#include <mutex>

#include "internal.h"
#include "../../include/jtrlan.h"

namespace {

constexpr int64_t kPartials = JTRLAN_NOALLOC_MAX_PARTIALS;  // doubles of per-block partials
constexpr int kCols = JTRLAN_NOALLOC_MAX_COLS;
constexpr int kMaxDevices = 64;

// Layout: [kPartials doubles: partials][kCols doubles: lambda][kCols doubles: norms][kCols ints: cols]
struct NoAllocScratch {
  double partials[kPartials];
  double lambda[kCols];
  double norms[kCols];
  int cols[kCols];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_addr[kMaxDevices] = {};

jtrlan_status noalloc_fail(jtrlan_status s, const char* what, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess)
    snprintf(buf, sizeof buf, "jtrlan_residual_norms_noalloc: %s: %s", what, cudaGetErrorString(e));
  else
    snprintf(buf, sizeof buf, "jtrlan_residual_norms_noalloc: %s", what);
  jtr::set_last_error(buf);
  return s;
}

__global__ void iota_kernel(int* cols, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) cols[i] = i;
}

// The device address of g_noalloc_scratch on the current device (looked up once per device).
jtrlan_status scratch_on_current_device(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(JTRLAN_ECUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(JTRLAN_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return noalloc_fail(JTRLAN_ECUDA, "cudaGetSymbolAddress", e);
    g_scratch_addr[dev] = (NoAllocScratch*)p;
  }
  *out = g_scratch_addr[dev];
  return JTRLAN_OK;
}

}  // namespace

extern "C" jtrlan_status jtrlan_residual_norms_noalloc(const jtrlan_operator* op, const void* X, int64_t ldx,
                                                       int ncols, const double* lambda, double* res,
                                                       void* cuda_stream) {
  using namespace jtr;
  if (!op || !X || !lambda || !res) return noalloc_fail(JTRLAN_EINVAL, "null argument");
  if (ncols <= 0) return noalloc_fail(JTRLAN_EINVAL, "ncols must be positive");
  if (op->dtype != JTRLAN_C128) return noalloc_fail(JTRLAN_EINVAL, "operator must be complex128 (no conversion buffer)");
  if (op->n <= 0 || (op->n & 1) || ldx < op->n) return noalloc_fail(JTRLAN_EINVAL, "need even n > 0 and ldx >= n");
  OpDev o{};
  o.kind = op->kind;
  o.n = op->n;
  o.h = op->n / 2;
  o.m0 = op->m0;
  o.kappa = op->kappa;
  o.vol = 1;
  if (op->kind == JTRLAN_STENCIL4D) {
    for (int d = 0; d < 4; ++d) {
      if (op->dims[d] < 1) return noalloc_fail(JTRLAN_EINVAL, "lattice extents must be >= 1");
      o.dims[d] = op->dims[d];
      o.vol *= op->dims[d];
    }
    if (op->n != 6 * o.vol) return noalloc_fail(JTRLAN_EINVAL, "stencil n must equal 6 * volume");
    if (!op->U || !op->W) return noalloc_fail(JTRLAN_EINVAL, "null link field");
    o.U = op->U;
    o.W = op->W;
  } else if (op->kind == JTRLAN_DENSE) {
    if (!op->a11 || !op->a12) return noalloc_fail(JTRLAN_EINVAL, "null dense block");
    o.a11 = op->a11;
    o.a12 = op->a12;
  } else {
    return noalloc_fail(JTRLAN_EINVAL, "unknown operator kind");
  }
  const int nblk = matvec_blocks(o);
  if (ncols > kCols) return noalloc_fail(JTRLAN_EINVAL, "ncols exceeds JTRLAN_NOALLOC_MAX_COLS");
  if ((int64_t)ncols * nblk > kPartials)
    return noalloc_fail(JTRLAN_EINVAL,
                        "ncols * blocks per product exceeds JTRLAN_NOALLOC_MAX_PARTIALS; pass fewer columns per call");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the call copies from pageable host memory and synchronises the stream, neither of which a
  // capturing stream allows: refuse before anything is enqueued
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return noalloc_fail(JTRLAN_ECUDA, "cudaStreamIsCapturing", e);
  if (cap != cudaStreamCaptureStatusNone)
    return noalloc_fail(JTRLAN_EINVAL, "the stream is being captured; this call cannot be captured");
  NoAllocScratch* sc = nullptr;
  jtrlan_status st = scratch_on_current_device(&sc);
  if (st != JTRLAN_OK) return st;
  // once work is enqueued, an error return first waits for that work (ignoring its status), so that
  // no kernel of this call still uses the shared array when the caller retries
  auto fail_after_enqueue = [&](const char* what, cudaError_t err) {
    cudaStreamSynchronize(s);
    return noalloc_fail(JTRLAN_ECUDA, what, err);
  };
  iota_kernel<<<1, 256, 0, s>>>(sc->cols, ncols);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(JTRLAN_ECUDA, "iota launch", e);
  e = cudaMemcpyAsync(sc->lambda, lambda, ncols * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail_after_enqueue("copy of lambda", e);
  e = launch_matvec<double>(o, (const double2*)X, nullptr, MV_RESID, sc->partials, sc->cols, sc->lambda, ncols, ldx,
                            nullptr, s);
  if (e != cudaSuccess) return fail_after_enqueue("residual kernel", e);
  e = launch_reduce_norms(sc->partials, nblk, ncols, sc->norms, s);
  if (e != cudaSuccess) return fail_after_enqueue("reduction kernel", e);
  e = cudaMemcpyAsync(res, sc->norms, ncols * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail_after_enqueue("copy of the norms", e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(JTRLAN_ECUDA, "stream synchronisation", e);
  return JTRLAN_OK;
}
