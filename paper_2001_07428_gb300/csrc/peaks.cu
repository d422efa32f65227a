// peaks.cu -- throughput loops that measure the arithmetic peaks the roofline figures divide by:
// FP64 FMA on the CUDA cores, FP64 matrix multiply-accumulate (mma.sync m8n8k4, the FP64 tensor
// path), and FP32 FMA.  Each kernel runs many independent accumulator chains per thread so that the
// pipe, not the dependency latency, limits it; the grid fills every SM.  Results are written only
// under a condition the data never meet, so the compiler keeps the arithmetic.
#include <cstdio>

#include "internal.h"
#include "../../include/jtrlan.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop_kernel(T* out, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == (T)-12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true for a, b below
}

// One warp-wide m8n8k4 FP64 MMA per instruction: D = A B + C with A 8x4, B 4x8, C/D 8x8; each lane
// holds one element of A and of B and two of C/D.  kChains independent accumulators per warp.
__global__ void __launch_bounds__(kThreads) dmma_loop_kernel(double* out, int iters, double a0, double b0) {
  double c[kChains][2];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k][0] = c[k][1] = (double)(threadIdx.x + k);
  const double a = a0 + 1e-9 * threadIdx.x, b = b0 - 1e-9 * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k][0] + c[k][1];
  if (s == -12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

jtrlan_status pk_fail(const char* what, cudaError_t e) {
  char buf[200];
  snprintf(buf, sizeof buf, "jtrlan_measure_peaks: %s: %s", what, cudaGetErrorString(e));
  jtr::set_last_error(buf);
  return JTRLAN_ECUDA;
}

// Best of `reps` timed launches (after one warm-up) of a kernel doing `flop` operations per launch.
template <typename Launch>
cudaError_t best_rate(Launch launch, double flop, int reps, cudaStream_t s, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  launch();
  float best = 1e30f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) *tflops = flop / (best * 1e-3) / 1e12;
  return e;
}

}  // namespace

extern "C" jtrlan_status jtrlan_measure_peaks(double* fp64_fma_tflops, double* fp64_mma_tflops, double* fp32_fma_tflops,
                                              void* cuda_stream) {
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return pk_fail("device query", e);
  const int grid = nsm * 8;                 // 8 blocks of 256 threads per SM
  const double threads = (double)grid * kThreads;
  void* buf = nullptr;
  if ((e = cudaMalloc(&buf, (size_t)grid * kThreads * sizeof(double))) != cudaSuccess)
    return pk_fail("cudaMalloc", e);
  const int it64 = 4096, it32 = 65536, itmma = 2048;
  double r64 = 0, rmma = 0, r32 = 0;
  e = best_rate([&] { fma_loop_kernel<double><<<grid, kThreads, 0, s>>>((double*)buf, it64, 0.999999, 1e-7); },
                2.0 * kChains * it64 * threads, 5, s, &r64);
  if (e == cudaSuccess)
    e = best_rate([&] { dmma_loop_kernel<<<grid, kThreads, 0, s>>>((double*)buf, itmma, 0.5, 0.25); },
                  2.0 * 8 * 8 * 4 * kChains * itmma * (threads / 32), 5, s, &rmma);
  if (e == cudaSuccess)
    e = best_rate([&] { fma_loop_kernel<float><<<grid, kThreads, 0, s>>>((float*)buf, it32, 0.9999f, 1e-7f); },
                  2.0 * kChains * it32 * threads, 5, s, &r32);
  cudaFree(buf);
  if (e != cudaSuccess) return pk_fail("timed loop", e);
  if (fp64_fma_tflops) *fp64_fma_tflops = r64;
  if (fp64_mma_tflops) *fp64_mma_tflops = rmma;
  if (fp32_fma_tflops) *fp32_fma_tflops = r32;
  return JTRLAN_OK;
}
