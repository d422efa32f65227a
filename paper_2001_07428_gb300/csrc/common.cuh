// common.cuh -- small device helpers shared by the libjtrlan kernels (complex arithmetic,
// reductions, the device-side state of one Lanczos step).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jtr {

// ------------------------------------------------------------------ complex numbers
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R re, R im) {
  cplx<R> z; z.x = re; z.y = im; return z;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }
// acc + a*b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}
// acc + conj(a)*b
template <typename C> __device__ __forceinline__ C cfmac(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
  return acc;
}
template <typename C> __device__ __forceinline__ double cabs2(C a) {
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}
// |a|^2 in the working precision (FP32 partial sums stay on the FP32 pipe)
template <typename C> __device__ __forceinline__ auto cabs2w(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a block of blockDim.x threads (multiple of 32, <= 1024); result valid in all threads.
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 doubles */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// 32-byte record of one Gram-Schmidt coefficient pair: c_v = v_i^H y and c_w = w_i^H y.
struct alignas(32) coef4 { double vr, vi, wr, wi; };

// Device-side state of the Lanczos step in flight (one per context).
struct StepState {
  double nrm[8];      // norms after the alpha subtraction (0) and after each GS pass (1..)
  double beta;        // accepted t_{j+1,j}
  double tmax;        // running max |t| of the current T-bar (breakdown scale)
  double alpha_im;    // Im(v_j^H A v_j), a diagnostic (reading: alpha is real)
  int done;           // the reorthogonalisation loop has exited for this step
  int status;         // 0 ok, 5 breakdown
  long long n_passes; // GS passes run (statistics)
  double units_first;  // sum over steps of (j+1) * n/2: row pair x column products of the first dot
  double units_dot;    // the same for the dot of every executed later pass
  double units_update; // the same for every executed update pass
  long long n_ritz_fallbacks;  // restarts whose Ritz fast path failed its checks (Jacobi used)
};

// Counter-based pseudo-random numbers (splitmix64, Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__host__ __device__ __forceinline__ double u01_sym(uint64_t x) {  // uniform in [-1, 1)
  return (double)(splitmix64(x) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

}  // namespace jtr
