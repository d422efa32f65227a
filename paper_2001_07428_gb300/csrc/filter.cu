// filter.cu -- the polynomial filter B = p(A) = sum_k g_k T_k((A - c I)/e) with real coefficients
// (Chebyshev three-term recurrence), and the Jackson-damped step coefficients used as its targets.
//
// B is Hermitian J-symmetric whenever A is (real coefficients: J p(A) J^{-1} = p(A^T) = p(A)^T,
// eq. (1)), so Algorithm 1 runs on it unchanged; its eigenvectors are those of A.
#include <math.h>

#include "internal.h"

namespace jtr {

namespace {

constexpr int kChebThreads = 256;

// One recurrence step over n complex entries:
//   t_next = sc (ax - c t_cur) - sp t_prev          (T_1: sc = 1/e, sp = 0; T_k: sc = 2/e, sp = 1)
//   acc    = g0 v + g t_next   (init)   or   acc += g t_next
// t_next may alias t_prev (each entry is read before it is written by the same thread).  With part
// set, each block also leaves the FP64 partial sum of conj(v) acc (the alpha of Algorithm 2).
template <typename R>
__global__ void __launch_bounds__(kChebThreads)
cheb_step_kernel(const cplx<R>* __restrict__ ax, const cplx<R>* __restrict__ t_cur, const cplx<R>* t_prev,
                 cplx<R>* t_next, cplx<R>* __restrict__ acc, const cplx<R>* __restrict__ v, int64_t n, R c, R sc,
                 R sp, R g, R g0, int init, double* __restrict__ part, float4* __restrict__ split_next) {
  double ar = 0.0, ai = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kChebThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kChebThreads) {
    const cplx<R> a = ax[i], t = t_cur[i];
    cplx<R> nx;
    nx.x = sc * (a.x - c * t.x);
    nx.y = sc * (a.y - c * t.y);
    if (sp != R(0)) {
      const cplx<R> p = t_prev[i];
      nx.x -= sp * p.x;
      nx.y -= sp * p.y;
    }
    t_next[i] = nx;
    if (split_next) {   // (hi, lo) copy of t_next for a compensated-FP32 product
      const float hx = (float)nx.x, hy = (float)nx.y;
      split_next[i] = make_float4(hx, hy, (float)((double)nx.x - (double)hx), (float)((double)nx.y - (double)hy));
    }
    cplx<R> s;
    if (init) {
      const cplx<R> vv = v[i];
      s.x = g0 * vv.x + g * nx.x;
      s.y = g0 * vv.y + g * nx.y;
    } else {
      s = acc[i];
      s.x += g * nx.x;
      s.y += g * nx.y;
    }
    acc[i] = s;
    if (part) {
      const cplx<R> vv = v[i];
      ar += (double)vv.x * (double)s.x + (double)vv.y * (double)s.y;
      ai += (double)vv.x * (double)s.y - (double)vv.y * (double)s.x;
    }
  }
  if (part) {
    __shared__ double red[2][kChebThreads / 32];
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][w] = ar;
      red[1][w] = ai;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < kChebThreads / 32; ++q) {
        sr += red[0][q];
        si += red[1][q];
      }
      ((double2*)part)[blockIdx.x] = make_double2(sr, si);
    }
  }
}

// Jackson-damped Chebyshev coefficients of the step [x <= tau] (Weisse et al., Rev. Mod. Phys. 78,
// 275 (2006), N = degree + 1 moments): out[i][k] = j_k c_k(tau_i), c_0 = (pi - acos tau)/pi,
// c_k = -2 sin(k acos tau)/(pi k).
__global__ void damped_step_kernel(const double* __restrict__ tau, int count, int degree, float* __restrict__ out) {
  const int total = count * (degree + 1);
  const double pi = 3.141592653589793;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / (degree + 1), k = e - i * (degree + 1);
    const double th = acos(fmin(1.0, fmax(-1.0, tau[i])));
    const double c = k == 0 ? (pi - th) / pi : -2.0 * sin(k * th) / (pi * k);
    const int N = degree + 1;
    const double q = pi / (N + 1);
    const double j = ((N - k + 1) * cos(q * k) + sin(q * k) / tan(q)) / (N + 1);
    out[e] = (float)(j * c);
  }
}

// out[0] = sum_i Re(part[i]) (fixed order): the Rayleigh quotient from conj(x) A x partials.
__global__ void sum_re_kernel(const double2* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i].x;
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    out[0] = t;
  }
}

// Per-block partial sums of |y_i - lambda x_i|^2 (FP64).
__global__ void __launch_bounds__(kChebThreads)
resid_part_kernel(const double2* __restrict__ y, const double2* __restrict__ x, const double* __restrict__ lam, int64_t n,
                  double* __restrict__ part) {
  const double l = *lam;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kChebThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kChebThreads) {
    const double2 a = y[i], b = x[i];
    const double dr = a.x - l * b.x, di = a.y - l * b.y;
    acc += dr * dr + di * di;
  }
  __shared__ double red[kChebThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kChebThreads / 32; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

}  // namespace

int cheb_blocks(int64_t n) {
  const int64_t b = (n + kChebThreads - 1) / kChebThreads;
  return (int)(b < 1216 ? b : 1216);
}

template <typename R>
cudaError_t launch_cheb_step(const void* ax, const void* t_cur, const void* t_prev, void* t_next, void* acc,
                             const void* v, int64_t n, double c, double sc, double sp, double g, double g0, int init,
                             double* part, void* split_next, cudaStream_t s) {
  cheb_step_kernel<R><<<cheb_blocks(n), kChebThreads, 0, s>>>(
      (const cplx<R>*)ax, (const cplx<R>*)t_cur, (const cplx<R>*)t_prev, (cplx<R>*)t_next, (cplx<R>*)acc,
      (const cplx<R>*)v, n, (R)c, (R)sc, (R)sp, (R)g, (R)g0, init, part, (float4*)split_next);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_step<float>(const void*, const void*, const void*, void*, void*, const void*, int64_t,
                                             double, double, double, double, double, int, double*, void*,
                                             cudaStream_t);
template cudaError_t launch_cheb_step<double>(const void*, const void*, const void*, void*, void*, const void*,
                                              int64_t, double, double, double, double, double, int, double*, void*,
                                              cudaStream_t);

cudaError_t launch_sum_re(const double* part, int nblk, double* out, cudaStream_t s) {
  sum_re_kernel<<<1, 256, 0, s>>>((const double2*)part, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_resid_part(const void* y, const void* x, const double* lam, int64_t n, double* part,
                              cudaStream_t s) {
  resid_part_kernel<<<cheb_blocks(n), kChebThreads, 0, s>>>((const double2*)y, (const double2*)x, lam, n, part);
  return cudaGetLastError();
}

cudaError_t launch_damped_step(const double* tau, int count, int degree, float* out, cudaStream_t s) {
  const int total = count * (degree + 1);
  if (total <= 0) return cudaSuccess;
  damped_step_kernel<<<(total + 255) / 256, 256, 0, s>>>(tau, count, degree, out);
  return cudaGetLastError();
}

}  // namespace jtr
