// cg.cu -- conjugate gradients for the invert mode of Algorithm 1: y = A^{-1} b for a Hermitian
// positive definite J-symmetric A in FP64, the Lanczos product of that mode (Sec. 4 solves the inner
// systems with CG).
//
// Hestenes-Stiefel CG from x_0 = 0: with r = b - A x and p the search direction,
//   alpha = r^H r / p^H A p,  x += alpha p,  r -= alpha A p,  beta = r_new^H r_new / r^H r,  p = r + beta p,
// until ||r|| <= rtol ||b||.  For Hermitian A every alpha and beta is real, so x is a real
// polynomial in A applied to b and the approximate inverse keeps A's J-symmetry (eq. (1)): the
// Lanczos vectors stay in their half-subspace.
//
// The scalars live in device memory (CgState) and are formed by one-block kernels, so iterations
// are enqueued back to back; the host reads the state every few iterations.  Once an iteration has
// converged (or found p^H A p <= 0) every later kernel of the solve leaves x, r and p unchanged.

#include <cuda_runtime.h>

#include "internal.h"

namespace jtr {
namespace {

constexpr int kCgThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;   // valid in thread 0
}

// x = 0, r = p = b; per-block partial sums of |b|^2
__global__ void __launch_bounds__(kCgThreads)
cg_init_kernel(const double2* __restrict__ b, double2* __restrict__ x, double2* __restrict__ r,
               double2* __restrict__ p, int64_t n, double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCgThreads) {
    const double2 v = b[i];
    x[i] = make_double2(0.0, 0.0);
    r[i] = v;
    p[i] = v;
    acc += v.x * v.x + v.y * v.y;
  }
  __shared__ double red[kCgThreads / 32];
  const double t = block_sum_d(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void cg_start_kernel(const double* __restrict__ part, int nblk, double rtol, CgState* st) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  __shared__ double red[32];
  const double t = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    st->rr = t;
    st->rr0 = t;
    st->tol2 = rtol * rtol * t;
    st->alpha = st->beta = 0.0;
    st->iters = 0;
    st->fail = 0;
    st->done = t == 0.0 ? 1 : 0;   // b = 0: x = 0 is exact
  }
}

// alpha = r^H r / p^H A p from the product's partials of p^H (A p)
__global__ void cg_alpha_kernel(const double2* __restrict__ part, int nblk, CgState* st) {
  if (st->done) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i].x;
  __shared__ double red[32];
  const double pap = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    if (!(pap > 0.0)) {   // A is not positive definite on p (or p is zero)
      st->fail = 1;
      st->done = 1;
    } else {
      st->alpha = st->rr / pap;
    }
  }
}

// x += alpha p, r -= alpha q; per-block partial sums of |r|^2
__global__ void __launch_bounds__(kCgThreads)
cg_xr_kernel(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
             const double2* __restrict__ q, int64_t n, const CgState* __restrict__ st, double* __restrict__ part) {
  if (st->done) return;   // the same value for every block: set before this launch or not at all
  const double a = st->alpha;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCgThreads) {
    const double2 pv = p[i], qv = q[i];
    double2 xv = x[i], rv = r[i];
    xv.x = fma(a, pv.x, xv.x);
    xv.y = fma(a, pv.y, xv.y);
    rv.x = fma(-a, qv.x, rv.x);
    rv.y = fma(-a, qv.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    acc += rv.x * rv.x + rv.y * rv.y;
  }
  __shared__ double red[kCgThreads / 32];
  const double t = block_sum_d(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void cg_beta_kernel(const double* __restrict__ part, int nblk, CgState* st) {
  if (st->done) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  __shared__ double red[32];
  const double rr = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    st->iters += 1;
    st->beta = rr / st->rr;
    st->rr = rr;
    if (rr <= st->tol2) st->done = 1;
  }
}

// p = r + beta p
__global__ void __launch_bounds__(kCgThreads)
cg_p_kernel(double2* __restrict__ p, const double2* __restrict__ r, int64_t n, const CgState* __restrict__ st) {
  if (st->done) return;
  const double bt = st->beta;
  for (int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCgThreads) {
    const double2 rv = r[i];
    double2 pv = p[i];
    pv.x = fma(bt, pv.x, rv.x);
    pv.y = fma(bt, pv.y, rv.y);
    p[i] = pv;
  }
}

// per-block partial sums of v^H y (double2), the alpha of the Lanczos step
__global__ void __launch_bounds__(kCgThreads)
vhy_part_kernel(const double2* __restrict__ v, const double2* __restrict__ y, int64_t n, double2* __restrict__ part) {
  double re = 0.0, im = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCgThreads) {
    const double2 a = v[i], b = y[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  __shared__ double red[kCgThreads / 32];
  const double tr = block_sum_d(re, red);
  __syncthreads();
  const double ti = block_sum_d(im, red);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(tr, ti);
}

}  // namespace

int cg_blocks(int64_t n) {
  const int64_t b = (n + kCgThreads - 1) / kCgThreads;
  return (int)(b < 1216 ? b : 1216);
}

cudaError_t launch_cg_init(const void* b, void* x, void* r, void* p, int64_t n, double* part, double rtol, CgState* st,
                           cudaStream_t s) {
  const int nb = cg_blocks(n);
  cg_init_kernel<<<nb, kCgThreads, 0, s>>>((const double2*)b, (double2*)x, (double2*)r, (double2*)p, n, part);
  cg_start_kernel<<<1, 256, 0, s>>>(part, nb, rtol, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_alpha(const double* pq_part, int nblk, CgState* st, cudaStream_t s) {
  cg_alpha_kernel<<<1, 256, 0, s>>>((const double2*)pq_part, nblk, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(void* x, void* r, void* p, const void* q, int64_t n, double* part, CgState* st,
                             cudaStream_t s) {
  const int nb = cg_blocks(n);
  cg_xr_kernel<<<nb, kCgThreads, 0, s>>>((double2*)x, (double2*)r, (const double2*)p, (const double2*)q, n, st, part);
  cg_beta_kernel<<<1, 256, 0, s>>>(part, nb, st);
  cg_p_kernel<<<nb, kCgThreads, 0, s>>>((double2*)p, (const double2*)r, n, st);
  return cudaGetLastError();
}

cudaError_t launch_vhy_part(const void* v, const void* y, int64_t n, double* part, cudaStream_t s) {
  vhy_part_kernel<<<cg_blocks(n), kCgThreads, 0, s>>>((const double2*)v, (const double2*)y, n, (double2*)part);
  return cudaGetLastError();
}

}  // namespace jtr
