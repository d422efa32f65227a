// ritz_dev.cuh -- device routines of the Ritz solve shared by ritz.cu (one problem, one warp per
// Ritz pair) and batch.cu (many problems, one CTA each).
#pragma once

#include <math.h>

#include "common.cuh"

namespace jtr {
namespace {

// ------------------------------------------------------------------ fast path: bisection + inverse iteration
// T-bar after a thick restart has the structure (0-based, k = restart size):
//   t_ii = d_i (i < k)          kept Ritz values
//   t_ki = t_ik = b_i (i < k)   the arrow row of the Krylov-Schur form
//   t_jj = alpha_j, t_{j,j+1} = t_{j+1,j} = beta_j (k <= j < m)   Lanczos tridiagonal
// Eliminating the diagonal part first keeps this an O(m) LDL^T factorisation of T - sigma I:
//   pi_i = d_i - sigma (i < k);  pi_k = alpha_k - sigma - sum_i b_i^2 / pi_i;
//   pi_j = alpha_j - sigma - beta_{j-1}^2 / pi_{j-1} (j > k)
// and by Sylvester's law of inertia the number of negative pivots is the number of eigenvalues
// below sigma.  Each wanted eigenvalue gets one warp: FP32 multisection on this count (32 shifts
// per round), then FP64 inverse iteration with Rayleigh-quotient shifts for the eigenvector and
// eigenvalue, then an FP64 inertia check on both sides of the result.  A separate one-block
// kernel checks residuals and orthogonality; if anything fails, the Jacobi kernel recomputes all.
struct TbarView {
  const double* T;
  int ld, m, k;
  __device__ __forceinline__ double diag(int j) const { return T[(size_t)j * ld + j]; }
  __device__ __forceinline__ double arrow(int i) const { return T[(size_t)k * ld + i]; }     // i < k
  __device__ __forceinline__ double off(int j) const { return T[(size_t)(j + 1) * ld + j]; } // j >= k
};

template <typename F>
__device__ __noinline__ int inertia(const TbarView& t, F sigma, F pivmin) {
  int neg = 0;
  F s = 0;
  for (int i = 0; i < t.k; ++i) {
    F p = (F)t.diag(i) - sigma;
    if (fabs(p) < pivmin) p = -pivmin;
    neg += p < 0;
    const F b = (F)t.arrow(i);
    s += b * b / p;
  }
  F p = (F)t.diag(t.k) - sigma - s;
  if (fabs(p) < pivmin) p = -pivmin;
  neg += p < 0;
  for (int j = t.k + 1; j < t.m; ++j) {
    const F b = (F)t.off(j - 1);
    p = (F)t.diag(j) - sigma - b * b / p;
    if (fabs(p) < pivmin) p = -pivmin;
    neg += p < 0;
  }
  return neg;
}

// Warp-cooperative solve of (T - sigma I) x = z in place (z: right-hand side on entry, in shared
// memory); ipiv receives the reciprocal pivots.  The k eliminations of the diagonal part are
// independent and run across the lanes; the tridiagonal part is a serial chain on lane 0.  On this
// part one FP64 warp instruction holds the FP64 pipe for ~16 cycles whatever the active mask, so
// the serial chain does one division per index and multiplies by stored reciprocals elsewhere.
__device__ __noinline__ void shifted_solve_warp(const TbarView& t, double sigma, double pivmin, double* z, double* ipiv) {
  const int k = t.k, m = t.m, lane = threadIdx.x & 31;
  double s = 0.0, sr = 0.0;
  for (int i = lane; i < k; i += 32) {
    double p = t.diag(i) - sigma;
    if (fabs(p) < pivmin) p = (p < 0 ? -pivmin : pivmin);
    const double ip = 1.0 / p;
    ipiv[i] = ip;
    const double b = t.arrow(i);
    s += b * b * ip;
    sr += b * z[i] * ip;
  }
  s = warp_sum(s);
  sr = warp_sum(sr);
  if (lane == 0) {
    double p = t.diag(k) - sigma - s;
    if (fabs(p) < pivmin) p = (p < 0 ? -pivmin : pivmin);
    double ip = 1.0 / p;
    ipiv[k] = ip;
    double zp = z[k] - sr;
    z[k] = zp;
    for (int j = k + 1; j < m; ++j) {
      const double b = t.off(j - 1);
      const double l = b * ip;
      double q = t.diag(j) - sigma - b * l;
      if (fabs(q) < pivmin) q = (q < 0 ? -pivmin : pivmin);
      ip = 1.0 / q;
      ipiv[j] = ip;
      zp = z[j] - l * zp;
      z[j] = zp;
    }
    double zn = z[m - 1] * ipiv[m - 1];
    z[m - 1] = zn;
    for (int j = m - 2; j >= k; --j) {
      zn = (z[j] - t.off(j) * zn) * ipiv[j];
      z[j] = zn;
    }
  }
  __syncwarp();
  const double zk = z[k];
  for (int i = lane; i < k; i += 32) z[i] = (z[i] - t.arrow(i) * zk) * ipiv[i];
  __syncwarp();
}

// Warp-cooperative FP64 inertia count of T - sigma I (same elimination order as above).
__device__ int inertia_warp(const TbarView& t, double sigma, double pivmin) {
  const int k = t.k, m = t.m, lane = threadIdx.x & 31;
  double s = 0.0;
  int neg = 0;
  for (int i = lane; i < k; i += 32) {
    double p = t.diag(i) - sigma;
    if (fabs(p) < pivmin) p = -pivmin;
    neg += p < 0;
    const double b = t.arrow(i);
    s += b * b / p;
  }
  s = warp_sum(s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) neg += __shfl_xor_sync(0xffffffffu, neg, o);
  if (lane == 0) {
    double p = t.diag(k) - sigma - s;
    if (fabs(p) < pivmin) p = -pivmin;
    neg += p < 0;
    for (int j = k + 1; j < m; ++j) {
      const double b = t.off(j - 1);
      p = t.diag(j) - sigma - b * b / p;
      if (fabs(p) < pivmin) p = -pivmin;
      neg += p < 0;
    }
  }
  return __shfl_sync(0xffffffffu, neg, 0);
}

__device__ double warp_normalize(double* z, int m) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < m; i += 32) s += z[i] * z[i];
  s = warp_sum(s);
  const double inv = 1.0 / sqrt(s);
  __syncwarp();
  for (int i = lane; i < m; i += 32) z[i] *= inv;
  __syncwarp();
  return s;
}

// (T z)_i for all i, lane-parallel, into tz.
__device__ void warp_apply(const TbarView& t, const double* z, double* tz) {
  const int lane = threadIdx.x & 31, k = t.k, m = t.m;
  for (int i = lane; i < m; i += 32) {
    double v;
    if (i < k) {
      v = t.diag(i) * z[i] + t.arrow(i) * z[k];
    } else {
      v = t.diag(i) * z[i];
      if (i == k) {
        for (int q = 0; q < k; ++q) v += t.arrow(q) * z[q];
      } else {
        v += t.off(i - 1) * z[i - 1];
      }
      if (i + 1 < m) v += t.off(i) * z[i + 1];
    }
    tz[i] = v;
  }
  __syncwarp();
}

// One warp computes the eigenpair of index r (ascending order) of the T-bar held in T (ld ldt, m x m,
// restart size k): FP32 multisection on the inertia count, FP64 inverse iteration with Rayleigh-
// quotient shifts, and an FP64 inertia check on both sides.  z, piv, tz: warp-private scratch of m
// doubles each.  Writes the normalised eigenvector to zout (m doubles) and returns the eigenvalue,
// or NaN if the inertia check fails.
__device__ double ritz_pair_warp(const double* T, int ldt, int m, int k, int r, double* z, double* piv, double* tz,
                                 double* zout) {
  const int lane = threadIdx.x & 31;
  const TbarView t{T, ldt, m, k};
  // Gershgorin interval and scale
  double glo = 1e300, ghi = -1e300;
  for (int j = lane; j < m; j += 32) {
    double rad = 0.0;
    if (j < k) rad = fabs(t.arrow(j));
    else {
      if (j == k) for (int q = 0; q < k; ++q) rad += fabs(t.arrow(q));
      else rad += fabs(t.off(j - 1));
      if (j + 1 < m) rad += fabs(t.off(j));
    }
    glo = fmin(glo, t.diag(j) - rad);
    ghi = fmax(ghi, t.diag(j) + rad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  glo -= 1e-6 * tnorm + 1e-300;
  ghi += 1e-6 * tnorm + 1e-300;
  // FP32 multisection: 32 shifts per round, keep [lo, hi] with count(lo) <= r < count(hi)
  float lo = (float)glo, hi = (float)ghi;
  const float pmin32 = (float)(tnorm * 1e-30) + 1e-30f;
  for (int round = 0; round < 8; ++round) {
    const float w = (hi - lo) / 33.0f;
    const float sig = lo + w * (float)(lane + 1);
    const int cnt = inertia<float>(t, sig, pmin32);
    const unsigned below = __ballot_sync(0xffffffffu, cnt <= r);   // shifts still at or below lambda_r
    const int nb = __popc(below);                                   // counts are monotone in the shift
    const float nlo = nb > 0 ? __shfl_sync(0xffffffffu, sig, nb - 1) : lo;
    const float nhi = nb < 32 ? __shfl_sync(0xffffffffu, sig, nb) : hi;
    lo = nlo;
    hi = nhi;
    if (hi - lo <= 4.0f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
  }
  const double lo64 = (double)lo, hi64 = (double)hi;
  const double slack = 1e-6 * tnorm;             // FP32 rounding of T moves eigenvalues by ~6e-8 ||T||
  double sigma = 0.5 * (lo64 + hi64);
  const double pivmin = 1e-18 * tnorm + 1e-300;
  // FP64 inverse iteration from a fixed pseudo-random start, three solves, each followed by a
  // Rayleigh quotient that becomes the next shift (kept only while inside the FP32 bracket)
  for (int j = lane; j < m; j += 32) z[j] = u01_sym(0x9E37ull * (uint64_t)(r + 1) + (uint64_t)j) + 0.5;
  __syncwarp();
  warp_normalize(z, m);
  double lambda = sigma;
  for (int it = 0; it < 3; ++it) {
    shifted_solve_warp(t, sigma, pivmin, z, piv);
    warp_normalize(z, m);
    warp_apply(t, z, tz);
    double q = 0.0;
    for (int j = lane; j < m; j += 32) q += z[j] * tz[j];
    lambda = warp_sum(q);
    if (lambda >= lo64 - slack && lambda <= hi64 + slack) sigma = lambda;
  }
  // FP64 inertia on both sides: lambda must be the r-th eigenvalue (Sylvester)
  const double delta = 1e-9 * tnorm;
  const int c_lo = inertia_warp(t, lambda - delta, pivmin);
  const int c_hi = inertia_warp(t, lambda + delta, pivmin);
  for (int j = lane; j < m; j += 32) zout[j] = z[j];
  return (c_lo <= r && c_hi >= r + 1 && lambda == lambda) ? lambda : NAN;
}

}  // namespace
}  // namespace jtr
