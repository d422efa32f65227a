// batch.cu -- many dense Hermitian J-symmetric problems of uneven size in one persistent launch.
//
// Each CTA takes instances from a queue (largest first, an atomic counter) and runs the whole of
// Algorithm 1 (TRLAN-JSYM) with the Lanczos step of Algorithm 2 for one instance at a time, with all
// control on the device: dense J-matvec (eq. (4): one read of A11, A12 serves both halves), alpha,
// classical Gram-Schmidt against V and W = J V^* repeated by the sqrt(2) test, the FP64 Ritz solve of
// ritz_dev.cuh (one warp per pair, verified; a one-CTA Jacobi if a check fails), the rotation of the
// kept columns, true residuals, the converged-first ordering and the shrink of eq. (29).
//
// Template parameter DF: false -- plain FP64 arithmetic; true -- the matvec, the Gram-Schmidt inner
// products and updates, and the rotation in compensated FP32 ("double-float", see gsdf.cu) on
// (hi, lo) copies of A and of the basis, with FP64 vectors, alpha/beta, Ritz solve and residuals.
//
// Per CTA: T-bar, the Ritz vectors of T-bar, the current v_j and y in shared memory; V
// (n_max x (m+1)) and the rotation target (n_max x kk, FP64) in a per-CTA global slot.  Bounded loops only (restarts <= max_restarts, GS
// passes <= gs_passes, Jacobi sweeps <= 40).
#include <math.h>

#include "internal.h"
#include "ritz_dev.cuh"
#include "../../include/jtrlan.h"

namespace jtr {

namespace {

// ------------------------------------------------------------------ compensated FP32 helpers
__device__ __forceinline__ void b_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void b_df_acc(float& s, float& e, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  const float cross = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  float t, te;
  b_two_sum(s, p, t, te);
  s = t;
  e = __fadd_rn(e, __fadd_rn(te, __fadd_rn(pe, cross)));
}
__device__ __forceinline__ float4 b_split(double2 v) {
  const float hx = (float)v.x, hy = (float)v.y;
  return make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}
__device__ __forceinline__ double2 b_join(float4 f) {
  return make_double2((double)f.x + (double)f.z, (double)f.y + (double)f.w);
}
// complex (s, e)[2] += a * b and += conj(a) * b, a and b as (hi.re, hi.im, lo.re, lo.im)
__device__ __forceinline__ void b_cacc(float* s, float* e, float4 a, float4 b, float sign = 1.f) {
  b_df_acc(s[0], e[0], sign * a.x, sign * a.z, b.x, b.z);
  b_df_acc(s[0], e[0], -sign * a.y, -sign * a.w, b.y, b.w);
  b_df_acc(s[1], e[1], sign * a.x, sign * a.z, b.y, b.w);
  b_df_acc(s[1], e[1], sign * a.y, sign * a.w, b.x, b.z);
}
__device__ __forceinline__ void b_caccc(float* s, float* e, float4 a, float4 b, float sign = 1.f) {
  b_df_acc(s[0], e[0], sign * a.x, sign * a.z, b.x, b.z);
  b_df_acc(s[0], e[0], sign * a.y, sign * a.w, b.y, b.w);
  b_df_acc(s[1], e[1], sign * a.x, sign * a.z, b.y, b.w);
  b_df_acc(s[1], e[1], -sign * a.y, -sign * a.w, b.x, b.z);
}
constexpr int kMaxM = kBatchMaxM;
constexpr int kMaxNev = kBatchMaxNev;

// (s, e) += (s2, e2) in compensated FP32
__device__ __forceinline__ void df_add(float& s, float& e, float s2, float e2) {
  float t, te;
  b_two_sum(s, s2, t, te);
  s = t;
  e = __fadd_rn(e, __fadd_rn(e2, te));
}
// One level of a reduce-scatter across lanes at distance o: a lane with `upper` set keeps the
// second of the two values (lo, hi) and receives its partner's copy of it; the other keeps the first.
__device__ __forceinline__ void df_xchg(float lo_s, float lo_e, float hi_s, float hi_e, bool upper, int o, float& ks,
                                        float& ke) {
  const float ss = upper ? lo_s : hi_s, se = upper ? lo_e : hi_e;
  ks = upper ? hi_s : lo_s;
  ke = upper ? hi_e : lo_e;
  const float rs = __shfl_xor_sync(0xffffffffu, ss, o), re = __shfl_xor_sync(0xffffffffu, se, o);
  df_add(ks, ke, rs, re);
}
// Warp sums of 8 compensated values: on return lane L holds the total of value (L >> 2) & 7.
__device__ __forceinline__ double df_reduce8(const float* s, const float* e) {
  const int lane = threadIdx.x & 31;
  float s4[4], e4[4], s2[2], e2[2], s1, e1;
#pragma unroll
  for (int k = 0; k < 4; ++k) df_xchg(s[k], e[k], s[4 + k], e[4 + k], lane & 16, 16, s4[k], e4[k]);
#pragma unroll
  for (int k = 0; k < 2; ++k) df_xchg(s4[k], e4[k], s4[2 + k], e4[2 + k], lane & 8, 8, s2[k], e2[k]);
  df_xchg(s2[0], e2[0], s2[1], e2[1], lane & 4, 4, s1, e1);
#pragma unroll
  for (int o = 2; o > 0; o >>= 1) df_add(s1, e1, __shfl_xor_sync(0xffffffffu, s1, o), __shfl_xor_sync(0xffffffffu, e1, o));
  return (double)s1 + (double)e1;
}
// Warp sums of 4 compensated values: on return lane L holds the total of value (L >> 3) & 3.
__device__ __forceinline__ double df_reduce4(const float* s, const float* e) {
  const int lane = threadIdx.x & 31;
  float s2[2], e2[2], s1, e1;
#pragma unroll
  for (int k = 0; k < 2; ++k) df_xchg(s[k], e[k], s[2 + k], e[2 + k], lane & 16, 16, s2[k], e2[k]);
  df_xchg(s2[0], e2[0], s2[1], e2[1], lane & 8, 8, s1, e1);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) df_add(s1, e1, __shfl_xor_sync(0xffffffffu, s1, o), __shfl_xor_sync(0xffffffffu, e1, o));
  return (double)s1 + (double)e1;
}

// O(m) per-instance state; the O(m^2) and O(n) arrays are in dynamic shared memory (BatchSmem).
struct Shared {
  double coef[(kMaxM + 1) * 4];
  float4 coef4[(kMaxM + 1) * 2];
  double red[64];
  double lam[kMaxM], lamv[kMaxM], arrow[kMaxM];
  double ev[kMaxNev], res[kMaxNev], res_est[kMaxNev], locked_ev[kMaxNev], locked_res[kMaxNev];
  int perm[kMaxM], ord[kMaxNev], conv[kMaxNev];
  int ok, status, icnv, k, nlocked, inst;
  double tmax;
};

__host__ __device__ inline size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

// Dynamic shared memory: T-bar ((m+1)^2), Z (m x kk) and its (hi, lo) float split Zf, the Ritz
// scratch (float T-bar, brackets, the lanes' interleaved vectors and pivots), the Gram-Schmidt
// partial sums (8 floats per thread), then the vectors x, y
// (FP64) and x4 ((hi, lo) copy of x, and of y during Gram-Schmidt), whose space the Jacobi fallback
// reuses for its two m x m arrays.
struct BatchSmem {
  size_t T, Z, Zf, Tf, br, zb, part, vec, total;
  __host__ __device__ BatchSmem(int64_t nmax, int m, int kk, int threads) {
    T = 0;
    Z = T + up16(sizeof(double) * (m + 1) * (m + 1));
    Zf = Z + up16(sizeof(double) * m * kk);
    Tf = Zf + up16(sizeof(float2) * m * kk);
    br = Tf + up16(sizeof(float) * 3 * m);
    zb = br + up16(sizeof(float) * 2 * kk);
    part = zb + up16(sizeof(double) * 2 * 32 * m * ((kk + 31) / 32));
    vec = part + up16(sizeof(float) * 8 * threads);
    const size_t vb = (size_t)nmax * (2 * sizeof(double2) + sizeof(float4));
    const size_t jb = 2 * sizeof(double) * m * m;
    total = vec + up16(vb > jb ? vb : jb);
  }
};

// ------------------------------------------------------------------ block reductions
__device__ double blk_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[32] = t;
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// Double-float y = A x: each warp takes two of its rows at a time (r0 and r0 + nw share the loads of
// x), walks the 32-column chunks of both with the next chunk's A loads issued before the current
// chunk's arithmetic, and reduces the 8 row sums with one reduce-scatter.
__device__ void cta_matvec_df(const float4* A11, const float4* A12, int64_t h, const float4* x4, double2* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int C = (int)((h + 31) >> 5);
  const int R = (w < h) ? (int)((h - 1 - w) / nw) + 1 : 0;
  const int total = ((R + 1) >> 1) * C;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fetch = [&](int q, int u, float4& a0, float4& b0, float4& a1, float4& b1) {
    const int64_t c = lane + 32 * u;
    const int64_t r0 = w + (int64_t)(2 * q) * nw, r1 = r0 + nw;
    a0 = b0 = a1 = b1 = z4;
    if (c < h) {
      a0 = A11[r0 * h + c];
      b0 = A12[r0 * h + c];
      if (r1 < h) {
        a1 = A11[r1 * h + c];
        b1 = A12[r1 * h + c];
      }
    }
  };
  float4 ca0, cb0, ca1, cb1;
  if (total > 0) fetch(0, 0, ca0, cb0, ca1, cb1);
  float s[8], e[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) s[k] = e[k] = 0.f;
  int q = 0, u = 0;
  for (int it = 0; it < total; ++it) {
    int qn = q, un = u + 1;
    if (un == C) {
      un = 0;
      ++qn;
    }
    float4 na0 = z4, nb0 = z4, na1 = z4, nb1 = z4;
    if (it + 1 < total) fetch(qn, un, na0, nb0, na1, nb1);
    const int64_t c = lane + 32 * u;
    if (c < h) {
      const float4 x1 = x4[c], x2 = x4[h + c];
      b_cacc(&s[0], &e[0], ca0, x1);          // y1 = A11 x1 + A12 x2
      b_cacc(&s[0], &e[0], cb0, x2);
      b_caccc(&s[2], &e[2], ca0, x2);         // y2 = conj(A11) x2 - conj(A12) x1
      b_caccc(&s[2], &e[2], cb0, x1, -1.f);
      b_cacc(&s[4], &e[4], ca1, x1);
      b_cacc(&s[4], &e[4], cb1, x2);
      b_caccc(&s[6], &e[6], ca1, x2);
      b_caccc(&s[6], &e[6], cb1, x1, -1.f);
    }
    if (u == C - 1) {
      const double v = df_reduce8(s, e);
      const int idx = lane >> 2;
      const int64_t row = w + (int64_t)(2 * q + (idx >> 2)) * nw;
      if ((lane & 3) == 0 && row < h) {
        const int comp = idx & 3;               // y1.re, y1.im, y2.re, y2.im
        ((double*)y)[comp < 2 ? 2 * row + comp : 2 * (h + row) + comp - 2] = v;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] = e[k] = 0.f;
    }
    ca0 = na0;
    cb0 = nb0;
    ca1 = na1;
    cb1 = nb1;
    q = qn;
    u = un;
  }
}

// y = A x (dense block form); x and y in shared memory (FP64), A rows from global.  Returns the
// block-wide Re/Im of x^H y in (*ar, *ai) when requested.
// The same with one row per warp at a time (the tile shape the autotuner may pick for small orders):
// four sums, one reduce-scatter per row.
__device__ void cta_matvec_df1(const float4* A11, const float4* A12, int64_t h, const float4* x4, double2* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int C = (int)((h + 31) >> 5);
  const int R = (w < h) ? (int)((h - 1 - w) / nw) + 1 : 0;
  const int total = R * C;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fetch = [&](int q, int u, float4& a0, float4& b0) {
    const int64_t c = lane + 32 * u;
    const int64_t r0 = w + (int64_t)q * nw;
    a0 = b0 = z4;
    if (c < h) {
      a0 = A11[r0 * h + c];
      b0 = A12[r0 * h + c];
    }
  };
  float4 ca0, cb0;
  if (total > 0) fetch(0, 0, ca0, cb0);
  float s[4], e[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = e[k] = 0.f;
  int q = 0, u = 0;
  for (int it = 0; it < total; ++it) {
    int qn = q, un = u + 1;
    if (un == C) {
      un = 0;
      ++qn;
    }
    float4 na0 = z4, nb0 = z4;
    if (it + 1 < total) fetch(qn, un, na0, nb0);
    const int64_t c = lane + 32 * u;
    if (c < h) {
      const float4 x1 = x4[c], x2 = x4[h + c];
      b_cacc(&s[0], &e[0], ca0, x1);          // y1 = A11 x1 + A12 x2
      b_cacc(&s[0], &e[0], cb0, x2);
      b_caccc(&s[2], &e[2], ca0, x2);         // y2 = conj(A11) x2 - conj(A12) x1
      b_caccc(&s[2], &e[2], cb0, x1, -1.f);
    }
    if (u == C - 1) {
      const double v = df_reduce4(s, e);      // lane L holds sum (L >> 3) & 3
      const int64_t row = w + (int64_t)q * nw;
      if ((lane & 7) == 0) {
        const int comp = lane >> 3;           // y1.re, y1.im, y2.re, y2.im
        ((double*)y)[comp < 2 ? 2 * row + comp : 2 * (h + row) + comp - 2] = v;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) s[k] = e[k] = 0.f;
    }
    ca0 = na0;
    cb0 = nb0;
    q = qn;
    u = un;
  }
}

template <bool DF, int MVR>
__device__ void cta_matvec(const BatchArgs& a, int64_t h, int64_t off, const double2* x, const float4* x4, double2* y,
                           double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (DF) {
    if constexpr (MVR == 1)
      cta_matvec_df1((const float4*)a.A11 + off, (const float4*)a.A12 + off, h, x4, y);
    else
      cta_matvec_df((const float4*)a.A11 + off, (const float4*)a.A12 + off, h, x4, y);
  } else if constexpr (MVR == 2) {   // two rows per warp (r and r + nw) sharing the loads of x
    for (int64_t r = w; r < h; r += 2 * nw) {
      const int64_t r2 = r + nw;
      const bool two = r2 < h;
      const double2* r11 = (const double2*)a.A11 + off + r * h;
      const double2* r12 = (const double2*)a.A12 + off + r * h;
      const double2* s11 = (const double2*)a.A11 + off + (two ? r2 : r) * h;
      const double2* s12 = (const double2*)a.A12 + off + (two ? r2 : r) * h;
      double2 y1 = make_double2(0, 0), y2 = make_double2(0, 0), z1 = make_double2(0, 0), z2 = make_double2(0, 0);
      for (int64_t c = lane; c < h; c += 32) {
        const double2 x1 = x[c], x2 = x[h + c];
        const double2 a11 = r11[c], a12 = r12[c];
        y1 = cfma(a11, x1, y1);
        y1 = cfma(a12, x2, y1);
        y2 = cfmac(a11, x2, y2);
        y2 = cfmac(make_double2(-a12.x, -a12.y), x1, y2);
        if (two) {
          const double2 b11 = s11[c], b12 = s12[c];
          z1 = cfma(b11, x1, z1);
          z1 = cfma(b12, x2, z1);
          z2 = cfmac(b11, x2, z2);
          z2 = cfmac(make_double2(-b12.x, -b12.y), x1, z2);
        }
      }
      const double v0 = warp_sum(y1.x), v1 = warp_sum(y1.y), v2 = warp_sum(y2.x), v3 = warp_sum(y2.y);
      const double u0 = warp_sum(z1.x), u1 = warp_sum(z1.y), u2 = warp_sum(z2.x), u3 = warp_sum(z2.y);
      if (lane == 0) {
        y[r] = make_double2(v0, v1);
        y[h + r] = make_double2(v2, v3);
        if (two) {
          y[r2] = make_double2(u0, u1);
          y[h + r2] = make_double2(u2, u3);
        }
      }
    }
  } else {
    for (int64_t r = w; r < h; r += nw) {
      const double2* r11 = (const double2*)a.A11 + off + r * h;
      const double2* r12 = (const double2*)a.A12 + off + r * h;
      double2 y1 = make_double2(0, 0), y2 = make_double2(0, 0);
      for (int64_t c = lane; c < h; c += 32) {
        const double2 a11 = r11[c], a12 = r12[c], x1 = x[c], x2 = x[h + c];
        y1 = cfma(a11, x1, y1);
        y1 = cfma(a12, x2, y1);
        y2 = cfmac(a11, x2, y2);
        y2 = cfmac(make_double2(-a12.x, -a12.y), x1, y2);
      }
      const double v0 = warp_sum(y1.x), v1 = warp_sum(y1.y), v2 = warp_sum(y2.x), v3 = warp_sum(y2.y);
      if (lane == 0) {
        y[r] = make_double2(v0, v1);
        y[h + r] = make_double2(v2, v3);
      }
    }
  }
  __syncthreads();
}

// c_v = V^H y and c_w = W^H y for columns 0..j (warp w takes columns w, w + nw, ...), into coef;
// the double-float form first splits y once into y4 and also leaves (hi, lo) splits of the
// coefficients in coef4 (c_v of column i at 2i, c_w at 2i + 1), so no FP64 work is left per element.
// The double-float form walks (column, 32-row chunk) pairs with the next chunk's loads issued before
// the current chunk's arithmetic and reduces the 4 sums of a column with one reduce-scatter.
template <bool DF>
__device__ void cta_dot(const void* Vv, int64_t n, int64_t h, int j, const double2* y, float4* y4, double* coef,
                        float4* coef4) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (DF) {
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) y4[p] = b_split(y[p]);
    __syncthreads();
    const float4* V = (const float4*)Vv;
    const int C = (int)((h + 31) >> 5);
    const int ncol = (w <= j) ? (j - w) / nw + 1 : 0;
    const int total = ncol * C;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto fetch = [&](int t, int u, float4& v1, float4& v2) {
      const int64_t p = lane + 32 * u;
      const int64_t i = w + (int64_t)t * nw;
      v1 = v2 = z4;
      if (p < h) {
        v1 = V[i * n + p];
        v2 = V[i * n + h + p];
      }
    };
    float4 c1, c2;
    if (total > 0) fetch(0, 0, c1, c2);
    float sv[4] = {0.f, 0.f, 0.f, 0.f}, ev[4] = {0.f, 0.f, 0.f, 0.f};   // c_v re, im, c_w re, im
    int t = 0, u = 0;
    for (int it = 0; it < total; ++it) {
      int tn = t, un = u + 1;
      if (un == C) {
        un = 0;
        ++tn;
      }
      float4 n1 = z4, n2 = z4;
      if (it + 1 < total) fetch(tn, un, n1, n2);
      const int64_t p = lane + 32 * u;
      if (p < h) {
        const float4 y1 = y4[p], y2 = y4[h + p];
        b_caccc(&sv[0], &ev[0], c1, y1);       // c_v = sum conj(v1) y1 + conj(v2) y2
        b_caccc(&sv[0], &ev[0], c2, y2);
        b_cacc(&sv[2], &ev[2], c1, y2);        // c_w = sum v1 y2 - v2 y1
        b_cacc(&sv[2], &ev[2], c2, y1, -1.f);
      }
      if (u == C - 1) {
        const double v = df_reduce4(sv, ev);
        const int i = w + t * nw;
        if ((lane & 7) == 0) coef[4 * i + (lane >> 3)] = v;
#pragma unroll
        for (int k = 0; k < 4; ++k) sv[k] = ev[k] = 0.f;
      }
      c1 = n1;
      c2 = n2;
      t = tn;
      u = un;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      coef4[2 * i] = b_split(make_double2(coef[4 * i], coef[4 * i + 1]));
      coef4[2 * i + 1] = b_split(make_double2(coef[4 * i + 2], coef[4 * i + 3]));
    }
  } else {
    for (int i = w; i <= j; i += nw) {
      const double2* vi = (const double2*)Vv + (int64_t)i * n;
      double2 cv = make_double2(0, 0), cw = make_double2(0, 0);
      for (int64_t p = lane; p < h; p += 32) {
        const double2 v1 = vi[p], v2 = vi[h + p], y1 = y[p], y2 = y[h + p];
        cv = cfmac(v1, y1, cv);
        cv = cfmac(v2, y2, cv);
        cw = cfma(v1, y2, cw);
        cw = cfma(make_double2(-v2.x, -v2.y), y1, cw);
      }
      const double c0 = warp_sum(cv.x), c1 = warp_sum(cv.y), c2 = warp_sum(cw.x), c3 = warp_sum(cw.y);
      if (lane == 0) {
        coef[4 * i] = c0;
        coef[4 * i + 1] = c1;
        coef[4 * i + 2] = c2;
        coef[4 * i + 3] = c3;
      }
    }
  }
  __syncthreads();
}

// y -= V c_v + W c_w; returns ||y||^2 (block-wide).  FP64: each thread a row pair.  Double-float:
// the CTA's threads form G = blockDim / hp groups of hp >= h threads (h rounded up to 32); group g
// takes columns g, g + G, ... for every row pair, with the next column's loads issued before the
// current one's arithmetic; groups 1 .. G-1 leave their compensated partial sums in `part`
// (8 floats per thread) and group 0 adds them and updates y.
template <bool DF>
__device__ double cta_update(const void* Vv, int64_t n, int64_t h, int j, const double* coef, const float4* coef4,
                             double2* y, float* part, double* red, int gs_groups) {
  double nrm = 0.0;
  if constexpr (DF) {
    const float4* V = (const float4*)Vv;
    // compensated sums of V c_v + W c_w over columns g0, g0 + G, ... <= j for row pair p
    auto accumulate = [&](int64_t p, int g0, int G, float* s, float* e) {
#pragma unroll
      for (int k = 0; k < 4; ++k) s[k] = e[k] = 0.f;
      if (g0 > j) return;
      float4 v1 = V[(int64_t)g0 * n + p], v2 = V[(int64_t)g0 * n + h + p];
      for (int i = g0; i <= j; i += G) {
        float4 n1 = v1, n2 = v2;
        if (i + G <= j) {
          n1 = V[(int64_t)(i + G) * n + p];
          n2 = V[(int64_t)(i + G) * n + h + p];
        }
        const float4 cv = coef4[2 * i], cw = coef4[2 * i + 1];
        b_cacc(&s[0], &e[0], v1, cv);          // (V c_v + W c_w)_1 = v1 c_v - conj(v2) c_w
        b_caccc(&s[0], &e[0], v2, cw, -1.f);
        b_cacc(&s[2], &e[2], v2, cv);          // (V c_v + W c_w)_2 = v2 c_v + conj(v1) c_w
        b_caccc(&s[2], &e[2], v1, cw);
        v1 = n1;
        v2 = n2;
      }
    };
    auto apply = [&](int64_t p, const float* s, const float* e) {
      double2 y1 = y[p], y2 = y[h + p];
      y1.x -= (double)s[0] + (double)e[0];
      y1.y -= (double)s[1] + (double)e[1];
      y2.x -= (double)s[2] + (double)e[2];
      y2.y -= (double)s[3] + (double)e[3];
      y[p] = y1;
      y[h + p] = y2;
      nrm += cabs2(y1) + cabs2(y2);
    };
    const int hp = (int)(((h + 31) >> 5) << 5);
    float s[4], e[4];
    if (hp <= (int)blockDim.x) {               // one sweep: G groups of hp threads
      int G = (int)blockDim.x / hp;
      if (gs_groups > 0 && G > gs_groups) G = gs_groups;   // tile shape: fewer, longer column walks
      const int g = (int)threadIdx.x / hp, tl = (int)threadIdx.x - g * hp;
      const bool active = g < G && tl < h;
      if (active) accumulate(tl, g, G, s, e);
      if (G > 1) {
        if (active && g > 0) {
          float* pp = part + (size_t)8 * ((g - 1) * hp + tl);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            pp[k] = s[k];
            pp[4 + k] = e[k];
          }
        }
        __syncthreads();
        if (active && g == 0)
          for (int gg = 1; gg < G; ++gg) {
            const float* pp = part + (size_t)8 * ((gg - 1) * hp + tl);
#pragma unroll
            for (int k = 0; k < 4; ++k) df_add(s[k], e[k], pp[k], pp[4 + k]);
          }
      }
      if (active && g == 0) apply(tl, s, e);
    } else {
      for (int64_t p = threadIdx.x; p < h; p += blockDim.x) {
        accumulate(p, 0, 1, s, e);
        apply(p, s, e);
      }
    }
  } else {
    for (int64_t p = threadIdx.x; p < h; p += blockDim.x) {
      double2 y1 = y[p], y2 = y[h + p];
      const double2* V = (const double2*)Vv;
      double2 a1 = make_double2(0, 0), a2 = make_double2(0, 0);
      for (int i = 0; i <= j; ++i) {
        const double2 v1 = V[(int64_t)i * n + p], v2 = V[(int64_t)i * n + h + p];
        const double2 cv = make_double2(coef[4 * i], coef[4 * i + 1]), cw = make_double2(coef[4 * i + 2], coef[4 * i + 3]);
        a1 = cfma(v1, cv, a1);
        a1 = cfmac(v2, make_double2(-cw.x, -cw.y), a1);
        a2 = cfma(v2, cv, a2);
        a2 = cfmac(v1, cw, a2);
      }
      y1.x -= a1.x; y1.y -= a1.y; y2.x -= a2.x; y2.y -= a2.y;
      y[p] = y1;
      y[h + p] = y2;
      nrm += cabs2(y1) + cabs2(y2);
    }
  }
  return blk_sum(nrm, red);
}

// Vt[:, c] = V Z[:, c] for c in [c0, c1), rows 2n real (FP64 target); the double-float form reads
// Z as (hi, lo) float pairs from Zf.
template <bool DF>
__device__ void cta_rotate(const void* Vv, int64_t n, int m, const double* Z, const float2* Zf, int c0, int c1,
                           double2* Vt) {
  for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
    for (int cb = c0; cb < c1; cb += 4) {
      double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
      float sr[4] = {0, 0, 0, 0}, er[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0}, ei[4] = {0, 0, 0, 0};
      for (int i = 0; i < m; ++i) {
        if (!DF) {
          const double2 v = ((const double2*)Vv)[(int64_t)i * n + p];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (cb + q < c1) {
              const double z = Z[(size_t)(cb + q) * m + i];
              ar[q] = fma(v.x, z, ar[q]);
              ai[q] = fma(v.y, z, ai[q]);
            }
          }
        } else {
          const float4 v = ((const float4*)Vv)[(int64_t)i * n + p];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (cb + q < c1) {
              const float2 z = Zf[(size_t)(cb + q) * m + i];
              b_df_acc(sr[q], er[q], v.x, v.z, z.x, z.y);
              b_df_acc(si[q], ei[q], v.y, v.w, z.x, z.y);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (cb + q < c1) {
          Vt[(int64_t)(cb + q) * n + p] = DF ? make_double2((double)sr[q] + (double)er[q], (double)si[q] + (double)ei[q])
                                             : make_double2(ar[q], ai[q]);
        }
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ Ritz solve, lane per pair
// T-bar as three float arrays (diagonal d, arrow a of the kept part, Lanczos off-diagonal e), so the
// FP32 multisection reads no FP64 value.
__device__ __forceinline__ int inertia_f32(const float* d, const float* a, const float* e, int m, int k, float sigma,
                                           float pivmin) {
  int neg = 0;
  float s = 0.f;
  for (int i = 0; i < k; ++i) {
    float p = d[i] - sigma;
    if (fabsf(p) < pivmin) p = -pivmin;
    neg += p < 0.f;
    s += a[i] * a[i] / p;
  }
  float p = d[k] - sigma - s;
  if (fabsf(p) < pivmin) p = -pivmin;
  neg += p < 0.f;
  for (int j = k + 1; j < m; ++j) {
    const float b = e[j - 1];
    p = d[j] - sigma - b * b / p;
    if (fabsf(p) < pivmin) p = -pivmin;
    neg += p < 0.f;
  }
  return neg;
}

// Serial FP64 LDL^T pass over T-bar - sigma I in the order of ritz_dev.cuh (kept part, the arrow
// row, then the tridiagonal chain): returns the number of negative pivots.
__device__ __forceinline__ int inertia_f64_serial(const TbarView& t, double sigma, double pivmin) {
  int neg = 0;
  double s = 0.0;
  for (int i = 0; i < t.k; ++i) {
    double p = t.diag(i) - sigma;
    if (fabs(p) < pivmin) p = -pivmin;
    neg += p < 0.0;
    const double b = t.arrow(i);
    s += b * b / p;
  }
  double p = t.diag(t.k) - sigma - s;
  if (fabs(p) < pivmin) p = -pivmin;
  neg += p < 0.0;
  for (int j = t.k + 1; j < t.m; ++j) {
    const double b = t.off(j - 1);
    p = t.diag(j) - sigma - b * b / p;
    if (fabs(p) < pivmin) p = -pivmin;
    neg += p < 0.0;
  }
  return neg;
}

// One lane's solve of (T - sigma I) x = z in place; z and ip are this lane's columns of interleaved
// arrays (element q at [32 q]).
__device__ __forceinline__ void solve_serial(const TbarView& t, double sigma, double pivmin, double* z, double* ip) {
  const int k = t.k, m = t.m;
  double s = 0.0, sr = 0.0;
  for (int i = 0; i < k; ++i) {
    double p = t.diag(i) - sigma;
    if (fabs(p) < pivmin) p = (p < 0 ? -pivmin : pivmin);
    const double r = 1.0 / p;
    ip[32 * i] = r;
    const double b = t.arrow(i);
    s += b * b * r;
    sr += b * z[32 * i] * r;
  }
  double p = t.diag(k) - sigma - s;
  if (fabs(p) < pivmin) p = (p < 0 ? -pivmin : pivmin);
  double r = 1.0 / p;
  ip[32 * k] = r;
  double zp = z[32 * k] - sr;
  z[32 * k] = zp;
  for (int j = k + 1; j < m; ++j) {
    const double b = t.off(j - 1);
    const double l = b * r;
    double q = t.diag(j) - sigma - b * l;
    if (fabs(q) < pivmin) q = (q < 0 ? -pivmin : pivmin);
    r = 1.0 / q;
    ip[32 * j] = r;
    zp = z[32 * j] - l * zp;
    z[32 * j] = zp;
  }
  double zn = z[32 * (m - 1)] * ip[32 * (m - 1)];
  z[32 * (m - 1)] = zn;
  for (int j = m - 2; j >= k; --j) {
    zn = (z[32 * j] - t.off(j) * zn) * ip[32 * j];
    z[32 * j] = zn;
  }
  const double zk = z[32 * k];
  for (int i = 0; i < k; ++i) z[32 * i] = (z[32 * i] - t.arrow(i) * zk) * ip[32 * i];
}

// z^T T z and z^T z for one lane's interleaved z.
__device__ __forceinline__ void rayleigh_serial(const TbarView& t, const double* z, double& ztz, double& zz) {
  const int k = t.k, m = t.m;
  double a = 0.0, n2 = 0.0;
  const double zk = z[32 * k];
  for (int i = 0; i < k; ++i) {
    const double zi = z[32 * i];
    a += zi * (t.diag(i) * zi + 2.0 * t.arrow(i) * zk);
    n2 += zi * zi;
  }
  for (int j = k; j < m; ++j) {
    const double zj = z[32 * j];
    a += t.diag(j) * zj * zj;
    if (j + 1 < m) a += 2.0 * t.off(j) * zj * z[32 * (j + 1)];
    n2 += zj * zj;
  }
  ztz = a;
  zz = n2;
}

// ||T z - lambda z||^2 for one lane's interleaved z.
__device__ __forceinline__ double resid2_serial(const TbarView& t, const double* z, double lambda) {
  const int k = t.k, m = t.m;
  const double zk = z[32 * k];
  double r2 = 0.0, ak = 0.0;
  for (int i = 0; i < k; ++i) {
    const double zi = z[32 * i];
    const double v = t.diag(i) * zi + t.arrow(i) * zk - lambda * zi;
    r2 += v * v;
    ak += t.arrow(i) * zi;
  }
  for (int j = k; j < m; ++j) {
    double v = (t.diag(j) - lambda) * z[32 * j];
    if (j == k) v += ak;
    else v += t.off(j - 1) * z[32 * (j - 1)];
    if (j + 1 < m) v += t.off(j) * z[32 * (j + 1)];
    r2 += v * v;
  }
  return r2;
}

// The kk wanted eigenpairs of the leading m x m block of T-bar (restart size k), sorted toward the
// wanted end, into lam and Z (column-major, ld m).  FP32 multisection on the inertia count of a float
// copy of T-bar brackets each eigenvalue (one warp per pair, 32 shifts a round); then each pair gets
// one LANE for the FP64 part -- inverse iteration with Rayleigh-quotient shifts (three solves), the
// inertia check on both sides of the result (Sylvester), and the residual and norm checks -- so each
// FP64 warp instruction serves up to 32 pairs.  *ok is cleared if any check fails.
// Scratch: Tf (3m floats), br (2 kk floats), zb and ipb (32 m doubles per group of 32 pairs).
__device__ void cta_ritz(const double* T, int ldt, int m, int k, int kk, int which, double tmax, float* Tf, float* br,
                         double* zb, double* ipb, double* lam, double* Z, double* red, int* ok) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const TbarView t{T, ldt, m, k};
  float* d = Tf;
  float* a = Tf + m;
  float* e = Tf + 2 * m;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    d[j] = (float)t.diag(j);
    a[j] = j < k ? (float)t.arrow(j) : 0.f;
    e[j] = (j >= k && j + 1 < m) ? (float)t.off(j) : 0.f;
  }
  if (w == 0) {   // Gershgorin interval
    double glo = 1e300, ghi = -1e300;
    for (int j = lane; j < m; j += 32) {
      double rad = 0.0;
      if (j < k) rad = fabs(t.arrow(j));
      else {
        if (j == k)
          for (int q = 0; q < k; ++q) rad += fabs(t.arrow(q));
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
    if (lane == 0) {
      const double tn = fmax(fabs(glo), fabs(ghi));
      red[40] = glo - (1e-6 * tn + 1e-300);
      red[41] = ghi + (1e-6 * tn + 1e-300);
      red[42] = tn;
    }
  }
  __syncthreads();
  const double tnorm = red[42];
  const float pmin32 = (float)(tnorm * 1e-30) + 1e-30f;
  for (int i = w; i < kk; i += nw) {   // FP32 multisection, keep count(lo) <= r < count(hi)
    const int r = (which == JTRLAN_LARGEST) ? m - 1 - i : i;
    float lo = (float)red[40], hi = (float)red[41];
    for (int round = 0; round < 8; ++round) {
      const float wd = (hi - lo) / 33.0f;
      const float sig = lo + wd * (float)(lane + 1);
      const int cnt = inertia_f32(d, a, e, m, k, sig, pmin32);
      const unsigned below = __ballot_sync(0xffffffffu, cnt <= r);
      const int nb = __popc(below);
      const float nlo = nb > 0 ? __shfl_sync(0xffffffffu, sig, nb - 1) : lo;
      const float nhi = nb < 32 ? __shfl_sync(0xffffffffu, sig, nb) : hi;
      lo = nlo;
      hi = nhi;
      if (hi - lo <= 4.0f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
    }
    if (lane == 0) {
      br[2 * i] = lo;
      br[2 * i + 1] = hi;
    }
  }
  __syncthreads();
  const int groups = (kk + 31) / 32;
  if (w < groups) {
    const int i = 32 * w + lane;
    if (i < kk) {
      const int r = (which == JTRLAN_LARGEST) ? m - 1 - i : i;
      double* z = zb + (size_t)w * 32 * m + lane;
      double* ip = ipb + (size_t)w * 32 * m + lane;
      const double lo64 = (double)br[2 * i], hi64 = (double)br[2 * i + 1];
      const double slack = 1e-6 * tnorm;           // FP32 rounding of T moves eigenvalues by ~6e-8 ||T||
      const double pivmin = 1e-18 * tnorm + 1e-300;
      double sigma = 0.5 * (lo64 + hi64);
      double nrm = 0.0;
      for (int q = 0; q < m; ++q) {
        const double v = u01_sym(0x9E37ull * (uint64_t)(r + 1) + (uint64_t)q) + 0.5;
        z[32 * q] = v;
        nrm += v * v;
      }
      double inv = 1.0 / sqrt(nrm);
      for (int q = 0; q < m; ++q) z[32 * q] *= inv;
      double lambda = sigma;
      for (int it = 0; it < 3; ++it) {
        solve_serial(t, sigma, pivmin, z, ip);
        double ztz, zz;
        rayleigh_serial(t, z, ztz, zz);
        inv = 1.0 / sqrt(zz);
        for (int q = 0; q < m; ++q) z[32 * q] *= inv;
        lambda = ztz / zz;
        if (lambda >= lo64 - slack && lambda <= hi64 + slack) sigma = lambda;
      }
      const double delta = 1e-9 * tnorm;
      const int c_lo = inertia_f64_serial(t, lambda - delta, pivmin);
      const int c_hi = inertia_f64_serial(t, lambda + delta, pivmin);
      const double r2 = resid2_serial(t, z, lambda);
      double nn = 0.0;
      for (int q = 0; q < m; ++q) {
        const double v = z[32 * q];
        Z[(size_t)i * m + q] = v;
        nn += v * v;
      }
      lam[i] = lambda;
      const bool good = c_lo <= r && c_hi >= r + 1 && lambda == lambda && sqrt(r2) <= 1e-11 * fmax(tmax, 1e-300) &&
                        fabs(nn - 1.0) <= 1e-12;
      if (!good) *ok = 0;
    }
  }
  __syncthreads();
}

// One-CTA cyclic Jacobi (sequential pairs, parallel row/column updates) for the fallback; sorts the
// kk pairs nearest the wanted end into lam / Z (column-major, ld m).  A: m*m scratch, Q: m*m.
__device__ void cta_jacobi(const double* T, int ld, int m, int kk, int which, double* A, double* Q, double* lam,
                           double* Z, int* idx) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e % m;
    A[e] = T[r * ld + c];
    Q[e] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ double cs[2];
  __shared__ int rotated;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        if (threadIdx.x == 0) {
          const double app = A[p * m + p], aqq = A[q * m + q], apq = A[p * m + q];
          double c = 1.0, s = 0.0;
          if (fabs(apq) > 1e-17 * (fabs(app) + fabs(aqq)) && fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            rotated = 1;
          }
          cs[0] = c; cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          for (int l = threadIdx.x; l < m; l += blockDim.x) {   // rows p, q
            const double ap = A[p * m + l], aq = A[q * m + l];
            A[p * m + l] = c * ap - s * aq;
            A[q * m + l] = s * ap + c * aq;
          }
          __syncthreads();
          for (int l = threadIdx.x; l < m; l += blockDim.x) {   // columns p, q and Q
            const double ap = A[l * m + p], aq = A[l * m + q];
            A[l * m + p] = c * ap - s * aq;
            A[l * m + q] = s * ap + c * aq;
            const double zp = Q[l * m + p], zq = Q[l * m + q];
            Q[l * m + p] = c * zp - s * zq;
            Q[l * m + q] = s * zp + c * zq;
          }
          __syncthreads();
        }
      }
    }
    __syncthreads();
    if (!rotated) break;
  }
  if (threadIdx.x == 0) {   // selection by rank toward the wanted end
    for (int i = 0; i < m; ++i) idx[i] = i;
    for (int i = 0; i < kk; ++i) {
      int best = i;
      for (int q = i + 1; q < m; ++q) {
        const double lq = A[idx[q] * m + idx[q]], lb = A[idx[best] * m + idx[best]];
        if (which == JTRLAN_LARGEST ? lq > lb : lq < lb) best = q;
      }
      const int t = idx[i]; idx[i] = idx[best]; idx[best] = t;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * m; e += blockDim.x) {
    const int c = e / m, l = e % m;
    Z[(size_t)c * m + l] = Q[l * m + idx[c]];
  }
  for (int c = threadIdx.x; c < kk; c += blockDim.x) lam[c] = A[idx[c] * m + idx[c]];
  __syncthreads();
}

// MVR: rows of the product a warp takes at once (the tile shape jtrlan_batch_set_tiles selects; a
// template parameter, so that each instance holds one code path and its registers).
template <bool DF, int MVR>
__global__ void __launch_bounds__(kBatchMaxThreads) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Shared S;
  const int m = a.m, nev = a.nev, kk = a.kk, ldt = m + 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const BatchSmem L(a.nmax, m, kk, blockDim.x);
  double* T = (double*)(dyn + L.T);
  double* Z = (double*)(dyn + L.Z);
  float2* Zf = (float2*)(dyn + L.Zf);
  float* Tf = (float*)(dyn + L.Tf);
  float* brk = (float*)(dyn + L.br);
  double* zb = (double*)(dyn + L.zb);
  float* part = (float*)(dyn + L.part);
  double2* x = (double2*)(dyn + L.vec);             // v_j (FP64), nmax
  double2* y = x + a.nmax;                          // the vector being built, nmax
  float4* x4 = (float4*)(y + a.nmax);               // v_j as (hi, lo), nmax (double-float form)
  void* V = (char*)a.Vslots + (size_t)blockIdx.x * a.nmax * (m + 1) * 16;
  double2* Vt = (double2*)a.Tslots + (size_t)blockIdx.x * a.nmax * kk;
  const double sqrt2 = 1.4142135623730951;
  while (true) {
    if (threadIdx.x == 0) S.inst = atomicAdd(a.queue, 1);
    __syncthreads();
    const int qi = S.inst;
    __syncthreads();
    if (qi >= a.count) break;
    const int inst = a.order[qi];
    const int64_t h = a.h[inst], n = 2 * h, off = a.a_off[inst];
    auto vcol = [&](int c) -> char* { return (char*)V + (size_t)c * n * 16; };
    auto store_v = [&](int c, int64_t p, double2 v) {
      if (DF) ((float4*)vcol(c))[p] = b_split(v);
      else ((double2*)vcol(c))[p] = v;
    };
    // ---- v_1 = (1, ..., 1) / sqrt(n) (Algorithm 1); T-bar = 0
    const double v0 = 1.0 / sqrt((double)n);
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) store_v(0, p, make_double2(v0, 0.0));
    for (int e = threadIdx.x; e < ldt * ldt; e += blockDim.x) T[e] = 0.0;
    if (threadIdx.x == 0) {
      S.k = 0; S.icnv = 0; S.status = 0; S.tmax = 0.0; S.nlocked = 0;
    }
    __syncthreads();
    int n_mv = 0, n_res = 0, restarts = 0, n_fb = 0, n_gs = 0;
    bool converged = false;
    long long tp[kBatchPhases] = {0, 0, 0, 0, 0}, tlast = (a.prof && threadIdx.x == 0) ? clock64() : 0;
    // SM cycles since the last mark, charged to phase ph (thread 0, after a barrier)
    auto mark = [&](int ph) {
      if (a.prof && threadIdx.x == 0) {
        const long long t = clock64();
        tp[ph] += t - tlast;
        tlast = t;
      }
    };
    for (; restarts < a.max_restarts; ++restarts) {
      const int k = S.k;
      // ---- Algorithm 2: Lanczos steps k .. m-1
      for (int j = k; j < m; ++j) {
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
          if (DF) {
            const float4 v = ((const float4*)vcol(j))[p];
            x4[p] = v;
            x[p] = b_join(v);
          } else {
            x[p] = ((const double2*)vcol(j))[p];
          }
        }
        __syncthreads();
        cta_matvec<DF, MVR>(a, h, off, x, x4, y, S.red);
        ++n_mv;
        double al = 0.0;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) al += x[p].x * y[p].x + x[p].y * y[p].y;
        al = blk_sum(al, S.red);                                  // t_{j,j} = Re(v_j^H A v_j)
        double nrm = 0.0;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
          double2 t = y[p];
          t.x -= al * x[p].x;
          t.y -= al * x[p].y;
          y[p] = t;
          nrm += cabs2(t);
        }
        double b0 = sqrt(blk_sum(nrm, S.red)), b1 = b0;
        mark(0);
        for (int pass = 0; pass < a.gs_passes; ++pass) {         // against W_j and V_j, sqrt(2) test
          cta_dot<DF>(V, n, h, j, y, x4, S.coef, S.coef4);
          b1 = sqrt(cta_update<DF>(V, n, h, j, S.coef, S.coef4, y, part, S.red, a.gs_groups));
          ++n_gs;
          if (sqrt2 * b1 > b0) break;
          b0 = b1;
        }
        const double tmax = fmax(S.tmax, fmax(fabs(al), b1));
        const bool brk = !(b1 > 1e-14 * fmax(tmax, 1.0));
        const double inv = brk ? 0.0 : 1.0 / b1;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) store_v(j + 1, p, make_double2(y[p].x * inv, y[p].y * inv));
        __syncthreads();
        if (threadIdx.x == 0) {
          T[j * ldt + j] = al;
          T[(j + 1) * ldt + j] = b1;
          if (j + 1 < m) T[j * ldt + j + 1] = b1;
          S.tmax = tmax;
          if (brk) S.status = JTRLAN_EBREAKDOWN;
        }
        __syncthreads();
        mark(1);
        if (S.status != 0) break;
      }
      if (S.status != 0) break;
      // ---- Rayleigh-Ritz: the kk wanted pairs of T_m, one warp each, each checked
      const double beta_m = T[m * ldt + m - 1];
      if (threadIdx.x == 0) S.ok = 1;
      __syncthreads();
      cta_ritz(T, ldt, m, k, kk, a.which, S.tmax, Tf, brk, zb, zb + (size_t)32 * m * ((kk + 31) / 32), S.lam, Z,
               S.red, &S.ok);
      for (int i = w; i + 1 < kk; i += nw) {   // ordered toward the wanted end, neighbours orthogonal
        double d = 0.0;
        for (int q = lane; q < m; q += 32) d += Z[(size_t)i * m + q] * Z[(size_t)(i + 1) * m + q];
        d = warp_sum(d);
        const bool mono = (a.which == JTRLAN_LARGEST) ? S.lam[i] > S.lam[i + 1] : S.lam[i] < S.lam[i + 1];
        if (lane == 0 && (!mono || !(fabs(d) <= 1e-9))) S.ok = 0;
      }
      __syncthreads();
      if (!S.ok) {
        cta_jacobi(T, ldt, m, kk, a.which, (double*)x, (double*)x + m * m, S.lam, Z, S.perm);
        ++n_fb;
      }
      mark(2);
      // ---- V_m Z for the nev candidates; Krylov-Schur arrow t_{m+1,i} = beta_m z_{m,i}
      if (DF) {
        for (int e = threadIdx.x; e < kk * m; e += blockDim.x) {
          const float zh = (float)Z[e];
          Zf[e] = make_float2(zh, (float)(Z[e] - (double)zh));
        }
        __syncthreads();
      }
      cta_rotate<DF>(V, n, m, Z, Zf, 0, nev, Vt);
      if (threadIdx.x == 0) {
        for (int i = 0; i < kk; ++i) {
          S.lamv[i] = S.lam[i];
          S.arrow[i] = beta_m * Z[(size_t)i * m + m - 1];
        }
        for (int i = 0; i < nev; ++i) {
          S.ev[i] = S.lamv[i];
          S.res_est[i] = fabs(S.arrow[i]);
          S.res[i] = INFINITY;
          S.conv[i] = 0;
        }
      }
      __syncthreads();
      mark(3);
      // ---- true residuals of the candidates whose estimate passes (locked pairs keep theirs)
      for (int i = 0; i < nev; ++i) {
        if (!(S.res_est[i] < a.tol)) continue;
        int hit = -1;
        if (S.res_est[i] < 1e-3 * a.tol)
          for (int q = 0; q < S.nlocked; ++q)
            if (fabs(S.ev[i] - S.locked_ev[q]) <= 1e-12 * fmax(1.0, fabs(S.ev[i]))) {
              hit = q;
              break;
            }
        __syncthreads();
        if (hit >= 0) {
          if (threadIdx.x == 0) {
            S.res[i] = S.locked_res[hit];
            S.conv[i] = 1;
          }
          continue;
        }
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
          const double2 v = Vt[(int64_t)i * n + p];
          x[p] = v;
          if (DF) x4[p] = b_split(v);
        }
        __syncthreads();
        cta_matvec<DF, MVR>(a, h, off, x, x4, y, S.red);
        ++n_res;
        double rr = 0.0;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
          const double dr = y[p].x - S.ev[i] * x[p].x, di = y[p].y - S.ev[i] * x[p].y;
          rr += dr * dr + di * di;
        }
        rr = sqrt(blk_sum(rr, S.red));
        if (threadIdx.x == 0) {
          S.res[i] = rr;
          S.conv[i] = rr < a.tol;
        }
      }
      __syncthreads();
      mark(4);
      // ---- converged pairs to the top (stable), lock them, k of eq. (29)
      if (threadIdx.x == 0) {
        int wpos = 0;
        for (int i = 0; i < nev; ++i)
          if (S.conv[i]) S.perm[wpos++] = i;
        const int icnv = wpos;
        for (int i = 0; i < nev; ++i)
          if (!S.conv[i]) S.perm[wpos++] = i;
        for (int i = nev; i < kk; ++i) S.perm[i] = i;
        double ev2[kMaxNev], res2[kMaxNev], lam2[kMaxM], arr2[kMaxM];
        for (int i = 0; i < kk; ++i) {
          lam2[i] = S.lamv[S.perm[i]];
          arr2[i] = S.arrow[S.perm[i]];
        }
        for (int i = 0; i < nev; ++i) {
          ev2[i] = S.ev[S.perm[i]];
          res2[i] = S.res[S.perm[i]];
        }
        for (int i = 0; i < kk; ++i) {
          S.lamv[i] = lam2[i];
          S.arrow[i] = arr2[i];
        }
        for (int i = 0; i < nev; ++i) {
          S.ev[i] = ev2[i];
          S.res[i] = res2[i];
        }
        for (int i = 0; i < icnv; ++i) {
          S.arrow[i] = 0.0;
          S.locked_ev[i] = S.ev[i];
          S.locked_res[i] = S.res[i];
        }
        S.nlocked = icnv;
        S.icnv = icnv;
        S.k = min(icnv + a.mwin, m - 1);
      }
      __syncthreads();
      if (S.icnv == nev) {
        converged = true;
        break;
      }
      // ---- shrink: kept columns (rotated, permuted) into V, v_{k+1} = v_{m+1}, arrowhead T-bar
      const int knew = S.k;
      cta_rotate<DF>(V, n, m, Z, Zf, nev, knew, Vt);
      for (int c = 0; c < knew; ++c)
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) store_v(c, p, Vt[(int64_t)S.perm[c] * n + p]);
      for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
        if (DF) ((float4*)vcol(knew))[p] = ((const float4*)vcol(m))[p];
        else ((double2*)vcol(knew))[p] = ((const double2*)vcol(m))[p];
      }
      for (int e = threadIdx.x; e < ldt * ldt; e += blockDim.x) T[e] = 0.0;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tm = 0.0;
        for (int i = 0; i < knew; ++i) {
          T[i * ldt + i] = S.lamv[i];
          T[knew * ldt + i] = S.arrow[i];
          T[i * ldt + knew] = S.arrow[i];
          tm = fmax(tm, fmax(fabs(S.lamv[i]), fabs(S.arrow[i])));
        }
        S.tmax = tm;
      }
      __syncthreads();
      mark(3);
    }
    // ---- results, sorted toward the wanted end (stable)
    if (threadIdx.x == 0) {
      int st = S.status;
      if (st == 0 && !converged) st = JTRLAN_ENOCONV;
      for (int i = 0; i < nev; ++i) S.ord[i] = i;
      for (int i = 1; i < nev; ++i) {
        const int t = S.ord[i];
        int q = i - 1;
        while (q >= 0 && ((a.which == JTRLAN_LARGEST) ? S.ev[S.ord[q]] < S.ev[t] : S.ev[S.ord[q]] > S.ev[t])) {
          S.ord[q + 1] = S.ord[q];
          --q;
        }
        S.ord[q + 1] = t;
      }
      for (int i = 0; i < nev; ++i) {
        a.out_ev[(size_t)inst * nev + i] = S.ev[S.ord[i]];
        a.out_res[(size_t)inst * nev + i] = S.res[S.ord[i]];
      }
      int* os = a.out_stats + (size_t)kBatchStats * inst;
      os[0] = n_mv;
      os[1] = restarts + (converged ? 1 : 0);
      os[2] = st;
      os[3] = n_res;
      os[4] = n_fb;
      os[5] = n_gs;
      if (a.prof)
        for (int q = 0; q < kBatchPhases; ++q) a.prof[(size_t)kBatchPhases * inst + q] = tp[q];
    }
    __syncthreads();
    if (converged && a.out_vec) {   // column c: Vt[:, perm[ord[c]]] (the candidates were permuted)
      double2* out = (double2*)a.out_vec + a.vec_off[inst];
      for (int c = 0; c < nev; ++c) {
        const int src = S.perm[S.ord[c]];
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) out[(int64_t)c * n + p] = Vt[(int64_t)src * n + p];
      }
    }
    __syncthreads();
  }
}

__global__ void split_df_inplace_kernel(double2* A, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = A[i];
    ((float4*)A)[i] = b_split(v);
  }
}

__global__ void c64_to_c128_batch_kernel(const float2* in, double2* out, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

}  // namespace

size_t batch_smem_bytes(int64_t nmax, int m, int kk, int threads) { return BatchSmem(nmax, m, kk, threads).total; }

namespace {
const void* batch_fn(bool df, int mv_rows) {
  if (df) return mv_rows == 1 ? (const void*)batch_kernel<true, 1> : (const void*)batch_kernel<true, 2>;
  return mv_rows == 2 ? (const void*)batch_kernel<false, 2> : (const void*)batch_kernel<false, 1>;
}
}  // namespace

cudaError_t batch_occupancy(bool df, int mv_rows, int threads, size_t smem, int* blocks) {
  const void* f = batch_fn(df, mv_rows);
  cudaError_t e = allow_dyn_smem(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, threads, smem);
}

cudaError_t launch_batch(bool df, const BatchArgs& a, int grid, int threads, cudaStream_t s) {
  const size_t sm = batch_smem_bytes(a.nmax, a.m, a.kk, threads);
  if (df) {
    if (a.mv_rows == 1) batch_kernel<true, 1><<<grid, threads, sm, s>>>(a);
    else batch_kernel<true, 2><<<grid, threads, sm, s>>>(a);
  } else {
    if (a.mv_rows == 2) batch_kernel<false, 2><<<grid, threads, sm, s>>>(a);
    else batch_kernel<false, 1><<<grid, threads, sm, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_df_inplace(void* A, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  split_df_inplace_kernel<<<1024, 256, 0, s>>>((double2*)A, count);
  return cudaGetLastError();
}

cudaError_t launch_c64_to_c128(const void* in, void* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  c64_to_c128_batch_kernel<<<1024, 256, 0, s>>>((const float2*)in, (double2*)out, count);
  return cudaGetLastError();
}

}  // namespace jtr
