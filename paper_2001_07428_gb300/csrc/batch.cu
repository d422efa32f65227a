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
// warp-wide compensated sum; the result (as FP64) in every lane
__device__ __forceinline__ double b_warp_df_sum(float s, float e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float so = __shfl_xor_sync(0xffffffffu, s, o), eo = __shfl_xor_sync(0xffffffffu, e, o);
    float t, te;
    b_two_sum(s, so, t, te);
    s = t;
    e = __fadd_rn(e, __fadd_rn(te, eo));
  }
  return (double)s + (double)e;
}

constexpr int kMaxM = kBatchMaxM;
constexpr int kMaxNev = kBatchMaxNev;

// O(m) per-instance state; the O(m^2) and O(n) arrays are in dynamic shared memory (BatchSmem).
struct Shared {
  double coef[(kMaxM + 1) * 4];
  double red[64];
  double lam[kMaxM], lamv[kMaxM], arrow[kMaxM];
  double ev[kMaxNev], res[kMaxNev], res_est[kMaxNev], locked_ev[kMaxNev], locked_res[kMaxNev];
  int perm[kMaxM], ord[kMaxNev], conv[kMaxNev];
  int ok, status, icnv, k, nlocked, inst;
  double tmax;
};

__host__ __device__ inline size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

// Dynamic shared memory: T-bar ((m+1)^2), Z (m x kk), the warps' Ritz scratch (3m each), then the
// vectors x, y (FP64) and x4 ((hi, lo) copy of x), whose space the Jacobi fallback reuses for its
// two m x m arrays.
struct BatchSmem {
  size_t T, Z, rs, vec, total;
  __host__ __device__ BatchSmem(int64_t nmax, int m, int kk, int threads) {
    T = 0;
    Z = T + up16(sizeof(double) * (m + 1) * (m + 1));
    rs = Z + up16(sizeof(double) * m * kk);
    vec = rs + up16(sizeof(double) * 3 * m * (threads / 32));
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

// y = A x (dense block form); x and y in shared memory (FP64), A rows from global.  Returns the
// block-wide Re/Im of x^H y in (*ar, *ai) when requested.
template <bool DF>
__device__ void cta_matvec(const BatchArgs& a, int64_t h, int64_t off, const double2* x, const float4* x4, double2* y,
                           double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t r = w; r < h; r += nw) {
    double v[4];
    if (!DF) {
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
      v[0] = warp_sum(y1.x); v[1] = warp_sum(y1.y); v[2] = warp_sum(y2.x); v[3] = warp_sum(y2.y);
    } else {
      const float4* r11 = (const float4*)a.A11 + off + r * h;
      const float4* r12 = (const float4*)a.A12 + off + r * h;
      float s1[2] = {0.f, 0.f}, e1[2] = {0.f, 0.f}, s2[2] = {0.f, 0.f}, e2[2] = {0.f, 0.f};
      for (int64_t c = lane; c < h; c += 32) {
        const float4 a11 = r11[c], a12 = r12[c], x1 = x4[c], x2 = x4[h + c];
        b_cacc(s1, e1, a11, x1);
        b_cacc(s1, e1, a12, x2);
        b_caccc(s2, e2, a11, x2);
        b_caccc(s2, e2, a12, x1, -1.f);
      }
      v[0] = b_warp_df_sum(s1[0], e1[0]); v[1] = b_warp_df_sum(s1[1], e1[1]);
      v[2] = b_warp_df_sum(s2[0], e2[0]); v[3] = b_warp_df_sum(s2[1], e2[1]);
    }
    if (lane == 0) {
      y[r] = make_double2(v[0], v[1]);
      y[h + r] = make_double2(v[2], v[3]);
    }
  }
  __syncthreads();
}

// c_v = V^H y and c_w = W^H y for columns 0..j (warp w takes columns w, w + nw, ...), into coef.
template <bool DF>
__device__ void cta_dot(const void* Vv, int64_t n, int64_t h, int j, const double2* y, double* coef) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i <= j; i += nw) {
    double c[4];
    if (!DF) {
      const double2* vi = (const double2*)Vv + (int64_t)i * n;
      double2 cv = make_double2(0, 0), cw = make_double2(0, 0);
      for (int64_t p = lane; p < h; p += 32) {
        const double2 v1 = vi[p], v2 = vi[h + p], y1 = y[p], y2 = y[h + p];
        cv = cfmac(v1, y1, cv);
        cv = cfmac(v2, y2, cv);
        cw = cfma(v1, y2, cw);
        cw = cfma(make_double2(-v2.x, -v2.y), y1, cw);
      }
      c[0] = warp_sum(cv.x); c[1] = warp_sum(cv.y); c[2] = warp_sum(cw.x); c[3] = warp_sum(cw.y);
    } else {
      const float4* vi = (const float4*)Vv + (int64_t)i * n;
      float sv[2] = {0.f, 0.f}, ev[2] = {0.f, 0.f}, sw[2] = {0.f, 0.f}, ew[2] = {0.f, 0.f};
      for (int64_t p = lane; p < h; p += 32) {
        const float4 v1 = vi[p], v2 = vi[h + p];
        const float4 y1 = b_split(y[p]), y2 = b_split(y[h + p]);
        b_caccc(sv, ev, v1, y1);
        b_caccc(sv, ev, v2, y2);
        b_cacc(sw, ew, v1, y2);
        b_cacc(sw, ew, v2, y1, -1.f);
      }
      c[0] = b_warp_df_sum(sv[0], ev[0]); c[1] = b_warp_df_sum(sv[1], ev[1]);
      c[2] = b_warp_df_sum(sw[0], ew[0]); c[3] = b_warp_df_sum(sw[1], ew[1]);
    }
    if (lane == 0) {
      coef[4 * i] = c[0]; coef[4 * i + 1] = c[1]; coef[4 * i + 2] = c[2]; coef[4 * i + 3] = c[3];
    }
  }
  __syncthreads();
}

// y -= V c_v + W c_w (each thread a row pair); returns ||y||^2 (block-wide).
template <bool DF>
__device__ double cta_update(const void* Vv, int64_t n, int64_t h, int j, const double* coef, double2* y,
                             double* red) {
  double nrm = 0.0;
  for (int64_t p = threadIdx.x; p < h; p += blockDim.x) {
    double2 y1 = y[p], y2 = y[h + p];
    if (!DF) {
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
    } else {
      const float4* V = (const float4*)Vv;
      float s1[2] = {0.f, 0.f}, e1[2] = {0.f, 0.f}, s2[2] = {0.f, 0.f}, e2[2] = {0.f, 0.f};
      for (int i = 0; i <= j; ++i) {
        const float4 v1 = V[(int64_t)i * n + p], v2 = V[(int64_t)i * n + h + p];
        const float4 cv = b_split(make_double2(coef[4 * i], coef[4 * i + 1]));
        const float4 cw = b_split(make_double2(coef[4 * i + 2], coef[4 * i + 3]));
        b_cacc(s1, e1, v1, cv);
        b_caccc(s1, e1, v2, cw, -1.f);
        b_cacc(s2, e2, v2, cv);
        b_caccc(s2, e2, v1, cw);
      }
      y1.x -= (double)s1[0] + (double)e1[0]; y1.y -= (double)s1[1] + (double)e1[1];
      y2.x -= (double)s2[0] + (double)e2[0]; y2.y -= (double)s2[1] + (double)e2[1];
    }
    y[p] = y1;
    y[h + p] = y2;
    nrm += cabs2(y1) + cabs2(y2);
  }
  return blk_sum(nrm, red);
}

// Vt[:, c] = V Z[:, c] for c in [c0, c1), rows 2n real (FP64 target).
template <bool DF>
__device__ void cta_rotate(const void* Vv, int64_t n, int m, const double* Z, int c0, int c1, double2* Vt) {
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
              const double z = Z[(size_t)(cb + q) * m + i];
              const float zh = (float)z, zl = (float)(z - (double)zh);
              b_df_acc(sr[q], er[q], v.x, v.z, zh, zl);
              b_df_acc(si[q], ei[q], v.y, v.w, zh, zl);
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

template <bool DF>
__global__ void __launch_bounds__(kBatchMaxThreads) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Shared S;
  const int m = a.m, nev = a.nev, kk = a.kk, ldt = m + 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const BatchSmem L(a.nmax, m, kk, blockDim.x);
  double* T = (double*)(dyn + L.T);
  double* Z = (double*)(dyn + L.Z);
  double* rs = (double*)(dyn + L.rs);
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
    int n_mv = 0, n_res = 0, restarts = 0;
    bool converged = false;
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
        cta_matvec<DF>(a, h, off, x, x4, y, S.red);
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
        for (int pass = 0; pass < a.gs_passes; ++pass) {         // against W_j and V_j, sqrt(2) test
          cta_dot<DF>(V, n, h, j, y, S.coef);
          b1 = sqrt(cta_update<DF>(V, n, h, j, S.coef, y, S.red));
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
        if (S.status != 0) break;
      }
      if (S.status != 0) break;
      // ---- Rayleigh-Ritz: the kk wanted pairs of T_m, one warp each, each checked
      const double beta_m = T[m * ldt + m - 1];
      if (threadIdx.x == 0) S.ok = 1;
      __syncthreads();
      for (int i = w; i < kk; i += nw) {
        const int r = (a.which == JTRLAN_LARGEST) ? m - 1 - i : i;
        double* zs = rs + (size_t)w * 3 * m;
        double* zi = Z + (size_t)i * m;
        const double l = ritz_pair_warp(T, ldt, m, k, r, zs, zs + m, zs + 2 * m, zi);
        warp_apply(TbarView{T, ldt, m, k}, zi, zs + 2 * m);
        double rr = 0.0, nn = 0.0;
        for (int q = lane; q < m; q += 32) {
          const double d = zs[2 * m + q] - l * zi[q];
          rr += d * d;
          nn += zi[q] * zi[q];
        }
        rr = warp_sum(rr);
        nn = warp_sum(nn);
        if (lane == 0) {
          S.lam[i] = l;
          if (!(l == l) || !(sqrt(rr) <= 1e-11 * fmax(S.tmax, 1e-300)) || !(fabs(nn - 1.0) <= 1e-12)) S.ok = 0;
        }
        __syncwarp();
      }
      __syncthreads();
      for (int i = w; i + 1 < kk; i += nw) {   // ordered toward the wanted end, neighbours orthogonal
        double d = 0.0;
        for (int q = lane; q < m; q += 32) d += Z[(size_t)i * m + q] * Z[(size_t)(i + 1) * m + q];
        d = warp_sum(d);
        const bool mono = (a.which == JTRLAN_LARGEST) ? S.lam[i] > S.lam[i + 1] : S.lam[i] < S.lam[i + 1];
        if (lane == 0 && (!mono || !(fabs(d) <= 1e-9))) S.ok = 0;
      }
      __syncthreads();
      if (!S.ok) cta_jacobi(T, ldt, m, kk, a.which, (double*)x, (double*)x + m * m, S.lam, Z, S.perm);
      // ---- V_m Z for the nev candidates; Krylov-Schur arrow t_{m+1,i} = beta_m z_{m,i}
      cta_rotate<DF>(V, n, m, Z, 0, nev, Vt);
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
        cta_matvec<DF>(a, h, off, x, x4, y, S.red);
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
      cta_rotate<DF>(V, n, m, Z, nev, knew, Vt);
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
      a.out_stats[4 * inst] = n_mv;
      a.out_stats[4 * inst + 1] = restarts + (converged ? 1 : 0);
      a.out_stats[4 * inst + 2] = st;
      a.out_stats[4 * inst + 3] = n_res;
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

cudaError_t batch_occupancy(bool df, int threads, size_t smem, int* blocks) {
  cudaError_t e = df ? cudaFuncSetAttribute(batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                     : cudaFuncSetAttribute(batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return df ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_kernel<true>, threads, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_kernel<false>, threads, smem);
}

cudaError_t launch_batch(bool df, const BatchArgs& a, int grid, int threads, cudaStream_t s) {
  const size_t sm = batch_smem_bytes(a.nmax, a.m, a.kk, threads);
  if (df) batch_kernel<true><<<grid, threads, sm, s>>>(a);
  else batch_kernel<false><<<grid, threads, sm, s>>>(a);
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
