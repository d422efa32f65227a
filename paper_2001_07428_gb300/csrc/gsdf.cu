// gsdf.cu -- the Gram-Schmidt part of Algorithm 2 in compensated FP32 ("double-float") arithmetic,
// for the mixed-precision forms.
//
// On this GPU the FP64 pipe runs at 1/64 of the FP32 rate, and in plain FP64 the reorthogonalisation
// against V and W = J V^* is bound by it.  Here the basis is stored as pairs of FP32 numbers,
// v = hi + lo (hi = fl32(v), lo = fl32(v - hi): 48 significant bits), the products use the exact
// FMA split p + e = a*b (Dekker 1971; e = fma(a, b, -p)), and the sums use Knuth's TwoSum with the
// rounding errors carried in a second accumulator (the Dot2 scheme of Ogita, Rump & Oishi 2005).
// The inner products and the update come out with errors of a few 1e-15 relative to ||v|| ||y||,
// which keeps V^H V = I and V^H W = O at FP64 level; the vector y itself, alpha, beta, the norms,
// the matvec, the Ritz solve and the residuals stay in FP64.
//
// Layout: V4[col * n + i] = {hi.re, hi.im, lo.re, lo.im} (float4); xbuf holds v_j in FP64 for the
// FP64 matvec.  The kernel sequence and the device-side exit test mirror gs.cu.
#include <cooperative_groups.h>

#include "internal.h"

namespace jtr {

namespace {

constexpr int kThreads = 256;
constexpr int kGroups = kThreads / 32;
// Dot kernels: one column per warp chunk (measured best on GB300 at 16^4: 2.2x faster than 8-column
// chunks).  Their shared memory (the split of y over a block's rows) holds them to two blocks per SM
// on the largest lattices, so they may use up to 128 registers: room for the pipelined loads.
constexpr int kCols = 1;             // columns per warp chunk in the dot kernels (4 * kCols <= 32)
constexpr int kDotMinBlocks = 2;
constexpr double kSqrt2 = 1.4142135623730951;

// ------------------------------------------------------------------ error-free building blocks
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {   // s + e = a + b
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, e) += (ah + al) * (bh + bl): ah * bh split exactly into the sum (TwoSum) and its rounding
// error, the cross terms ah * bl and al * bh (first order) fused into the error sum -- 12 FP32 ops.
__device__ __forceinline__ void df_acc(float& s, float& e, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  float t, te;
  two_sum(s, p, t, te);
  s = t;
  e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fadd_rn(e, __fadd_rn(te, pe))));
}
__device__ __forceinline__ void df_sub(float& s, float& e, float ah, float al, float bh, float bl) {
  df_acc(s, e, -ah, -al, bh, bl);
}
// (s, e) += a * (bh + bl) for an a that is exact in FP32 (a complex64 link): the exact split of
// a * bh into the sum, a * bl and the rounding errors into e -- 11 FP32 operations.
__device__ __forceinline__ void df_acc_xa(float& s, float& e, float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  const float pe = __fmaf_rn(a, bh, -p);
  float t, te;
  two_sum(s, p, t, te);
  s = t;
  e = __fmaf_rn(a, bl, __fadd_rn(e, __fadd_rn(te, pe)));
}

__device__ __forceinline__ float4 split(double2 v) {
  const float hx = (float)v.x, hy = (float)v.y;
  return make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}
__device__ __forceinline__ double2 join(float4 f) {
  return make_double2((double)f.x + (double)f.z, (double)f.y + (double)f.w);
}

// ------------------------------------------------------------------ inner products (one pass)
// c_v,i = sum_p conj(v1) y1 + conj(v2) y2 and c_w,i = sum_p (v1 y2 - v2 y1) for columns 0..j over
// rows [p0, p1); y has been split into ys (shared, [2][rows]).  Warp q takes chunks of 8 columns;
// each lane keeps 8 x 4 (sum, error) pairs, combines them to FP64 and the warp transposes them
// through shared memory so that lane k adds up accumulator k.
// 16 compensated products of one row pair (v1, v2) of a column with (y1, y2) into the four sums.
__device__ __forceinline__ void dfdot_row(float* s, float* e, float4 v1, float4 v2, float4 y1, float4 y2) {
  // Re c_v: v1.x y1.x + v1.y y1.y + v2.x y2.x + v2.y y2.y
  df_acc(s[0], e[0], v1.x, v1.z, y1.x, y1.z);
  df_acc(s[0], e[0], v1.y, v1.w, y1.y, y1.w);
  df_acc(s[0], e[0], v2.x, v2.z, y2.x, y2.z);
  df_acc(s[0], e[0], v2.y, v2.w, y2.y, y2.w);
  // Im c_v: v1.x y1.y - v1.y y1.x + v2.x y2.y - v2.y y2.x
  df_acc(s[1], e[1], v1.x, v1.z, y1.y, y1.w);
  df_sub(s[1], e[1], v1.y, v1.w, y1.x, y1.z);
  df_acc(s[1], e[1], v2.x, v2.z, y2.y, y2.w);
  df_sub(s[1], e[1], v2.y, v2.w, y2.x, y2.z);
  // Re c_w: v1.x y2.x - v1.y y2.y - v2.x y1.x + v2.y y1.y
  df_acc(s[2], e[2], v1.x, v1.z, y2.x, y2.z);
  df_sub(s[2], e[2], v1.y, v1.w, y2.y, y2.w);
  df_sub(s[2], e[2], v2.x, v2.z, y1.x, y1.z);
  df_acc(s[2], e[2], v2.y, v2.w, y1.y, y1.w);
  // Im c_w: v1.x y2.y + v1.y y2.x - v2.x y1.y - v2.y y1.x
  df_acc(s[3], e[3], v1.x, v1.z, y2.y, y2.w);
  df_acc(s[3], e[3], v1.y, v1.w, y2.x, y2.z);
  df_sub(s[3], e[3], v2.x, v2.z, y1.y, y1.w);
  df_sub(s[3], e[3], v2.y, v2.w, y1.x, y1.z);
}

// ------------------------------------------------------------------ inner products (one pass)
// c_v,i = sum_p conj(v1) y1 + conj(v2) y2 and c_w,i = sum_p (v1 y2 - v2 y1) for columns 0..j over
// rows [p0, p1); y has been split into ys (shared, [2][rows]).  Warp q takes one column at a time
// (q, q + 8, ...); each lane walks four rows at a time and keeps 4 (sum, error) pairs, combines them
// to FP64 and the warp transposes them through shared memory so that lane k adds up accumulator k.
// Pipelined (the separate launches, two blocks per SM): the next four rows' eight loads of V are
// issued before the current four rows' arithmetic, so each warp keeps 8 KB in flight.
template <bool Pipelined>
__device__ void dfdot_body(const GSArgs& a, int64_t p0, int64_t p1, const float4* ys, float* red, int rb) {
  static_assert(kCols == 1, "one column per warp chunk");
  const float4* V = (const float4*)a.V;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t n = a.n, h = a.h, rows = p1 - p0;
  float* wred_s = red + (size_t)q * 2 * (4 * kCols) * 33;   // sums, then rounding errors, [4 kCols][33]
  float* wred_e = wred_s + (4 * kCols) * 33;
  for (int c0 = q; c0 <= a.j; c0 += kGroups) {
    float s[1][4], e[1][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) s[0][t] = e[0][t] = 0.f;
    const int ncol = 1;
    const float4* vi = V + (int64_t)c0 * n + p0;
    int64_t r0 = lane;
    if (Pipelined) {
      if (r0 + 96 < rows) {
        float4 a1[4], a2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a1[u] = vi[r0 + 32 * u];
          a2[u] = vi[h + r0 + 32 * u];
        }
        for (;;) {
          const int64_t rn = r0 + 128;
          const bool more = rn + 96 < rows;
          float4 b1[4], b2[4];
          if (more) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              b1[u] = vi[rn + 32 * u];
              b2[u] = vi[h + rn + 32 * u];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) dfdot_row(s[0], e[0], a1[u], a2[u], ys[r0 + 32 * u], ys[rows + r0 + 32 * u]);
          r0 = rn;
          if (!more) break;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            a1[u] = b1[u];
            a2[u] = b2[u];
          }
        }
      }
    } else {
      // four rows per lane: their eight loads of V are issued before the arithmetic, so a warp keeps
      // 4 KB in flight (the basis is read from HBM once per pass and the y tile sits in shared memory)
      for (; r0 + 96 < rows; r0 += 128) {
        float4 v1u[4], v2u[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v1u[u] = vi[r0 + 32 * u];
          v2u[u] = vi[h + r0 + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) dfdot_row(s[0], e[0], v1u[u], v2u[u], ys[r0 + 32 * u], ys[rows + r0 + 32 * u]);
      }
    }
    for (int64_t r = r0; r < rows; r += 32) dfdot_row(s[0], e[0], vi[r], vi[h + r], ys[r], ys[rows + r]);
#pragma unroll
    for (int c = 0; c < kCols; ++c)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        wred_s[(4 * c + t) * 33 + lane] = s[c][t];
        wred_e[(4 * c + t) * 33 + lane] = e[c][t];
      }
    __syncwarp();
    // lane k adds up accumulator k over the 32 lanes, still compensated; one FP64 conversion
    float S = 0.f, E = 0.f;
    if (lane < 4 * kCols) {
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        float t, te;
        two_sum(S, wred_s[lane * 33 + l], t, te);
        S = t;
        E = __fadd_rn(E, __fadd_rn(te, wred_e[lane * 33 + l]));
      }
    }
    __syncwarp();
    const int c = lane >> 2, t = lane & 3;
    if (lane < 4 * kCols && c < ncol)
      a.part_dot[((int64_t)(c0 + c) * a.nblk + rb) * 4 + t] = (double)S + (double)E;
  }
}

// shared-memory layout of the dot kernels: ys [2 * rows_per_block] float4, then the reduction buffer
__device__ __forceinline__ void split_rows(const GSArgs& a, int64_t p0, int64_t p1, float4* ys) {
  const double2* y = (const double2*)a.y;
  const int64_t rows = p1 - p0;
  for (int64_t r = threadIdx.x; r < rows; r += kThreads) {
    ys[r] = split(y[p0 + r]);
    ys[rows + r] = split(y[a.h + p0 + r]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, kDotMinBlocks)
gsdf_first_kernel(GSArgs a, const double2* __restrict__ x, const double2* __restrict__ alpha_part, int n_alpha_part) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double sh[32];
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_alpha_part; i += kThreads) {
    ar += alpha_part[i].x;
    ai += alpha_part[i].y;
  }
  ar = block_sum(ar, sh);
  ai = block_sum(ai, sh);
  const int j = a.j;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.T[(int64_t)j * a.ldt + j] = ar;                 // t_{j,j} (its real part)
    StepState* st = a.st;
    st->alpha_im = ai;
    st->done = 0;
    double tm = fmax(st->tmax, fabs(ar));
    if (j > 0) tm = fmax(tm, fabs(a.T[(int64_t)j * a.ldt + j - 1]));
    st->tmax = tm;
    st->n_passes += 1;
    st->units_first += (double)(j + 1) * (double)a.h;
  }
  double2* y = (double2*)a.y;
  const int64_t h = a.h;
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
  double nrm = 0.0;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {   // y -= alpha v_j, exactly in FP64
    double2 y1 = y[p], y2 = y[h + p];
    const double2 v1 = x[p], v2 = x[h + p];
    y1.x -= ar * v1.x; y1.y -= ar * v1.y;
    y2.x -= ar * v2.x; y2.y -= ar * v2.y;
    y[p] = y1;
    y[h + p] = y2;
    nrm += cabs2(y1) + cabs2(y2);
  }
  nrm = block_sum(nrm, sh);
  if (threadIdx.x == 0) a.part_nrm[blockIdx.x] = nrm;
  float4* ys = (float4*)dyn;
  float* red = (float*)(ys + 2 * a.rows_per_block);
  split_rows(a, p0, p1, ys);
  dfdot_body<true>(a, p0, p1, ys, red, blockIdx.x);
}

__global__ void __launch_bounds__(kThreads, kDotMinBlocks) gsdf_dot_kernel(GSArgs a, int pass) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double sh[32];
  __shared__ int s_skip;
  StepState* st = a.st;
  if (threadIdx.x == 0) s_skip = st->done;
  __syncthreads();
  if (s_skip) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < a.nblk; b += kThreads) s += a.part_nrm[b];
  const double nrm_prev = sqrt(block_sum(s, sh));   // b1 after pass - 1
  const double ref = st->nrm[pass - 2];              // b0 before pass - 1
  if (kSqrt2 * nrm_prev > ref) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->nrm[pass - 1] = nrm_prev;
      st->beta = nrm_prev;
      st->done = 1;
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->nrm[pass - 1] = nrm_prev;
    st->n_passes += 1;
    st->units_dot += (double)(a.j + 1) * (double)a.h;
  }
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, a.h);
  float4* ys = (float4*)dyn;
  float* red = (float*)(ys + 2 * a.rows_per_block);
  split_rows(a, p0, p1, ys);
  dfdot_body<true>(a, p0, p1, ys, red, blockIdx.x);
}

// The update's coefficients in shared memory, classified once per launch (every block alike):
// column i is "large" when some component of c_v or c_w exceeds thr = 2^-23 ||y|| / ((j+1)(j+4)).
// Large columns are applied in compensated FP32 from their (hi, lo) splits scf[2i], scf[2i+1]; the
// others enter one plain FP32 sum through csm[i] = (c_v.re, c_v.im, c_w.re, c_w.im) rounded to FP32
// (zero for a large column), with the hi parts of V.  Each term of that sum is off by at most
// (j + 4) 2^-24 of |v c| (product, the dropped lo parts, the recursive sum), so the whole plain part
// errs by at most (j+4) 2^-24 sum_i |c_i| <= 2^-47 ||y||, the level of the compensated dots' own
// error.  (With 2^-27, a 2^-51 bound, the rounding-size coefficients of the filtered phase lay just
// above the threshold once the filter's products carried their sums at about 2^-41, and most columns
// took the compensated path: 1.10 against 0.67 ms an update at 24^3 x 48.)
// In a Lanczos step nearly every coefficient is of rounding size (exactly, only beta_{j-1} and, after
// a restart, the arrow couplings are not), so the update costs about one read of V instead of 16
// compensated products per row pair and column.
struct UpdCoef {
  float4* scf;          // [2 (m+1)] (hi, lo) splits of c_v, c_w
  float4* csm;          // [m+1] FP32 coefficients of the plain sum (zero for large columns)
  unsigned char* big;   // [m+1] 1 for a large column
};

__device__ __forceinline__ void classify_coefs(const coef4* coef, int j, double ynorm, UpdCoef u) {
  const double thr = ldexp(ynorm, -23) / ((double)(j + 1) * (double)(j + 4));
  for (int i = threadIdx.x; i <= j; i += kThreads) {
    const coef4 c = coef[i];
    u.scf[2 * i] = split(make_double2(c.vr, c.vi));
    u.scf[2 * i + 1] = split(make_double2(c.wr, c.wi));
    const bool large = fmax(fmax(fabs(c.vr), fabs(c.vi)), fmax(fabs(c.wr), fabs(c.wi))) > thr;
    u.big[i] = large ? 1 : 0;
    u.csm[i] = large ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4((float)c.vr, (float)c.vi, (float)c.wr, (float)c.wi);
  }
}

// y -= V c_v + W c_w over rows [p0, p1): warp q owns rows p0 + 32 q + lane, then + 256, ...; the
// small columns go into a plain FP32 sum (four columns' loads in flight), the large ones into a
// compensated one; both are converted once and applied to y in FP64 by the warp that owns the row:
// no cross-warp reduction and no barrier.  Returns this thread's share of ||y||^2.  The branch
// depends only on the block's row range, so it is uniform across the block (dfupdate_split has
// barriers).  Blocks with fewer than 256 rows (the small lattices' cooperative partition) take
// dfupdate_split instead, so that no warp idles; it applies every column in compensated FP32.
__device__ double dfupdate_split(const GSArgs& a, int64_t p0, int64_t p1, const float4* scf, float (*red_s)[32][4],
                                 float (*red_e)[32][4]);
__device__ double dfupdate_rows(const GSArgs& a, int64_t p0, int64_t p1, UpdCoef u, float (*red_s)[32][4],
                                float (*red_e)[32][4]) {
  if (p1 - p0 < 32 * kGroups) return dfupdate_split(a, p0, p1, u.scf, red_s, red_e);
  const float4* V = (const float4*)a.V;
  double2* y = (double2*)a.y;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t n = a.n, h = a.h;
  const int j = a.j;
  const float4* scf = u.scf;
  double nrm = 0.0;
  for (int64_t p = p0 + 32 * q + lane; p < p1; p += 32 * kGroups) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f}, sp[4] = {0.f, 0.f, 0.f, 0.f};
    int i = 0;
    for (; i + 3 <= j; i += 4) {
      float4 v1u[4], v2u[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        v1u[t] = V[(int64_t)(i + t) * n + p];
        v2u[t] = V[(int64_t)(i + t) * n + h + p];
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float4 v1 = v1u[t], v2 = v2u[t], c = u.csm[i + t];   // c = (cv.re, cv.im, cw.re, cw.im)
        // y1 correction: v1 c_v - conj(v2) c_w;  y2 correction: v2 c_v + conj(v1) c_w
        sp[0] = __fmaf_rn(v1.x, c.x, sp[0]); sp[0] = __fmaf_rn(-v1.y, c.y, sp[0]);
        sp[0] = __fmaf_rn(-v2.x, c.z, sp[0]); sp[0] = __fmaf_rn(-v2.y, c.w, sp[0]);
        sp[1] = __fmaf_rn(v1.x, c.y, sp[1]); sp[1] = __fmaf_rn(v1.y, c.x, sp[1]);
        sp[1] = __fmaf_rn(-v2.x, c.w, sp[1]); sp[1] = __fmaf_rn(v2.y, c.z, sp[1]);
        sp[2] = __fmaf_rn(v2.x, c.x, sp[2]); sp[2] = __fmaf_rn(-v2.y, c.y, sp[2]);
        sp[2] = __fmaf_rn(v1.x, c.z, sp[2]); sp[2] = __fmaf_rn(v1.y, c.w, sp[2]);
        sp[3] = __fmaf_rn(v2.x, c.y, sp[3]); sp[3] = __fmaf_rn(v2.y, c.x, sp[3]);
        sp[3] = __fmaf_rn(v1.x, c.w, sp[3]); sp[3] = __fmaf_rn(-v1.y, c.z, sp[3]);
      }
    }
    for (; i <= j; ++i) {
      const float4 v1 = V[(int64_t)i * n + p], v2 = V[(int64_t)i * n + h + p], c = u.csm[i];
      sp[0] = __fmaf_rn(v1.x, c.x, sp[0]); sp[0] = __fmaf_rn(-v1.y, c.y, sp[0]);
      sp[0] = __fmaf_rn(-v2.x, c.z, sp[0]); sp[0] = __fmaf_rn(-v2.y, c.w, sp[0]);
      sp[1] = __fmaf_rn(v1.x, c.y, sp[1]); sp[1] = __fmaf_rn(v1.y, c.x, sp[1]);
      sp[1] = __fmaf_rn(-v2.x, c.w, sp[1]); sp[1] = __fmaf_rn(v2.y, c.z, sp[1]);
      sp[2] = __fmaf_rn(v2.x, c.x, sp[2]); sp[2] = __fmaf_rn(-v2.y, c.y, sp[2]);
      sp[2] = __fmaf_rn(v1.x, c.z, sp[2]); sp[2] = __fmaf_rn(v1.y, c.w, sp[2]);
      sp[3] = __fmaf_rn(v2.x, c.y, sp[3]); sp[3] = __fmaf_rn(v2.y, c.x, sp[3]);
      sp[3] = __fmaf_rn(v1.x, c.w, sp[3]); sp[3] = __fmaf_rn(-v1.y, c.z, sp[3]);
    }
    for (i = 0; i <= j; ++i) {     // the large columns, compensated (uniform branch: same column for all)
      if (!u.big[i]) continue;
      const float4 v1 = V[(int64_t)i * n + p], v2 = V[(int64_t)i * n + h + p];
      const float4 cv = scf[2 * i], cw = scf[2 * i + 1];
      df_acc(s[0], e[0], v1.x, v1.z, cv.x, cv.z);  df_sub(s[0], e[0], v1.y, v1.w, cv.y, cv.w);
      df_sub(s[0], e[0], v2.x, v2.z, cw.x, cw.z);  df_sub(s[0], e[0], v2.y, v2.w, cw.y, cw.w);
      df_acc(s[1], e[1], v1.x, v1.z, cv.y, cv.w);  df_acc(s[1], e[1], v1.y, v1.w, cv.x, cv.z);
      df_sub(s[1], e[1], v2.x, v2.z, cw.y, cw.w);  df_acc(s[1], e[1], v2.y, v2.w, cw.x, cw.z);
      df_acc(s[2], e[2], v2.x, v2.z, cv.x, cv.z);  df_sub(s[2], e[2], v2.y, v2.w, cv.y, cv.w);
      df_acc(s[2], e[2], v1.x, v1.z, cw.x, cw.z);  df_acc(s[2], e[2], v1.y, v1.w, cw.y, cw.w);
      df_acc(s[3], e[3], v2.x, v2.z, cv.y, cv.w);  df_acc(s[3], e[3], v2.y, v2.w, cv.x, cv.z);
      df_acc(s[3], e[3], v1.x, v1.z, cw.y, cw.w);  df_sub(s[3], e[3], v1.y, v1.w, cw.x, cw.z);
    }
    double2 y1 = y[p], y2 = y[h + p];
    y1.x -= ((double)s[0] + (double)e[0]) + (double)sp[0];
    y1.y -= ((double)s[1] + (double)e[1]) + (double)sp[1];
    y2.x -= ((double)s[2] + (double)e[2]) + (double)sp[2];
    y2.y -= ((double)s[3] + (double)e[3]) + (double)sp[3];
    y[p] = y1;
    y[h + p] = y2;
    nrm += cabs2(y1) + cabs2(y2);
  }
  return nrm;
}

// y -= V c_v + W c_w with every 32-row chunk shared by all warps: warp q takes columns q, q + 8, ...,
// the eight compensated partial sums are added (still compensated) by warp 0, which updates y in FP64.
__device__ double dfupdate_split(const GSArgs& a, int64_t p0, int64_t p1, const float4* scf, float (*red_s)[32][4],
                                 float (*red_e)[32][4]) {
  const float4* V = (const float4*)a.V;
  double2* y = (double2*)a.y;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t n = a.n, h = a.h;
  const int j = a.j;
  double nrm = 0.0;
  for (int64_t pb = p0; pb < p1; pb += 32) {
    const int64_t p = pb + lane;
    const bool ok = p < p1;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
    if (ok) {
      for (int i = q; i <= j; i += kGroups) {
        const float4 v1 = V[(int64_t)i * n + p], v2 = V[(int64_t)i * n + h + p];
        const float4 cv = scf[2 * i], cw = scf[2 * i + 1];
        df_acc(s[0], e[0], v1.x, v1.z, cv.x, cv.z);  df_sub(s[0], e[0], v1.y, v1.w, cv.y, cv.w);
        df_sub(s[0], e[0], v2.x, v2.z, cw.x, cw.z);  df_sub(s[0], e[0], v2.y, v2.w, cw.y, cw.w);
        df_acc(s[1], e[1], v1.x, v1.z, cv.y, cv.w);  df_acc(s[1], e[1], v1.y, v1.w, cv.x, cv.z);
        df_sub(s[1], e[1], v2.x, v2.z, cw.y, cw.w);  df_acc(s[1], e[1], v2.y, v2.w, cw.x, cw.z);
        df_acc(s[2], e[2], v2.x, v2.z, cv.x, cv.z);  df_sub(s[2], e[2], v2.y, v2.w, cv.y, cv.w);
        df_acc(s[2], e[2], v1.x, v1.z, cw.x, cw.z);  df_acc(s[2], e[2], v1.y, v1.w, cw.y, cw.w);
        df_acc(s[3], e[3], v2.x, v2.z, cv.y, cv.w);  df_acc(s[3], e[3], v2.y, v2.w, cv.x, cv.z);
        df_acc(s[3], e[3], v1.x, v1.z, cw.y, cw.w);  df_sub(s[3], e[3], v1.y, v1.w, cw.x, cw.z);
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      red_s[q][lane][t] = s[t];
      red_e[q][lane][t] = e[t];
    }
    __syncthreads();
    if (q == 0 && ok) {
      double c[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float S = red_s[0][lane][t], E = red_e[0][lane][t];
#pragma unroll
        for (int g = 1; g < kGroups; ++g) {
          float u, ue;
          two_sum(S, red_s[g][lane][t], u, ue);
          S = u;
          E = __fadd_rn(E, __fadd_rn(ue, red_e[g][lane][t]));
        }
        c[t] = (double)S + (double)E;
      }
      double2 y1 = y[p], y2 = y[h + p];
      y1.x -= c[0]; y1.y -= c[1];
      y2.x -= c[2]; y2.y -= c[3];
      y[p] = y1;
      y[h + p] = y2;
      nrm += cabs2(y1) + cabs2(y2);
    }
    __syncthreads();
  }
  return nrm;
}

__global__ void __launch_bounds__(kThreads) gsdf_update_kernel(GSArgs a, int pass) {
  extern __shared__ float4 scf[];                       // per column: {cv hi/lo}, {cw hi/lo}; then csm, big
  __shared__ double sh[32];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = a.st->done;
  __syncthreads();
  if (s_skip) return;
  const int j = a.j;
  UpdCoef u{scf, scf + 2 * (j + 1), (unsigned char*)(scf + 3 * (j + 1))};
  classify_coefs(a.coef, j, a.st->nrm[pass - 1], u);   // ||y|| before this update (b0, or the last pass's)
  if (blockIdx.x == 0 && threadIdx.x == 0) a.st->units_update += (double)(j + 1) * (double)a.h;
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, a.h);
  __shared__ float red_s[kGroups][32][4], red_e[kGroups][32][4];
  const double nrm = block_sum(dfupdate_rows(a, p0, p1, u, red_s, red_e), sh);
  if (threadIdx.x == 0) a.part_nrm[blockIdx.x] = nrm;
}

// v_{j+1} = y / beta stored split into V4[:, j+1] and in FP64 into x (the next matvec input).
__global__ void __launch_bounds__(kThreads) gsdf_normalize_kernel(GSArgs a, double2* __restrict__ x) {
  __shared__ double sh[32];
  StepState* st = a.st;
  const int done = st->done;
  double beta;
  if (done) {
    beta = st->beta;
  } else {
    double s = 0.0;
    for (int b = threadIdx.x; b < a.nblk; b += kThreads) s += a.part_nrm[b];
    beta = sqrt(block_sum(s, sh));
  }
  const double tmax = st->tmax;
  const bool brk = !(beta > 1e-14 * fmax(tmax, 1.0));
  const double inv = brk ? 0.0 : 1.0 / beta;
  const double2* y = (const double2*)a.y;
  float4* v = (float4*)a.V + (int64_t)(a.j + 1) * a.n;
  const int64_t h = a.h;
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {
    const double2 y1 = y[p], y2 = y[h + p];
    const double2 v1 = make_double2(y1.x * inv, y1.y * inv), v2 = make_double2(y2.x * inv, y2.y * inv);
    v[p] = split(v1);
    v[h + p] = split(v2);
    x[p] = v1;
    x[h + p] = v2;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int j = a.j;
    a.T[(int64_t)(j + 1) * a.ldt + j] = beta;
    if (j + 1 < a.m) a.T[(int64_t)j * a.ldt + j + 1] = beta;
    if (brk) st->status = 5;
  }
}

// ------------------------------------------------------------------ one cooperative launch per step
// The compensated-FP32 Gram-Schmidt of one Lanczos step (alpha, every pass with the sqrt(2) test,
// normalisation) as one cooperative launch, like gs_step_coop_kernel in gs.cu: grid-wide barriers
// where the multi-kernel path ends one launch and starts the next; each block walks row blocks
// rb = blockIdx.x, blockIdx.x + gridDim.x, ... of the same partition; every block takes the test from
// the same partials in the same order; nrm2 holds two slots of nblk norm partials.

__device__ __forceinline__ double coop_norm_df(const double* part, int nblk, double* sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads) s += part[b];
  return sqrt(block_sum(s, sh));
}

__global__ void __launch_bounds__(kThreads, 3)
gsdf_step_coop_kernel(GSArgs a, double2* __restrict__ x, const double2* __restrict__ alpha_part, int n_alpha_part,
                      int passes, double* __restrict__ nrm2) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double sh[32];
  __shared__ float red_s[kGroups][32][4], red_e[kGroups][32][4];
  float4* ys = (float4*)dyn;
  float* red = (float*)(ys + 2 * a.rows_per_block);
  float4* scf = (float4*)(red + kGroups * 2 * (4 * kCols) * 33);
  const UpdCoef upd{scf, scf + 2 * (a.m + 1), (unsigned char*)(scf + 3 * (a.m + 1))};
  const int j = a.j;
  const int64_t h = a.h;
  const int nblk = a.nblk;
  StepState* st = a.st;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_alpha_part; i += kThreads) {
    ar += alpha_part[i].x;
    ai += alpha_part[i].y;
  }
  ar = block_sum(ar, sh);
  ai = block_sum(ai, sh);
  double tmax = fmax(st->tmax, fabs(ar));
  if (j > 0) tmax = fmax(tmax, fabs(a.T[(int64_t)j * a.ldt + j - 1]));
  if (lead) {
    a.T[(int64_t)j * a.ldt + j] = ar;
    st->alpha_im = ai;
    st->done = 0;
    st->tmax = tmax;
    st->n_passes += 1;
    st->units_first += (double)(j + 1) * (double)h;
  }
  double2* y = (double2*)a.y;
  for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {   // y -= alpha v_j in FP64; b0; pass-1 dots
    const int64_t p0 = (int64_t)rb * a.rows_per_block;
    const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
    double nrm = 0.0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {
      double2 y1 = y[p], y2 = y[h + p];
      const double2 v1 = x[p], v2 = x[h + p];
      y1.x -= ar * v1.x; y1.y -= ar * v1.y;
      y2.x -= ar * v2.x; y2.y -= ar * v2.y;
      y[p] = y1;
      y[h + p] = y2;
      nrm += cabs2(y1) + cabs2(y2);
    }
    nrm = block_sum(nrm, sh);
    if (threadIdx.x == 0) nrm2[rb] = nrm;
    split_rows(a, p0, p1, ys);
    dfdot_body<false>(a, p0, p1, ys, red, rb);
    __syncthreads();                                       // ys and red are reused by the next row block
  }
  double bref = 0.0, beta = 0.0;
  for (int pass = 1;; ++pass) {
    grid.sync();
    if (pass == 1) {
      bref = coop_norm_df(nrm2, nblk, sh);
      if (lead) st->nrm[0] = bref;
    }
    for (int c = blockIdx.x; c <= j; c += gridDim.x) {
      const coef4* src = (const coef4*)a.part_dot + (int64_t)c * nblk;
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int b = threadIdx.x; b < nblk; b += kThreads) {
        const coef4 cc = src[b];
        s0 += cc.vr; s1 += cc.vi; s2 += cc.wr; s3 += cc.wi;
      }
      s0 = block_sum(s0, sh); s1 = block_sum(s1, sh); s2 = block_sum(s2, sh); s3 = block_sum(s3, sh);
      if (threadIdx.x == 0) {
        coef4 cc; cc.vr = s0; cc.vi = s1; cc.wr = a.no_w ? 0.0 : s2; cc.wi = a.no_w ? 0.0 : s3;
        a.coef[c] = cc;
      }
    }
    grid.sync();
    classify_coefs(a.coef, j, bref, upd);                 // bref: ||y|| before this update
    __syncthreads();
    double* slot = nrm2 + (size_t)(pass & 1) * nblk;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
      const int64_t p0 = (int64_t)rb * a.rows_per_block;
      const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
      const double nb = block_sum(dfupdate_rows(a, p0, p1, upd, red_s, red_e), sh);
      if (threadIdx.x == 0) slot[rb] = nb;
    }
    if (lead) st->units_update += (double)(j + 1) * (double)h;
    grid.sync();
    const double b1 = coop_norm_df(slot, nblk, sh);
    if (lead && pass < 8) st->nrm[pass] = b1;
    if (kSqrt2 * b1 > bref || pass >= passes) {
      beta = b1;
      break;
    }
    bref = b1;
    if (lead) {
      st->n_passes += 1;
      st->units_dot += (double)(j + 1) * (double)h;
    }
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
      const int64_t p0 = (int64_t)rb * a.rows_per_block;
      const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
      split_rows(a, p0, p1, ys);
      dfdot_body<false>(a, p0, p1, ys, red, rb);
      __syncthreads();
    }
  }
  const bool brk = !(beta > 1e-14 * fmax(tmax, 1.0));
  const double inv = brk ? 0.0 : 1.0 / beta;
  float4* v = (float4*)a.V + (int64_t)(j + 1) * a.n;
  for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
    const int64_t p0 = (int64_t)rb * a.rows_per_block;
    const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {
      const double2 y1 = y[p], y2 = y[h + p];
      const double2 v1 = make_double2(y1.x * inv, y1.y * inv), v2 = make_double2(y2.x * inv, y2.y * inv);
      v[p] = split(v1);
      v[h + p] = split(v2);
      x[p] = v1;
      x[h + p] = v2;
    }
  }
  if (lead) {
    a.T[(int64_t)(j + 1) * a.ldt + j] = beta;
    if (j + 1 < a.m) a.T[(int64_t)j * a.ldt + j + 1] = beta;
    st->beta = beta;
    st->done = 1;
    if (brk) st->status = 5;
  }
}

// ------------------------------------------------------------------ basis conversions
__global__ void df_from_fp64_kernel(const double2* in, float4* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = split(in[i]);
}
__global__ void fp64_from_df_kernel(const float4* in, double2* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = join(in[i]);
}
// V4[:, c] = split(Vsrc[:, perm[c]]) for c < k and V4[:, k] = V4[:, m].
__global__ void shrink_df_kernel(float4* V, const double2* Vsrc, int64_t n, const int* perm, int k, int m) {
  const int c = blockIdx.y;
  float4* dst = V + (int64_t)c * n;
  if (c < k) {
    const double2* src = Vsrc + (int64_t)perm[c] * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      dst[i] = split(src[i]);
  } else {
    const float4* src = V + (int64_t)m * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      dst[i] = src[i];
  }
}
// out[:, c] = V4[:, order[c]] (FP64) and, with partners, out[:, nev + c] = J conj(...).
__global__ void gather_pairs_df_kernel(const float4* V, int64_t n, const int* order, int nev, int partners,
                                       double2* out) {
  const int c = blockIdx.y;
  const int64_t h = n / 2;
  const float4* src = V + (int64_t)order[c] * n;
  double2* dst = out + (int64_t)c * n;
  double2* dstp = out + (int64_t)(nev + c) * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < h; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x1 = join(src[i]), x2 = join(src[h + i]);
    dst[i] = x1;
    dst[h + i] = x2;
    if (partners) {
      dstp[i] = make_double2(-x2.x, x2.y);
      dstp[h + i] = make_double2(x1.x, -x1.y);
    }
  }
}

// Vout (FP64, 2n x kk real view) = V4 * Z in compensated FP32: V is already (hi, lo), Z is split
// into (hi, lo) as it is staged, every multiply-add is df_acc, and each output is (sum + error)
// converted once to FP64.  The restart rotation is the one dense contraction of the method; on the
// FP32 pipes it runs at several times the FP64 rate with FP64-level accuracy (K = m <= 1023).
__global__ void __launch_bounds__(256)
rotate_df_kernel(const float4* __restrict__ V, int64_t n, int m, const double* __restrict__ Z, int kk,
                 double* __restrict__ out) {
  constexpr int BM = 64, BN = 32, BK = 16;
  __shared__ float2 As[BK][BM];      // (hi, lo) of the real view of V
  __shared__ float2 Bs[BK][BN];      // (hi, lo) of Z
  const int64_t rows = 2 * n;
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tr = tid % 16, tc = tid / 16;   // rows tr + 16 i (i < 4), cols tc + 16 j (j < 2)
  float s[4][2], e[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) s[i][0] = s[i][1] = e[i][0] = e[i][1] = 0.f;
  for (int k0 = 0; k0 < m; k0 += BK) {
    for (int q = tid; q < BK * BM; q += 256) {
      const int kx = q / BM, r = q % BM;
      const int64_t gr = row0 + r;
      float2 val = make_float2(0.f, 0.f);
      if (gr < rows && k0 + kx < m) {
        const float4 f = V[(int64_t)(k0 + kx) * n + (gr >> 1)];
        val = (gr & 1) ? make_float2(f.y, f.w) : make_float2(f.x, f.z);
      }
      As[kx][r] = val;
    }
    for (int q = tid; q < BK * BN; q += 256) {
      const int kx = q / BN, c = q % BN;
      float2 val = make_float2(0.f, 0.f);
      if (k0 + kx < m && col0 + c < kk) {
        const double z = Z[(int64_t)(col0 + c) * m + k0 + kx];
        const float zh = (float)z;
        val = make_float2(zh, (float)(z - (double)zh));
      }
      Bs[kx][c] = val;
    }
    __syncthreads();
#pragma unroll 4
    for (int x = 0; x < BK; ++x) {
      float2 av[4], bv[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[x][tr + 16 * i];
      bv[0] = Bs[x][tc];
      bv[1] = Bs[x][tc + 16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        df_acc(s[i][0], e[i][0], av[i].x, av[i].y, bv[0].x, bv[0].y);
        df_acc(s[i][1], e[i][1], av[i].x, av[i].y, bv[1].x, bv[1].y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + tr + 16 * i;
    if (gr >= rows) continue;
#pragma unroll
    for (int jx = 0; jx < 2; ++jx) {
      const int gc = col0 + tc + 16 * jx;
      if (gc < kk) out[(int64_t)gc * rows + gr] = (double)s[i][jx] + (double)e[i][jx];
    }
  }
}

// ------------------------------------------------------------------ double-float stencil matvec
// y (FP64) = A x for x given as (hi, lo) pairs (a column of the mixed basis), links given as (hi, lo)
// pairs in structure-of-arrays layout L[(mu*9 + e)*V + s] (float4 per complex).  One thread per
// (site, colour) as in the FP32 kernel.  The product of the Lanczos steps and of the certifying
// residuals and Rayleigh quotients (stencil_df_kernel) makes every complex multiply-add four df_acc
// (Dot2), so its result has FP64-level accuracy while the arithmetic runs on the FP32 pipes; the
// filter's fused Chebyshev steps (stencil_df_cheb_kernel) carry the sums as biased blocks instead.
// With `part` non-null the block partials of x^H y (FP64) are written for alpha.
constexpr int kDfSites = 64;
constexpr int kDfMinBlocks = 4;   // 4 x 192 threads per SM (measured best of 2..6 at 16^4)

// Dot2 form: every product split exactly and added by TwoSum (11 FP32 operations with a complex64
// link, 12 with a (hi, lo) link).
__device__ __forceinline__ void cdf_acc(float* s, float* e, float4 a, float4 b) {   // (re, im) += a * b
  df_acc(s[0], e[0], a.x, a.z, b.x, b.z);
  df_sub(s[0], e[0], a.y, a.w, b.y, b.w);
  df_acc(s[1], e[1], a.x, a.z, b.y, b.w);
  df_acc(s[1], e[1], a.y, a.w, b.x, b.z);
}
__device__ __forceinline__ void cdf_accc(float* s, float* e, float4 a, float4 b) {  // += conj(a) * b
  df_acc(s[0], e[0], a.x, a.z, b.x, b.z);
  df_acc(s[0], e[0], a.y, a.w, b.y, b.w);
  df_acc(s[1], e[1], a.x, a.z, b.y, b.w);
  df_sub(s[1], e[1], a.y, a.w, b.x, b.z);
}
// The same for a link exact in FP32 (a = (re, im), no low part).
__device__ __forceinline__ void cdf_acc(float* s, float* e, float2 a, float4 b) {
  df_acc_xa(s[0], e[0], a.x, b.x, b.z);
  df_acc_xa(s[0], e[0], -a.y, b.y, b.w);
  df_acc_xa(s[1], e[1], a.x, b.y, b.w);
  df_acc_xa(s[1], e[1], a.y, b.x, b.z);
}
__device__ __forceinline__ void cdf_accc(float* s, float* e, float2 a, float4 b) {
  df_acc_xa(s[0], e[0], a.x, b.x, b.z);
  df_acc_xa(s[0], e[0], a.y, b.y, b.w);
  df_acc_xa(s[1], e[1], a.x, b.y, b.w);
  df_acc_xa(s[1], e[1], -a.y, b.x, b.z);
}
// ------------------------------------------------------------------ block sums at a fixed bias
// The hopping sum of one direction mu is 12 complex products per colour row whose magnitudes are
// known before they are added (sum |a| |bh|, from the high parts of the operands).  Such sums can be
// carried at a fixed bias: S = 1.5 sigma + (sum so far), sigma a power of two >= 2.125 times the bound
// of the sum, keeps S inside [sigma, 2 sigma).  The FMA t = fl(S + a bh) then needs no TwoSum: t - S
// is exactly the amount added (both lie in one binade, Sterbenz), and a bh minus that amount -- the
// FMA's rounding error, at most half an ulp of sigma -- goes, rounded once, into the error sum e
// together with a bl.  5 FP32 operations a product (6 with a (hi, lo) link) against 11 (12) for the
// Dot2 form.  The bound grows direction by direction; before each direction S moves to the bias of
// the grown bound (rebias: exact up to the part it hands to e), and at the end S - 1.5 sigma is the
// exact high part.  The error sum now collects terms of the size of an ulp of sigma rather than of the
// partial sums, so the result is about 16 times less accurate than Dot2: an exact emulation of the
// sequence (fractions) over 300 random 48-term sums gave at most 2^-40.8 of sum |a| |bh|, against
// 2^-44.8 for the Dot2 form.  The filter's Chebyshev steps use it (their products only shape the
// Krylov space; every pair is accepted on A's residual, computed with the Dot2 form).

// 1.5 sigma for the smallest power of two sigma >= 2.125 bound, with sigma in [2^-100, 2^126] (a bound
// below 2^-100 only ever meets products that small; one above 2^125 does not occur for the
// normalised vectors of the method).
__device__ __forceinline__ float bias_of(float bound) {
  const float v = fminf(fmaxf(2.125f * bound, 7.8886091e-31f), 8.5070592e+37f);
  const uint32_t p2 = (__float_as_uint(v) + 0x007fffffu) & 0x7f800000u;   // next power of two >= v
  return __uint_as_float(p2 | 0x00400000u);                               // 1.5 * sigma
}
// (S, e) += a * (bh + bl), a exact in FP32 (a complex64 link)
__device__ __forceinline__ void bias_acc(float& S, float& e, float a, float bh, float bl) {
  const float t = __fmaf_rn(a, bh, S);
  e = __fmaf_rn(a, bl, __fadd_rn(e, __fmaf_rn(a, bh, -__fsub_rn(t, S))));
  S = t;
}
// (S, e) += (ah + al) * (bh + bl): the same with al * bh in the error sum
__device__ __forceinline__ void bias_acc(float& S, float& e, float ah, float al, float bh, float bl) {
  const float t = __fmaf_rn(ah, bh, S);
  e = __fmaf_rn(al, bh, __fmaf_rn(ah, bl, __fadd_rn(e, __fmaf_rn(ah, bh, -__fsub_rn(t, S)))));
  S = t;
}
// (re, im) += a * b and += conj(a) * b for b = (hi.re, hi.im, lo.re, lo.im)
__device__ __forceinline__ void cbias_acc(float* S, float* e, float2 a, float4 b) {
  bias_acc(S[0], e[0], a.x, b.x, b.z);
  bias_acc(S[0], e[0], -a.y, b.y, b.w);
  bias_acc(S[1], e[1], a.x, b.y, b.w);
  bias_acc(S[1], e[1], a.y, b.x, b.z);
}
__device__ __forceinline__ void cbias_accc(float* S, float* e, float2 a, float4 b) {
  bias_acc(S[0], e[0], a.x, b.x, b.z);
  bias_acc(S[0], e[0], a.y, b.y, b.w);
  bias_acc(S[1], e[1], a.x, b.y, b.w);
  bias_acc(S[1], e[1], -a.y, b.x, b.z);
}
__device__ __forceinline__ void cbias_acc(float* S, float* e, float4 a, float4 b) {
  bias_acc(S[0], e[0], a.x, a.z, b.x, b.z);
  bias_acc(S[0], e[0], -a.y, -a.w, b.y, b.w);
  bias_acc(S[1], e[1], a.x, a.z, b.y, b.w);
  bias_acc(S[1], e[1], a.y, a.w, b.x, b.z);
}
__device__ __forceinline__ void cbias_accc(float* S, float* e, float4 a, float4 b) {
  bias_acc(S[0], e[0], a.x, a.z, b.x, b.z);
  bias_acc(S[0], e[0], a.y, a.w, b.y, b.w);
  bias_acc(S[1], e[1], a.x, a.z, b.y, b.w);
  bias_acc(S[1], e[1], -a.y, -a.w, b.x, b.z);
}
__device__ __forceinline__ float4 cneg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
// |re| + |im| of the high part
__device__ __forceinline__ float l1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ float l1(float4 a) { return fabsf(a.x) + fabsf(a.y); }

// Moves S from bias bo = 1.5 sigma_o to bn = 1.5 sigma_n (sigma_n >= sigma_o, |S - bo| < sigma_o / 2):
// S - bo is exact (Sterbenz), adding bn rounds to the new binade's ulp, and what that rounding
// dropped, (S - bo) - (t - bn), is exact and goes into e.  With sigma_n = sigma_o nothing moves.
__device__ __forceinline__ void rebias(float& S, float& e, float bo, float bn) {
  const float d = __fsub_rn(S, bo);
  const float t = __fadd_rn(d, bn);
  e = __fadd_rn(e, __fsub_rn(d, __fsub_rn(t, bn)));
  S = t;
}

// The hopping sums of site s, colour a, in compensated FP32: (ys1, ye1) and (ys2, ye2) for the U
// terms of y1 and y2, (ws1, we1) and (ws2, we2) for the W terms (kappa not yet applied).
struct DfSums {
  float ys1[2], ye1[2], ys2[2], ye2[2], ws1[2], we1[2], ws2[2], we2[2];
};

// A link as stored: a (hi, lo) float4 pair, or a float2 exact in FP32 (complex64 links), for which
// the products take the shorter exact-multiplier form.

// The sums in the Dot2 form (the certifying product: residuals and Rayleigh quotients).
template <typename LinkT>
__device__ __forceinline__ void stencil_df_sums_dot2(const OpDev& op, const float4* __restrict__ x, int s, int a,
                                                DfSums& r) {
  const int vol = (int)op.vol;
  const int64_t h = op.h;
  const LinkT* U = (const LinkT*)op.U;
  const LinkT* W = (const LinkT*)op.W;
  const float4* x1 = x;
  const float4* x2 = x + h;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    r.ys1[c] = r.ye1[c] = r.ys2[c] = r.ye2[c] = 0.f;
    r.ws1[c] = r.we1[c] = r.ws2[c] = r.we2[c] = 0.f;
  }
  const int d0 = op.dims[0], d1 = op.dims[1], d2 = op.dims[2], d3 = op.dims[3];
  // the site's coordinates, once (x fastest)
  const int r1 = s / d0, r2 = r1 / d1;
  const int x0 = s - r1 * d0, x1c = r1 - r2 * d1, x2c = r2 % d2, x3c = r2 / d2;
  int stride = 1;
  // the direction loop stays rolled: unrolled, its 4 x 3 x 8 compensated products overflowed the
  // instruction cache (ncu: "no instruction" stalls as frequent as memory stalls); extents and
  // coordinates are selected in registers, not indexed
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int L = mu == 0 ? d0 : mu == 1 ? d1 : mu == 2 ? d2 : d3;
    const int c = mu == 0 ? x0 : mu == 1 ? x1c : mu == 2 ? x2c : x3c;
    const int sp = (c == L - 1) ? s - (L - 1) * stride : s + stride;
    const int sm = (c == 0) ? s + (L - 1) * stride : s - stride;
    stride *= L;
    const LinkT* Um = U + (int64_t)mu * 9 * vol;
    const LinkT* Wm = W + (int64_t)mu * 9 * vol;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 p1 = x1[3 * sp + b], p2 = x2[3 * sp + b];
      const float4 m1 = x1[3 * sm + b], m2 = x2[3 * sm + b];
      const LinkT uf = Um[(a * 3 + b) * vol + s];    // U(s)_{ab}
      const LinkT ub = Um[(b * 3 + a) * vol + sm];   // U(s-mu)_{ba}
      const LinkT wf = Wm[(a * 3 + b) * vol + s];    // W(s)_{ab}
      const LinkT wb = Wm[(b * 3 + a) * vol + sm];   // W(s-mu)_{ba}
      cdf_acc(r.ys1, r.ye1, uf, p1);           // U(s) x1(s+mu)
      cdf_accc(r.ys1, r.ye1, ub, m1);          // U(s-mu)^H x1(s-mu)
      cdf_accc(r.ys2, r.ye2, uf, p2);          // U(s)^* x2(s+mu)
      cdf_acc(r.ys2, r.ye2, ub, m2);           // U(s-mu)^T x2(s-mu)
      cdf_acc(r.ws1, r.we1, wf, p2);           // W(s) x2(s+mu)
      cdf_acc(r.ws1, r.we1, cneg(wb), m2);     // -W(s-mu)^T x2(s-mu)
      cdf_accc(r.ws2, r.we2, cneg(wf), p1);    // -W(s)^* x1(s+mu)
      cdf_accc(r.ws2, r.we2, wb, m1);          // +W(s-mu)^H x1(s-mu)
    }
  }
}

// The sums as biased blocks, one per direction (the Chebyshev steps of the filter).
template <typename LinkT>
__device__ __forceinline__ void stencil_df_sums_biased(const OpDev& op, const float4* __restrict__ x, int s, int a,
                                                DfSums& r) {
  const int vol = (int)op.vol;
  const int64_t h = op.h;
  const LinkT* U = (const LinkT*)op.U;
  const LinkT* W = (const LinkT*)op.W;
  const float4* x1 = x;
  const float4* x2 = x + h;
  // running sums held at a bias (S) with their error sums (e); one bound for the two U sums and one
  // for the two W sums (sum |a| |bh| over both, over the blocks so far: at most twice either's own)
  float ou = bias_of(0.f), ow = ou;
  float bu = 0.f, bw = 0.f;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    r.ys1[c] = r.ys2[c] = r.ws1[c] = r.ws2[c] = ou;
    r.ye1[c] = r.ye2[c] = r.we1[c] = r.we2[c] = 0.f;
  }
  const int d0 = op.dims[0], d1 = op.dims[1], d2 = op.dims[2], d3 = op.dims[3];
  // the site's coordinates, once (x fastest)
  const int r1 = s / d0, r2 = r1 / d1;
  const int x0 = s - r1 * d0, x1c = r1 - r2 * d1, x2c = r2 % d2, x3c = r2 / d2;
  int stride = 1;
  // the direction loop stays rolled: unrolled, its 4 x 3 x 8 compensated products overflowed the
  // instruction cache (ncu: "no instruction" stalls as frequent as memory stalls); extents and
  // coordinates are selected in registers, not indexed
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int L = mu == 0 ? d0 : mu == 1 ? d1 : mu == 2 ? d2 : d3;
    const int c = mu == 0 ? x0 : mu == 1 ? x1c : mu == 2 ? x2c : x3c;
    const int sp = (c == L - 1) ? s - (L - 1) * stride : s + stride;
    const int sm = (c == 0) ? s + (L - 1) * stride : s - stride;
    stride *= L;
    const LinkT* Um = U + (int64_t)mu * 9 * vol;
    const LinkT* Wm = W + (int64_t)mu * 9 * vol;
    // the block's bound first (high parts only), then its products: the operands are read twice
    // (the second time from L1) rather than held, which would spill
    const float2* x1h = reinterpret_cast<const float2*>(x1);
    const float2* x2h = reinterpret_cast<const float2*>(x2);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float nuf = l1(Um[(a * 3 + b) * vol + s]), nub = l1(Um[(b * 3 + a) * vol + sm]);
      const float nwf = l1(Wm[(a * 3 + b) * vol + s]), nwb = l1(Wm[(b * 3 + a) * vol + sm]);
      const float np = l1(x1h[2 * (3 * sp + b)]) + l1(x2h[2 * (3 * sp + b)]);
      const float nm = l1(x1h[2 * (3 * sm + b)]) + l1(x2h[2 * (3 * sm + b)]);
      bu = fmaf(nuf, np, fmaf(nub, nm, bu));
      bw = fmaf(nwf, np, fmaf(nwb, nm, bw));
    }
    {
      const float nu = bias_of(bu), nw = bias_of(bw);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        rebias(r.ys1[q], r.ye1[q], ou, nu);
        rebias(r.ys2[q], r.ye2[q], ou, nu);
        rebias(r.ws1[q], r.we1[q], ow, nw);
        rebias(r.ws2[q], r.we2[q], ow, nw);
      }
      ou = nu; ow = nw;
    }
    auto products = [&](int b) {
      const float4 p1 = x1[3 * sp + b], p2 = x2[3 * sp + b];
      const float4 m1 = x1[3 * sm + b], m2 = x2[3 * sm + b];
      const LinkT uf = Um[(a * 3 + b) * vol + s];    // U(s)_{ab}
      const LinkT ub = Um[(b * 3 + a) * vol + sm];   // U(s-mu)_{ba}
      const LinkT wf = Wm[(a * 3 + b) * vol + s];    // W(s)_{ab}
      const LinkT wb = Wm[(b * 3 + a) * vol + sm];   // W(s-mu)_{ba}
      cbias_acc(r.ys1, r.ye1, uf, p1);           // U(s) x1(s+mu)
      cbias_accc(r.ys1, r.ye1, ub, m1);          // U(s-mu)^H x1(s-mu)
      cbias_accc(r.ys2, r.ye2, uf, p2);          // U(s)^* x2(s+mu)
      cbias_acc(r.ys2, r.ye2, ub, m2);           // U(s-mu)^T x2(s-mu)
      cbias_acc(r.ws1, r.we1, wf, p2);           // W(s) x2(s+mu)
      cbias_acc(r.ws1, r.we1, cneg(wb), m2);     // -W(s-mu)^T x2(s-mu)
      cbias_accc(r.ws2, r.we2, cneg(wf), p1);    // -W(s)^* x1(s+mu)
      cbias_accc(r.ws2, r.we2, wb, m1);          // +W(s-mu)^H x1(s-mu)
    };
    if constexpr (sizeof(LinkT) == sizeof(float2)) {
#pragma unroll
      for (int b = 0; b < 3; ++b) products(b);
    } else {   // (hi, lo) links: unrolled, the operands of the three b spill at 80 registers
#pragma unroll 1
      for (int b = 0; b < 3; ++b) products(b);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {   // the high parts without their bias (exact)
    r.ys1[q] = __fsub_rn(r.ys1[q], ou);
    r.ys2[q] = __fsub_rn(r.ys2[q], ou);
    r.ws1[q] = __fsub_rn(r.ws1[q], ow);
    r.ws2[q] = __fsub_rn(r.ws2[q], ow);
  }
}

template <typename LinkT>
__global__ void __launch_bounds__(3 * kDfSites, kDfMinBlocks)
stencil_df_kernel(OpDev op, const float4* __restrict__ x, double2* __restrict__ Y, double* __restrict__ part) {
  __shared__ double sh[32];
  const int vol = (int)op.vol;
  const int64_t h = op.h;
  const int s = blockIdx.x * kDfSites + (threadIdx.x % kDfSites);
  const int a = threadIdx.x / kDfSites;
  double c0 = 0.0, c1 = 0.0;
  if (s < vol) {
    DfSums r;
    stencil_df_sums_dot2<LinkT>(op, x, s, a, r);
    const int64_t e1 = 3 * (int64_t)s + a;
    const double2 xa = join(x[e1]), xb = join(x[h + e1]);
    const double kap = op.kappa, m0 = op.m0;
    const double2 o1 = make_double2((double)r.ys1[0] + (double)r.ye1[0] + kap * ((double)r.ws1[0] + (double)r.we1[0]) + m0 * xa.x,
                                    (double)r.ys1[1] + (double)r.ye1[1] + kap * ((double)r.ws1[1] + (double)r.we1[1]) + m0 * xa.y);
    const double2 o2 = make_double2((double)r.ys2[0] + (double)r.ye2[0] + kap * ((double)r.ws2[0] + (double)r.we2[0]) + m0 * xb.x,
                                    (double)r.ys2[1] + (double)r.ye2[1] + kap * ((double)r.ws2[1] + (double)r.we2[1]) + m0 * xb.y);
    Y[e1] = o1;
    Y[h + e1] = o2;
    if (part) {
      c0 = xa.x * o1.x + xa.y * o1.y + xb.x * o2.x + xb.y * o2.y;
      c1 = xa.x * o1.y - xa.y * o1.x + xb.x * o2.y - xb.y * o2.x;
    }
  }
  if (part) {
    c0 = block_sum(c0, sh);
    c1 = block_sum(c1, sh);
    if (threadIdx.x == 0) ((double2*)part)[blockIdx.x] = make_double2(c0, c1);
  }
}

// ------------------------------------------------------------------ float-float scalars
// hi + lo with |lo| <= ulp(hi)/2; the operations below keep about 48 significant bits.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_norm(float s, float e) {   // two_sum renormalisation
  ff r;
  two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {   // exact split of hi * hi plus first-order cross terms
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  ff r;
  r.hi = __fadd_rn(p, e);                                   // fast two-sum: |p| >= |e|
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, p));
  return r;
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_re(float4 v) { return ff{v.x, v.z}; }
__device__ __forceinline__ ff ff_im(float4 v) { return ff{v.y, v.w}; }

// Constants of one Chebyshev step as float-float pairs.
struct ChebConsts {
  ff kappa, m0, c, sc, g, g0;
};

// One step of the Chebyshev recurrence for B = p(A) fused into the compensated-FP32 product t -> A t
// (x = t_k, the current recurrence vector, as (hi, lo)):
//   t_next = sc (A t - c t) - t_prev     (t_prev omitted when null)
//   acc    = g0 v + g t_next (init)   or   acc += g t_next
// all in float-float arithmetic on the FP32 pipe, the hopping sums as biased blocks (one per direction;
// 5 FP32 operations a product); t_next and acc are stored as (hi, lo) float4, so t_next feeds the next
// product directly.  On 24^3 x 48 this took a launch from 322 to about 255 us (the step from 12.2 to
// 10.5 s, the same products and restarts); on the last step acc goes out in FP64 to y, with the
// per-block partials of conj(v) y (the alpha of Algorithm 2).  t_next may alias t_prev (the same
// thread reads an entry before writing it); neighbours are read from x only.
template <typename LinkT>
__global__ void __launch_bounds__(3 * kDfSites, kDfMinBlocks)
stencil_df_cheb_kernel(OpDev op, const float4* __restrict__ x, const float4* t_prev, float4* t_next,
                       float4* __restrict__ acc, const float4* __restrict__ v, double2* __restrict__ y,
                       double* __restrict__ part, ChebConsts k, int init, int last) {
  __shared__ double sh[32];
  const int vol = (int)op.vol;
  const int64_t h = op.h;
  const int s = blockIdx.x * kDfSites + (threadIdx.x % kDfSites);
  const int a = threadIdx.x / kDfSites;
  double c0 = 0.0, c1 = 0.0;
  if (s < vol) {
    DfSums r;
    stencil_df_sums_biased<LinkT>(op, x, s, a, r);
    const int64_t e1 = 3 * (int64_t)s + a;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t e = e1 + (half ? h : 0);
      const float* ys = half ? r.ys2 : r.ys1;
      const float* ye = half ? r.ye2 : r.ye1;
      const float* ws = half ? r.ws2 : r.ws1;
      const float* we = half ? r.we2 : r.we1;
      const float4 xt = x[e];
      const float4 tp = t_prev ? t_prev[e] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 ac = init ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[e];
      const float4 vv = (init || last) ? v[e] : make_float4(0.f, 0.f, 0.f, 0.f);
      ff nx[2], an[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const ff xc = c ? ff_im(xt) : ff_re(xt);
        // (A t)_c = U sums + kappa W sums + m0 t
        ff u = ff_add(ff_norm(ys[c], ye[c]), ff_mul(k.kappa, ff_norm(ws[c], we[c])));
        u = ff_add(u, ff_mul(k.m0, xc));
        ff d = ff_mul(k.sc, ff_add(u, ff_neg(ff_mul(k.c, xc))));
        if (t_prev) d = ff_add(d, ff_neg(c ? ff_im(tp) : ff_re(tp)));
        nx[c] = d;
        const ff gn = ff_mul(k.g, d);
        an[c] = init ? ff_add(ff_mul(k.g0, c ? ff_im(vv) : ff_re(vv)), gn) : ff_add(c ? ff_im(ac) : ff_re(ac), gn);
      }
      t_next[e] = make_float4(nx[0].hi, nx[1].hi, nx[0].lo, nx[1].lo);
      if (last) {
        const double2 o = make_double2((double)an[0].hi + (double)an[0].lo, (double)an[1].hi + (double)an[1].lo);
        y[e] = o;
        const double2 vd = join(vv);
        c0 += vd.x * o.x + vd.y * o.y;
        c1 += vd.x * o.y - vd.y * o.x;
      } else {
        acc[e] = make_float4(an[0].hi, an[1].hi, an[0].lo, an[1].lo);
      }
    }
  }
  if (last) {
    c0 = block_sum(c0, sh);
    c1 = block_sum(c1, sh);
    if (threadIdx.x == 0) ((double2*)part)[blockIdx.x] = make_double2(c0, c1);
  }
}

// FP64 links [4][V][9] -> (hi, lo) structure-of-arrays [4][9][V].
__global__ void links_df_kernel(const double2* in, float4* out, int64_t vol) {
  const int64_t total = 36 * vol;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q % vol, me = q / vol, mu = me / 9, e = me % 9;
    out[q] = split(in[(mu * vol + s) * 9 + e]);
  }
}

inline int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 1216 ? 1216 : (g < 1 ? 1 : g));
}

size_t dot_smem(const GSArgs& a) {
  return (size_t)2 * a.rows_per_block * sizeof(float4) + (size_t)kGroups * 2 * (4 * kCols) * 33 * sizeof(float);
}

}  // namespace

cudaError_t launch_gsdf_first(const GSArgs& a, const void* x, const double2* alpha_part, int n_alpha_part,
                              cudaStream_t s) {
  const size_t sm = dot_smem(a);
  cudaError_t e = allow_dyn_smem((const void*)gsdf_first_kernel, (size_t)sm);
  if (e != cudaSuccess) return e;
  gsdf_first_kernel<<<a.nblk, kThreads, sm, s>>>(a, (const double2*)x, alpha_part, n_alpha_part);
  return cudaGetLastError();
}

size_t gsdf_coop_smem(const GSArgs& a) {
  return dot_smem(a) + (size_t)3 * (a.m + 1) * sizeof(float4) + (size_t)(a.m + 1);
}

cudaError_t gsdf_coop_occupancy(const GSArgs& a, int* per_sm) {
  int dev = 0, coop = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  const size_t sm = gsdf_coop_smem(a);
  if ((e = allow_dyn_smem((const void*)gsdf_step_coop_kernel, (size_t)sm)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gsdf_step_coop_kernel, kThreads, sm)) != cudaSuccess)
    return e;
  *per_sm = coop ? per : 0;
  return cudaSuccess;
}

cudaError_t launch_gsdf_step_coop(const GSArgs& a, void* x, const double2* alpha_part, int n_alpha_part, int passes,
                                  double* nrm2, int grid, cudaStream_t s) {
  GSArgs aa = a;
  double2* xx = (double2*)x;
  const double2* ap = alpha_part;
  int na = n_alpha_part, ps = passes;
  double* nr = nrm2;
  void* args[] = {&aa, &xx, &ap, &na, &ps, &nr};
  return cudaLaunchCooperativeKernel((const void*)gsdf_step_coop_kernel, dim3(grid), dim3(kThreads), args,
                                     gsdf_coop_smem(a), s);
}

cudaError_t launch_gsdf_dot(const GSArgs& a, int pass, cudaStream_t s) {
  const size_t sm = dot_smem(a);
  cudaError_t e = allow_dyn_smem((const void*)gsdf_dot_kernel, (size_t)sm);
  if (e != cudaSuccess) return e;
  gsdf_dot_kernel<<<a.nblk, kThreads, sm, s>>>(a, pass);
  return cudaGetLastError();
}

cudaError_t launch_gsdf_update(const GSArgs& a, int pass, cudaStream_t s) {
  const size_t sm = (size_t)(a.j + 1) * 3 * sizeof(float4) + (size_t)(a.j + 1);
  gsdf_update_kernel<<<a.nblk, kThreads, sm, s>>>(a, pass);
  return cudaGetLastError();
}

cudaError_t launch_gsdf_normalize(const GSArgs& a, void* x, cudaStream_t s) {
  gsdf_normalize_kernel<<<a.nblk, kThreads, 0, s>>>(a, (double2*)x);
  return cudaGetLastError();
}

cudaError_t launch_df_from_fp64(const void* in, void* out, int64_t n, cudaStream_t s) {
  df_from_fp64_kernel<<<grid_for(n), 256, 0, s>>>((const double2*)in, (float4*)out, n);
  return cudaGetLastError();
}

cudaError_t launch_fp64_from_df(const void* in, void* out, int64_t n, cudaStream_t s) {
  fp64_from_df_kernel<<<grid_for(n), 256, 0, s>>>((const float4*)in, (double2*)out, n);
  return cudaGetLastError();
}

cudaError_t launch_shrink_df(void* V, const void* Vsrc, int64_t n, const int* perm, int k, int m, cudaStream_t s) {
  dim3 grid(grid_for(n) / 4 + 1, k + 1);
  shrink_df_kernel<<<grid, 256, 0, s>>>((float4*)V, (const double2*)Vsrc, n, perm, k, m);
  return cudaGetLastError();
}

cudaError_t launch_gather_pairs_df(const void* V, int64_t n, const int* order, int nev, int partners, void* out,
                                   cudaStream_t s) {
  dim3 grid(grid_for(n / 2) / 4 + 1, nev);
  gather_pairs_df_kernel<<<grid, 256, 0, s>>>((const float4*)V, n, order, nev, partners, (double2*)out);
  return cudaGetLastError();
}

int matvec_df_blocks(const OpDev& op) { return (int)((op.vol + kDfSites - 1) / kDfSites); }

cudaError_t launch_matvec_df(const OpDev& op, const void* x, void* y, double* part, cudaStream_t s) {
  if (op.links32)
    stencil_df_kernel<float2><<<matvec_df_blocks(op), 3 * kDfSites, 0, s>>>(op, (const float4*)x, (double2*)y, part);
  else
    stencil_df_kernel<float4><<<matvec_df_blocks(op), 3 * kDfSites, 0, s>>>(op, (const float4*)x, (double2*)y, part);
  return cudaGetLastError();
}

cudaError_t launch_matvec_df_cheb(const OpDev& op, const void* x, const void* t_prev, void* t_next, void* acc,
                                  const void* v, void* y, double* part, double kappa, double m0, double c, double sc,
                                  double g, double g0, int init, int last, cudaStream_t s) {
  auto f = [](double d) { const float hi = (float)d; return ff{hi, (float)(d - (double)hi)}; };
  ChebConsts k{f(kappa), f(m0), f(c), f(sc), f(g), f(g0)};
  if (op.links32)
    stencil_df_cheb_kernel<float2><<<matvec_df_blocks(op), 3 * kDfSites, 0, s>>>(
        op, (const float4*)x, (const float4*)t_prev, (float4*)t_next, (float4*)acc, (const float4*)v, (double2*)y,
        part, k, init, last);
  else
    stencil_df_cheb_kernel<float4><<<matvec_df_blocks(op), 3 * kDfSites, 0, s>>>(
        op, (const float4*)x, (const float4*)t_prev, (float4*)t_next, (float4*)acc, (const float4*)v, (double2*)y,
        part, k, init, last);
  return cudaGetLastError();
}

cudaError_t launch_links_df(const void* in, void* out, int64_t vol, cudaStream_t s) {
  links_df_kernel<<<1024, 256, 0, s>>>((const double2*)in, (float4*)out, vol);
  return cudaGetLastError();
}

cudaError_t launch_rotate_df(const void* V, int64_t n, int m, const double* Z, int kk, void* Vout, cudaStream_t s) {
  dim3 grid((unsigned)((2 * n + 63) / 64), (unsigned)((kk + 31) / 32));
  rotate_df_kernel<<<grid, 256, 0, s>>>((const float4*)V, n, m, Z, kk, (double*)Vout);
  return cudaGetLastError();
}

}  // namespace jtr
