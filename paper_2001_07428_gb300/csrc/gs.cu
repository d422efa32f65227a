// gs.cu -- the Gram-Schmidt part of the Lanczos step with J-symmetry (Algorithm 2).
//
// After y = A v_j (matvec.cu, which also leaves per-block partials of v_j^H y):
//   t_{j,j} = Re(v_j^H y); y -= t_{j,j} v_j; b0 = ||y||
//   repeat: orthogonalise y against W_j = J V_j^* and V_j; b1 = ||y||;
//           stop when sqrt(2) b1 > b0, else b0 = b1           (gamma = sqrt(2))
//   t_{j+1,j} = b1; v_{j+1} = y / b1                          (reading: divide by the final norm)
//
// W is never stored.  With v_i = [v1; v2] and w_i = J v_i^* = [-v2^*; v1^*]:
//   c_v,i = v_i^H y = sum_p conj(v1) y1 + conj(v2) y2
//   c_w,i = w_i^H y = sum_p (v1 y2 - v2 y1)          (no conjugate)
//   y -= v_i c_v,i + w_i c_w,i:  y1 -= v1 c_v - conj(v2) c_w,  y2 -= v2 c_v + conj(v1) c_w
// so one read of V gives both projections (classical Gram-Schmidt over [W_j, V_j], repeated by the
// same sqrt(2) test as the paper's modified Gram-Schmidt loop).
//
// The data-dependent repeat runs without host synchronisation: every pass is launched, and each
// kernel of a pass returns at once when the device-side flag st->done says the loop has exited.
// All reductions use a fixed order, so results are reproducible run to run.
#include <cooperative_groups.h>

#include "internal.h"

namespace jtr {

namespace {

constexpr int kGsThreads = 256;   // 8 warps: lane = row pair in a tile of 32, warp = column group
constexpr int kColGroups = kGsThreads / 32;
constexpr int kRedThreads = 128;
constexpr double kSqrt2 = 1.4142135623730951;

// c_v and c_w for columns 0..j over rows [p0, p1) of this block, written as per-block partials.
// Warp q takes chunks of 8 consecutive columns (q*8, q*8 + 64, ...); each lane accumulates the
// 8 x 4 real sums of its rows, then the warp transposes the 32 accumulators through shared memory
// so that lane k adds up accumulator k: 31 adds per 32 results instead of 5-step shuffle trees
// per result (on this GPU one FP64 warp instruction holds the FP64 pipe for ~16 cycles).
// FP64 takes 4 columns per chunk (16 accumulators: about 80 registers, 3 blocks of 256 threads per
// SM, so the usual grid runs in one wave); FP32 keeps 8.
template <typename P>
__host__ __device__ constexpr int dot_cols() { return sizeof(P) == 8 ? 4 : 8; }
// shared memory of the dot kernels' transposed reduction: [8 warps][4 dot_cols][33]
template <typename P>
__host__ __device__ constexpr size_t dot_smem() { return (size_t)kColGroups * 4 * dot_cols<P>() * 33 * sizeof(P); }

// R: storage type of V and y; P: arithmetic type of the projections (P = float on FP64 data is the
// mixed form's FP32 inner product).
template <typename R, typename P = R>
__device__ __forceinline__ void dot_body(const GSArgs& a, int64_t p0, int64_t p1, P* red /* [8 warps][4 dot_cols][33] */,
                                         int rb) {
  using C = cplx<R>;
  using Q = cplx<P>;
  const C* V = (const C*)a.V;
  const C* y = (const C*)a.y;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t n = a.n, h = a.h;
  constexpr int NC = dot_cols<P>();
  constexpr int NA = 4 * NC;                     // accumulators per lane (32 or 16)
  P* wred = red + (size_t)q * NA * 33;
  double* out = a.part_dot;
  for (int c0 = NC * q; c0 <= a.j; c0 += NC * kColGroups) {
    P acc[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = (P)0;
    const int ncol = min(NC, a.j + 1 - c0);
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const C yy1 = y[p], yy2 = y[h + p];
      const Q y1 = mk<P>((P)yy1.x, (P)yy1.y), y2 = mk<P>((P)yy2.x, (P)yy2.y);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < ncol) {
          const C* vi = V + (int64_t)(c0 + c) * n;
          const C vv1 = vi[p], vv2 = vi[h + p];
          const Q v1 = mk<P>((P)vv1.x, (P)vv1.y), v2 = mk<P>((P)vv2.x, (P)vv2.y);
          // c_v += conj(v1) y1 + conj(v2) y2 ;  c_w += v1 y2 - v2 y1
          acc[c][0] = fma(v1.x, y1.x, fma(v1.y, y1.y, fma(v2.x, y2.x, fma(v2.y, y2.y, acc[c][0]))));
          acc[c][1] = fma(v1.x, y1.y, fma(-v1.y, y1.x, fma(v2.x, y2.y, fma(-v2.y, y2.x, acc[c][1]))));
          acc[c][2] = fma(v1.x, y2.x, fma(-v1.y, y2.y, fma(-v2.x, y1.x, fma(v2.y, y1.y, acc[c][2]))));
          acc[c][3] = fma(v1.x, y2.y, fma(v1.y, y2.x, fma(-v2.x, y1.y, fma(-v2.y, y1.x, acc[c][3]))));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int t = 0; t < 4; ++t) wred[(4 * c + t) * 33 + lane] = acc[c][t];
    __syncwarp();
    // accumulator row = lane % NA; 32 / NA lanes share a row, each adding NA of its 32 entries
    const int row = lane % NA, part = lane / NA;
    P sum = (P)0;
#pragma unroll 8
    for (int l = 0; l < NA; ++l) sum += wred[row * 33 + part * NA + l];
#pragma unroll
    for (int o = NA; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __syncwarp();
    const int c = row >> 2, t = row & 3;
    if (lane < NA && c < ncol) out[((int64_t)(c0 + c) * a.nblk + rb) * 4 + t] = (double)sum;
  }
}

// First pass: alpha from the matvec partials, y -= alpha v_j, b0 partials, then the dot products.
template <typename R, typename P = R>
__global__ void __launch_bounds__(kGsThreads, 3)
gs_first_kernel(GSArgs a, const double2* __restrict__ alpha_part, int n_alpha_part) {
  using C = cplx<R>;
  __shared__ double sh[32];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_alpha_part; i += kGsThreads) {
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
  const R alpha = (R)ar;
  const C* vj = (const C*)a.V + (int64_t)j * a.n;
  C* y = (C*)a.y;
  const int64_t h = a.h;
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
  R nrm_r = 0;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kGsThreads) {
    C y1 = y[p], y2 = y[h + p];
    const C v1 = vj[p], v2 = vj[h + p];
    y1.x -= alpha * v1.x; y1.y -= alpha * v1.y;
    y2.x -= alpha * v2.x; y2.y -= alpha * v2.y;
    y[p] = y1;
    y[h + p] = y2;
    nrm_r += cabs2w(y1) + cabs2w(y2);
  }
  const double nrm = block_sum((double)nrm_r, sh);  // its barriers also publish the y writes to the whole block
  if (threadIdx.x == 0) a.part_nrm[blockIdx.x] = nrm;
  dot_body<R, P>(a, p0, p1, (P*)dyn_smem, blockIdx.x);
}

// Later passes: first finish the test of the previous pass, then the dot products.
template <typename R>
__global__ void __launch_bounds__(kGsThreads, 3) gs_dot_kernel(GSArgs a, int pass) {
  __shared__ double sh[32];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ int s_skip;
  StepState* st = a.st;
  if (threadIdx.x == 0) s_skip = st->done;
  __syncthreads();
  if (s_skip) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < a.nblk; b += kGsThreads) s += a.part_nrm[b];
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
  dot_body<R>(a, p0, p1, (R*)dyn_smem, blockIdx.x);
}

// Reduce the dot partials of every column (one block per column); with `first`, block j+1 also
// reduces b0.
__global__ void __launch_bounds__(kRedThreads) gs_reduce_kernel(GSArgs a, int first) {
  __shared__ double sh[32];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = first ? 0 : a.st->done;
  __syncthreads();
  if (s_skip) return;
  const int col = blockIdx.x;
  if (col <= a.j) {
    const coef4* src = (const coef4*)a.part_dot + (int64_t)col * a.nblk;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int b = threadIdx.x; b < a.nblk; b += kRedThreads) {
      const coef4 c = src[b];
      s0 += c.vr; s1 += c.vi; s2 += c.wr; s3 += c.wi;
    }
    s0 = block_sum(s0, sh); s1 = block_sum(s1, sh); s2 = block_sum(s2, sh); s3 = block_sum(s3, sh);
    if (threadIdx.x == 0) {
      coef4 c; c.vr = s0; c.vi = s1; c.wr = a.no_w ? 0.0 : s2; c.wi = a.no_w ? 0.0 : s3;
      a.coef[col] = c;
    }
  } else {
    double s = 0.0;
    for (int b = threadIdx.x; b < a.nblk; b += kRedThreads) s += a.part_nrm[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) a.st->nrm[0] = sqrt(s);
  }
}

// y -= V c_v + W c_w over this block's rows; partial ||y||^2.
template <typename R>
__global__ void __launch_bounds__(kGsThreads) gs_update_kernel(GSArgs a) {
  using C = cplx<R>;
  extern __shared__ coef4 sc[];
  __shared__ C red1[kColGroups][32], red2[kColGroups][32];
  __shared__ double sh[32];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = a.st->done;
  __syncthreads();
  if (s_skip) return;
  const int j = a.j;
  for (int i = threadIdx.x; i <= j; i += kGsThreads) sc[i] = a.coef[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) a.st->units_update += (double)(j + 1) * (double)a.h;
  __syncthreads();
  const C* V = (const C*)a.V;
  C* y = (C*)a.y;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t n = a.n, h = a.h;
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
  R nrm_r = 0;
  for (int64_t pb = p0; pb < p1; pb += 32) {
    const int64_t p = pb + lane;
    const bool ok = p < p1;
    C acc1 = mk<R>(0, 0), acc2 = mk<R>(0, 0);
    if (ok) {
      for (int i = q; i <= j; i += kColGroups) {
        const C* vi = V + (int64_t)i * n;
        const C v1 = vi[p], v2 = vi[h + p];
        const C cv = mk<R>((R)sc[i].vr, (R)sc[i].vi);
        const C cw = mk<R>((R)sc[i].wr, (R)sc[i].wi);
        const C ncw = mk<R>(-cw.x, -cw.y);
        acc1 = cfma(v1, cv, acc1);      //  v1 c_v
        acc1 = cfmac(v2, ncw, acc1);    // -conj(v2) c_w
        acc2 = cfma(v2, cv, acc2);      //  v2 c_v
        acc2 = cfmac(v1, cw, acc2);     // +conj(v1) c_w
      }
    }
    red1[q][lane] = acc1;
    red2[q][lane] = acc2;
    __syncthreads();
    if (q == 0 && ok) {
      C s1 = red1[0][lane], s2 = red2[0][lane];
#pragma unroll
      for (int g = 1; g < kColGroups; ++g) { s1 = cadd(s1, red1[g][lane]); s2 = cadd(s2, red2[g][lane]); }
      const C y1 = csub(y[p], s1), y2 = csub(y[h + p], s2);
      y[p] = y1;
      y[h + p] = y2;
      nrm_r += cabs2w(y1) + cabs2w(y2);
    }
    __syncthreads();
  }
  const double nrm = block_sum((double)nrm_r, sh);
  if (threadIdx.x == 0) a.part_nrm[blockIdx.x] = nrm;
}

// v_{j+1} = y / beta; t_{j+1,j} = beta; breakdown check.
template <typename R>
__global__ void __launch_bounds__(kGsThreads) gs_normalize_kernel(GSArgs a) {
  using C = cplx<R>;
  __shared__ double sh[32];
  StepState* st = a.st;
  const int done = st->done;
  double beta;
  if (done) {
    beta = st->beta;
  } else {  // the pass cap was reached: keep the norm after the last pass
    double s = 0.0;
    for (int b = threadIdx.x; b < a.nblk; b += kGsThreads) s += a.part_nrm[b];
    beta = sqrt(block_sum(s, sh));
  }
  const double tmax = st->tmax;
  const bool brk = !(beta > 1e-14 * fmax(tmax, 1.0));
  const R inv = brk ? (R)0 : (R)(1.0 / beta);
  const C* y = (const C*)a.y;
  C* v = (C*)a.V + (int64_t)(a.j + 1) * a.n;
  const int64_t h = a.h;
  const int64_t p0 = (int64_t)blockIdx.x * a.rows_per_block;
  const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kGsThreads) {
    v[p] = cscale(y[p], inv);
    v[h + p] = cscale(y[h + p], inv);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int j = a.j;
    a.T[(int64_t)(j + 1) * a.ldt + j] = beta;        // t_{j+1,j}
    if (j + 1 < a.m) a.T[(int64_t)j * a.ldt + j + 1] = beta;
    if (brk) st->status = 5;
  }
}

template <typename R>
__global__ void fill_ones_kernel(cplx<R>* v, int64_t n, R val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = mk<R>(val, (R)0);
}

template <typename R>
__global__ void fill_random_kernel(cplx<R>* v, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = mk<R>((R)u01_sym(seed + 2 * (uint64_t)i), (R)u01_sym(seed + 2 * (uint64_t)i + 1));
}

// v64 = sum of the first ncol columns of an FP32 basis (ld n), promoted to FP64.
__global__ void sum_columns_kernel(const float2* X, int64_t n, int ncol, double2* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < ncol; ++c) {
      const float2 v = X[(int64_t)c * n + i];
      re += v.x;
      im += v.y;
    }
    out[i] = make_double2(re, im);
  }
}

__global__ void c128_to_c64_kernel(const double2* in, float2* out, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// FP64 links [4][V][9] -> FP32 structure-of-arrays [4][9][V].
__global__ void links_soa_kernel(const double2* in, float2* out, int64_t vol) {
  const int64_t total = 36 * vol;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q % vol;
    const int64_t me = q / vol;            // mu * 9 + e
    const int64_t mu = me / 9, e = me % 9;
    const double2 v = in[(mu * vol + s) * 9 + e];
    out[q] = make_float2((float)v.x, (float)v.y);
  }
}

template <typename R>
__global__ void sumsq_kernel(const cplx<R>* v, int64_t n, double* part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += cabs2(v[i]);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename R>
__global__ void scale_by_norm_kernel(cplx<R>* v, int64_t n, const double* part, int nblk) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = block_sum(s, sh);
  const R inv = (R)(1.0 / sqrt(s));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = cscale(v[i], inv);
}

template <typename R>
__global__ void jsym_check_kernel(const cplx<R>* v, const cplx<R>* y, int64_t h, double* out) {
  __shared__ double sh[32];
  double wr = 0, wi = 0, yy = 0, vv = 0;
  for (int64_t p = threadIdx.x; p < h; p += blockDim.x) {
    const cplx<R> v1 = v[p], v2 = v[h + p], y1 = y[p], y2 = y[h + p];
    // w^H y with w = J v^*: sum (v1 y2 - v2 y1)
    wr += (double)v1.x * y2.x - (double)v1.y * y2.y - ((double)v2.x * y1.x - (double)v2.y * y1.y);
    wi += (double)v1.x * y2.y + (double)v1.y * y2.x - ((double)v2.x * y1.y + (double)v2.y * y1.x);
    yy += cabs2(y1) + cabs2(y2);
    vv += cabs2(v1) + cabs2(v2);
  }
  wr = block_sum(wr, sh); wi = block_sum(wi, sh); yy = block_sum(yy, sh); vv = block_sum(vv, sh);
  if (threadIdx.x == 0) { out[0] = wr; out[1] = wi; out[2] = yy; out[3] = vv; }
}

}  // namespace

// ------------------------------------------------------------------ one cooperative launch per step
// The whole Gram-Schmidt part of one Lanczos step (alpha, y -= alpha v_j, every pass of dot, reduce and
// update with the sqrt(2) test, normalisation) in a single cooperative launch: the grid synchronises
// where the multi-kernel path ends one launch and starts the next, and each block walks row blocks
// rb = blockIdx.x, blockIdx.x + gridDim.x, ... of the same partition (so partials, summation orders
// and results do not depend on the grid size).  Every block computes the norms of the test from the
// same partials in the same order, so all blocks take the same decision.  nrm2 holds two slots of
// nblk norm partials, alternating between passes.
template <typename R>
__device__ R update_rows(const GSArgs& a, int64_t p0, int64_t p1, const coef4* sc, cplx<R> (*red1)[32],
                         cplx<R> (*red2)[32]) {
  using C = cplx<R>;
  const C* V = (const C*)a.V;
  C* y = (C*)a.y;
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t n = a.n, h = a.h;
  const int j = a.j;
  R nrm_r = 0;
  for (int64_t pb = p0; pb < p1; pb += 32) {
    const int64_t p = pb + lane;
    const bool ok = p < p1;
    C acc1 = mk<R>(0, 0), acc2 = mk<R>(0, 0);
    if (ok) {
      for (int i = q; i <= j; i += kColGroups) {
        const C* vi = V + (int64_t)i * n;
        const C v1 = vi[p], v2 = vi[h + p];
        const C cv = mk<R>((R)sc[i].vr, (R)sc[i].vi);
        const C cw = mk<R>((R)sc[i].wr, (R)sc[i].wi);
        const C ncw = mk<R>(-cw.x, -cw.y);
        acc1 = cfma(v1, cv, acc1);
        acc1 = cfmac(v2, ncw, acc1);
        acc2 = cfma(v2, cv, acc2);
        acc2 = cfmac(v1, cw, acc2);
      }
    }
    red1[q][lane] = acc1;
    red2[q][lane] = acc2;
    __syncthreads();
    if (q == 0 && ok) {
      C s1 = red1[0][lane], s2 = red2[0][lane];
#pragma unroll
      for (int g = 1; g < kColGroups; ++g) { s1 = cadd(s1, red1[g][lane]); s2 = cadd(s2, red2[g][lane]); }
      const C y1 = csub(y[p], s1), y2 = csub(y[h + p], s2);
      y[p] = y1;
      y[h + p] = y2;
      nrm_r += cabs2w(y1) + cabs2w(y2);
    }
    __syncthreads();
  }
  return nrm_r;
}

// sqrt of the sum of nblk partials, the same fixed order in every block
__device__ __forceinline__ double coop_norm(const double* part, int nblk, double* sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kGsThreads) s += part[b];
  return sqrt(block_sum(s, sh));
}

template <typename R>
__global__ void __launch_bounds__(kGsThreads, 3)
gs_step_coop_kernel(GSArgs a, const double2* __restrict__ alpha_part, int n_alpha_part, int passes,
                    double* __restrict__ nrm2) {
  using C = cplx<R>;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32];
  __shared__ C red1[kColGroups][32], red2[kColGroups][32];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  R* dred = (R*)dyn_smem;
  coef4* sc = (coef4*)(dyn_smem + dot_smem<R>());
  const int j = a.j;
  const int64_t h = a.h;
  const int nblk = a.nblk;
  StepState* st = a.st;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  // alpha = Re(v_j^H A v_j) from the product's partials (every block, same order)
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_alpha_part; i += kGsThreads) {
    ar += alpha_part[i].x;
    ai += alpha_part[i].y;
  }
  ar = block_sum(ar, sh);
  ai = block_sum(ai, sh);
  double tmax = st->tmax;
  tmax = fmax(tmax, fabs(ar));
  if (j > 0) tmax = fmax(tmax, fabs(a.T[(int64_t)j * a.ldt + j - 1]));
  if (lead) {
    a.T[(int64_t)j * a.ldt + j] = ar;
    st->alpha_im = ai;
    st->done = 0;
    st->tmax = tmax;
    st->n_passes += 1;
    st->units_first += (double)(j + 1) * (double)h;
  }
  const R alpha = (R)ar;
  const C* vj = (const C*)a.V + (int64_t)j * a.n;
  C* y = (C*)a.y;
  for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {   // y -= alpha v_j; b0 partials; pass-1 dots
    const int64_t p0 = (int64_t)rb * a.rows_per_block;
    const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
    R nrm_r = 0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kGsThreads) {
      C y1 = y[p], y2 = y[h + p];
      const C v1 = vj[p], v2 = vj[h + p];
      y1.x -= alpha * v1.x; y1.y -= alpha * v1.y;
      y2.x -= alpha * v2.x; y2.y -= alpha * v2.y;
      y[p] = y1;
      y[h + p] = y2;
      nrm_r += cabs2w(y1) + cabs2w(y2);
    }
    const double nb = block_sum((double)nrm_r, sh);
    if (threadIdx.x == 0) nrm2[rb] = nb;
    dot_body<R, R>(a, p0, p1, dred, rb);
  }
  double bref = 0.0, beta = 0.0;
  for (int pass = 1;; ++pass) {
    grid.sync();                                           // dot partials and norm partials complete
    if (pass == 1) {
      bref = coop_norm(nrm2, nblk, sh);                    // b0
      if (lead) st->nrm[0] = bref;
    }
    for (int c = blockIdx.x; c <= j; c += gridDim.x) {     // coefficients of column c
      const coef4* src = (const coef4*)a.part_dot + (int64_t)c * nblk;
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int b = threadIdx.x; b < nblk; b += kGsThreads) {
        const coef4 cc = src[b];
        s0 += cc.vr; s1 += cc.vi; s2 += cc.wr; s3 += cc.wi;
      }
      s0 = block_sum(s0, sh); s1 = block_sum(s1, sh); s2 = block_sum(s2, sh); s3 = block_sum(s3, sh);
      if (threadIdx.x == 0) {
        coef4 cc; cc.vr = s0; cc.vi = s1; cc.wr = a.no_w ? 0.0 : s2; cc.wi = a.no_w ? 0.0 : s3;
        a.coef[c] = cc;
      }
    }
    grid.sync();                                           // coefficients complete
    for (int i = threadIdx.x; i <= j; i += kGsThreads) sc[i] = a.coef[i];
    __syncthreads();
    double* slot = nrm2 + (size_t)(pass & 1) * nblk;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
      const int64_t p0 = (int64_t)rb * a.rows_per_block;
      const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
      const double nb = block_sum((double)update_rows<R>(a, p0, p1, sc, red1, red2), sh);
      if (threadIdx.x == 0) slot[rb] = nb;
    }
    if (lead) st->units_update += (double)(j + 1) * (double)h;
    grid.sync();                                           // updated y and its norm partials complete
    const double b1 = coop_norm(slot, nblk, sh);
    if (lead && pass < 8) st->nrm[pass] = b1;
    if (kSqrt2 * b1 > bref || pass >= passes) {            // the sqrt(2) test, or the pass cap
      beta = b1;
      break;
    }
    bref = b1;
    if (lead) {
      st->n_passes += 1;
      st->units_dot += (double)(j + 1) * (double)h;
    }
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {  // dots of the next pass on this block's rows
      const int64_t p0 = (int64_t)rb * a.rows_per_block;
      const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
      dot_body<R, R>(a, p0, p1, dred, rb);
    }
  }
  // normalise: v_{j+1} = y / beta, t_{j+1,j} = beta; breakdown below 1e-14 max(max|t|, 1)
  const bool brk = !(beta > 1e-14 * fmax(tmax, 1.0));
  const R inv = brk ? (R)0 : (R)(1.0 / beta);
  C* v = (C*)a.V + (int64_t)(j + 1) * a.n;
  for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
    const int64_t p0 = (int64_t)rb * a.rows_per_block;
    const int64_t p1 = min(p0 + (int64_t)a.rows_per_block, h);
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kGsThreads) {
      v[p] = cscale(y[p], inv);
      v[h + p] = cscale(y[h + p], inv);
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

int gs_blocks(int64_t h, int* rows_per_block) {
  // Row tiles of 32 row pairs, about four blocks per SM.
  const int64_t tiles = (h + 31) / 32;
  const int64_t target = 4 * 152;
  const int64_t tpb = (tiles + target - 1) / target;
  const int rpb = (int)(32 * (tpb < 1 ? 1 : tpb));
  if (rows_per_block) *rows_per_block = rpb;
  return (int)((h + rpb - 1) / rpb);
}


template <typename R>
cudaError_t launch_gs_first(const GSArgs& a, const double2* alpha_part, int n_alpha_part, cudaStream_t s) {
  if (dot_smem<R>() > 48 * 1024) {  // per device, so set on every launch (cheap)
    cudaError_t e = allow_dyn_smem((const void*)gs_first_kernel<R>, (size_t)dot_smem<R>());
    if (e != cudaSuccess) return e;
  }
  gs_first_kernel<R><<<a.nblk, kGsThreads, dot_smem<R>(), s>>>(a, alpha_part, n_alpha_part);
  return cudaGetLastError();
}

cudaError_t launch_gs_reduce(const GSArgs& a, int first, cudaStream_t s) {
  gs_reduce_kernel<<<a.j + 1 + (first ? 1 : 0), kRedThreads, 0, s>>>(a, first);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gs_update(const GSArgs& a, cudaStream_t s) {
  gs_update_kernel<R><<<a.nblk, kGsThreads, (size_t)(a.j + 1) * sizeof(coef4), s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gs_dot(const GSArgs& a, int pass, cudaStream_t s) {
  if (dot_smem<R>() > 48 * 1024) {
    cudaError_t e = allow_dyn_smem((const void*)gs_dot_kernel<R>, (size_t)dot_smem<R>());
    if (e != cudaSuccess) return e;
  }
  gs_dot_kernel<R><<<a.nblk, kGsThreads, dot_smem<R>(), s>>>(a, pass);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gs_normalize(const GSArgs& a, cudaStream_t s) {
  gs_normalize_kernel<R><<<a.nblk, kGsThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fill_ones(void* v, int64_t n, cudaStream_t s) {
  fill_ones_kernel<R><<<256, 256, 0, s>>>((cplx<R>*)v, n, (R)(1.0 / sqrt((double)n)));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fill_random(void* v, int64_t n, uint64_t seed, cudaStream_t s) {
  fill_random_kernel<R><<<256, 256, 0, s>>>((cplx<R>*)v, n, seed);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_normalize_col(void* v, int64_t n, double* part, int nblk, cudaStream_t s) {
  sumsq_kernel<R><<<nblk, 256, 0, s>>>((const cplx<R>*)v, n, part);
  scale_by_norm_kernel<R><<<nblk, 256, 0, s>>>((cplx<R>*)v, n, part, nblk);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_jsym_check(const void* v, const void* y, int64_t h, double* out, cudaStream_t s) {
  jsym_check_kernel<R><<<1, 1024, 0, s>>>((const cplx<R>*)v, (const cplx<R>*)y, h, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_columns(const void* X32, int64_t n, int ncol, void* out64, cudaStream_t s) {
  sum_columns_kernel<<<1024, 256, 0, s>>>((const float2*)X32, n, ncol, (double2*)out64);
  return cudaGetLastError();
}

cudaError_t launch_c128_to_c64(const void* in, void* out, int64_t count, cudaStream_t s) {
  c128_to_c64_kernel<<<1024, 256, 0, s>>>((const double2*)in, (float2*)out, count);
  return cudaGetLastError();
}

cudaError_t launch_links_soa(const void* in, void* out, int64_t vol, cudaStream_t s) {
  links_soa_kernel<<<1024, 256, 0, s>>>((const double2*)in, (float2*)out, vol);
  return cudaGetLastError();
}

template <typename R>
size_t gs_coop_smem(int m) { return dot_smem<R>() + (size_t)(m + 1) * sizeof(coef4); }

template <typename R>
cudaError_t gs_coop_occupancy(int m, int* per_sm) {
  int dev = 0, coop = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  const size_t sm = gs_coop_smem<R>(m);
  if ((e = allow_dyn_smem((const void*)gs_step_coop_kernel<R>, (size_t)sm)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gs_step_coop_kernel<R>, kGsThreads, sm)) != cudaSuccess)
    return e;
  *per_sm = coop ? per : 0;
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_gs_step_coop(const GSArgs& a, const double2* alpha_part, int n_alpha_part, int passes,
                                double* nrm2, int grid, cudaStream_t s) {
  GSArgs aa = a;
  const double2* ap = alpha_part;
  int na = n_alpha_part, ps = passes;
  double* nr = nrm2;
  void* args[] = {&aa, &ap, &na, &ps, &nr};
  return cudaLaunchCooperativeKernel((const void*)gs_step_coop_kernel<R>, dim3(grid), dim3(kGsThreads), args,
                                     gs_coop_smem<R>(a.m), s);
}
template cudaError_t gs_coop_occupancy<double>(int, int*);
template cudaError_t gs_coop_occupancy<float>(int, int*);
template cudaError_t launch_gs_step_coop<double>(const GSArgs&, const double2*, int, int, double*, int, cudaStream_t);
template cudaError_t launch_gs_step_coop<float>(const GSArgs&, const double2*, int, int, double*, int, cudaStream_t);
template cudaError_t launch_gs_first<double>(const GSArgs&, const double2*, int, cudaStream_t);
template cudaError_t launch_gs_first<float>(const GSArgs&, const double2*, int, cudaStream_t);
template cudaError_t launch_gs_update<float>(const GSArgs&, cudaStream_t);
template cudaError_t launch_gs_dot<float>(const GSArgs&, int, cudaStream_t);
template cudaError_t launch_gs_normalize<float>(const GSArgs&, cudaStream_t);
template cudaError_t launch_fill_ones<float>(void*, int64_t, cudaStream_t);
template cudaError_t launch_normalize_col<float>(void*, int64_t, double*, int, cudaStream_t);
template cudaError_t launch_gs_update<double>(const GSArgs&, cudaStream_t);
template cudaError_t launch_gs_dot<double>(const GSArgs&, int, cudaStream_t);
template cudaError_t launch_gs_normalize<double>(const GSArgs&, cudaStream_t);
template cudaError_t launch_fill_ones<double>(void*, int64_t, cudaStream_t);
template cudaError_t launch_fill_random<double>(void*, int64_t, uint64_t, cudaStream_t);
template cudaError_t launch_fill_random<float>(void*, int64_t, uint64_t, cudaStream_t);
template cudaError_t launch_normalize_col<double>(void*, int64_t, double*, int, cudaStream_t);
template cudaError_t launch_jsym_check<double>(const void*, const void*, int64_t, double*, cudaStream_t);

}  // namespace jtr
