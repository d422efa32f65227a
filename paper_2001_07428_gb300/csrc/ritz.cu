// ritz.cu -- the restart of Algorithm 1 on the device: Rayleigh-Ritz solve of T_m, the basis
// rotation V_m := V_m Z_m (Corollary 2 keeps V and W = J V^* orthogonal under it), the shrink to
// k + 1 vectors with v_{k+1} = v_{m+1}, and the output gather with partners y = J x^* (eq. (2)).
#include "internal.h"
#include "ritz_dev.cuh"
#include "../../include/jtrlan.h"

namespace jtr {

namespace {

// ------------------------------------------------------------------ cyclic Jacobi, one CTA
// T_m = Z Lambda Z^T for the real symmetric m x m leading block of T-bar (arrowhead plus
// tridiagonal).  Parallel Jacobi: each round applies mp/2 disjoint plane rotations chosen by the
// round-robin ordering (player 0 fixed, the others rotate), so a sweep of mp-1 rounds visits every
// pair once.  Rotation angles follow Rutishauser's stable formulas (Golub & Van Loan, sym.schur2).
// An odd m is padded with one decoupled index.  Sweeps stop when no off-diagonal entry exceeds
// 1e-17 (|a_pp| + |a_qq|) -- i.e. T is diagonal to working precision -- or after 60 sweeps.
constexpr int kRitzThreads = 1024;
constexpr int kMaxPairs = 512;

__global__ void __launch_bounds__(kRitzThreads)
ritz_jacobi_kernel(const double* __restrict__ T, int ldt, int m, int which, double* __restrict__ lam,
                   double* __restrict__ Zout, double* __restrict__ work, int use_smem, const int* __restrict__ gate,
                   long long* __restrict__ fallbacks) {
  extern __shared__ double dsm[];
  if (gate && *gate == 0) return;   // the fast path succeeded
  if (fallbacks && threadIdx.x == 0) *fallbacks += 1;
  __shared__ double rc[kMaxPairs], rs[kMaxPairs], rt[kMaxPairs], rapp[kMaxPairs], raqq[kMaxPairs],
      rapq[kMaxPairs];
  __shared__ int rp[kMaxPairs], rq[kMaxPairs];
  __shared__ int s_rot;
  __shared__ int rank_of[2 * kMaxPairs];
  const int mp = m + (m & 1);
  const int half = mp / 2;
  double* A = use_smem ? dsm : work;
  double* Z = A + (size_t)mp * mp;
  const int tid = threadIdx.x;
  for (int e = tid; e < mp * mp; e += kRitzThreads) {
    const int r = e / mp, c = e % mp;
    A[e] = (r < m && c < m) ? T[(size_t)r * ldt + c] : 0.0;
    Z[e] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      for (int k = tid; k < half; k += kRitzThreads) {
        // round-robin pairing: position 0 holds player 0, positions 1..mp-1 rotate
        const int a = (k == 0) ? 0 : ((k - 1 + round) % (mp - 1)) + 1;
        const int b = ((mp - 2 - k + round) % (mp - 1)) + 1;
        const int p = min(a, b), q = max(a, b);
        const double app = A[p * mp + p], aqq = A[q * mp + q], apq = A[p * mp + q];
        double c = 1.0, s = 0.0, t = 0.0;
        if (fabs(apq) > 1e-17 * (fabs(app) + fabs(aqq)) && fabs(apq) > 1e-300) {
          const double tau = (aqq - app) / (2.0 * apq);
          t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
          s_rot = 1;
        }
        rp[k] = p; rq[k] = q; rc[k] = c; rs[k] = s; rt[k] = t;
        rapp[k] = app; raqq[k] = aqq; rapq[k] = apq;
      }
      __syncthreads();
      // rows p, q  <-  J^T A
      for (int e = tid; e < half * mp; e += kRitzThreads) {
        const int k = e / mp, l = e % mp;
        if (rs[k] == 0.0) continue;
        const int p = rp[k], q = rq[k];
        const double c = rc[k], s = rs[k];
        const double ap = A[p * mp + l], aq = A[q * mp + l];
        A[p * mp + l] = c * ap - s * aq;
        A[q * mp + l] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q  <-  A J,  Z <- Z J
      for (int e = tid; e < half * mp; e += kRitzThreads) {
        const int k = e / mp, l = e % mp;
        if (rs[k] == 0.0) continue;
        const int p = rp[k], q = rq[k];
        const double c = rc[k], s = rs[k];
        const double ap = A[l * mp + p], aq = A[l * mp + q];
        A[l * mp + p] = c * ap - s * aq;
        A[l * mp + q] = s * ap + c * aq;
        const double zp = Z[l * mp + p], zq = Z[l * mp + q];
        Z[l * mp + p] = c * zp - s * zq;
        Z[l * mp + q] = s * zp + c * zq;
      }
      __syncthreads();
      for (int k = tid; k < half; k += kRitzThreads) {
        if (rs[k] == 0.0) continue;
        const int p = rp[k], q = rq[k];
        A[p * mp + q] = 0.0;
        A[q * mp + p] = 0.0;
        A[p * mp + p] = rapp[k] - rt[k] * rapq[k];
        A[q * mp + q] = raqq[k] + rt[k] * rapq[k];
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  // sort the m eigenvalues toward the wanted end (stable in the index)
  for (int i = tid; i < m; i += kRitzThreads) {
    const double li = A[i * mp + i];
    int r = 0;
    for (int k = 0; k < m; ++k) {
      const double lk = A[k * mp + k];
      const bool before = (which == JTRLAN_LARGEST) ? (lk > li) : (lk < li);
      if (before || (lk == li && k < i)) ++r;
    }
    rank_of[r] = i;
  }
  __syncthreads();
  for (int r = tid; r < m; r += kRitzThreads) lam[r] = A[rank_of[r] * mp + rank_of[r]];
  for (int e = tid; e < m * m; e += kRitzThreads) {
    const int c = e / m, l = e % m;  // Zout column-major: component l of eigenvector c
    Zout[(size_t)c * m + l] = Z[l * mp + rank_of[c]];
  }
}

constexpr int kBisectWarps = 4;

__global__ void __launch_bounds__(32 * kBisectWarps)
ritz_bisect_kernel(const double* __restrict__ T, int ldt, int m, int k, int kk, int which, double* __restrict__ lam,
                   double* __restrict__ Zout, int* __restrict__ ok) {
  extern __shared__ double rsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kBisectWarps + warp;
  if (i >= kk) return;
  double* z = rsm + (size_t)warp * 3 * m;
  const int r = (which == JTRLAN_LARGEST) ? m - 1 - i : i;   // index in ascending order
  const double lambda = ritz_pair_warp(T, ldt, m, k, r, z, z + m, z + 2 * m, Zout + (size_t)i * m);
  if (lane == 0) {
    lam[i] = lambda;
    ok[i] = (lambda == lambda) ? 1 : 0;
  }
}

// One block: residual ||T z_i - lambda_i z_i||, orthogonality of neighbours, the per-pair inertia
// flags; sets *fallback (read by the Jacobi kernel).
__global__ void __launch_bounds__(256)
ritz_check_kernel(const double* __restrict__ T, int ldt, int m, int k, int kk, int which, const double* __restrict__ lam,
                  const double* __restrict__ Z, const int* __restrict__ ok, int* __restrict__ fallback) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const TbarView t{T, ldt, m, k};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double tn = 0.0;
  for (int j = 0; j < m; ++j) tn = fmax(tn, fabs(t.diag(j)));
  for (int i = warp; i < kk; i += 8) {
    const double* z = Z + (size_t)i * m;
    double res = 0.0, dot = 0.0, nn = 0.0;
    for (int j = lane; j < m; j += 32) {
      double v = t.diag(j) * z[j];
      if (j < k) v += t.arrow(j) * z[k];
      else {
        if (j == k) for (int q = 0; q < k; ++q) v += t.arrow(q) * z[q];
        else v += t.off(j - 1) * z[j - 1];
        if (j + 1 < m) v += t.off(j) * z[j + 1];
      }
      v -= lam[i] * z[j];
      res += v * v;
      nn += z[j] * z[j];
      if (i + 1 < kk) dot += z[j] * Z[(size_t)(i + 1) * m + j];
    }
    res = warp_sum(res); dot = warp_sum(dot); nn = warp_sum(nn);
    if (lane == 0) {
      bool good = ok[i] && sqrt(res) <= 1e-11 * fmax(tn, 1e-300) && fabs(nn - 1.0) <= 1e-12 && fabs(dot) <= 1e-9;
      if (i + 1 < kk) good = good && ((which == JTRLAN_LARGEST) ? lam[i] > lam[i + 1] : lam[i] < lam[i + 1]);
      if (!good) atomicExch(&bad, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *fallback = bad;
}

// ------------------------------------------------------------------ rotation V_m Z
// Real GEMM on the interleaved view: V as a (2n x m) real matrix (column-major, ld 2n) times
// Z (m x kk) gives Vout (2n x kk).  FP64: a 64 x 32 output tile per block, 8 outputs per thread.
template <typename R>
__global__ void __launch_bounds__(256)
rotate_kernel(const R* __restrict__ V, int64_t rows, int m, const double* __restrict__ Z, int kk, R* __restrict__ out) {
  constexpr int BM = 64, BN = 32, BK = 16;
  __shared__ R As[BK][BM];
  __shared__ double Bs[BK][BN];
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tr = tid % 16, tc = tid / 16;  // 4 rows (tr, tr+16, ...) x 2 cols (tc, tc+16)
  double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int k0 = 0; k0 < m; k0 += BK) {
    for (int e = tid; e < BK * BM; e += 256) {
      const int kk_ = e / BM, r = e % BM;
      const int64_t gr = row0 + r;
      As[kk_][r] = (gr < rows && k0 + kk_ < m) ? V[(int64_t)(k0 + kk_) * rows + gr] : (R)0;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk_ = e / BN, c = e % BN;
      Bs[kk_][c] = (k0 + kk_ < m && col0 + c < kk) ? Z[(int64_t)(col0 + c) * m + k0 + kk_] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int x = 0; x < BK; ++x) {
      double a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = (double)As[x][tr + 16 * i];
      b[0] = Bs[x][tc];
      b[1] = Bs[x][tc + 16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = fma(a[i], b[0], acc[i][0]);
        acc[i][1] = fma(a[i], b[1], acc[i][1]);
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
      if (gc < kk) out[(int64_t)gc * rows + gr] = (R)acc[i][jx];
    }
  }
}

// FP32 rotation for the mixed-precision phase: Z rounded to FP32, FP32 accumulation.
__global__ void __launch_bounds__(256)
rotate32_kernel(const float* __restrict__ V, int64_t rows, int m, const double* __restrict__ Z, int kk,
                float* __restrict__ out) {
  constexpr int BM = 128, BN = 32, BK = 16;
  __shared__ float As[BK][BM];
  __shared__ float Bs[BK][BN];
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tr = tid % 32, tc = tid / 32;  // rows tr + 32 i (i < 4), cols tc + 8 j (j < 4)
  float acc[4][4] = {};
  for (int k0 = 0; k0 < m; k0 += BK) {
    for (int e = tid; e < BK * BM; e += 256) {
      const int kx = e / BM, r = e % BM;
      const int64_t gr = row0 + r;
      As[kx][r] = (gr < rows && k0 + kx < m) ? V[(int64_t)(k0 + kx) * rows + gr] : 0.f;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kx = e / BN, c = e % BN;
      Bs[kx][c] = (k0 + kx < m && col0 + c < kk) ? (float)Z[(int64_t)(col0 + c) * m + k0 + kx] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int x = 0; x < BK; ++x) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[x][tr + 32 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[x][tc + 8 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + tr + 32 * i;
    if (gr >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tc + 8 * j;
      if (gc < kk) out[(int64_t)gc * rows + gr] = acc[i][j];
    }
  }
}

template <typename R>
__global__ void shrink_kernel(cplx<R>* V, const cplx<R>* Vsrc, int64_t n, const int* perm, int k, int m) {
  const int c = blockIdx.y;
  const cplx<R>* src = (c < k) ? Vsrc + (int64_t)perm[c] * n : V + (int64_t)m * n;
  cplx<R>* dst = V + (int64_t)c * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

template <typename R>
__global__ void gather_pairs_kernel(const cplx<R>* V, int64_t n, const int* order, int nev, int partners,
                                    cplx<R>* out) {
  const int c = blockIdx.y;
  const int64_t h = n / 2;
  const cplx<R>* src = V + (int64_t)order[c] * n;
  cplx<R>* dst = out + (int64_t)c * n;
  cplx<R>* dstp = out + (int64_t)(nev + c) * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < h; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx<R> x1 = src[i], x2 = src[h + i];
    dst[i] = x1;
    dst[h + i] = x2;
    if (partners) {  // J x^* = [-x2^*; x1^*]
      dstp[i] = mk<R>(-x2.x, x2.y);
      dstp[h + i] = mk<R>(x1.x, -x1.y);
    }
  }
}

__global__ void reduce_norms_kernel(const double* part, int nblk, double* out) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(int64_t)c * nblk + b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[c] = sqrt(s);
}

__global__ void report_kernel(const double* lam, const double* Z, int m, const double* T, int ldt,
                              const StepState* st, double* rep) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    rep[i] = lam[i];
    rep[m + i] = Z[(int64_t)i * m + (m - 1)];   // z_{m,i}: last component of eigenvector i
  }
  if (threadIdx.x == 0) {
    rep[2 * m] = T[(int64_t)m * ldt + m - 1];    // t_{m+1,m} = beta_m
    rep[2 * m + 1] = (double)st->status;
    rep[2 * m + 2] = (double)st->n_passes;
    rep[2 * m + 3] = st->tmax;
    rep[2 * m + 4] = st->units_first;
    rep[2 * m + 5] = st->units_dot;
    rep[2 * m + 6] = st->units_update;
    rep[2 * m + 7] = (double)st->n_ritz_fallbacks;
  }
}

inline int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 1216 ? 1216 : (g < 1 ? 1 : g));
}

}  // namespace

cudaError_t launch_ritz(const double* T, int ldt, int m, int k, int kk, int which, double* lam, double* Z,
                        int* flags, cudaStream_t s) {
  if (m < 1 || m > 2 * kMaxPairs - 1 || k < 0 || k >= m || kk < 1 || kk > m) return cudaErrorInvalidValue;
  int* ok = flags + 1;        // kk per-pair flags
  int* fallback = flags;      // 1: run the Jacobi kernel
  const size_t bsm = (size_t)kBisectWarps * 3 * m * sizeof(double);
  if (bsm > 48 * 1024) {
    cudaError_t e = allow_dyn_smem((const void*)ritz_bisect_kernel, (size_t)bsm);
    if (e != cudaSuccess) return e;
  }
  ritz_bisect_kernel<<<(kk + kBisectWarps - 1) / kBisectWarps, 32 * kBisectWarps, bsm, s>>>(T, ldt, m, k, kk, which, lam,
                                                                                            Z, ok);
  ritz_check_kernel<<<1, 256, 0, s>>>(T, ldt, m, k, kk, which, lam, Z, ok, fallback);
  return cudaGetLastError();
}

static cudaError_t jacobi_launch(const double* T, int ldt, int m, int which, double* lam, double* Z, double* work,
                                 const int* gate, long long* fallbacks, cudaStream_t s) {
  if (m < 1 || m > 2 * kMaxPairs - 1) return cudaErrorInvalidValue;
  const int mp = m + (m & 1);
  const size_t bytes = (size_t)2 * mp * mp * sizeof(double);
  const int use_smem = bytes <= 160 * 1024;
  if (use_smem) {
    cudaError_t e = allow_dyn_smem((const void*)ritz_jacobi_kernel, (size_t)bytes);
    if (e != cudaSuccess) return e;
  }
  ritz_jacobi_kernel<<<1, kRitzThreads, use_smem ? bytes : 0, s>>>(T, ldt, m, which, lam, Z, work, use_smem, gate,
                                                                   fallbacks);
  return cudaGetLastError();
}

cudaError_t launch_ritz_fallback(const double* T, int ldt, int m, int which, double* lam, double* Z, double* work,
                                 const int* flags, long long* fallbacks, cudaStream_t s) {
  return jacobi_launch(T, ldt, m, which, lam, Z, work, flags, fallbacks, s);
}

cudaError_t launch_ritz_jacobi(const double* T, int ldt, int m, int which, double* lam, double* Z, double* work,
                               cudaStream_t s) {
  return jacobi_launch(T, ldt, m, which, lam, Z, work, nullptr, nullptr, s);
}

template <typename R>
cudaError_t launch_rotate(const void* V, int64_t n, int m, const double* Z, int kk, void* Vout, cudaStream_t s) {
  const int64_t rows = 2 * n;
  if constexpr (sizeof(R) == sizeof(float)) {
    dim3 grid((unsigned)((rows + 127) / 128), (unsigned)((kk + 31) / 32));
    rotate32_kernel<<<grid, 256, 0, s>>>((const float*)V, rows, m, Z, kk, (float*)Vout);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((kk + 31) / 32));
  rotate_kernel<R><<<grid, 256, 0, s>>>((const R*)V, rows, m, Z, kk, (R*)Vout);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_shrink(void* V, const void* Vsrc, int64_t n, const int* perm, int k, int m, cudaStream_t s) {
  dim3 grid(grid_for(n) / 4 + 1, k + 1);
  shrink_kernel<R><<<grid, 256, 0, s>>>((cplx<R>*)V, (const cplx<R>*)Vsrc, n, perm, k, m);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gather_pairs(const void* V, int64_t n, const int* order, int nev, int partners, void* out,
                                cudaStream_t s) {
  dim3 grid(grid_for(n / 2) / 4 + 1, nev);
  gather_pairs_kernel<R><<<grid, 256, 0, s>>>((const cplx<R>*)V, n, order, nev, partners, (cplx<R>*)out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_norms(const double* part, int nblk, int ncol, double* out, cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  reduce_norms_kernel<<<ncol, 128, 0, s>>>(part, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_report(const double* lam, const double* Z, int m, const double* T, int ldt, const StepState* st,
                          double* rep, cudaStream_t s) {
  report_kernel<<<1, 256, 0, s>>>(lam, Z, m, T, ldt, st, rep);
  return cudaGetLastError();
}

template cudaError_t launch_rotate<double>(const void*, int64_t, int, const double*, int, void*, cudaStream_t);
template cudaError_t launch_rotate<float>(const void*, int64_t, int, const double*, int, void*, cudaStream_t);
template cudaError_t launch_shrink<float>(void*, const void*, int64_t, const int*, int, int, cudaStream_t);
template cudaError_t launch_shrink<double>(void*, const void*, int64_t, const int*, int, int, cudaStream_t);
template cudaError_t launch_gather_pairs<double>(const void*, int64_t, const int*, int, int, void*, cudaStream_t);

}  // namespace jtr
