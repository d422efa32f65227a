// matvec.cu -- the J-symmetric operator y = A x (Algorithm 2, "v_{j+1} = A v_j").
//
// A = [[A11, A12], [A12^H, A11^T]] (Sec. 1, eq. (4)).  Only A11 and A12 are stored; the
// second block row is applied through conjugation, y2 = conj(A11 conj(x2) - A12 conj(x1)),
// so one read of A11/A12 (dense) or of the links U, W (stencil) serves both halves.
//
// Stencil blocks (periodic 4D lattice, three colours):
//   (A11 p)(s) = m0 p(s) + sum_mu [U_mu(s) p(s+mu) + U_mu(s-mu)^H p(s-mu)]
//   (A12 p)(s) = kappa sum_mu [W_mu(s) p(s+mu) - W_mu(s-mu)^T p(s-mu)]
// hence, per site s and colour a,
//   y1 = m0 x1 + sum_mu [U(s) x1(s+mu) + U(s-mu)^H x1(s-mu)] + kappa [W(s) x2(s+mu) - W(s-mu)^T x2(s-mu)]
//   y2 = m0 x2 + sum_mu [U(s)^* x2(s+mu) + U(s-mu)^T x2(s-mu)] - kappa [W(s)^* x1(s+mu) - W(s-mu)^H x1(s-mu)]
//
// FP64 on this GPU is arithmetic-bound (about 2 DFMA per clock per SM), so the FP64 kernel
// spreads one site over 24 threads -- (half, colour, direction) -- to keep every SM busy at
// small volumes; the four direction threads are adjacent lanes and meet through shuffles.
#include "internal.h"
#include "../../include/jtrlan.h"

namespace jtr {

namespace {

constexpr int kMvThreads = 256;

template <typename R, int MODE>
__global__ void __launch_bounds__(kMvThreads)
stencil_kernel(OpDev op, const cplx<R>* __restrict__ X, cplx<R>* __restrict__ Y, double* __restrict__ part,
               const int* __restrict__ cand, const double* __restrict__ lam, int64_t ldx) {
  using C = cplx<R>;
  __shared__ double sh[32];
  const int64_t vol = op.vol, h = op.h;
  const int64_t t = (int64_t)blockIdx.x * kMvThreads + threadIdx.x;
  const int col = blockIdx.y;
  const C* x = X + (MODE == MV_RESID ? (int64_t)cand[col] * ldx : 0);
  // warp w takes half = w & 1 of the 8 (site, colour) items (w >> 1) * 8 + lane / 4, one direction
  // per lane: the half is warp-uniform, so the two halves' code paths never diverge inside a warp
  const int lane = (int)(t & 31);
  const int64_t w = t >> 5;
  const int mu = lane & 3;
  const int half = (int)(w & 1);
  const int64_t item = (w >> 1) * 8 + (lane >> 2);   // 3 s + a
  const int a = (int)(item % 3);
  const int64_t s = item / 3;
  const bool active = item < 3 * vol;

  C accU = mk<R>(0, 0), accW = mk<R>(0, 0);
  if (active) {
    const int d0 = op.dims[0], d1 = op.dims[1], d2 = op.dims[2], d3 = op.dims[3];
    const int64_t stride = mu == 0 ? 1 : mu == 1 ? (int64_t)d0 : mu == 2 ? (int64_t)d0 * d1 : (int64_t)d0 * d1 * d2;
    const int L = mu == 0 ? d0 : mu == 1 ? d1 : mu == 2 ? d2 : d3;
    const int c = (int)((s / stride) % L);
    const int64_t sp = (c == L - 1) ? s - (int64_t)(L - 1) * stride : s + stride;
    const int64_t sm = (c == 0) ? s + (int64_t)(L - 1) * stride : s - stride;
    const C* U = (const C*)op.U;
    const C* W = (const C*)op.W;
    const C* Uf = U + ((int64_t)mu * vol + s) * 9;
    const C* Ub = U + ((int64_t)mu * vol + sm) * 9;
    const C* Wf = W + ((int64_t)mu * vol + s) * 9;
    const C* Wb = W + ((int64_t)mu * vol + sm) * 9;
    const C* x1 = x;
    const C* x2 = x + h;
    if (half == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        accU = cfma(Uf[a * 3 + b], x1[3 * sp + b], accU);    // U(s) x1(s+mu)
        accU = cfmac(Ub[b * 3 + a], x1[3 * sm + b], accU);   // U(s-mu)^H x1(s-mu)
        accW = cfma(Wf[a * 3 + b], x2[3 * sp + b], accW);    // W(s) x2(s+mu)
        C wb = Wb[b * 3 + a];
        wb.x = -wb.x; wb.y = -wb.y;
        accW = cfma(wb, x2[3 * sm + b], accW);               // -W(s-mu)^T x2(s-mu)
      }
    } else {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        accU = cfmac(Uf[a * 3 + b], x2[3 * sp + b], accU);   // U(s)^* x2(s+mu)
        accU = cfma(Ub[b * 3 + a], x2[3 * sm + b], accU);    // U(s-mu)^T x2(s-mu)
        C wf = Wf[a * 3 + b];
        wf.x = -wf.x; wf.y = -wf.y;
        accW = cfmac(wf, x1[3 * sp + b], accW);              // -W(s)^* x1(s+mu)
        accW = cfmac(Wb[b * 3 + a], x1[3 * sm + b], accW);   // +W(s-mu)^H x1(s-mu)
      }
    }
  }
  const R kap = (R)op.kappa;
  C acc = mk<R>(accU.x + kap * accW.x, accU.y + kap * accW.y);
  // sum over the four direction lanes
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);

  double c0 = 0.0, c1 = 0.0;
  if (active && mu == 0) {
    const int64_t e = (int64_t)half * h + 3 * s + a;
    const C xe = x[e];
    const R m0 = (R)op.m0;
    acc.x += m0 * xe.x;
    acc.y += m0 * xe.y;
    if (MODE != MV_RESID) Y[e] = acc;
    if (MODE == MV_ALPHA) {  // conj(x_e) * y_e
      c0 = (double)xe.x * acc.x + (double)xe.y * acc.y;
      c1 = (double)xe.x * acc.y - (double)xe.y * acc.x;
    } else if (MODE == MV_RESID) {
      const double l = lam[col];
      const double rr = (double)acc.x - l * (double)xe.x, ri = (double)acc.y - l * (double)xe.y;
      c0 = rr * rr + ri * ri;
    }
  }
  if (MODE == MV_ALPHA) {
    c0 = block_sum(c0, sh);
    c1 = block_sum(c1, sh);
    if (threadIdx.x == 0) ((double2*)part)[blockIdx.x] = make_double2(c0, c1);
  } else if (MODE == MV_RESID) {
    c0 = block_sum(c0, sh);
    if (threadIdx.x == 0) part[(int64_t)col * gridDim.x + blockIdx.x] = c0;
  }
}

// FP32 (mixed-precision) stencil, HBM-bound: one thread per (site, colour a) computes y1[a] and
// y2[a].  The three colour threads of a site split its 144 incident link words (row a of U(s),
// W(s) and column a of U(s-mu), W(s-mu) for each direction) with no overlap, which keeps the live
// state small.  A block holds all three colours of 128 consecutive sites (warps are colour-uniform):
// element (r, c) of a link is read forward by colour r of its site and backward by colour c of the
// next site along mu, at most ~54 blocks later, so the second read hits L2 and DRAM sees each link
// once.  Links are stored structure-of-arrays, L[(mu*9 + e)*V + s], so every link load of a warp
// is one contiguous 256-byte segment.  Index arithmetic is 32-bit.
// 64 sites (192 threads) per block and at least 5 resident blocks per SM: measured best on GB300
// (4.8 TB/s at 24^3 x 48), with each direction's 24 loads issued before its arithmetic.
constexpr int kSitesPerBlock = 64;
constexpr int kSiteThreads = 3 * kSitesPerBlock;
constexpr int kSiteMinBlocks = 5;

template <int MODE>
__global__ void __launch_bounds__(kSiteThreads, kSiteMinBlocks)
stencil_site_kernel(OpDev op, const float2* __restrict__ X, float2* __restrict__ Y, double* __restrict__ part,
                    const int* __restrict__ cand, const double* __restrict__ lam, int64_t ldx) {
  __shared__ double sh[32];
  const int vol = (int)op.vol;
  const int64_t h = op.h;
  const int s = blockIdx.x * kSitesPerBlock + (threadIdx.x % kSitesPerBlock);
  const int a = threadIdx.x / kSitesPerBlock;
  const int col = blockIdx.y;
  const float2* x = X + (MODE == MV_RESID ? (int64_t)cand[col] * ldx : 0);
  double c0 = 0.0, c1 = 0.0;
  if (s < vol) {
    const float2* U = (const float2*)op.U;
    const float2* W = (const float2*)op.W;
    const float2* x1 = x;
    const float2* x2 = x + h;
    float2 y1 = make_float2(0.f, 0.f), y2 = y1, w1 = y1, w2 = y1;
    int coord[4];
    {
      int r = s;
#pragma unroll
      for (int d = 0; d < 3; ++d) { coord[d] = r % op.dims[d]; r /= op.dims[d]; }
      coord[3] = r;
    }
    int stride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int L = op.dims[mu];
      const int c = coord[mu];
      const int sp = (c == L - 1) ? s - (L - 1) * stride : s + stride;
      const int sm = (c == 0) ? s + (L - 1) * stride : s - stride;
      stride *= L;
      const float2* Um = U + (int64_t)mu * 9 * vol;
      const float2* Wm = W + (int64_t)mu * 9 * vol;
      float2 P1[3], P2[3], M1[3], M2[3], UF[3], UB[3], WF[3], WB[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        UF[b] = Um[(a * 3 + b) * vol + s];
        UB[b] = Um[(b * 3 + a) * vol + sm];
        WF[b] = Wm[(a * 3 + b) * vol + s];
        WB[b] = Wm[(b * 3 + a) * vol + sm];
      }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        P1[b] = x1[3 * sp + b]; P2[b] = x2[3 * sp + b];
        M1[b] = x1[3 * sm + b]; M2[b] = x2[3 * sm + b];
      }
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 p1 = P1[b], p2 = P2[b], m1 = M1[b], m2 = M2[b];
        // uf = U(s)_{ab}, ub = U(s-mu)_{ba}, wf = W(s)_{ab}, wb = W(s-mu)_{ba}
        const float2 uf = UF[b], ub = UB[b], wf = WF[b], wb = WB[b];
        y1 = cfma(uf, p1, y1);                          // U(s) x1(s+mu)
        y1 = cfmac(ub, m1, y1);                         // U(s-mu)^H x1(s-mu)
        y2 = cfmac(uf, p2, y2);                         // U(s)^* x2(s+mu)
        y2 = cfma(ub, m2, y2);                          // U(s-mu)^T x2(s-mu)
        w1 = cfma(wf, p2, w1);                          // W(s) x2(s+mu)
        w1 = cfma(make_float2(-wb.x, -wb.y), m2, w1);   // -W(s-mu)^T x2(s-mu)
        w2 = cfmac(make_float2(-wf.x, -wf.y), p1, w2);  // -W(s)^* x1(s+mu)
        w2 = cfmac(wb, m1, w2);                         // +W(s-mu)^H x1(s-mu)
      }
    }
    const float kap = (float)op.kappa, m0 = (float)op.m0;
    const int64_t e1 = 3 * (int64_t)s + a;
    const float2 xa = x1[e1], xb = x2[e1];
    const float2 o1 = make_float2(y1.x + kap * w1.x + m0 * xa.x, y1.y + kap * w1.y + m0 * xa.y);
    const float2 o2 = make_float2(y2.x + kap * w2.x + m0 * xb.x, y2.y + kap * w2.y + m0 * xb.y);
    if (MODE != MV_RESID) { Y[e1] = o1; Y[h + e1] = o2; }
    if (MODE == MV_ALPHA) {
      c0 = (double)(xa.x * o1.x + xa.y * o1.y + xb.x * o2.x + xb.y * o2.y);
      c1 = (double)(xa.x * o1.y - xa.y * o1.x + xb.x * o2.y - xb.y * o2.x);
    } else if (MODE == MV_RESID) {
      const float l = (float)lam[col];
      const float r0 = o1.x - l * xa.x, r1 = o1.y - l * xa.y, r2 = o2.x - l * xb.x, r3 = o2.y - l * xb.y;
      c0 = (double)(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    }
  }
  const int64_t blk = blockIdx.x;     // block index within one product
  const int64_t nblk = gridDim.x;
  if (MODE == MV_ALPHA) {
    c0 = block_sum(c0, sh);
    c1 = block_sum(c1, sh);
    if (threadIdx.x == 0) ((double2*)part)[blk] = make_double2(c0, c1);
  } else if (MODE == MV_RESID) {
    c0 = block_sum(c0, sh);
    if (threadIdx.x == 0) part[(int64_t)col * nblk + blk] = c0;
  }
}

// Dense: one warp per row r of the blocks; y1[r] and y2[r] from one read of row r of A11, A12.
constexpr int kDenseRowsPerBlock = kMvThreads / 32;

template <typename R, int MODE>
__global__ void __launch_bounds__(kMvThreads)
dense_kernel(OpDev op, const cplx<R>* __restrict__ X, cplx<R>* __restrict__ Y, double* __restrict__ part,
             const int* __restrict__ cand, const double* __restrict__ lam, int64_t ldx) {
  using C = cplx<R>;
  __shared__ double sh[32];
  const int64_t h = op.h;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * kDenseRowsPerBlock + (threadIdx.x >> 5);
  const int col = blockIdx.y;
  const C* x = X + (MODE == MV_RESID ? (int64_t)cand[col] * ldx : 0);
  const C* A11 = (const C*)op.a11;
  const C* A12 = (const C*)op.a12;
  C y1 = mk<R>(0, 0), y2 = mk<R>(0, 0);
  if (row < h) {
    const C* r11 = A11 + row * h;
    const C* r12 = A12 + row * h;
    for (int64_t c = lane; c < h; c += 32) {
      const C a11 = r11[c], a12 = r12[c], x1 = x[c], x2 = x[h + c];
      y1 = cfma(a11, x1, y1);             // A11 x1
      y1 = cfma(a12, x2, y1);             // A12 x2
      y2 = cfmac(a11, x2, y2);            // A11^T x2 = conj(A11) x2 (A11 Hermitian)
      C na12 = a12; na12.x = -na12.x; na12.y = -na12.y;
      y2 = cfmac(na12, x1, y2);           // A12^H x1 = -conj(A12) x1 (A12 skew-symmetric)
    }
  }
  double v[4] = {(double)y1.x, (double)y1.y, (double)y2.x, (double)y2.y};
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = warp_sum(v[k]);
  double c0 = 0.0, c1 = 0.0;
  if (row < h && lane == 0) {
    const C o1 = mk<R>((R)v[0], (R)v[1]), o2 = mk<R>((R)v[2], (R)v[3]);
    const C x1 = x[row], x2 = x[h + row];
    if (MODE != MV_RESID) { Y[row] = o1; Y[h + row] = o2; }
    if (MODE == MV_ALPHA) {
      c0 = (double)x1.x * o1.x + (double)x1.y * o1.y + (double)x2.x * o2.x + (double)x2.y * o2.y;
      c1 = (double)x1.x * o1.y - (double)x1.y * o1.x + (double)x2.x * o2.y - (double)x2.y * o2.x;
    } else if (MODE == MV_RESID) {
      const double l = lam[col];
      const double a0 = v[0] - l * x1.x, a1 = v[1] - l * x1.y, a2 = v[2] - l * x2.x, a3 = v[3] - l * x2.y;
      c0 = a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3;
    }
  }
  if (MODE == MV_ALPHA) {
    c0 = block_sum(c0, sh);
    c1 = block_sum(c1, sh);
    if (threadIdx.x == 0) ((double2*)part)[blockIdx.x] = make_double2(c0, c1);
  } else if (MODE == MV_RESID) {
    c0 = block_sum(c0, sh);
    if (threadIdx.x == 0) part[(int64_t)col * gridDim.x + blockIdx.x] = c0;
  }
}

template <typename R, int MODE>
cudaError_t launch_mode(const OpDev& op, const cplx<R>* x, cplx<R>* y, double* part, const int* cand,
                        const double* lam, int ncand, int64_t ldx, int nblk, cudaStream_t s) {
  dim3 grid(nblk, MODE == MV_RESID ? ncand : 1);
  if (op.kind == JTRLAN_STENCIL4D) {
    if constexpr (sizeof(R) == sizeof(float))
      stencil_site_kernel<MODE><<<grid, kSiteThreads, 0, s>>>(op, x, y, part, cand, lam, ldx);
    else
      stencil_kernel<R, MODE><<<grid, kMvThreads, 0, s>>>(op, x, y, part, cand, lam, ldx);
  } else {
    dense_kernel<R, MODE><<<grid, kMvThreads, 0, s>>>(op, x, y, part, cand, lam, ldx);
  }
  return cudaGetLastError();
}

}  // namespace

int matvec_blocks(const OpDev& op) {
  if (op.kind == JTRLAN_STENCIL4D) {
    if (op.fp32) return (int)((op.vol + kSitesPerBlock - 1) / kSitesPerBlock);
    return (int)((64 * ((3 * op.vol + 7) / 8) + kMvThreads - 1) / kMvThreads);   // 2 warps per 8 items
  }
  return (int)((op.h + kDenseRowsPerBlock - 1) / kDenseRowsPerBlock);
}

template <typename R>
cudaError_t launch_matvec(const OpDev& op, const cplx<R>* x, cplx<R>* y, MvMode mode, double* part,
                          const int* cand, const double* lam, int ncand, int64_t ldx, int* nblk_out,
                          cudaStream_t s) {
  const int nblk = matvec_blocks(op);
  if (nblk_out) *nblk_out = nblk;
  if (mode == MV_RESID && ncand <= 0) return cudaSuccess;
  switch (mode) {
    case MV_PLAIN: return launch_mode<R, MV_PLAIN>(op, x, y, part, cand, lam, ncand, ldx, nblk, s);
    case MV_ALPHA: return launch_mode<R, MV_ALPHA>(op, x, y, part, cand, lam, ncand, ldx, nblk, s);
    default: return launch_mode<R, MV_RESID>(op, x, y, part, cand, lam, ncand, ldx, nblk, s);
  }
}

template cudaError_t launch_matvec<double>(const OpDev&, const double2*, double2*, MvMode, double*, const int*,
                                           const double*, int, int64_t, int*, cudaStream_t);
template cudaError_t launch_matvec<float>(const OpDev&, const float2*, float2*, MvMode, double*, const int*,
                                          const double*, int, int64_t, int*, cudaStream_t);

}  // namespace jtr
