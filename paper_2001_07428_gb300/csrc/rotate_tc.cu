// rotate_tc.cu -- the restart rotation V_m Z of a compensated-FP32 basis on the 5th-generation
// tensor cores (tcgen05.mma, BF16 operands, FP32 accumulators in tensor memory).
//
// The rotation is the thick-restart step of Algorithm 1 (the kept Ritz vectors are V_m times the
// eigenvectors Z of T_m) and the one dense contraction of the method: in the real view,
// C (2n x kk) = V (2n x m) Z (m x kk), with V held as (hi, lo) FP32 pairs and Z in FP64.  The
// tensor cores have no FP64 kind, so both operands are written as exact sums of BF16 digits (an
// Ozaki-type splitting, Ozaki et al., Numer. Algorithms 59 (2012)):
//   x = 2^E sum_{s<7} a_s 2^(-7(s+1)) + r,   a_s integers, |a_0| <= 128, |a_s| <= 64 (s >= 1),
//   |r| <= 2^(E-50),
// with one exponent E per row of V (|x| < 2^E along the row) and one, F, per column of Z.  A digit
// has at most 8 significant bits, so it is exact in BF16 and a digit product is exact in FP32.
// For the d-th accumulator P_d = sum_k sum_{s+t=d} a_s b_t every partial sum is an integer of
// magnitude below m * 9 * 2^12 < 2^24 (m <= 455; shared memory limits this kernel to m <= 320), so the
// tensor core adds without rounding.  The 28
// digit pairs with s + t <= 6 feed 7 accumulators (one per d); the epilogue forms
// sum_d 2^(-7d) P_d in float-float and scales it by 2^(E + F - 14).  Each dropped pair (s + t >= 7)
// and each digit remainder is below 2^-49 of max_k |V_rk| max_k |Z_kc| per product, the accuracy of
// the compensated-FP32 CUDA-core kernel this replaces.
//
// Kernel structure (one persistent CTA per SM, 416 threads, warp-specialised):
//   * warp 12, one lane: loads the BF16 digits of its 32 columns of Z (all of K, built once by
//     tc_zslice_kernel) into shared memory with bulk copies, then issues the 28 MMAs of every
//     K = 16 chunk and commits them to mbarriers;
//   * warps 4..11, two groups of four taking alternate chunks: read the (hi, lo) rows of V, split
//     them into digits and write the BF16 digit planes into a ring of shared-memory stages in the
//     canonical no-swizzle K-major layout (8 x 16-byte core matrices);
//   * warps 0..3: read the 7 accumulators of a finished tile from tensor memory (one row per
//     thread), combine, scale and write FP64 results; two accumulator sets (2 x 224 of the 512
//     columns) let the epilogue of one tile overlap the MMAs of the next.
// Every mbarrier wait is bounded: past about two seconds the CTA records an error code, every role
// leaves its loop, tensor memory is freed and the kernel returns.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace jtr {
namespace {

constexpr int kTcRows = 128;                       // real rows of V per tile (M of the MMA)
constexpr int kTcCols = 32;                        // columns of Z per tile (N of the MMA)
constexpr int kTcK = 16;                           // K of one BF16 MMA
constexpr int kDig = 7;                            // digits per operand
constexpr int kPlaneA = kTcRows * kTcK * 2;        // one digit plane of one A chunk: 4096 bytes
constexpr int kPlaneB = kTcCols * kTcK * 2;        // one digit plane of one B chunk: 1024 bytes
constexpr int kStageA = kDig * kPlaneA;            // 28672 bytes
constexpr int kChunkB = kDig * kPlaneB;            // 7168 bytes
constexpr int kAccSet = 256;                       // TMEM columns per accumulator set (7 x 32 used)
constexpr int kEpiWarps = 4, kProdWarps = 8;
constexpr int kMmaWarp = kEpiWarps + kProdWarps;   // 12
constexpr int kThreads = (kMmaWarp + 1) * 32;      // 416
constexpr int kProdGroup = 128;                    // threads of one producer group
constexpr long long kSpinCycles = 4000000000LL;    // about 2 s at the GB300 SM clock

struct TcBars {
  unsigned long long full[4];      // stage written by a producer group (128 arrivals)
  unsigned long long empty[4];     // stage consumed by the MMAs (tcgen05.commit)
  unsigned long long accfull[2];   // accumulator set complete (tcgen05.commit)
  unsigned long long accempty[2];  // accumulator set read by the epilogue (128 arrivals)
  unsigned long long bimg;         // Z digits landed (bulk-copy transaction count)
  uint32_t tmem;                   // tensor-memory base address written by tcgen05.alloc
  int abort;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity; false (after recording `code`) if it does not complete
// within kSpinCycles or another role has given up.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, TcBars* bars, int* err, int code) {
  const long long t0 = clock64();
  while (!mbar_try(a, parity)) {
    if (*(volatile int*)&bars->abort) return false;
    if (clock64() - t0 > kSpinCycles) {
      *(volatile int*)&bars->abort = 1;
      atomicCAS(err, 0, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension byte offset (the
// stride between core matrices along K), stride-dimension byte offset (between 8-row groups along
// M or N), the fixed version bits 46-48 = 0b001, no swizzling.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 consecutive 32-bit columns of this warp's 32 lanes: register j of lane i = column (col + j),
// lane (lane base + i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 2^e as a float, e in [-126, 127]
__device__ __forceinline__ float exp2f_int(int e) { return __int_as_float((e + 127) << 23); }

// The seven digits of x = (hi + lo) 2^(-E) * 128 (|hi| < 2^E, |lo| <= 2^-23 |hi|): a_0 = rint(p), then
// p <- 128 (p - a_s), each step exact in FP32.  lo enters through two exact TwoSum folds (before digits
// 2 and 4) and a last plain add before digit 6 (its rounding lies below the discarded remainder);
// every digit after the first stays within [-64, 64].
__device__ __forceinline__ void split7(float hi, float lo, float sc, float (&a)[7]) {
  float p = hi * sc, q = lo * sc;
  a[0] = rintf(p); p = (p - a[0]) * 128.f;
  a[1] = rintf(p); p = (p - a[1]) * 128.f;
  {
    const float y = q * 16384.f, s = p + y, bb = s - p;
    q = (p - (s - bb)) + (y - bb);
    p = s;
  }
  a[2] = rintf(p); p = (p - a[2]) * 128.f;
  a[3] = rintf(p); p = (p - a[3]) * 128.f;
  {
    const float y = q * 16384.f, s = p + y, bb = s - p;
    q = (p - (s - bb)) + (y - bb);
    p = s;
  }
  a[4] = rintf(p); p = (p - a[4]) * 128.f;
  a[5] = rintf(p); p = (p - a[5]) * 128.f;
  a[6] = rintf(p + q * 16384.f);
}

// (hi, lo) -> (fl(hi + lo), the exact rest): exact when |lo| <= |hi| or hi = 0, and the same
// arithmetic in the row-exponent pass and in the digit producers.
__device__ __forceinline__ float2 renorm(float hi, float lo) {
  const float s = hi + lo;
  return make_float2(s, lo - (s - hi));
}

// Two digits as packed BF16, element k in the low half.  A digit is an integer of at most 8
// significant bits, so its BF16 form is exactly the upper half of its FP32 bits.
__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  return __byte_perm(__float_as_uint(lo_k), __float_as_uint(hi_k), 0x7632);
}

// (h, l) <- (h, l) 2^-7 + P exactly up to float-float rounding.
__device__ __forceinline__ void df_horner(float& h, float& l, float P) {
  const float hs = h * 0.0078125f, ls = l * 0.0078125f;
  const float s = P + hs, bb = s - P;
  const float e = (P - (s - bb)) + (hs - bb);
  const float t = ls + e;
  h = s + t;
  l = t - (h - s);
}

// (h + l) 2^es in FP64; the scaling stays in FP32 (exact, no underflow of l) for |es| <= 100.  (An
// integer assembly of the FP64 bits, which avoids the FP64 pipe, measured slower on GB300.)
__device__ __forceinline__ double tc_combine(float h, float l, int es) {
  if (es >= -100 && es <= 100) {
    const float sc = exp2f_int(es);
    return (double)(h * sc) + (double)(l * sc);
  }
  return ((double)h + (double)l) * __longlong_as_double((long long)(es + 1023) << 52);
}

__global__ void __launch_bounds__(kThreads, 1)
rotate_tc_kernel(const float4* __restrict__ V, int64_t n, int m, int nkc, int nst, const int8_t* __restrict__ Erow,
                 const uint8_t* __restrict__ Bimg, const int* __restrict__ Ecol, int kk, int ntn, int ngrp,
                 int64_t mtiles, double* __restrict__ out, int* err, int selftest) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Bs = sm;                                  // nkc chunks x 7 planes x 1 KB
  uint8_t* As = Bs + (size_t)nkc * kChunkB;          // nst stages x 7 planes x 4 KB
  TcBars* bars = (TcBars*)(As + (size_t)nst * kStageA);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = blockIdx.x % ntn, grp = blockIdx.x / ntn;
  const int64_t rows = 2 * n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(saddr(&bars->full[s]), kProdGroup);
      mbar_init(saddr(&bars->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(saddr(&bars->accfull[b]), 1);
      mbar_init(saddr(&bars->accempty[b]), kEpiWarps * 32);
    }
    mbar_init(saddr(&bars->bimg), 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&bars->tmem)),
                 "r"(2 * kAccSet)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem;

  if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue (one lane)
    if (lane == 0) {
      const uint32_t bbar = saddr(&bars->bimg);
      mbar_expect_tx(bbar, (uint32_t)(nkc * kChunkB));
      const uint8_t* src = Bimg + (size_t)nt * nkc * kChunkB;
      for (int kc = 0; kc < nkc; ++kc) bulk_g2s(saddr(Bs + (size_t)kc * kChunkB), src + (size_t)kc * kChunkB, kChunkB, bbar);
      bool ok = mbar_wait(bbar, 0, bars, err, 1);
      constexpr uint32_t idesc = idesc_bf16(kTcRows, kTcCols);
      int64_t g = 0;
      int it = 0;
      for (int64_t mt = grp; ok && mt < mtiles; mt += ngrp, ++it) {
        const int buf = it & 1;
        if (it >= 2) {
          ok = mbar_wait(saddr(&bars->accempty[buf]), ((it >> 1) - 1) & 1, bars, err, 2);
          if (!ok) break;
          tc_fence_after();
        }
        const uint32_t dbase = tmem + (uint32_t)(buf * kAccSet);
        for (int kc = 0; kc < nkc; ++kc, ++g) {
          const int st = (int)(g % nst);
          ok = mbar_wait(saddr(&bars->full[st]), (uint32_t)((g / nst) & 1), bars, err, 3);
          if (!ok) break;
          tc_fence_after();
          const uint32_t a0 = saddr(As + (size_t)st * kStageA);
          const uint32_t b0 = saddr(Bs + (size_t)kc * kChunkB);
#pragma unroll
          for (int d = 0; d < kDig; ++d)
#pragma unroll
            for (int s = 0; s <= d; ++s)
              umma_bf16(dbase + (uint32_t)(d * kTcCols), sdesc(a0 + s * kPlaneA, 128, 256),
                        sdesc(b0 + (d - s) * kPlaneB, 128, 256), idesc, (kc | s) != 0);
          umma_commit(saddr(&bars->empty[st]));
        }
        if (!ok) break;
        // selftest: the first tile's accumulator barrier is never signalled, so the epilogue's bounded
        // wait runs out (the failure path, exercised without a fault)
        if (!(selftest && it == 0)) umma_commit(saddr(&bars->accfull[buf]));
      }
    }
    __syncwarp();
  } else if (warp >= kEpiWarps) {
    // ---------------------------------------------------------------- digit producers
    const int pw = (warp - kEpiWarps) & 3, pg = (warp - kEpiWarps) >> 2;
    const int il = pw * 16 + (lane & 15);   // complex row of the tile (real rows 2 il, 2 il + 1)
    const int kh = lane >> 4;               // which 8 of the chunk's 16 k
    const int sel = (lane >> 2) & 1;        // store order of the two rows (conflict-free banks)
    int64_t g = 0;
    bool ok = true;
    for (int64_t mt = grp; ok && mt < mtiles; mt += ngrp) {
      const int64_t gi = mt * (kTcRows / 2) + il;
      const bool live = gi < n;
      char2 e2 = make_char2(0, 0);
      if (live) e2 = reinterpret_cast<const char2*>(Erow)[gi];
      const float sre = exp2f_int(7 - (int)e2.x), sim = exp2f_int(7 - (int)e2.y);
      for (int kc = 0; kc < nkc; ++kc, ++g) {
        if ((int)(g & 1) != pg) continue;
        const int st = (int)(g % nst);
        if (g >= nst && !mbar_wait(saddr(&bars->empty[st]), (uint32_t)(((g / nst) - 1) & 1), bars, err, 4)) {
          ok = false;
          break;
        }
        const int k0 = kc * kTcK + kh * 8;
        float4 f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          f[e] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (live && k0 + e < m) f[e] = V[(int64_t)(k0 + e) * n + gi];
        }
        uint32_t pr[kDig][4], pi[kDig][4];   // digit planes of the real and imaginary rows, 8 k each
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          float ar0[7], ar1[7], ai0[7], ai1[7];
          const float2 r0 = renorm(f[e].x, f[e].z), r1 = renorm(f[e + 1].x, f[e + 1].z);
          const float2 i0 = renorm(f[e].y, f[e].w), i1 = renorm(f[e + 1].y, f[e + 1].w);
          split7(r0.x, r0.y, sre, ar0);
          split7(r1.x, r1.y, sre, ar1);
          split7(i0.x, i0.y, sim, ai0);
          split7(i1.x, i1.y, sim, ai1);
#pragma unroll
          for (int s = 0; s < kDig; ++s) {
            pr[s][e >> 1] = pack_bf16(ar0[s], ar1[s]);
            pi[s][e >> 1] = pack_bf16(ai0[s], ai1[s]);
          }
        }
        uint8_t* sa = As + (size_t)st * kStageA;
#pragma unroll
        for (int s = 0; s < kDig; ++s) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int comp = j ^ sel;
            const int r = 2 * il + comp;
            const uint4 wr = make_uint4(pr[s][0], pr[s][1], pr[s][2], pr[s][3]);
            const uint4 wi = make_uint4(pi[s][0], pi[s][1], pi[s][2], pi[s][3]);
            const uint4 w = comp ? wi : wr;
            *reinterpret_cast<uint4*>(sa + s * kPlaneA + ((r >> 3) * 2 + kh) * 128 + (r & 7) * 16) = w;
          }
        }
        fence_proxy_async();
        mbar_arrive(saddr(&bars->full[st]));
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int row = warp * 32 + lane;
    int it = 0;
    for (int64_t mt = grp; mt < mtiles; mt += ngrp, ++it) {
      const int buf = it & 1;
      // tcgen05.ld is warp-collective: one lane waits and the whole warp takes its result
      bool ok = true;
      if (lane == 0) ok = mbar_wait(saddr(&bars->accfull[buf]), (uint32_t)((it >> 1) & 1), bars, err, 5);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * kAccSet);
      float h[32], l[32];
      uint32_t v[32];
      tmem_ld32(ta + 6 * kTcCols, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) { h[j] = __uint_as_float(v[j]); l[j] = 0.f; }
#pragma unroll
      for (int d = 5; d >= 0; --d) {
        tmem_ld32(ta + (uint32_t)(d * kTcCols), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) df_horner(h[j], l[j], __uint_as_float(v[j]));
      }
      tc_fence_before();
      mbar_arrive(saddr(&bars->accempty[buf]));   // every epilogue thread: 128 arrivals
      const int64_t r = mt * kTcRows + row;
      if (r < rows) {
        const int er = (int)Erow[r];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = nt * kTcCols + j;
          if (c < kk) out[(int64_t)c * rows + r] = tc_combine(h[j], l[j], er + __ldg(Ecol + c) - 14);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccSet) : "memory");
  }
}

// E of every real row: |x| < 2^E for all k, from the largest biased exponent of the renormalised hi
// (|hi + lo| <= 2^E then holds too, lo being at most half an ulp of hi); clamped to [-120, 127] (a row whose entries
// all lie below 2^-120 is resolved to 2^-169 absolute).
__global__ void tc_rowexp_kernel(const float4* __restrict__ V, int64_t n, int m, int8_t* __restrict__ Erow) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t br = 0, bi = 0;
    int k = 0;
    for (; k + 4 <= m; k += 4) {
      float4 f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) f[u] = V[(int64_t)(k + u) * n + i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        br = max(br, __float_as_uint(renorm(f[u].x, f[u].z).x) & 0x7f800000u);
        bi = max(bi, __float_as_uint(renorm(f[u].y, f[u].w).x) & 0x7f800000u);
      }
    }
    for (; k < m; ++k) {
      const float4 f = V[(int64_t)k * n + i];
      br = max(br, __float_as_uint(renorm(f.x, f.z).x) & 0x7f800000u);
      bi = max(bi, __float_as_uint(renorm(f.y, f.w).x) & 0x7f800000u);
    }
    const int er = min(max((int)(br >> 23) - 126, -120), 127);
    const int ei = min(max((int)(bi >> 23) - 126, -120), 127);
    reinterpret_cast<char2*>(Erow)[i] = make_char2((signed char)er, (signed char)ei);
  }
}

// The BF16 digit planes of Z, one block per column c of the padded width ntn * 32, in the order the
// rotation kernel copies them: [column tile][K chunk][digit][core matrix (n/8, k/8)][8 x 8].
// F_c: |z| < 2^F_c down the column (from the largest biased FP64 exponent), clamped to [-880, 120].
// The split runs in FP64 and is exact at every step.
__global__ void tc_zslice_kernel(const double* __restrict__ Z, int m, int kk, int nkc, uint16_t* __restrict__ Bimg,
                                 int* __restrict__ Ecol) {
  const int c = blockIdx.x;
  __shared__ unsigned int smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  unsigned int lm = 0;
  if (c < kk)
    for (int k = threadIdx.x; k < m; k += blockDim.x)
      lm = max(lm, (unsigned int)((__double_as_longlong(Z[(int64_t)c * m + k]) >> 52) & 0x7ff));
  atomicMax(&smax, lm);
  __syncthreads();
  const int F = min(max((int)smax - 1022, -880), 120);
  if (threadIdx.x == 0) Ecol[c] = F;
  const double sc = __longlong_as_double((long long)(7 - F + 1023) << 52);
  const int nt = c / kTcCols, cn = c % kTcCols, ni = cn >> 3, nr = cn & 7;
  for (int k = threadIdx.x; k < nkc * kTcK; k += blockDim.x) {
    double zz = (c < kk && k < m) ? Z[(int64_t)c * m + k] * sc : 0.0;
    const int kc = k / kTcK, ki = (k % kTcK) >> 3, ke = k & 7;
    uint16_t* dst = Bimg + ((size_t)(nt * nkc + kc) * kDig) * (kPlaneB / 2) + (ni * 2 + ki) * 64 + nr * 8 + ke;
#pragma unroll
    for (int t = 0; t < kDig; ++t) {
      const double a = rint(zz);
      zz = (zz - a) * 128.0;
      dst[t * (kPlaneB / 2)] = __bfloat16_as_ushort(__float2bfloat16_rn((float)a));
    }
  }
}

}  // namespace

int tc_rotate_max_m() { return 320; }

size_t tc_rotate_bytes(int64_t n, int m, int kk_max) {
  const int nkc = (m + kTcK - 1) / kTcK, ntn = (kk_max + kTcCols - 1) / kTcCols;
  return (size_t)2 * n + 256 + (size_t)ntn * nkc * kChunkB + 256 + (size_t)ntn * kTcCols * sizeof(int) + 256;
}

TcWork tc_rotate_carve(void* base, int64_t n, int m, int kk_max) {
  const int nkc = (m + kTcK - 1) / kTcK, ntn = (kk_max + kTcCols - 1) / kTcCols;
  uint8_t* p = (uint8_t*)base;
  auto take = [&](size_t bytes) { uint8_t* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  TcWork w;
  w.Erow = (int8_t*)take((size_t)2 * n);
  w.Bimg = (uint8_t*)take((size_t)ntn * nkc * kChunkB);
  w.Ecol = (int*)take((size_t)ntn * kTcCols * sizeof(int));
  w.err = (int*)take(sizeof(int) * 4);
  w.n = n;
  w.m = m;
  w.kk_max = kk_max;
  return w;
}

cudaError_t launch_rotate_tc(const void* V, int64_t n, int m, const double* Z, int kk, void* out, const TcWork& w,
                             bool fresh_rowexp, cudaStream_t s, int selftest) {
  if (m < 1 || m > tc_rotate_max_m() || kk < 1 || kk > w.kk_max || n != w.n || m != w.m) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;   // per device: queried on every call (cheap), as is the attribute below
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e0 != cudaSuccess) return e0;
  const int nkc = (m + kTcK - 1) / kTcK, ntn = (kk + kTcCols - 1) / kTcCols;
  const int64_t mtiles = (2 * n + kTcRows - 1) / kTcRows;
  if (fresh_rowexp) {
    const int64_t nb = std::min<int64_t>((n + 255) / 256, (int64_t)nsm * 8);
    tc_rowexp_kernel<<<(unsigned)nb, 256, 0, s>>>((const float4*)V, n, m, w.Erow);
  }
  tc_zslice_kernel<<<ntn * kTcCols, 128, 0, s>>>(Z, m, kk, nkc, (uint16_t*)w.Bimg, w.Ecol);
  const size_t bbytes = (size_t)nkc * kChunkB;
  const size_t cap = 232448;   // opt-in dynamic shared memory per block
  const size_t fixed = bbytes + 1024 + sizeof(TcBars) + 64;
  int nst = (int)std::min<size_t>(4, (cap - fixed) / kStageA);
  if (nst < 2) return cudaErrorInvalidValue;
  size_t smem = fixed + (size_t)nst * kStageA;
  if (smem < 120 * 1024) smem = 120 * 1024;   // one CTA per SM: each holds all 512 tensor-memory columns
  {
    cudaError_t e = allow_dyn_smem((const void*)rotate_tc_kernel, smem);
    if (e != cudaSuccess) return e;
  }
  const int ngrp = (int)std::min<int64_t>(std::max(1, nsm / ntn), mtiles);
  rotate_tc_kernel<<<ntn * ngrp, kThreads, smem, s>>>((const float4*)V, n, m, nkc, nst, w.Erow, w.Bimg, w.Ecol, kk,
                                                       ntn, ngrp, mtiles, (double*)out, w.err, selftest);
  return cudaGetLastError();
}

}  // namespace jtr
