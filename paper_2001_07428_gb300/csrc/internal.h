// internal.h -- host-side launchers shared between the translation units of libjtrlan.
// Not part of the public ABI (that is include/jtrlan.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace jtr {

// Allows `bytes` of dynamic shared memory for kernel `func` on the current device: raises the
// kernel's cap once per device to the opt-in maximum (thread-safe); cudaErrorInvalidValue if `bytes`
// exceeds that maximum.
cudaError_t allow_dyn_smem(const void* func, size_t bytes);

// Description of the operator as the kernels see it (device pointers owned by the context).
struct OpDev {
  int kind;            // JTRLAN_DENSE / JTRLAN_STENCIL4D
  int64_t n;           // vector length
  int64_t h;           // n / 2
  int dims[4];
  int64_t vol;
  double m0, kappa;
  const void* a11;     // dense blocks (h x h row-major), working precision
  const void* a12;
  const void* U;       // stencil links: FP64 [4][V][9]; FP32 structure-of-arrays [4][9][V]
  const void* W;
  int fp32;            // 1: FP32 operator (float2 links / blocks), 0: FP64
  int links32;         // compensated-FP32 stencil: 1 = links exact in FP32 (float2 SoA, the caller's
                       // complex64 links), 0 = (hi, lo) float4 SoA
};

// Modes of the matvec kernels.
enum MvMode { MV_PLAIN = 0, MV_ALPHA = 1, MV_RESID = 2 };

// y = A x.  MV_ALPHA also writes per-block partial sums of x^H y to part (double2[nblk]).
// MV_RESID takes ncand columns x_c = X[:, cand[c]] (ld = n), computes ||A x_c - lam[c] x_c||^2
// per block into part[c * nblk + b] (double) and writes no y.  Returns the per-column block
// count (nblk) through *nblk_out.
template <typename R>
cudaError_t launch_matvec(const OpDev& op, const cplx<R>* x, cplx<R>* y, MvMode mode, double* part,
                          const int* cand, const double* lam, int ncand, int64_t ldx,
                          int* nblk_out, cudaStream_t s);
int matvec_blocks(const OpDev& op);  // nblk of launch_matvec for one column

// Lanczos-step Gram-Schmidt against [V, W] with W = J V^* implicit (Algorithm 2).
struct GSArgs {
  const void* V;       // n x (m+1) complex, ld = n, working precision
  int64_t n, h;
  void* y;             // the vector being orthogonalised (n complex)
  int j;               // current column: v_j = V[:, j]; columns 0..j take part
  double* part_dot;    // [(m+1)][nblk] coef4 partials
  double* part_nrm;    // [nblk] partial squared norms
  coef4* coef;         // [(m+1)] reduced coefficients
  StepState* st;
  double* T;           // T-bar, (m+1) x (m+1) row-major
  int ldt;             // m + 1
  int m;
  int nblk;            // blocks of the row-parallel GS kernels
  int no_w;            // nonzero: plain TRLAN (Gram-Schmidt against V only, W removed)
  int rows_per_block;  // row pairs per block (multiple of 32)
};
int gs_blocks(int64_t h, int* rows_per_block);

// The kernels of one Lanczos step's reorthogonalisation, in launch order:
//   first, reduce(first=1), update, {dot(pass), reduce(0), update} for pass = 2..P, normalize.
template <typename R>
cudaError_t launch_gs_first(const GSArgs& a, const double2* alpha_part, int n_alpha_part, cudaStream_t s);
cudaError_t launch_gs_reduce(const GSArgs& a, int first, cudaStream_t s);
template <typename R>
cudaError_t launch_gs_update(const GSArgs& a, cudaStream_t s);
template <typename R>
cudaError_t launch_gs_dot(const GSArgs& a, int pass, cudaStream_t s);
template <typename R>
cudaError_t launch_gs_normalize(const GSArgs& a, cudaStream_t s);

// Mixed forms: the same Gram-Schmidt sequence in compensated FP32 ("double-float") arithmetic on a
// basis stored as float4 {hi.re, hi.im, lo.re, lo.im} (gsdf.cu); y, alpha, beta and norms in FP64.
// x is the FP64 copy of v_j (the matvec input), rewritten with v_{j+1} by the normalisation.
cudaError_t launch_gsdf_first(const GSArgs& a, const void* x, const double2* alpha_part, int n_alpha_part,
                              cudaStream_t s);
cudaError_t launch_gsdf_dot(const GSArgs& a, int pass, cudaStream_t s);
cudaError_t launch_gsdf_update(const GSArgs& a, int pass, cudaStream_t s);   // pass: 1 after the first dots
cudaError_t launch_gsdf_normalize(const GSArgs& a, void* x, cudaStream_t s);
cudaError_t launch_df_from_fp64(const void* in, void* out, int64_t n, cudaStream_t s);
cudaError_t launch_fp64_from_df(const void* in, void* out, int64_t n, cudaStream_t s);
cudaError_t launch_shrink_df(void* V, const void* Vsrc, int64_t n, const int* perm, int k, int m, cudaStream_t s);
cudaError_t launch_gather_pairs_df(const void* V, int64_t n, const int* order, int nev, int partners, void* out,
                                   cudaStream_t s);
cudaError_t launch_rotate_df(const void* V, int64_t n, int m, const double* Z, int kk, void* Vout, cudaStream_t s);
// Conjugate gradients for the invert mode (cg.cu): y = A^{-1} b for Hermitian positive definite A.
struct CgState {
  double rr, rr0, alpha, beta, tol2;   // r^H r, |b|^2, the step scalars, (rtol |b|)^2
  int done, iters, fail;               // converged (or failed); iterations; p^H A p <= 0 seen
  double cnorm;                        // ||A v_{m+1}|| of the invert-mode residual estimate
  double zero;                         // 0.0, the lambda of a plain norm through launch_resid_part
};
int cg_blocks(int64_t n);
// x = 0, r = p = b, and the state from |b|^2 (cg_blocks(n) partials in part)
cudaError_t launch_cg_init(const void* b, void* x, void* r, void* p, int64_t n, double* part, double rtol, CgState* st,
                           cudaStream_t s);
// alpha from the partials of p^H (A p) that launch_matvec(MV_ALPHA) left for p
cudaError_t launch_cg_alpha(const double* pq_part, int nblk, CgState* st, cudaStream_t s);
// x += alpha p, r -= alpha q, beta and the convergence test, p = r + beta p
cudaError_t launch_cg_update(void* x, void* r, void* p, const void* q, int64_t n, double* part, CgState* st,
                             cudaStream_t s);
// cg_blocks(n) partials (double2) of v^H y
cudaError_t launch_vhy_part(const void* v, const void* y, int64_t n, double* part, cudaStream_t s);

// Restart rotation of a (hi, lo) basis on the tensor cores (rotate_tc.cu): BF16 digit splitting of
// both operands, exact FP32 accumulation of every digit pair, FP64 result as launch_rotate_df.
struct TcWork {
  int8_t* Erow = nullptr;   // 2n row exponents of V
  uint8_t* Bimg = nullptr;  // BF16 digit planes of Z, ceil(kk_max/32) x ceil(m/16) x 7168 bytes
  int* Ecol = nullptr;      // column exponents of Z
  int* err = nullptr;       // nonzero: a bounded wait in the rotation kernel ran out
  int64_t n = 0;
  int m = 0, kk_max = 0;
};
int tc_rotate_max_m();
size_t tc_rotate_bytes(int64_t n, int m, int kk_max);
TcWork tc_rotate_carve(void* base, int64_t n, int m, int kk_max);
// fresh_rowexp: recompute the row exponents of V (false: V is unchanged since the last call)
// selftest = 1: the first tile's accumulator barrier is never signalled, so a bounded wait runs out and
// w.err is set (the failure path, without a fault; the output is then undefined).
cudaError_t launch_rotate_tc(const void* V, int64_t n, int m, const double* Z, int kk, void* out, const TcWork& w,
                             bool fresh_rowexp, cudaStream_t s, int selftest = 0);
// Stencil y (FP64) = A x with x and the links as (hi, lo) pairs; part (may be null) receives the
// block partials of x^H y.  op.U / op.W: (hi, lo) links, structure-of-arrays [4][9][V].
int matvec_df_blocks(const OpDev& op);
cudaError_t launch_matvec_df(const OpDev& op, const void* x, void* y, double* part, cudaStream_t s);
// One Chebyshev step of B = p(A) fused into the compensated-FP32 stencil product (x, t_prev, t_next,
// acc, v: (hi, lo) float4 vectors; t_next may alias t_prev): t_next = sc (A x - c x) - t_prev,
// acc = g0 v + g t_next (init) or acc += g t_next; on the last step acc goes to y (FP64) with
// matvec_df_blocks(op) double2 partials of conj(v) y in part.
cudaError_t launch_matvec_df_cheb(const OpDev& op, const void* x, const void* t_prev, void* t_next, void* acc,
                                  const void* v, void* y, double* part, double kappa, double m0, double c, double sc,
                                  double g, double g0, int init, int last, cudaStream_t s);
cudaError_t launch_links_df(const void* in, void* out, int64_t vol, cudaStream_t s);

// Kernel classes for the optional per-kernel profile.
enum KernelTag {
  K_MATVEC = 0, K_GS_FIRST, K_GS_REDUCE, K_GS_UPDATE, K_GS_DOT, K_GS_NORMALIZE, K_RITZ, K_ROTATE,
  K_RESID, K_SHRINK, K_OTHER, K_RITZ_FALLBACK, K_FILTER, K_GS_STEP, K_CG, K_NTAGS
};
template <typename R>
cudaError_t launch_fill_ones(void* v, int64_t n, cudaStream_t s);
template <typename R>
cudaError_t launch_normalize_col(void* v, int64_t n, double* part, int nblk, cudaStream_t s);

// Ritz solve of the leading m x m block of T-bar (FP64): the kk eigenpairs nearest the wanted
// end, sorted toward it, into lam[0..kk) and Z[:, 0..kk) (m x m column-major, ld m).  k is the size
// of the kept (arrow) part.  Fast path: bisection + inverse iteration, one warp per pair, checked;
// on any failed check the one-CTA Jacobi kernel recomputes all m pairs.  flags >= kk + 1 ints,
// work >= 2*mp*mp doubles (mp = m rounded up to even).  *nlaunch receives the kernel count.
cudaError_t launch_ritz(const double* T, int ldt, int m, int k, int kk, int which, double* lam, double* Z,
                        int* flags, cudaStream_t s);
// The Jacobi fallback after launch_ritz: runs only if launch_ritz's checks failed (flags[0] != 0),
// and then counts the event in *fallbacks.
cudaError_t launch_ritz_fallback(const double* T, int ldt, int m, int which, double* lam, double* Z, double* work,
                                 const int* flags, long long* fallbacks, cudaStream_t s);
// The Jacobi kernel alone (all m pairs).
cudaError_t launch_ritz_jacobi(const double* T, int ldt, int m, int which, double* lam, double* Z, double* work,
                               cudaStream_t s);

// Vout[:, 0:kk] = V[:, 0:m] * Z[:, 0:kk] (V complex n x m, ld n; Z real m x kk, ld m).
template <typename R>
cudaError_t launch_rotate(const void* V, int64_t n, int m, const double* Z, int kk, void* Vout,
                          cudaStream_t s);
// V[:, c] = Vsrc[:, perm[c]] for c < k and V[:, k] = V[:, m] (restart shrink, Algorithm 1).
template <typename R>
cudaError_t launch_shrink(void* V, const void* Vsrc, int64_t n, const int* perm, int k, int m,
                          cudaStream_t s);
// out[:, c] = V[:, order[c]] and, if partners, out[:, nev + c] = J conj(V[:, order[c]]).
template <typename R>
cudaError_t launch_gather_pairs(const void* V, int64_t n, const int* order, int nev, int partners,
                                void* out, cudaStream_t s);
// Column sums of squares partials -> sqrt into out[c] (c < ncol), partials [ncol][nblk].
cudaError_t launch_reduce_norms(const double* part, int nblk, int ncol, double* out, cudaStream_t s);
// Lemma 1 check partials: sum (v1 y2 - v2 y1), ||y||^2, ||v||^2 over all rows -> out[4].
template <typename R>
cudaError_t launch_jsym_check(const void* v, const void* y, int64_t h, double* out, cudaStream_t s);
template <typename R>
cudaError_t launch_fill_random(void* v, int64_t n, uint64_t seed, cudaStream_t s);
// Gathers lam[0..m), Z[m-1, 0..m), T[m][m-1], st->status into rep[2m + 2].
cudaError_t launch_report(const double* lam, const double* Z, int m, const double* T, int ldt,
                          const StepState* st, double* rep, cudaStream_t s);

// Mixed precision helpers: out64 = sum of the first ncol FP32 columns (promoted); FP64 -> FP32
// copies; FP64 links [4][V][9] to FP32 structure-of-arrays [4][9][V].
cudaError_t launch_sum_columns(const void* X32, int64_t n, int ncol, void* out64, cudaStream_t s);
cudaError_t launch_c128_to_c64(const void* in, void* out, int64_t count, cudaStream_t s);
cudaError_t launch_links_soa(const void* in, void* out, int64_t vol, cudaStream_t s);

// ------------------------------------------------------------------ batched dense solver (batch.cu)
// Launch arguments of the persistent kernel: instance i has order n = 2 h[i]; its A11 and A12 are
// h x h row-major at a_off[i] in the packed arrays (double2, or float4 (hi, lo) in the double-float
// form).  Per CTA slot: V of nmax x (m + 1) 16-byte elements and an FP64 rotation target of
// nmax x kk.  Results: out_ev / out_res [count][nev] sorted toward the wanted end, out_stats
// [count][kBatchStats] = {Lanczos products, outer iterations, status, residual products, Ritz
// fallbacks, Gram-Schmidt passes}, out_vec at vec_off[i] (n x nev FP64 columns, written once
// converged), prof (optional) [count][kBatchPhases] SM cycles per phase.  queue: work counter.
struct BatchArgs {
  int count;
  const int* order;
  const int64_t* h;
  const int64_t* a_off;
  const void* A11;
  const void* A12;
  void* Vslots;
  void* Tslots;
  int64_t nmax;
  int m, nev, mwin, kk, which, gs_passes, max_restarts;
  double tol;
  double* out_ev;
  double* out_res;
  int* out_stats;
  void* out_vec;
  const int64_t* vec_off;
  long long* prof;
  int* queue;
  int mv_rows;     // tile: rows of the product a warp takes at once (1 or 2; they share the loads of x)
  int gs_groups;   // tile: most thread groups splitting the columns of the compensated update (0: all that fit)
};
constexpr int kBatchStats = 6;
constexpr int kBatchPhases = 5;   // Lanczos product + alpha, Gram-Schmidt, Ritz, rotation + shrink, residuals
constexpr int kBatchMaxM = 64;
constexpr int kBatchMaxNev = 32;
constexpr int kBatchMaxThreads = 512;
size_t batch_smem_bytes(int64_t nmax, int m, int kk, int threads);
cudaError_t batch_occupancy(bool df, int mv_rows, int threads, size_t smem, int* blocks_per_sm);
cudaError_t launch_batch(bool df, const BatchArgs& a, int grid, int threads, cudaStream_t s);
// In place: each double2 element becomes the float4 (hi.re, hi.im, lo.re, lo.im) with hi = fl32(x),
// lo = fl32(x - hi).
cudaError_t launch_split_df_inplace(void* A, int64_t count, cudaStream_t s);
cudaError_t launch_c64_to_c128(const void* in, void* out, int64_t count, cudaStream_t s);

// ------------------------------------------------------------------ polynomial filter (filter.cu)
// One step of the Chebyshev recurrence for B = p(A) = sum_k g_k T_k((A - c I)/e) over n complex
// entries of type R: t_next = sc (ax - c t_cur) - sp t_prev; acc = g0 v + g t_next (init) or
// acc += g t_next; t_next may alias t_prev.  part (optional): cheb_blocks(n) double2 partials of
// conj(v) acc.  split_next (optional): float4 (hi, lo) copy of t_next.
int cheb_blocks(int64_t n);
template <typename R>
cudaError_t launch_cheb_step(const void* ax, const void* t_cur, const void* t_prev, void* t_next, void* acc,
                             const void* v, int64_t n, double c, double sc, double sp, double g, double g0, int init,
                             double* part, void* split_next, cudaStream_t s);
// out[0] = sum of the real parts of nblk double2 partials.
cudaError_t launch_sum_re(const double* part, int nblk, double* out, cudaStream_t s);
// cheb_blocks(n) partial sums of |y - lam[0] x|^2 (FP64 complex vectors).
cudaError_t launch_resid_part(const void* y, const void* x, const double* lam, int64_t n, double* part,
                              cudaStream_t s);
// out[i][k] (k <= degree) = Jackson-damped Chebyshev coefficients of the step [x <= tau[i]] (FP32).
cudaError_t launch_damped_step(const double* tau, int count, int degree, float* out, cudaStream_t s);

// The whole Gram-Schmidt part of one Lanczos step (alpha, every pass, normalisation) as one
// cooperative launch (gs.cu).  gs_coop_occupancy: resident blocks per SM for basis size m (0 if the
// device cannot launch cooperatively).  The launch's grid is a.nblk: one row block per CTA, all
// resident.  nrm2: 2 * a.nblk doubles of scratch.
template <typename R>
cudaError_t gs_coop_occupancy(int m, int* per_sm);
template <typename R>
cudaError_t launch_gs_step_coop(const GSArgs& a, const double2* alpha_part, int n_alpha_part, int passes,
                                double* nrm2, int grid, cudaStream_t s);

// The compensated-FP32 Gram-Schmidt of one Lanczos step as one cooperative launch (gsdf.cu); its
// shared memory, so its occupancy, depends on rows_per_block and m of `a`.
cudaError_t gsdf_coop_occupancy(const GSArgs& a, int* per_sm);
cudaError_t launch_gsdf_step_coop(const GSArgs& a, void* x, const double2* alpha_part, int n_alpha_part, int passes,
                                  double* nrm2, int grid, cudaStream_t s);

// Sets the thread-local text returned by jtrlan_last_error().
void set_last_error(const char* msg);

}  // namespace jtr
