/* jtrlan.h -- C ABI of libjtrlan: thick-restart Lanczos for Hermitian J-symmetric matrices
 * (TRLAN-JSYM) on one NVIDIA GB300 (sm_103a).
 *
 * Paper: T. Ishikawa and T. Sogabe, "A thick-restart Lanczos type method for Hermitian
 * J-symmetric eigenvalue problems" (arXiv:2001.07428).
 *
 * Problem (Sec. 1, eqs. (1), (2), (4)): A is Hermitian and J-symmetric, J A J^{-1} = A^T with
 * the canonical J = [[O, -I], [I, O]], so A = [[A11, A12], [A12^H, A11^T]] with A11^H = A11 and
 * A12^T = -A12.  Every eigenvalue is doubly degenerate and y = J x* pairs each eigenvector x
 * with a second one.  Algorithm 1 (TRLAN-JSYM) with the Lanczos step of Algorithm 2 finds the
 * nev wanted eigenvalues once each, searching only one of the two orthogonal half-spaces.
 *
 * Vector layout (canonical): n complex numbers, x = [x1; x2], each half n/2 long.  Complex
 * numbers are stored as interleaved (re, im) pairs: double2 for JTRLAN_C128, float2 for
 * JTRLAN_C64.  Matrices of vectors (eigenvectors) are column-major, one vector per column.
 *
 * Conventions for every call:
 *   - Every call returns a jtrlan_status and never throws or aborts across the ABI.
 *   - All GPU work is enqueued on the CUDA stream given to jtrlan_create (NULL = legacy
 *     default stream).  Calls that return host data synchronise that stream.
 *   - Pointers documented as "host or device" may be either: copies use unified addressing.
 *   - jtrlan_last_error() returns a thread-local text for the last failing call.
 */
#ifndef JTRLAN_H
#define JTRLAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JTRLAN_OK = 0,
  JTRLAN_EINVAL = 1,      /* invalid argument (sizes, parameters, null pointer) */
  JTRLAN_ENOMEM = 2,      /* device or host allocation failed */
  JTRLAN_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  JTRLAN_ENOTJSYM = 4,    /* the Lemma 1 self-check found the operator not J-symmetric */
  JTRLAN_EBREAKDOWN = 5,  /* Lanczos breakdown: beta below the breakdown threshold */
  JTRLAN_ENOCONV = 6,     /* max_restarts reached before nev pairs converged */
  JTRLAN_ETIMEOUT = 7,    /* a bounded device-side wait ran out (tensor-core rotation) */
  JTRLAN_ESTATE = 8       /* call out of order (e.g. pairs before a successful solve) */
} jtrlan_status;

enum { JTRLAN_DENSE = 0, JTRLAN_STENCIL4D = 1 };     /* jtrlan_operator.kind   */
enum { JTRLAN_C128 = 0, JTRLAN_C64 = 1 };            /* jtrlan_operator.dtype  */
enum { JTRLAN_SMALLEST = 0, JTRLAN_LARGEST = 1 };    /* jtrlan_params.which    */
enum { JTRLAN_FP64 = 0, JTRLAN_MIXED = 1, JTRLAN_MIXED_REORTH = 2 };  /* jtrlan_params.precision */

/* The operator A in the block form of eq. (4).
 *
 * kind = JTRLAN_DENSE: a11 and a12 are (n/2) x (n/2) row-major complex matrices (host or
 *   device), the blocks A11 (Hermitian) and A12 (skew-symmetric) of eq. (4).  Only these two
 *   blocks are read; A12^H and A11^T are applied through conjugation.
 * kind = JTRLAN_STENCIL4D: a periodic 4D lattice dims[0..3] = (Lx, Ly, Lz, Lt) with site index
 *   s = x + Lx*(y + Ly*(z + Lz*t)), three colours per site, n = 6 * Lx*Ly*Lz*Lt.  U and W are
 *   link fields of shape [4][V][3][3] row-major complex (host or device), direction mu = 0..3
 *   along x, y, z, t.  The blocks are
 *     (A11 p)(s) = m0 p(s) + sum_mu [U_mu(s) p(s+mu) + U_mu(s-mu)^H p(s-mu)],
 *     (A12 p)(s) = kappa * sum_mu [W_mu(s) p(s+mu) - W_mu(s-mu)^T p(s-mu)],
 *   which are Hermitian and skew-symmetric respectively, as eq. (4) requires.
 * dtype: storage precision of the caller's a11/a12 or U/W arrays (JTRLAN_C128 = double2,
 *   JTRLAN_C64 = float2).  jtrlan_create converts them to the precision the solve needs.
 * Ownership: jtrlan_create copies the operator into buffers the context owns; the caller may
 *   free or reuse its arrays as soon as jtrlan_create returns. */
typedef struct {
  int kind;
  int dtype;
  int64_t n;          /* vector length; even.  Stencil: must equal 6 * volume. */
  int dims[4];        /* stencil only */
  double m0;          /* stencil only: diagonal mass term of A11 */
  double kappa;       /* stencil only: strength of the A12 hopping term */
  const void* a11;    /* dense only */
  const void* a12;    /* dense only */
  const void* U;      /* stencil only */
  const void* W;      /* stencil only */
} jtrlan_operator;

/* Parameters of Algorithm 1.
 *   nev: wanted eigenvalues (one per J pair), 0 < nev < m.
 *   m: maximum Krylov dimension, m < n/2.  mwin: restart window, k = min(icnv + mwin, m - 1)
 *   (eq. (29)), 0 <= mwin.
 *   tol: convergence threshold on ||A x - lambda x|| with ||x|| = 1 (Algorithm 1, normal mode).
 *   which: JTRLAN_SMALLEST (smallest algebraic) or JTRLAN_LARGEST.
 *   precision: JTRLAN_FP64 -- plain FP64 arithmetic throughout.
 *     JTRLAN_MIXED_REORTH -- the basis V is stored as (hi, lo) FP32 pairs (about 48 significant
 *       bits) and the three steps that plain FP64 spends on the FP64 pipe run in compensated FP32
 *       ("double-float": exact FMA-split products, TwoSum-carried sums): the stencil product A v_j
 *       (on (hi, lo) links, or on the complex64 links themselves when dtype is JTRLAN_C64, which
 *       are exact in FP32; a dense operator keeps the FP64 product), the Gram-Schmidt passes
 *       against V and W = J V^*, and the restart rotation V_m Z (on the tensor cores by exact BF16
 *       digit splitting with FP32 accumulation in tensor memory when m <= 320 and rotate_simt is 0,
 *       else on the CUDA cores).  The vector y being orthogonalised, alpha/beta, the norms and the
 *       sqrt(2) test, the Ritz solve, the rotated Ritz vectors and the true residuals are FP64.
 *       Inside a certifying filter's Chebyshev steps on the stencil the hopping sums are carried as
 *       biased block sums instead of by TwoSum (about 2^-41 of sum |a| |x| against 2^-45): those
 *       products only shape the Krylov space, and every pair is still accepted on A's residual.
 *     JTRLAN_MIXED -- an FP32 phase (matvec, Gram-Schmidt and rotation in FP32; alpha/beta, Ritz
 *       solve and residual norms in FP64) run to max(tol, 1e-5 max|t|), then the JTRLAN_MIXED_REORTH
 *       solve started from the normalised sum of the FP32 Ritz vectors, run to tol.
 *     Results are FP64 in every mode.
 *   max_restarts: bound on outer iterations (N_conv); 0 selects 1000.
 *   gs_max_passes: bound on Gram-Schmidt passes per Lanczos step (Algorithm 2 has none);
 *     0 selects 3.
 *   v1: optional start vector (n complex128 numbers, whatever the operator's dtype; host or
 *     device), read by every jtrlan_solve; NULL gives v1 = (1, ..., 1)/sqrt(n) as in Algorithm 1.
 *     It is normalised by the library.
 *   check_jsym: if nonzero, jtrlan_create tests Lemma 1, |(J v*)^H A v| <= 1e-10 ||A v|| ||v||,
 *     on a fixed pseudo-random v and fails with JTRLAN_ENOTJSYM otherwise.
 *   profile: if nonzero, jtrlan_solve brackets every kernel launch with CUDA events on the context
 *     stream and sums the device time per kernel class (read with jtrlan_get_profile).  This adds
 *     two event records per launch; leave it off for timed runs.
 *   filter_degree, filter_coeffs, filter_lo, filter_hi (the paper has no filter): with d =
 *     filter_degree > 0 the FP32 phase of JTRLAN_MIXED runs Algorithm 1 on B = p(A) =
 *     sum_k g_k T_k((A - c I)/e), c = (lo + hi)/2, e = (hi - lo)/2, T_k the Chebyshev polynomials,
 *     wanting the LARGEST eigenvalues of B; real g_k keep B Hermitian J-symmetric.  That phase is
 *     judged by the Lanczos residual estimates |t_{m+1,i}| of B only (to 1e-5 max|t|); the second,
 *     unfiltered phase then starts from the sum of its Ritz vectors and certifies every pair with
 *     the true residual of A, so a poor filter costs time, never accuracy.  [lo, hi] should contain
 *     the spectrum (jtrlan_bounds estimates it); 1 <= d <= 1024.
 *   filter_final_degree, filter_final_coeffs: with d2 > 0 the certifying phase (the only phase of
 *     JTRLAN_FP64 and JTRLAN_MIXED_REORTH, the second of JTRLAN_MIXED) also runs on B2 = p2(A), same
 *     window, largest wanted, with FP64-accurate products; a Ritz vector x of B2 is accepted when
 *     ||A x - (x^H A x) x|| < tol (checked once B2's estimate is below 10 tol), and x^H A x is the
 *     eigenvalue reported.  Choose p2 strictly decreasing across the wanted eigenvalues: where p2 is
 *     flat, B2 cannot separate eigenvectors and the solve ends in JTRLAN_ENOCONV.
 *   invert, cg_tol, cg_max_iter: Algorithm 1's invert mode, for the smallest eigenvalues of a
 *     Hermitian positive definite J-symmetric A (Sec. 4 uses it with CG).  The Lanczos product is
 *     A^{-1} v_j, each applied by conjugate gradients from x = 0 to ||v_j - A x|| <= cg_tol; the
 *     wanted end is the largest eigenvalues lambda_i of T (those of A^{-1}); every restart takes
 *     c = ||A v_{m+1}|| and reports ev(i) = 1/lambda_i with the residual estimate
 *     res_est(i) = c |t_{m+1,i} ev(i)|, and the true residuals ||A v_i - ev(i) v_i|| use A itself.
 *     Needs which = JTRLAN_SMALLEST, precision = JTRLAN_FP64 and no filter; plain_trlan may be set
 *     (the TRLAN of the paper's comparison in invert mode).  A CG step with p^H A p <= 0 (A not
 *     positive definite) ends the solve in JTRLAN_EBREAKDOWN. */
typedef struct {
  int nev;
  int m;
  int mwin;
  double tol;
  int which;
  int precision;
  int max_restarts;
  int gs_max_passes;
  const void* v1;
  int check_jsym;
  int profile;        /* nonzero: time every kernel launch with CUDA events (jtrlan_get_profile) */
  int filter_degree;  /* 0: none; else the degree d of the polynomial filter (JTRLAN_MIXED only) */
  const double* filter_coeffs;  /* host, d + 1 Chebyshev coefficients g_0..g_d (copied at create) */
  double filter_lo, filter_hi;  /* the window [a, b] of the Chebyshev variable (A - c)/e */
  int filter_final_degree;      /* 0: none; else the degree of the certifying phase's filter */
  const double* filter_final_coeffs;  /* host, filter_final_degree + 1 coefficients (copied) */
  int plain_trlan;    /* nonzero: the standard TRLAN the paper compares against (Algorithms 1 and 2
                         with W removed: Gram-Schmidt against V only) */
  int rotate_simt;    /* nonzero: the restart rotation of a compensated-FP32 basis runs on the CUDA
                         cores (jtrlan_rotate_df path 1) instead of the tensor cores */
  int invert;         /* nonzero: Algorithm 1's invert mode (see below) */
  double cg_tol;      /* invert mode: relative residual ||b - A x|| / ||b|| of each CG solve (0: 1e-12) */
  int cg_max_iter;    /* invert mode: iterations per CG solve before JTRLAN_ENOCONV (0: 10000) */
  int gs_split;       /* nonzero: the Gram-Schmidt part of every Lanczos step runs as separate kernel
                         launches (first pass, reduction, update, later passes, normalisation) instead
                         of one cooperative launch.  The library takes this path by itself where a
                         cooperative launch is unavailable or one block's rows do not fit shared
                         memory; the switch exists so that the path can be exercised on any size.
                         Same arithmetic and results up to summation order. */
} jtrlan_params;

/* Counters of the last solve (Sec. 3 counts only the Lanczos-step products as N_MV). */
typedef struct {
  int64_t n_matvec;        /* N_MV: products A v_j inside Algorithm 2 */
  int64_t n_resid_matvec;  /* products for the true residuals of Algorithm 1 (not in N_MV) */
  int64_t n_gs_passes;     /* Gram-Schmidt passes over [V, W] */
  int n_restarts;          /* N_conv: outer iterations */
  int icnv;                /* converged pairs at exit */
  double solve_ms;         /* wall time of jtrlan_solve on the host clock */
  int64_t n_launches;      /* CUDA kernels launched by the solve */
  int n_ritz_fallbacks;    /* restarts whose fast Ritz solve failed a check (Jacobi used) */
  int n_restarts_fp32;     /* JTRLAN_MIXED: outer iterations of the FP32 phase (in n_restarts) */
  int64_t n_matvec_fp32;   /* JTRLAN_MIXED: products of the FP32 phase (included in n_matvec) */
  int64_t n_matvec_inner;  /* invert mode: products A p launched by the CG solves (N_MV counts the
                              A^{-1} v_j), plus one A v_{m+1} per restart */
  int64_t n_cg_iters;      /* invert mode: CG iterations to convergence, summed over the solves */
} jtrlan_stats;

/* Per-kernel-class profile of the last solve (filled when jtrlan_params.profile was set; the
 * launch counts are always filled).  work[] holds the algorithmic work of each class:
 *   "matvec": products A v (Lanczos steps) times the units of one product -- lattice sites for a
 *     stencil, (n/2)^2 block entries for a dense operator;
 *   "gs_first", "gs_dot", "gs_update": row-pair x basis-column products (each reads one complex
 *     number of each half of a basis vector and does four complex multiply-adds);
 *   "rotate": (2n) x m x kk real multiply-adds of V_m Z;  "resid": products A v as for "matvec";
 *   other classes: 0. */
#define JTRLAN_MAX_KERNEL_CLASSES 16
typedef struct {
  int n_classes;
  const char* names[JTRLAN_MAX_KERNEL_CLASSES];
  double ms[JTRLAN_MAX_KERNEL_CLASSES];
  int64_t launches[JTRLAN_MAX_KERNEL_CLASSES];
  double work[JTRLAN_MAX_KERNEL_CLASSES];
} jtrlan_profile;

typedef struct jtrlan_ctx jtrlan_ctx;  /* opaque; owned by the library */

/* Validates op and params, allocates the context's device buffers and copies the operator.
 * cuda_stream: a cudaStream_t (or NULL) on which every later call enqueues its work.
 * Errors: JTRLAN_EINVAL (odd n, n != 6V for a stencil, nev/m/mwin out of range, null
 * pointers), JTRLAN_ENOMEM, JTRLAN_ECUDA, JTRLAN_ENOTJSYM.  *out is NULL on failure. */
jtrlan_status jtrlan_create(const jtrlan_operator* op, const jtrlan_params* params,
                            void* cuda_stream, jtrlan_ctx** out);

/* y = A x in the canonical layout, both device pointers of n complex numbers: double2 for a
 * JTRLAN_FP64 context, float2 (the FP32 operator) for the two mixed modes.
 * Enqueued on the context stream; no sync.
 * This is the Algorithm 2 product A v_j.  Errors: JTRLAN_EINVAL (null), JTRLAN_ECUDA. */
jtrlan_status jtrlan_apply(jtrlan_ctx* ctx, const void* x, void* y);

/* Runs Algorithm 1 (TRLAN-JSYM) with the Lanczos step of Algorithm 2 until nev pairs have a
 * true residual below tol.  Synchronises the context stream once per restart.  stats may be
 * NULL.  Errors: JTRLAN_ENOCONV, JTRLAN_EBREAKDOWN, JTRLAN_ECUDA. */
jtrlan_status jtrlan_solve(jtrlan_ctx* ctx, jtrlan_stats* stats);

/* Copies the converged pairs of the last successful solve, sorted by eigenvalue (ascending for
 * JTRLAN_SMALLEST, descending for JTRLAN_LARGEST).
 *   evals: host array of nev doubles (may be NULL).
 *   evecs: host or device array, column-major n x nev (or n x 2nev if with_partners) of double2
 *     (FP64 in both precision modes); may be NULL.  With partners,
 *     column nev + i holds y_i = J x_i^* (eq. (2)).
 *   res: host array of nev doubles, the true residuals ||A x_i - lambda_i x_i|| (may be NULL).
 * Synchronises the context stream.  Errors: JTRLAN_ESTATE if no solve has succeeded. */
jtrlan_status jtrlan_pairs(jtrlan_ctx* ctx, int with_partners, double* evals, void* evecs,
                           double* res);

/* Copies the per-kernel profile of the last solve into *out.  Errors: JTRLAN_EINVAL (null). */
jtrlan_status jtrlan_get_profile(jtrlan_ctx* ctx, jtrlan_profile* out);

/* Frees everything the context owns (after synchronising its stream).  NULL is a no-op. */
void jtrlan_destroy(jtrlan_ctx* ctx);

/* y = p(A) x by the Chebyshev recurrence of the context's filter (window filter_lo..filter_hi):
 *   - a JTRLAN_MIXED context with an FP32-phase filter (filter_degree > 0): that filter with the FP32
 *     operator; x, y DEVICE complex64 vectors of n entries;
 *   - otherwise a context with a certifying filter (filter_final_degree > 0, or jtrlan_set_filter):
 *     that filter with the product the solve uses in its certifying phase (FP64, or on the stencil of
 *     the mixed forms the compensated-FP32 product fused with a float-float recurrence step); x, y
 *     DEVICE complex128 vectors of n entries.
 * x and y distinct.  Enqueued on the context stream; uses the context's filter buffers (no call on
 * the same context may overlap it).  Errors: JTRLAN_EINVAL (null, or no filter), JTRLAN_ECUDA. */
jtrlan_status jtrlan_apply_filter(jtrlan_ctx* ctx, const void* x, void* y);

/* Spectral bounds for a filter window (the paper has no counterpart): `steps` Lanczos steps of
 * Algorithm 2 on A (full reorthogonalisation, no restart) from a fixed pseudo-random start, in the
 * context's working precision (FP32 for JTRLAN_MIXED), then the Rayleigh-Ritz values of the
 * steps x steps tridiagonal in FP64.  *lo = theta_min - |beta_steps z_{steps,min}| (the smallest
 * Ritz value less its residual bound: an estimate of lambda_min), *hi = theta_max + beta_steps (an
 * estimate, not a guarantee, of an upper bound of lambda_max).  2 <= steps <= m.  Synchronises the
 * context stream.  Afterwards jtrlan_get_profile describes this call (its launches) until the next
 * solve.  Errors: JTRLAN_EINVAL,
 * JTRLAN_EBREAKDOWN, JTRLAN_ECUDA. */
jtrlan_status jtrlan_bounds(jtrlan_ctx* ctx, int steps, double* lo, double* hi);

/* Sets (or replaces) the certifying phase's filter of a context: the same as creating it with
 * filter_final_degree = degree, filter_final_coeffs = coeffs (host, degree + 1 Chebyshev coefficients
 * g_0..g_degree, copied) and the window [lo, hi], so that a later jtrlan_solve runs Algorithm 1 on
 * B = p(A) with every pair certified by the true residual of A (see jtrlan_params).  The window is
 * shared with the FP32-phase filter of JTRLAN_MIXED.  It lets one context serve a filter chosen per
 * solve (the learned filter: jtrlan_bounds on this context, the network, then this call) without
 * copying the operator again.  The first call on a context created without a certifying filter
 * allocates that phase's buffers (four vectors); later calls only copy coefficients.  Clears the
 * results of the last solve (jtrlan_pairs returns JTRLAN_ESTATE until the next solve).
 * Errors: JTRLAN_EINVAL (null, degree outside 1..1024, lo >= hi, a non-finite coefficient, an
 * invert-mode context), JTRLAN_ENOMEM. */
jtrlan_status jtrlan_set_filter(jtrlan_ctx* ctx, int degree, const double* coeffs, double lo, double hi);

/* Jackson-damped Chebyshev coefficients of the step [x <= tau_i] (Jackson damping as in Weisse et
 * al., Rev. Mod. Phys. 78, 275 (2006), N = degree + 1 moments), the targets of the learned filter:
 * tau: device, count doubles; out: device, count x (degree + 1) floats.  Enqueued on cuda_stream.
 * Errors: JTRLAN_EINVAL, JTRLAN_ECUDA. */
jtrlan_status jtrlan_damped_step(const double* tau, int count, int degree, float* out, void* cuda_stream);

/* Residual norms without device allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot call cudaMalloc --
 * an application whose own caching allocator already holds the device memory it may use, code
 * that must not let cudaMalloc's implicit synchronisation stall other streams, or a plug-in given
 * no allocation rights.  It computes res[i] = ||A x_i - lambda[i] x_i|| for the ncols columns x_i
 * of X, with the same kernels as the solver's convergence check, and allocates nothing: its
 * scratch lives in one static device array of 8 * JTRLAN_NOALLOC_MAX_PARTIALS + 20 *
 * JTRLAN_NOALLOC_MAX_COLS bytes (about 2 MiB) that every GPU which loads the library holds until the
 * process exits.
 *   op: the operator; dtype must be JTRLAN_C128 and a11/a12 or U/W must be DEVICE pointers (no
 *     copy or conversion is made).  X: device, n x ncols complex128, column-major with leading
 *     dimension ldx >= n.  lambda: host, ncols doubles.  res: host, ncols doubles (written).
 *   cuda_stream: the stream to run on (NULL = legacy default); the call synchronises it.  It copies
 *     from pageable host memory and synchronises, so it may not be made on a stream that is being
 *     captured into a CUDA graph: that returns JTRLAN_EINVAL before anything is enqueued.
 * Limits: ncols <= JTRLAN_NOALLOC_MAX_COLS and ncols * B <= JTRLAN_NOALLOC_MAX_PARTIALS, where B is
 *   the number of blocks of one product (stencil: ceil(64 ceil(3 V / 8) / 256), which is
 *   ceil(24 V / 256) when V is a multiple of 8; dense: ceil((n/2) / 8)).
 *   Larger requests fail with JTRLAN_EINVAL and a message naming the limit: split the columns.
 * The first call on a device looks up the array's device address there (cudaGetSymbolAddress with
 * that device current) and caches it for the life of the process; after a cudaDeviceReset (or any
 * other reset of the device's primary context) that address is stale, so do not use this call on a
 * device that has been reset in the same process.
 * All calls on a device share the one array, and every call overwrites all of it that it reads,
 * so nothing carries over between calls; calls whose GPU work overlaps (on different streams or
 * host threads) race on it and must be serialised by the caller.  When the call fails after it has
 * enqueued work, it waits for that work before returning, so a retry does not race with it.
 * Errors: JTRLAN_EINVAL (null pointers, sizes beyond the limits, unsupported dtype, a capturing
 * stream), JTRLAN_ECUDA. */
#define JTRLAN_NOALLOC_MAX_PARTIALS 262144
#define JTRLAN_NOALLOC_MAX_COLS 1024
jtrlan_status jtrlan_residual_norms_noalloc(const jtrlan_operator* op, const void* X, int64_t ldx,
                                            int ncols, const double* lambda, double* res,
                                            void* cuda_stream);

/* Restart rotation of a compensated-FP32 basis: out = V Z.
 *
 * The thick-restart step of Algorithm 1 keeps the Ritz vectors V_m Z, Z the eigenvectors of T_m;
 * this is that product for a basis held as (hi, lo) FP32 pairs, the layout of the
 * JTRLAN_MIXED_REORTH and JTRLAN_MIXED solvers, with an FP64 result.
 *   V: device, n x m complex numbers, column-major (column j at V + j n), each as float4
 *     (re_hi, im_hi, re_lo, im_lo), the value being hi + lo; |V| < 2^127.
 *   Z: device, m x kk FP64, column-major (column c at Z + c m); |Z| < 2^120.
 *   out: device, n x kk complex128, column-major, written; must not overlap V or Z.
 *   path: 0 = tensor cores (tcgen05, BF16 digit splitting with exact FP32 accumulation; needs
 *     m <= 320), 1 = compensated FP32 on the CUDA cores (any m), 2 = a self-test of the tensor-core
 *     kernel's failure path: one accumulator barrier is never signalled, the kernel's bounded wait
 *     (about 2 s) runs out, the kernel frees its tensor memory and returns, and the call returns
 *     JTRLAN_ETIMEOUT with out undefined; the stream stays usable.
 * Each entry agrees with the exact product of the given values to about 2^-49 m max_k |V_rk|
 * max_k |Z_kc| on either path (on path 0 a row of the real view whose entries all lie below 2^-120
 * is resolved to 2^-169 absolute instead; path 1 multiplies FP32 pairs, so there the bound needs
 * every nonzero product |V_rk Z_kc| above 2^-100 and every |Z| below 2^100).  The call allocates and frees its scratch (row and column exponents,
 * the BF16 digits of Z) and synchronises the stream.
 * Errors: JTRLAN_EINVAL (null pointers, n < 1, m < 1, kk < 1, path 0 or 2 with m > 320, path not 0/1/2),
 * JTRLAN_ENOMEM, JTRLAN_ECUDA, JTRLAN_ETIMEOUT (a bounded wait inside the tensor-core kernel ran
 * out; the stream stays usable). */
jtrlan_status jtrlan_rotate_df(const void* V, int64_t n, int m, const double* Z, int kk, void* out, int path,
                               void* cuda_stream);

/* ---- Batched dense solver: many independent dense operators of uneven order, one persistent launch.
 *
 * Algorithm 1 (TRLAN-JSYM) with the Lanczos step of Algorithm 2, as jtrlan_solve runs it on one
 * operator, applied to `count` dense Hermitian J-symmetric operators at once: one kernel launch (held
 * in a CUDA graph) in which each CTA takes instances, largest order first, from a device-side queue
 * and runs the whole method for one instance with all control on the device.  Each instance starts
 * from v_1 = (1, ..., 1)/sqrt(n) (Algorithm 1).  precision: JTRLAN_FP64 (plain FP64) or
 * JTRLAN_MIXED_REORTH (products, Gram-Schmidt and rotation in compensated FP32 on (hi, lo) pairs;
 * alpha/beta, the Ritz solve and the residuals in FP64).  */
typedef struct jtrlan_batch jtrlan_batch;  /* opaque; owned by the library */

typedef struct {
  int count;               /* instances in the batch */
  int n_ok;                /* instances that converged */
  int64_t n_matvec;        /* Lanczos-step products A v_j, all instances */
  int64_t n_resid_matvec;  /* products for true residuals, all instances */
  int max_restarts;        /* largest outer-iteration count of any instance */
  int grid;                /* CTAs of the persistent launch */
  int threads;             /* threads per CTA */
  int graph;               /* 1: the launch was replayed from a CUDA graph */
  double solve_ms;         /* device time of the launch (CUDA events on the library's stream) */
  int64_t n_ritz_fallbacks;  /* restarts whose fast Ritz solve failed a check (Jacobi used) */
  int64_t n_gs_passes;       /* Gram-Schmidt passes, all instances */
  double phase_frac[5];      /* params.profile only: share of CTA cycles in the Lanczos product,
                                Gram-Schmidt, Ritz solve, rotation + shrink, residual checks */
} jtrlan_batch_stats;

/* Copies `count` dense operators (ops[i].kind == JTRLAN_DENSE, even ops[i].n with m < n/2, blocks
 * host or device, complex128 or complex64, read during the call only) into one packed device array.
 * params holds nev, m, mwin, tol, which, precision, max_restarts, gs_max_passes and profile (per-phase
 * cycle counts, reported in jtrlan_batch_stats) for every instance; v1 must be NULL and check_jsym 0.  Limits: m <= 64, nev <= 32.  The library runs the batch on a
 * stream of its own, ordered after and before cuda_stream (NULL = legacy default) by events.
 * Errors: JTRLAN_EINVAL (a limit or a field out of range, naming it), JTRLAN_ENOMEM, JTRLAN_ECUDA.
 * *out is NULL on failure. */
jtrlan_status jtrlan_batch_create(int count, const jtrlan_operator* ops, const jtrlan_params* params,
                                  void* cuda_stream, jtrlan_batch** out);

/* Fixes the launch shape: threads per CTA (a multiple of 32 in [64, 512]) and CTAs per SM
 * (0 = as many as fit).  Errors: JTRLAN_EINVAL, JTRLAN_ECUDA. */
jtrlan_status jtrlan_batch_set_shape(jtrlan_batch* b, int threads, int ctas_per_sm);

/* Autotuner: solves the batch once per candidate launch shape (128, 256, 512 threads; 1 .. the
 * occupancy limit of CTAs per SM), timing each with CUDA events, then, at the fastest shape, once per
 * candidate tile shape (jtrlan_batch_set_tiles: 1 or 2 product rows per warp; in the compensated form
 * also all, 1, 2 or 4 update groups), and keeps the fastest of all for later solves (read the tiles
 * with jtrlan_batch_get_tiles).  Any output pointer may be NULL; *best_ms is the fastest time seen.
 * Leaves the results of the last candidate in place.  Errors: JTRLAN_EINVAL, JTRLAN_ECUDA. */
jtrlan_status jtrlan_batch_tune(jtrlan_batch* b, int* threads, int* ctas_per_sm, double* best_ms);

/* Tile shapes of the persistent kernel.  mv_rows: rows of the product A v that a warp takes at once
 * (1 or 2; two rows share the loads of v).  gs_groups (compensated form only): the most thread groups
 * that split the columns of the Gram-Schmidt update y -= V c_v + W c_w, each group walking the row
 * pairs of the instance (0: as many as the block holds; fewer groups give longer column walks and a
 * shorter cross-group sum).  Results agree up to summation order.  Defaults: mv_rows 2 (compensated)
 * or 1 (FP64), gs_groups 0.  Errors: JTRLAN_EINVAL (values out of range). */
jtrlan_status jtrlan_batch_set_tiles(jtrlan_batch* b, int mv_rows, int gs_groups);
jtrlan_status jtrlan_batch_get_tiles(jtrlan_batch* b, int* mv_rows, int* gs_groups);

/* Solves every instance in one persistent launch (captured once into a CUDA graph per launch shape,
 * replayed afterwards) and waits for it.  stats may be NULL.  Returns JTRLAN_OK if all instances
 * converged, else the status of the first failing one (JTRLAN_ENOCONV, JTRLAN_EBREAKDOWN); the
 * per-instance statuses are in jtrlan_batch_results.  Errors: JTRLAN_ECUDA. */
jtrlan_status jtrlan_batch_solve(jtrlan_batch* b, jtrlan_batch_stats* stats);

/* Host copies of the last solve, instance i at row i in creation order:
 *   evals, res: count x nev doubles, sorted by eigenvalue toward the wanted end, res the true
 *     residuals ||A x - lambda x|| (infinity where never tested);
 *   istats: count x JTRLAN_BATCH_STATS ints {Lanczos products, outer iterations, status, residual
 *     products, Ritz fallbacks, Gram-Schmidt passes}.
 * Any pointer may be NULL.  Errors: JTRLAN_ESTATE (no solve yet), JTRLAN_ECUDA. */
#define JTRLAN_BATCH_STATS 6
jtrlan_status jtrlan_batch_results(jtrlan_batch* b, double* evals, double* res, int* istats);

/* Eigenvectors of instance i (creation order) in the order of jtrlan_batch_results: column-major
 * n_i x nev complex128 (double2) into evecs (host or device).  Errors: JTRLAN_EINVAL (index),
 * JTRLAN_ESTATE (no solve, or instance i did not converge), JTRLAN_ECUDA. */
jtrlan_status jtrlan_batch_vectors(jtrlan_batch* b, int i, void* evecs);

/* Frees everything the batch owns (after synchronising its stream).  NULL is a no-op. */
void jtrlan_batch_destroy(jtrlan_batch* b);

/* ---- The learned filter's network (the paper has none): a 3-layer perceptron in FP32,
 *   A1 = tanh(X W1^T + b1), A2 = tanh(A1 W2^T + b2), Y = A2 W3^T + b3,
 * trained on the mean squared error L = mean((Y - T)^2) with Adam (Kingma and Ba, ICLR 2015;
 * b1 = 0.9, b2 = 0.999, eps = 1e-8), all in the library's CUDA kernels.  Parameters are one packed
 * FP32 vector: W1 (width x n_in, row-major), b1, W2 (width x width), b2, W3 (n_out x width), b3, of
 * jtrlan_mlp_param_count(n_in, width, n_out) floats.  Batches X (N x n_in) and T, Y (N x n_out) are
 * row-major FP32 DEVICE arrays.  Work runs on a stream of the network's own, ordered after and
 * before cuda_stream by events. */
typedef struct jtrlan_mlp jtrlan_mlp;  /* opaque; owned by the library */

int64_t jtrlan_mlp_param_count(int n_in, int width, int n_out);

/* Glorot-uniform weights (splitmix64 on the parameter index and seed), zero biases.
 * Errors: JTRLAN_EINVAL (sizes outside 1..4096), JTRLAN_ENOMEM, JTRLAN_ECUDA. */
jtrlan_status jtrlan_mlp_create(int n_in, int width, int n_out, uint64_t seed, void* cuda_stream,
                                jtrlan_mlp** out);

/* Copy the packed parameters out of / into the network (host or device pointer).  Setting them
 * also resets the Adam state. */
jtrlan_status jtrlan_mlp_get_params(jtrlan_mlp* net, float* theta);
jtrlan_status jtrlan_mlp_set_params(jtrlan_mlp* net, const float* theta);

/* Y = network(X) for N samples (enqueued, no synchronisation). */
jtrlan_status jtrlan_mlp_forward(jtrlan_mlp* net, const float* X, int N, float* Y);

/* The loss L of the batch and dL/dtheta (packed order) into grad (host or device, may be NULL) and
 * *loss (host, may be NULL); no parameter change.  Synchronises. */
jtrlan_status jtrlan_mlp_gradient(jtrlan_mlp* net, const float* X, const float* T, int N, float* grad,
                                  double* loss);

/* `steps` full-batch Adam steps at learning rate lr.  The step (forward, loss, back-propagation,
 * update) is captured once per (X, T, N) into a CUDA graph and replayed; loss_hist (host, `steps`
 * floats, may be NULL) receives the loss before each update.  Synchronises.
 * Errors: JTRLAN_EINVAL, JTRLAN_ENOMEM, JTRLAN_ECUDA. */
jtrlan_status jtrlan_mlp_train(jtrlan_mlp* net, const float* X, const float* T, int N, int steps, float lr,
                               float* loss_hist);

void jtrlan_mlp_destroy(jtrlan_mlp* net);

/* Measured arithmetic peaks of the current device, the denominators of roofline fractions (the
 * paper has no counterpart): best of five timed launches of throughput loops that fill every SM with
 * independent accumulator chains -- FP64 FMA on the CUDA cores, FP64 mma.sync m8n8k4 (the FP64 tensor
 * path), FP32 FMA -- in TFLOP/s (an FMA counts 2 flop).  Any output may be NULL.  Takes about 0.5 s;
 * allocates and frees a small scratch buffer; synchronises cuda_stream.  Errors: JTRLAN_ECUDA. */
jtrlan_status jtrlan_measure_peaks(double* fp64_fma_tflops, double* fp64_mma_tflops, double* fp32_fma_tflops,
                                   void* cuda_stream);

/* Static text for a status code. */
const char* jtrlan_status_string(jtrlan_status s);

/* Thread-local text describing the last failure on this host thread ("" if none). */
const char* jtrlan_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* JTRLAN_H */
