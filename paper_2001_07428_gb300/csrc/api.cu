// api.cu -- the C ABI of libjtrlan (include/jtrlan.h): context management and the host side of
// Algorithm 1 (TRLAN-JSYM).  Every vector operation runs in the kernels of matvec.cu, gs.cu and
// ritz.cu; the host keeps only the O(m) bookkeeping of the restart (which Ritz pairs to test,
// the converged-first ordering, k of eq. (29)) and reads back O(m) numbers once per restart.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "../../include/jtrlan.h"

using namespace jtr;

namespace {

thread_local std::string g_last_error;

}  // namespace

void jtr::set_last_error(const char* msg) { g_last_error = msg; }

namespace {

jtrlan_status fail(jtrlan_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define JT_CUDA(expr)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(e_ == cudaErrorMemoryAllocation ? JTRLAN_ENOMEM : JTRLAN_ECUDA,                  \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                             \
  } while (0)

__global__ void c64_to_c128_kernel(const float2* in, double2* out, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

const char* kTagNames[K_NTAGS] = {"matvec", "gs_first", "gs_reduce", "gs_update", "gs_dot", "gs_normalize",
                                  "ritz", "rotate", "resid", "shrink", "other", "ritz_fallback", "filter", "gs_step", "cg"};

// Optional per-launch CUDA-event timing, harvested at the host synchronisation points.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> tag;
  size_t used = 0;
  double ms[K_NTAGS] = {};
  cudaError_t begin(int t, cudaStream_t s) {
    if (!on) return cudaSuccess;
    if (2 * used + 2 > ev.size()) {
      const size_t add = 512;
      for (size_t i = 0; i < 2 * add; ++i) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
      }
      tag.resize(ev.size() / 2);
    }
    tag[used] = t;
    return cudaEventRecord(ev[2 * used], s);
  }
  cudaError_t end(cudaStream_t s) {
    if (!on) return cudaSuccess;
    cudaError_t r = cudaEventRecord(ev[2 * used + 1], s);
    ++used;
    return r;
  }
  cudaError_t harvest() {  // call after the stream has been synchronised
    for (size_t i = 0; i < used; ++i) {
      float f = 0.f;
      cudaError_t r = cudaEventElapsedTime(&f, ev[2 * i], ev[2 * i + 1]);
      if (r != cudaSuccess) return r;
      ms[tag[i]] += f;
    }
    used = 0;
    return cudaSuccess;
  }
  ~Profiler() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// Operator copy and Krylov basis in one working precision.
struct Phase {
  OpDev op{};
  OpDev opdf{};           // double-float phase, stencil: (hi, lo) links for the Lanczos products
  bool dfmv = false;      // use opdf for the Lanczos products
  void* V = nullptr;      // n x (m + 1); float4 (hi, lo) pairs in a double-float phase
  void* Vtmp = nullptr;   // n x kk (rotation target; FP64 in a double-float phase)
  void* y = nullptr;      // the vector being built
  void* x = nullptr;      // double-float phase: FP64 copy of v_j (the matvec input)
  bool df = false;        // basis stored as compensated FP32 pairs
  size_t cs = 0;          // bytes per complex number of V
  double* alpha_part = nullptr;
  double* resid_part = nullptr;
  int mv_nblk = 0;
  int which = JTRLAN_SMALLEST;  // the wanted end of this phase's operator
  bool filtered = false;        // the Lanczos product is B = p(A)
  bool certify = false;         // filtered phase judged by the true residual of A at x^H A x
  std::vector<double> fcoef;    // filter coefficients g_0..g_d
  void* fbuf[4] = {nullptr, nullptr, nullptr, nullptr};   // A t, two recurrence vectors, (hi, lo) copy
};

}  // namespace

struct jtrlan_ctx {
  jtrlan_operator opd{};
  jtrlan_params prm{};
  cudaStream_t stream = nullptr;
  OpDev op{};
  int64_t n = 0, h = 0;
  int m = 0, nev = 0, mwin = 0, kk = 0, max_restarts = 0, gs_passes = 0;
  bool mixed = false;              // JTRLAN_MIXED: an FP32 phase, then the FP64 phase
  std::vector<void*> owned;        // device allocations
  std::vector<void*> owned_host;   // pinned host allocations
  Phase p64, p32, pdf;             // FP64, FP32 and double-float phases (allocated as the mode needs)
  double* T = nullptr;
  double* lam = nullptr;
  double* Z = nullptr;
  double* ritz_ws = nullptr;
  int* ritz_flags = nullptr;
  double* work_ritz() { return ritz_ws; }
  double* part_dot = nullptr;
  double* part_nrm = nullptr;
  coef4* coef = nullptr;
  StepState* st = nullptr;
  double* d_res = nullptr;
  double* d_candlam = nullptr;
  int* d_cand = nullptr;
  int* d_perm = nullptr;
  int* d_order = nullptr;
  double* d_rep = nullptr;
  double* d_misc = nullptr;
  // pinned staging
  double* h_rep = nullptr;
  double* h_T = nullptr;
  double* h_res = nullptr;
  double* h_candlam = nullptr;
  int* h_cand = nullptr;
  int* h_perm = nullptr;
  int* h_order = nullptr;
  double* h_misc = nullptr;
  int gs_nblk = 0, gs_rpb = 0;
  int coop64 = 0, coop32 = 0, coopdf = 0;   // row blocks (= CTAs) of the cooperative Gram-Schmidt step; 0: not used
  int coop_rpb = 0, coop_rpb_df = 0;        // its rows per block
  bool invert = false;             // Algorithm 1's invert mode: the Lanczos product is A^{-1} v by CG
  void *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr;   // CG residual, direction, A p
  double* cg_part = nullptr;       // cg_blocks(n) partials
  double* cg_pq = nullptr;         // product partials of p^H A p (double2)
  CgState* cg_st = nullptr;
  CgState* h_cgst = nullptr;       // pinned copy
  int64_t cg_matvecs = 0, cg_iters = 0;
  cudaGraphExec_t cg_group = nullptr;   // kCgGroup CG iterations captured once (buffers are the context's)
  const void* cg_group_y = nullptr;     // the solution buffer the graph writes
  TcWork tc{};                     // scratch of the tensor-core rotation (compensated-FP32 basis)
  bool tc_on = false;
  int* h_tcerr = nullptr;          // pinned copy of its error flag
  double fc = 0.0, fe = 1.0;       // filter window centre and half-width
  Profiler prof;
  double work_base[3] = {};        // device work counters carried across solve phases
  int fallback_base = 0;
  int64_t gs_pass_base = 0;
  int64_t nl[K_NTAGS] = {};        // launches per kernel class in the last solve
  double work[K_NTAGS] = {};       // algorithmic work per kernel class in the last solve
  // results of the last solve
  bool solved = false;
  std::vector<double> ev, res;
  jtrlan_stats stats{};

  template <typename T_>
  jtrlan_status dalloc(T_** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return fail(JTRLAN_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    owned.push_back(q);
    *p = (T_*)q;
    return JTRLAN_OK;
  }
  template <typename T_>
  jtrlan_status halloc(T_** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMallocHost(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return fail(JTRLAN_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    owned_host.push_back(q);
    *p = (T_*)q;
    return JTRLAN_OK;
  }
  ~jtrlan_ctx() {
    cudaStreamSynchronize(stream);
    if (cg_group) cudaGraphExecDestroy(cg_group);
    for (void* p : owned) cudaFree(p);
    for (void* p : owned_host) cudaFreeHost(p);
  }
};

namespace {

#define JT_TRY(expr)                       \
  do {                                     \
    jtrlan_status s_ = (expr);             \
    if (s_ != JTRLAN_OK) return s_;        \
  } while (0)

// Copies `count` complex numbers of the caller's dtype (host or device) into an owned FP64 buffer.
jtrlan_status upload_c128(jtrlan_ctx* c, const void* src, int dtype, int64_t count, void** dst) {
  double2* d = nullptr;
  JT_TRY(c->dalloc(&d, (size_t)count * sizeof(double2)));
  if (dtype == JTRLAN_C128) {
    JT_CUDA(cudaMemcpyAsync(d, src, (size_t)count * sizeof(double2), cudaMemcpyDefault, c->stream));
  } else {
    float2* tmp = nullptr;
    JT_CUDA(cudaMallocAsync((void**)&tmp, (size_t)count * sizeof(float2), c->stream));
    JT_CUDA(cudaMemcpyAsync(tmp, src, (size_t)count * sizeof(float2), cudaMemcpyDefault, c->stream));
    c64_to_c128_kernel<<<1024, 256, 0, c->stream>>>(tmp, d, count);
    JT_CUDA(cudaGetLastError());
    JT_CUDA(cudaFreeAsync(tmp, c->stream));
  }
  *dst = d;
  return JTRLAN_OK;
}

jtrlan_status validate(const jtrlan_operator* op, const jtrlan_params* p) {
  if (!op || !p) return fail(JTRLAN_EINVAL, "null operator or params");
  if (op->n <= 0 || (op->n & 1)) return fail(JTRLAN_EINVAL, "n must be positive and even");
  if (op->dtype != JTRLAN_C128 && op->dtype != JTRLAN_C64) return fail(JTRLAN_EINVAL, "unknown dtype");
  if (op->kind == JTRLAN_STENCIL4D) {
    int64_t vol = 1;
    for (int d = 0; d < 4; ++d) {
      if (op->dims[d] < 1) return fail(JTRLAN_EINVAL, "lattice extents must be >= 1");
      vol *= op->dims[d];
    }
    if (op->n != 6 * vol) return fail(JTRLAN_EINVAL, "stencil n must equal 6 * volume");
    if (!op->U || !op->W) return fail(JTRLAN_EINVAL, "null link field");
  } else if (op->kind == JTRLAN_DENSE) {
    if (!op->a11 || !op->a12) return fail(JTRLAN_EINVAL, "null dense block");
  } else {
    return fail(JTRLAN_EINVAL, "unknown operator kind");
  }
  if (p->nev <= 0 || p->m <= p->nev) return fail(JTRLAN_EINVAL, "need 0 < nev < m");
  if ((int64_t)p->m >= op->n / 2) return fail(JTRLAN_EINVAL, "need m < n/2");
  if (p->m > 1023) return fail(JTRLAN_EINVAL, "m > 1023 is not supported by the Ritz kernel");
  if (p->mwin < 0) return fail(JTRLAN_EINVAL, "need mwin >= 0");
  if (!(p->tol > 0.0)) return fail(JTRLAN_EINVAL, "need tol > 0");
  if (p->which != JTRLAN_SMALLEST && p->which != JTRLAN_LARGEST) return fail(JTRLAN_EINVAL, "unknown which");
  if (p->precision != JTRLAN_FP64 && p->precision != JTRLAN_MIXED && p->precision != JTRLAN_MIXED_REORTH)
    return fail(JTRLAN_EINVAL, "unknown precision");
  if (p->gs_max_passes < 0 || p->gs_max_passes > 7) return fail(JTRLAN_EINVAL, "gs_max_passes must be 0..7");
  if (p->max_restarts < 0) return fail(JTRLAN_EINVAL, "max_restarts must be >= 0");
  if (p->filter_degree < 0 || p->filter_degree > 1024) return fail(JTRLAN_EINVAL, "filter_degree must be 0..1024");
  if (p->filter_final_degree < 0 || p->filter_final_degree > 1024)
    return fail(JTRLAN_EINVAL, "filter_final_degree must be 0..1024");
  if (p->filter_degree > 0) {
    if (p->precision != JTRLAN_MIXED) return fail(JTRLAN_EINVAL, "filter_degree applies to the FP32 phase of JTRLAN_MIXED");
    if (!p->filter_coeffs) return fail(JTRLAN_EINVAL, "null filter_coeffs");
  }
  if (p->filter_final_degree > 0 && !p->filter_final_coeffs) return fail(JTRLAN_EINVAL, "null filter_final_coeffs");
  if ((p->filter_degree > 0 || p->filter_final_degree > 0) && !(p->filter_lo < p->filter_hi))
    return fail(JTRLAN_EINVAL, "need filter_lo < filter_hi");
  if (p->invert) {
    if (p->precision != JTRLAN_FP64) return fail(JTRLAN_EINVAL, "invert mode runs in JTRLAN_FP64");
    if (p->which != JTRLAN_SMALLEST) return fail(JTRLAN_EINVAL, "invert mode finds the smallest eigenvalues");
    if (p->filter_degree > 0 || p->filter_final_degree > 0) return fail(JTRLAN_EINVAL, "invert mode takes no filter");
  }
  if (p->cg_tol < 0.0 || p->cg_max_iter < 0) return fail(JTRLAN_EINVAL, "need cg_tol >= 0 and cg_max_iter >= 0");
  return JTRLAN_OK;
}

// Turns the final phase (FP64, or double-float in the mixed forms) into the certifying filtered phase
// on B = p(A) with coefficients g_0..g_degree: buffers on the first call, coefficients every call.
jtrlan_status setup_certify(jtrlan_ctx* c, const double* coeffs, int degree) {
  Phase& ph = c->mixed ? c->pdf : c->p64;
  if (!ph.certify) {
    ph.filtered = true;
    ph.certify = true;
    ph.which = JTRLAN_LARGEST;
    for (int b = 0; b < 3; ++b) JT_TRY(c->dalloc(&ph.fbuf[b], (size_t)c->n * sizeof(double2)));
    JT_TRY(c->dalloc(&ph.fbuf[3], (size_t)c->n * sizeof(float4)));
    const int nb = std::max(cheb_blocks(c->n), ph.dfmv ? matvec_df_blocks(ph.opdf) : ph.mv_nblk);
    JT_TRY(c->dalloc(&ph.alpha_part, (size_t)nb * sizeof(double2)));
    JT_TRY(c->dalloc(&ph.resid_part, (size_t)std::max(nb, ph.mv_nblk * c->nev) * sizeof(double)));
  }
  ph.fcoef.assign(coeffs, coeffs + degree + 1);
  return JTRLAN_OK;
}

jtrlan_status create_impl(const jtrlan_operator* op, const jtrlan_params* prm, void* stream, jtrlan_ctx** out) {
  JT_TRY(validate(op, prm));
  jtrlan_ctx* c = new (std::nothrow) jtrlan_ctx();
  if (!c) return fail(JTRLAN_ENOMEM, "host allocation failed");
  *out = c;  // released by the caller on failure
  c->opd = *op;
  c->prm = *prm;
  c->stream = (cudaStream_t)stream;
  c->n = op->n;
  c->h = op->n / 2;
  c->m = prm->m;
  c->nev = prm->nev;
  c->mwin = prm->mwin;
  c->kk = std::min(prm->nev + prm->mwin, prm->m - 1);
  c->max_restarts = prm->max_restarts ? prm->max_restarts : 1000;
  c->gs_passes = prm->gs_max_passes ? prm->gs_max_passes : 3;
  c->mixed = prm->precision != JTRLAN_FP64;   // both mixed forms keep the FP32 operator
  OpDev& o = c->p64.op;
  o.kind = op->kind;
  o.n = c->n;
  o.h = c->h;
  o.m0 = op->m0;
  o.kappa = op->kappa;
  o.vol = 1;
  o.fp32 = 0;
  for (int d = 0; d < 4; ++d) { o.dims[d] = op->dims[d]; if (op->kind == JTRLAN_STENCIL4D) o.vol *= op->dims[d]; }
  if (op->kind == JTRLAN_STENCIL4D) {
    void *u = nullptr, *w = nullptr;
    JT_TRY(upload_c128(c, op->U, op->dtype, 4 * o.vol * 9, &u));
    JT_TRY(upload_c128(c, op->W, op->dtype, 4 * o.vol * 9, &w));
    o.U = u; o.W = w;
  } else {
    void *a = nullptr, *b = nullptr;
    JT_TRY(upload_c128(c, op->a11, op->dtype, c->h * c->h, &a));
    JT_TRY(upload_c128(c, op->a12, op->dtype, c->h * c->h, &b));
    o.a11 = a; o.a12 = b;
  }
  const int m = c->m;
  const int mp = m + (m & 1);
  c->gs_nblk = gs_blocks(c->h, &c->gs_rpb);
  auto make_phase = [&](Phase& ph, size_t cs) -> jtrlan_status {
    ph.cs = cs;
    ph.mv_nblk = matvec_blocks(ph.op);
    JT_TRY(c->dalloc(&ph.V, (size_t)c->n * (m + 1) * cs));
    JT_TRY(c->dalloc(&ph.Vtmp, (size_t)c->n * std::max(c->kk, 1) * cs));
    JT_TRY(c->dalloc(&ph.y, (size_t)c->n * cs));
    JT_TRY(c->dalloc(&ph.alpha_part, (size_t)ph.mv_nblk * sizeof(double2)));
    JT_TRY(c->dalloc(&ph.resid_part, (size_t)ph.mv_nblk * c->nev * sizeof(double)));
    return JTRLAN_OK;
  };
  if (!c->mixed) {
    JT_TRY(make_phase(c->p64, sizeof(double2)));
  } else {  // double-float phase on the FP64 operator
    c->pdf.op = o;
    c->pdf.df = true;
    JT_TRY(make_phase(c->pdf, sizeof(float4)));
    JT_TRY(c->dalloc(&c->pdf.x, (size_t)c->n * sizeof(double2)));
    if (op->kind == JTRLAN_STENCIL4D) {   // (hi, lo) links for the compensated-FP32 matvec
      OpDev& d = c->pdf.opdf;
      d = o;
      if (op->dtype == JTRLAN_C64) {
        // the caller's links are complex64, so they are exact in FP32: the compensated kernels read
        // the FP32 phase's structure-of-arrays copy (set below) as (hi, 0) pairs
        d.links32 = 1;
      } else {
        float4 *u = nullptr, *w = nullptr;
        JT_TRY(c->dalloc(&u, (size_t)36 * o.vol * sizeof(float4)));
        JT_TRY(c->dalloc(&w, (size_t)36 * o.vol * sizeof(float4)));
        JT_CUDA(launch_links_df(o.U, u, o.vol, c->stream));
        JT_CUDA(launch_links_df(o.W, w, o.vol, c->stream));
        d.U = u; d.W = w;
      }
      c->pdf.dfmv = true;
      const int nb = matvec_df_blocks(d);
      if (nb > c->pdf.mv_nblk) JT_TRY(c->dalloc(&c->pdf.alpha_part, (size_t)nb * sizeof(double2)));
    }
  }
  if (c->mixed && !prm->rotate_simt && m <= tc_rotate_max_m()) {   // restart rotation on the tensor cores
    void* base = nullptr;
    JT_TRY(c->dalloc(&base, tc_rotate_bytes(c->n, m, std::max(c->kk, 1))));
    c->tc = tc_rotate_carve(base, c->n, m, std::max(c->kk, 1));
    JT_CUDA(cudaMemsetAsync(c->tc.err, 0, sizeof(int), c->stream));
    JT_TRY(c->halloc(&c->h_tcerr, sizeof(int)));
    *c->h_tcerr = 0;
    c->tc_on = true;
  }
  if (c->mixed) {  // the FP32 operator: links re-laid out structure-of-arrays, or FP32 dense blocks
    OpDev& q = c->p32.op;
    q = o;
    q.fp32 = 1;
    if (op->kind == JTRLAN_STENCIL4D) {
      float2 *u = nullptr, *w = nullptr;
      JT_TRY(c->dalloc(&u, (size_t)36 * o.vol * sizeof(float2)));
      JT_TRY(c->dalloc(&w, (size_t)36 * o.vol * sizeof(float2)));
      JT_CUDA(launch_links_soa(o.U, u, o.vol, c->stream));
      JT_CUDA(launch_links_soa(o.W, w, o.vol, c->stream));
      q.U = u; q.W = w;
      if (c->pdf.opdf.links32) {
        c->pdf.opdf.U = u;
        c->pdf.opdf.W = w;
      }
    } else {
      float2 *a = nullptr, *b = nullptr;
      JT_TRY(c->dalloc(&a, (size_t)c->h * c->h * sizeof(float2)));
      JT_TRY(c->dalloc(&b, (size_t)c->h * c->h * sizeof(float2)));
      JT_CUDA(launch_c128_to_c64(o.a11, a, c->h * c->h, c->stream));
      JT_CUDA(launch_c128_to_c64(o.a12, b, c->h * c->h, c->stream));
      q.a11 = a; q.a12 = b;
    }
    if (prm->precision == JTRLAN_MIXED) {
      JT_TRY(make_phase(c->p32, sizeof(float2)));
      if (prm->filter_degree > 0) {   // B = p(A) in the FP32 phase: largest p wanted
        c->p32.filtered = true;
        c->p32.which = JTRLAN_LARGEST;
        c->p32.fcoef.assign(prm->filter_coeffs, prm->filter_coeffs + prm->filter_degree + 1);
        for (int b = 0; b < 3; ++b) JT_TRY(c->dalloc(&c->p32.fbuf[b], (size_t)c->n * sizeof(float2)));
        if (cheb_blocks(c->n) > c->p32.mv_nblk)
          JT_TRY(c->dalloc(&c->p32.alpha_part, (size_t)cheb_blocks(c->n) * sizeof(double2)));
      }
    } else {
      c->p32.mv_nblk = matvec_blocks(q);
    }
  }
  c->p64.which = c->pdf.which = prm->which;
  if (!c->p32.filtered) c->p32.which = prm->which;
  if (prm->invert) {   // Lanczos on A^{-1}: its largest eigenvalues are A's smallest
    c->invert = true;
    c->p64.which = JTRLAN_LARGEST;
    JT_TRY(c->dalloc(&c->cg_r, (size_t)c->n * sizeof(double2)));
    JT_TRY(c->dalloc(&c->cg_p, (size_t)c->n * sizeof(double2)));
    JT_TRY(c->dalloc(&c->cg_q, (size_t)c->n * sizeof(double2)));
    JT_TRY(c->dalloc(&c->cg_part, (size_t)cg_blocks(c->n) * sizeof(double)));
    JT_TRY(c->dalloc(&c->cg_pq, (size_t)c->p64.mv_nblk * sizeof(double2)));
    JT_TRY(c->dalloc(&c->cg_st, sizeof(CgState)));
    JT_TRY(c->halloc(&c->h_cgst, sizeof(CgState)));
    JT_CUDA(cudaMemsetAsync(c->cg_st, 0, sizeof(CgState), c->stream));
    if (cg_blocks(c->n) > c->p64.mv_nblk)
      JT_TRY(c->dalloc(&c->p64.alpha_part, (size_t)cg_blocks(c->n) * sizeof(double2)));
    if (cg_blocks(c->n) > c->p64.mv_nblk * c->nev)
      JT_TRY(c->dalloc(&c->p64.resid_part, (size_t)cg_blocks(c->n) * sizeof(double)));
  }
  c->fc = 0.5 * (prm->filter_lo + prm->filter_hi);
  c->fe = 0.5 * (prm->filter_hi - prm->filter_lo);
  if (prm->filter_final_degree > 0)   // the certifying phase on B = p(A), judged by A's residuals
    JT_TRY(setup_certify(c, prm->filter_final_coeffs, prm->filter_final_degree));
  {  // cooperative Gram-Schmidt step: its own row partition, one row block per resident CTA
    int dev = 0, nsm = 0;
    JT_CUDA(cudaGetDevice(&dev));
    JT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (c->h + 31) / 32;
    // rows per block and row blocks for per CTAs per SM, at least min_tpb tiles of 32 row pairs a block
    auto part = [&](int per, int* rpb, int* nb, int64_t min_tpb) {
      const int64_t G = (int64_t)per * nsm;
      int64_t tpb = (tiles + G - 1) / G;
      if (tpb < min_tpb) tpb = min_tpb;
      *rpb = (int)(32 * (tpb < 1 ? 1 : tpb));
      *nb = (int)((c->h + *rpb - 1) / *rpb);
    };
    int per = 0;
    if (!c->mixed) {
      JT_CUDA(gs_coop_occupancy<double>(m, &per));
      if (per > 0) part(per, &c->coop_rpb, &c->coop64, 1);
    }
    if (prm->precision == JTRLAN_MIXED) {
      JT_CUDA(gs_coop_occupancy<float>(m, &per));
      if (per > 0) part(per, &c->coop_rpb, &c->coop32, 1);
    }
    if (c->mixed) {   // the shared memory grows with rows_per_block: size it, then check it still fits
      GSArgs g{};
      g.m = m;
      g.rows_per_block = (int)(32 * ((tiles + 2 * nsm - 1) / (2 * nsm)));
      // too many rows for one CTA's shared memory (large lattices): keep the multi-kernel path
      if (gsdf_coop_occupancy(g, &per) != cudaSuccess) {
        cudaGetLastError();
        per = 0;
      }
      if (per > 0) {
        // at least 4 tiles a block: on small lattices fewer, fuller blocks pay less for the grid-wide
        // reductions (8^4: 77.6 -> 71.1 ms per solve; FP64 measured best at one tile a block)
        part(per, &c->coop_rpb_df, &c->coopdf, 4);
        g.rows_per_block = c->coop_rpb_df;
        if (gsdf_coop_occupancy(g, &per) != cudaSuccess) {
          cudaGetLastError();
          per = 0;
        }
        if ((int64_t)per * nsm < c->coopdf) c->coopdf = 0;
      }
    }
  }
  if (prm->gs_split) c->coop64 = c->coop32 = c->coopdf = 0;   // the separate-launch Gram-Schmidt path
  const int nblk_max = std::max(c->gs_nblk, std::max(std::max(c->coop64, c->coop32), c->coopdf));
  JT_TRY(c->dalloc(&c->T, (size_t)(m + 1) * (m + 1) * sizeof(double)));
  JT_TRY(c->dalloc(&c->lam, (size_t)m * sizeof(double)));
  JT_TRY(c->dalloc(&c->Z, (size_t)m * m * sizeof(double)));
  JT_TRY(c->dalloc(&c->ritz_ws, (size_t)2 * mp * mp * sizeof(double)));
  JT_TRY(c->dalloc(&c->ritz_flags, (size_t)(m + 1) * sizeof(int)));
  JT_TRY(c->dalloc(&c->part_dot, (size_t)(m + 1) * nblk_max * sizeof(coef4)));
  JT_TRY(c->dalloc(&c->part_nrm, (size_t)2 * nblk_max * sizeof(double)));   // two slots (cooperative step)
  JT_TRY(c->dalloc(&c->coef, (size_t)(m + 1) * sizeof(coef4)));
  JT_TRY(c->dalloc(&c->st, sizeof(StepState)));
  JT_TRY(c->dalloc(&c->d_res, (size_t)c->nev * sizeof(double)));
  JT_TRY(c->dalloc(&c->d_candlam, (size_t)c->nev * sizeof(double)));
  JT_TRY(c->dalloc(&c->d_cand, (size_t)c->nev * sizeof(int)));
  JT_TRY(c->dalloc(&c->d_perm, (size_t)m * sizeof(int)));
  JT_TRY(c->dalloc(&c->d_order, (size_t)c->nev * sizeof(int)));
  JT_TRY(c->dalloc(&c->d_rep, (size_t)(2 * m + 8) * sizeof(double)));  // lam, z_m, 8 scalars
  JT_TRY(c->dalloc(&c->d_misc, 16 * sizeof(double)));
  JT_TRY(c->halloc(&c->h_rep, (size_t)(2 * m + 8) * sizeof(double)));
  JT_TRY(c->halloc(&c->h_T, (size_t)(m + 1) * (m + 1) * sizeof(double)));
  JT_TRY(c->halloc(&c->h_res, (size_t)c->nev * sizeof(double)));
  JT_TRY(c->halloc(&c->h_candlam, (size_t)c->nev * sizeof(double)));
  JT_TRY(c->halloc(&c->h_cand, (size_t)c->nev * sizeof(int)));
  JT_TRY(c->halloc(&c->h_perm, (size_t)m * sizeof(int)));
  JT_TRY(c->halloc(&c->h_order, (size_t)c->nev * sizeof(int)));
  JT_TRY(c->halloc(&c->h_misc, 16 * sizeof(double)));
  if (prm->check_jsym) {  // Lemma 1: (J v^*)^H A v = 0 for any v
    Phase& ph = c->mixed ? c->pdf : c->p64;   // both have FP64 Vtmp and y
    JT_CUDA(launch_fill_random<double>(ph.Vtmp, c->n, 0x5eed1234ull, c->stream));
    JT_CUDA(launch_matvec<double>(o, (const double2*)ph.Vtmp, (double2*)ph.y, MV_PLAIN, nullptr, nullptr,
                                  nullptr, 0, 0, nullptr, c->stream));
    JT_CUDA(launch_jsym_check<double>(ph.Vtmp, ph.y, c->h, c->d_misc, c->stream));
    JT_CUDA(cudaMemcpyAsync(c->h_misc, c->d_misc, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    JT_CUDA(cudaStreamSynchronize(c->stream));
    const double wAv = std::hypot(c->h_misc[0], c->h_misc[1]);
    const double scale = std::sqrt(c->h_misc[2] * c->h_misc[3]);
    if (!(wAv <= 1e-10 * scale)) {
      char buf[160];
      std::snprintf(buf, sizeof buf, "Lemma 1 check failed: |(Jv*)^H A v| = %.3e vs ||Av|| ||v|| = %.3e", wAv, scale);
      return fail(JTRLAN_ENOTJSYM, buf);
    }
  }
  JT_CUDA(cudaStreamSynchronize(c->stream));
  return JTRLAN_OK;
}

inline void* col(void* base, int64_t n, int j, size_t cs) { return (char*)base + (size_t)j * n * cs; }

#define LAUNCH(tag, expr)                  \
  do {                                     \
    JT_CUDA(c->prof.begin((tag), s));      \
    JT_CUDA(expr);                         \
    JT_CUDA(c->prof.end(s));               \
    c->nl[(tag)] += 1;                     \
  } while (0)

// y = p(A) v by the Chebyshev recurrence (filter.cu): d products of A and d recurrence steps; the
// last step leaves the alpha partials of conj(v) y in part (cheb_blocks(n) of them) if given.
template <typename R>
jtrlan_status filter_apply(jtrlan_ctx* c, Phase& ph, const void* v, void* y, double* part) {
  using C = cplx<R>;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const int d = (int)ph.fcoef.size() - 1;
  const double* g = ph.fcoef.data();
  void* ax = ph.fbuf[0];
  void* B[2] = {ph.fbuf[1], ph.fbuf[2]};
  LAUNCH(K_MATVEC, launch_matvec<R>(ph.op, (const C*)v, (C*)ax, MV_PLAIN, nullptr, nullptr, nullptr, 0, 0, nullptr, s));
  LAUNCH(K_FILTER, launch_cheb_step<R>(ax, v, nullptr, B[1], y, v, n, c->fc, 1.0 / c->fe, 0.0, g[1], g[0], 1,
                                       d == 1 ? part : nullptr, nullptr, s));
  for (int k = 2; k <= d; ++k) {
    const void* tcur = B[(k - 1) & 1];                 // T_{k-1}
    const void* tprev = k == 2 ? v : B[k & 1];         // T_{k-2}
    void* tnext = B[k & 1];                            // T_k (over T_{k-2} from k = 3 on)
    LAUNCH(K_MATVEC, launch_matvec<R>(ph.op, (const C*)tcur, (C*)ax, MV_PLAIN, nullptr, nullptr, nullptr, 0, 0,
                                      nullptr, s));
    LAUNCH(K_FILTER, launch_cheb_step<R>(ax, tcur, tprev, tnext, y, v, n, c->fc, 2.0 / c->fe, 1.0, g[k], 0.0, 0,
                                         k == d ? part : nullptr, nullptr, s));
  }
  return JTRLAN_OK;
}

// The certifying phase's product y = p(A) v in FP64 vectors, v given in FP64 (v64) and, for the
// stencil double-float phase, as (hi, lo) pairs (vdf): there each recurrence step is fused into the
// compensated-FP32 product (float-float recurrence, (hi, lo) vectors between steps); otherwise FP64
// products and FP64 recurrence steps.  Alpha partials of conj(v) y in ph.alpha_part (cheb_blocks(n)).
jtrlan_status filter_apply_cert_io(jtrlan_ctx* c, Phase& ph, const void* v64, const void* vdf, void* y) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const int d = (int)ph.fcoef.size() - 1;
  const double* g = ph.fcoef.data();
  if (ph.dfmv) {
    void* acc = ph.fbuf[0];
    void* B[2] = {ph.fbuf[1], ph.fbuf[2]};
    const OpDev& o = ph.opdf;
    LAUNCH(K_MATVEC, launch_matvec_df_cheb(o, vdf, nullptr, B[1], acc, vdf, y, ph.alpha_part, o.kappa, o.m0, c->fc,
                                           1.0 / c->fe, g[1], g[0], 1, d == 1, s));
    for (int k = 2; k <= d; ++k)
      LAUNCH(K_MATVEC, launch_matvec_df_cheb(o, B[(k - 1) & 1], k == 2 ? vdf : B[k & 1], B[k & 1], acc, vdf, y,
                                             ph.alpha_part, o.kappa, o.m0, c->fc, 2.0 / c->fe, g[k], 0.0, 0, k == d,
                                             s));
    return JTRLAN_OK;
  }
  void* ax = ph.fbuf[0];
  void* B[2] = {ph.fbuf[1], ph.fbuf[2]};
  const void* v = v64;
  auto product = [&](const void* t64) -> jtrlan_status {
    LAUNCH(K_MATVEC, launch_matvec<double>(ph.op, (const double2*)t64, (double2*)ax, MV_PLAIN, nullptr, nullptr,
                                           nullptr, 0, 0, nullptr, s));
    return JTRLAN_OK;
  };
  JT_TRY(product(v));
  LAUNCH(K_FILTER, launch_cheb_step<double>(ax, v, nullptr, B[1], y, v, n, c->fc, 1.0 / c->fe, 0.0, g[1], g[0], 1,
                                            d == 1 ? ph.alpha_part : nullptr, nullptr, s));
  for (int k = 2; k <= d; ++k) {
    const void* tcur = B[(k - 1) & 1];
    const void* tprev = k == 2 ? v : B[k & 1];
    void* tnext = B[k & 1];
    JT_TRY(product(tcur));
    LAUNCH(K_FILTER, launch_cheb_step<double>(ax, tcur, tprev, tnext, y, v, n, c->fc, 2.0 / c->fe, 1.0, g[k], 0.0,
                                              0, k == d ? ph.alpha_part : nullptr, nullptr, s));
  }
  return JTRLAN_OK;
}

jtrlan_status filter_apply_cert(jtrlan_ctx* c, Phase& ph, int j) {
  const void* vj = col(ph.V, c->n, j, ph.cs);
  return filter_apply_cert_io(c, ph, ph.df ? ph.x : vj, vj, ph.y);   // v_j in FP64: ph.x beside a (hi, lo) basis
}

// Rayleigh quotient lam_out = x^H A x and residual res_out = ||A x - lam x|| of one FP64 column
// (device scalars), for the certifying filtered phase.
jtrlan_status rq_resid(jtrlan_ctx* c, Phase& ph, const void* x, double* lam_out, double* res_out) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  int nparts;
  if (ph.dfmv) {
    LAUNCH(K_RESID, launch_df_from_fp64(x, ph.fbuf[3], n, s));
    LAUNCH(K_RESID, launch_matvec_df(ph.opdf, ph.fbuf[3], ph.fbuf[0], ph.alpha_part, s));
    nparts = matvec_df_blocks(ph.opdf);
  } else {
    LAUNCH(K_RESID, launch_matvec<double>(ph.op, (const double2*)x, (double2*)ph.fbuf[0], MV_ALPHA, ph.alpha_part,
                                          nullptr, nullptr, 0, 0, nullptr, s));
    nparts = ph.mv_nblk;
  }
  LAUNCH(K_RESID, launch_sum_re(ph.alpha_part, nparts, lam_out, s));
  LAUNCH(K_RESID, launch_resid_part(ph.fbuf[0], x, lam_out, n, ph.resid_part, s));
  LAUNCH(K_RESID, launch_reduce_norms(ph.resid_part, cheb_blocks(n), 1, res_out, s));
  return JTRLAN_OK;
}

// y = A^{-1} b by conjugate gradients (cg.cu) on the FP64 operator, for the invert mode: iterations
// are enqueued in groups of kCgGroup, and the host reads the device state after each group.
constexpr int kCgGroup = 4;
jtrlan_status cg_solve(jtrlan_ctx* c, Phase& ph, const void* b, void* y) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const double rtol = c->prm.cg_tol > 0.0 ? c->prm.cg_tol : 1e-12;
  const int max_iter = c->prm.cg_max_iter > 0 ? c->prm.cg_max_iter : 10000;
  LAUNCH(K_CG, launch_cg_init(b, y, c->cg_r, c->cg_p, n, c->cg_part, rtol, c->cg_st, s));
  c->nl[K_CG] += 1;   // two kernels
  auto group = [&](cudaStream_t st) -> cudaError_t {
    for (int u = 0; u < kCgGroup; ++u) {
      cudaError_t e = launch_matvec<double>(ph.op, (const double2*)c->cg_p, (double2*)c->cg_q, MV_ALPHA, c->cg_pq,
                                            nullptr, nullptr, 0, 0, nullptr, st);
      if (e == cudaSuccess) e = launch_cg_alpha(c->cg_pq, ph.mv_nblk, c->cg_st, st);
      if (e == cudaSuccess) e = launch_cg_update(y, c->cg_r, c->cg_p, c->cg_q, n, c->cg_part, c->cg_st, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (!c->prof.on && (!c->cg_group || c->cg_group_y != y)) {
    // capture the group once, on a private stream (the caller's may be the legacy default stream,
    // which cannot be captured); the graph then replays on the context stream
    if (c->cg_group) {
      cudaGraphExecDestroy(c->cg_group);
      c->cg_group = nullptr;
    }
    cudaStream_t cap = nullptr;
    JT_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = group(cap);
      e = cudaStreamEndCapture(cap, &gr);
      if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->cg_group, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      c->cg_group = nullptr;
      return fail(JTRLAN_ECUDA, std::string("CG graph: ") + cudaGetErrorString(e));
    }
    c->cg_group_y = y;
  }
  for (int launched = 0;;) {
    if (c->prof.on) {   // the per-kernel profile needs every launch bracketed by events
      for (int u = 0; u < kCgGroup; ++u) {
        LAUNCH(K_CG, launch_matvec<double>(ph.op, (const double2*)c->cg_p, (double2*)c->cg_q, MV_ALPHA, c->cg_pq,
                                           nullptr, nullptr, 0, 0, nullptr, s));
        LAUNCH(K_CG, launch_cg_alpha(c->cg_pq, ph.mv_nblk, c->cg_st, s));
        LAUNCH(K_CG, launch_cg_update(y, c->cg_r, c->cg_p, c->cg_q, n, c->cg_part, c->cg_st, s));
        c->nl[K_CG] += 2;   // three kernels
      }
    } else {
      JT_CUDA(cudaGraphLaunch(c->cg_group, s));
      c->nl[K_CG] += 5 * kCgGroup;
    }
    launched += kCgGroup;
    c->cg_matvecs += kCgGroup;
    c->work[K_CG] += (double)kCgGroup * (c->opd.kind == JTRLAN_STENCIL4D ? (double)ph.op.vol : (double)c->h * c->h);
    JT_CUDA(cudaMemcpyAsync(c->h_cgst, c->cg_st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    JT_CUDA(cudaStreamSynchronize(s));
    if (c->h_cgst->fail)
      return fail(JTRLAN_EBREAKDOWN, "invert mode: a CG step found p^H A p <= 0 (A is not positive definite)");
    if (c->h_cgst->done) {
      c->cg_iters += c->h_cgst->iters;
      return JTRLAN_OK;
    }
    if (launched >= max_iter)
      return fail(JTRLAN_ENOCONV, "invert mode: CG did not reach cg_tol in cg_max_iter iterations");
  }
}

// Algorithm 2 steps j0 .. j1-1 of the phase (products, alpha, Gram-Schmidt against V and W with the
// sqrt(2) test, normalisation), enqueued without host synchronisation.  With `filtered` the product
// is B = p(A).
template <typename R>
jtrlan_status lanczos_steps(jtrlan_ctx* c, Phase& ph, GSArgs& a, int j0, int j1, bool filtered) {
  using C = cplx<R>;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const size_t cs = ph.cs;
  if (ph.df) LAUNCH(K_OTHER, launch_fp64_from_df(col(ph.V, n, j0, cs), ph.x, n, s));   // v_j0 in FP64
  const int mv_parts = c->invert ? cg_blocks(n)
                       : (filtered && !(ph.certify && ph.dfmv)) ? cheb_blocks(n)
                       : ph.dfmv ? matvec_df_blocks(ph.opdf) : ph.mv_nblk;
  for (int j = j0; j < j1; ++j) {
    if (filtered) {
      if constexpr (std::is_same<R, float>::value)
        JT_TRY(filter_apply<R>(c, ph, col(ph.V, n, j, cs), ph.y, ph.alpha_part));
      else
        JT_TRY(filter_apply_cert(c, ph, j));
    } else if (ph.dfmv) {   // compensated FP32 on the (hi, lo) column and links, FP64 result
      LAUNCH(K_MATVEC, launch_matvec_df(ph.opdf, col(ph.V, n, j, cs), ph.y, ph.alpha_part, s));
    } else if (c->invert) {   // invert mode: y = A^{-1} v_j by CG, then the partials of v_j^H y
      JT_TRY(cg_solve(c, ph, col(ph.V, n, j, cs), ph.y));
      LAUNCH(K_CG, launch_vhy_part(col(ph.V, n, j, cs), ph.y, n, ph.alpha_part, s));
    } else {
      const void* vj = ph.df ? ph.x : col(ph.V, n, j, cs);
      LAUNCH(K_MATVEC, launch_matvec<R>(ph.op, (const C*)vj, (C*)ph.y, MV_ALPHA, ph.alpha_part,
                                        nullptr, nullptr, 0, 0, nullptr, s));
    }
    a.j = j;
    if (ph.df) {
      // compensated FP32 reorthogonalisation of an FP64 vector against a (hi, lo) basis; see gsdf.cu
      if (c->coopdf > 0) {   // the whole step in one cooperative launch, on its own row partition
        GSArgs ac = a;
        ac.nblk = c->coopdf;
        ac.rows_per_block = c->coop_rpb_df;
        LAUNCH(K_GS_STEP, launch_gsdf_step_coop(ac, ph.x, (const double2*)ph.alpha_part, mv_parts, c->gs_passes,
                                                 c->part_nrm, c->coopdf, s));
        continue;
      }
      LAUNCH(K_GS_FIRST, launch_gsdf_first(a, ph.x, (const double2*)ph.alpha_part, mv_parts, s));
      LAUNCH(K_GS_REDUCE, launch_gs_reduce(a, 1, s));
      LAUNCH(K_GS_UPDATE, launch_gsdf_update(a, 1, s));
      for (int pass = 2; pass <= c->gs_passes; ++pass) {
        LAUNCH(K_GS_DOT, launch_gsdf_dot(a, pass, s));
        LAUNCH(K_GS_REDUCE, launch_gs_reduce(a, 0, s));
        LAUNCH(K_GS_UPDATE, launch_gsdf_update(a, pass, s));
      }
      LAUNCH(K_GS_NORMALIZE, launch_gsdf_normalize(a, ph.x, s));
    } else {
      const int coop = std::is_same<R, float>::value ? c->coop32 : c->coop64;
      if (coop > 0) {   // the whole step in one cooperative launch, on its own row partition
        GSArgs ac = a;
        ac.nblk = coop;
        ac.rows_per_block = c->coop_rpb;
        LAUNCH(K_GS_STEP, launch_gs_step_coop<R>(ac, (const double2*)ph.alpha_part, mv_parts, c->gs_passes,
                                                  c->part_nrm, coop, s));
        continue;
      }
      LAUNCH(K_GS_FIRST, launch_gs_first<R>(a, (const double2*)ph.alpha_part, mv_parts, s));
      LAUNCH(K_GS_REDUCE, launch_gs_reduce(a, 1, s));
      LAUNCH(K_GS_UPDATE, launch_gs_update<R>(a, s));
      for (int pass = 2; pass <= c->gs_passes; ++pass) {
        LAUNCH(K_GS_DOT, launch_gs_dot<R>(a, pass, s));
        LAUNCH(K_GS_REDUCE, launch_gs_reduce(a, 0, s));
        LAUNCH(K_GS_UPDATE, launch_gs_update<R>(a, s));
      }
      LAUNCH(K_GS_NORMALIZE, launch_gs_normalize<R>(a, s));
    }
  }
  return JTRLAN_OK;
}

// Algorithm 1 (TRLAN-JSYM) in working precision R from the start vector in ph.V[:, 0] (already
// normalised), until nev pairs have true residual < tol (tol_rel_tmax > 0: the phase tolerance is
// max(tol, tol_rel_tmax * max|t|), for the FP32 phase).  On success the converged Ritz vectors
// are ph.V[:, 0..nev) with eigenvalues ev and residuals res (converged-first order).
template <typename R>
jtrlan_status run_phase(jtrlan_ctx* c, Phase& ph, double tol, double tol_rel_tmax, int max_restarts,
                        jtrlan_stats& stt, std::vector<double>& ev, std::vector<double>& res, int* icnv_out) {
  using C = cplx<R>;
  const int m = c->m, nev = c->nev, ldt = m + 1, kk = c->kk;
  const int64_t n = c->n;
  const size_t cs = ph.cs;
  cudaStream_t s = c->stream;
  JT_CUDA(cudaMemsetAsync(c->st, 0, sizeof(StepState), s));
  JT_CUDA(cudaMemsetAsync(c->T, 0, (size_t)ldt * ldt * sizeof(double), s));
  GSArgs a{};
  a.V = ph.V; a.n = n; a.h = c->h; a.y = ph.y; a.part_dot = c->part_dot; a.part_nrm = c->part_nrm;
  a.coef = c->coef; a.st = c->st; a.T = c->T; a.ldt = ldt; a.m = m; a.nblk = c->gs_nblk;
  a.rows_per_block = c->gs_rpb;
  a.no_w = c->prm.plain_trlan ? 1 : 0;
  const double mv_units = ph.op.kind == JTRLAN_STENCIL4D ? (double)ph.op.vol : (double)c->h * (double)c->h;
  ev.assign(nev, 0.0);
  res.assign(nev, INFINITY);
  std::vector<double> res_est(nev), lamv(m), arrow(m);
  std::vector<double> rq(nev, 0.0);            // certifying filtered phase: x^H A x of each candidate
  std::vector<char> conv(nev);
  std::vector<int> perm(m);
  std::vector<double> locked_ev, locked_res, locked_rq;   // pairs locked at the previous restart
  int k = 0, icnv = 0;
  *icnv_out = 0;
  for (int restart = 0; restart < max_restarts; ++restart) {
    // ---- Algorithm 2: m - k Lanczos steps, no host synchronisation inside
    JT_TRY(lanczos_steps<R>(c, ph, a, k, m, ph.filtered));
    const int per_step = ph.filtered ? (int)ph.fcoef.size() - 1 : 1;   // products of A per Lanczos step
    stt.n_matvec += (int64_t)(m - k) * per_step;                         // invert mode: A^{-1} v_j
    if (!c->invert) c->work[K_MATVEC] += (double)(m - k) * per_step * mv_units;
    if (c->invert) {   // c = ||A v_{m+1}|| of the invert-mode residual estimates (Algorithm 1)
      const void* vm1 = col(ph.V, n, m, cs);
      LAUNCH(K_CG, launch_matvec<double>(ph.op, (const double2*)vm1, (double2*)c->cg_q, MV_PLAIN, nullptr, nullptr,
                                         nullptr, 0, 0, nullptr, s));
      LAUNCH(K_CG, launch_resid_part(c->cg_q, vm1, &c->cg_st->zero, n, ph.resid_part, s));
      LAUNCH(K_CG, launch_reduce_norms(ph.resid_part, cheb_blocks(n), 1, &c->cg_st->cnorm, s));
      c->cg_matvecs += 1;
      c->work[K_CG] += mv_units;
    }
    stt.n_restarts += 1;
    // ---- Rayleigh-Ritz (FP64): T_m = Z Lambda Z^T, the kk wanted pairs; V_m Z into Vtmp
    LAUNCH(K_RITZ, launch_ritz(c->T, ldt, m, k, kk, ph.which, c->lam, c->Z, c->ritz_flags, s));
    c->nl[K_RITZ] += 1;  // two kernels: bisection + inverse iteration, checks
    LAUNCH(K_RITZ_FALLBACK, launch_ritz_fallback(c->T, ldt, m, ph.which, c->lam, c->Z, c->work_ritz(),
                                                 c->ritz_flags, &c->st->n_ritz_fallbacks, s));
    // V_m Z, first the nev candidate columns (the rest once k of eq. (29) is known)
    const size_t tcs = ph.df ? sizeof(double2) : cs;   // element size of Vtmp
    auto rotate_cols = [&](int c0, int ncols) -> jtrlan_status {
      if (ncols <= 0) return JTRLAN_OK;
      void* out = (char*)ph.Vtmp + (size_t)c0 * n * tcs;
      const double* Zc = c->Z + (size_t)c0 * m;
      if (ph.df && c->tc_on)
        LAUNCH(K_ROTATE, launch_rotate_tc(ph.V, n, m, Zc, ncols, out, c->tc, c0 == 0, s));
      else if (ph.df)
        LAUNCH(K_ROTATE, launch_rotate_df(ph.V, n, m, Zc, ncols, out, s));
      else
        LAUNCH(K_ROTATE, launch_rotate<R>(ph.V, n, m, Zc, ncols, out, s));
      c->work[K_ROTATE] += 2.0 * (double)n * m * ncols;
      return JTRLAN_OK;
    };
    JT_TRY(rotate_cols(0, nev));
    LAUNCH(K_OTHER, launch_report(c->lam, c->Z, m, c->T, ldt, c->st, c->d_rep, s));
    JT_CUDA(cudaMemcpyAsync(c->h_rep, c->d_rep, (size_t)(2 * m + 8) * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (ph.df && c->tc_on) JT_CUDA(cudaMemcpyAsync(c->h_tcerr, c->tc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (c->invert) JT_CUDA(cudaMemcpyAsync(c->h_cgst, c->cg_st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    JT_CUDA(cudaStreamSynchronize(s));
    JT_CUDA(c->prof.harvest());
    if (ph.df && c->tc_on && *c->h_tcerr != 0)
      return fail(JTRLAN_ETIMEOUT, "tensor-core rotation: a bounded wait ran out (code " +
                                       std::to_string(*c->h_tcerr) + ")");
    stt.n_gs_passes += (int64_t)c->h_rep[2 * m + 2] - c->gs_pass_base;
    c->gs_pass_base = (int64_t)c->h_rep[2 * m + 2];
    c->work[K_GS_FIRST] = c->work_base[0] + c->h_rep[2 * m + 4];
    c->work[K_GS_DOT] = c->work_base[1] + c->h_rep[2 * m + 5];
    c->work[K_GS_UPDATE] = c->work_base[2] + c->h_rep[2 * m + 6];
    c->work[K_GS_STEP] = c->work[K_GS_FIRST] + c->work[K_GS_DOT] + c->work[K_GS_UPDATE];
    stt.n_ritz_fallbacks = c->fallback_base + (int)c->h_rep[2 * m + 7];
    if (c->h_rep[2 * m + 1] != 0.0) return fail(JTRLAN_EBREAKDOWN, "Lanczos breakdown: beta below 1e-14 max|T|");
    const double tmax = c->h_rep[2 * m + 3];
    const double tol_ph = std::max(tol, tol_rel_tmax * tmax);
    const double beta_m = c->h_rep[2 * m];
    for (int i = 0; i < kk; ++i) {
      lamv[i] = c->h_rep[i];
      arrow[i] = beta_m * c->h_rep[m + i];   // t_{m+1,i} = t_{m+1,m} z_{m,i}
    }
    int ncand = 0;
    std::vector<char> reused(nev, 0);
    const double cnorm = c->invert ? c->h_cgst->cnorm : 0.0;
    for (int i = 0; i < nev; ++i) {
      // invert mode: T holds A^{-1}'s Ritz values; ev(i) = 1/lambda_i, res_est(i) = c |t_{m+1,i} ev(i)|
      ev[i] = c->invert ? 1.0 / lamv[i] : lamv[i];
      res_est[i] = c->invert ? cnorm * std::fabs(arrow[i] * ev[i]) : std::fabs(arrow[i]);
      conv[i] = 0;                            // is_convd reset every outer iteration
      // a certifying filtered phase tests A's residual once B's estimate is near tol (B = p(A)
      // scales residuals by about |p'(lambda)|, so the estimate alone is neither necessary nor enough)
      if (!(res_est[i] < (ph.certify ? 10.0 * tol_ph : tol_ph))) continue;
      if (ph.filtered && !ph.certify) {   // B = p(A): judged by the estimate; the unfiltered phase certifies
        res[i] = res_est[i];
        conv[i] = 1;
        continue;
      }
      // A pair locked at the previous restart is decoupled in T-bar (t_{m+1,i} = 0), so the
      // Rayleigh-Ritz step returns it unchanged: keep its verified residual instead of another
      // product (reading R6b).
      int hit = -1;
      if (res_est[i] < 1e-3 * tol_ph)
        for (size_t q = 0; q < locked_ev.size(); ++q)
          if (std::fabs(ev[i] - locked_ev[q]) <= 1e-12 * std::max(1.0, std::fabs(ev[i]))) { hit = (int)q; break; }
      if (hit >= 0) {
        res[i] = locked_res[hit];
        rq[i] = locked_rq[hit];
        conv[i] = 1;
        reused[i] = 1;
        continue;
      }
      c->h_cand[ncand] = i; c->h_candlam[ncand] = ev[i]; ++ncand;
    }
    if (ncand > 0 && ph.certify) {  // x^H A x and ||A x - (x^H A x) x|| of each candidate (FP64)
      for (int q = 0; q < ncand; ++q)
        JT_TRY(rq_resid(c, ph, (char*)ph.Vtmp + (size_t)c->h_cand[q] * n * sizeof(double2), c->d_candlam + q,
                        c->d_res + q));
      JT_CUDA(cudaMemcpyAsync(c->h_res, c->d_res, ncand * sizeof(double), cudaMemcpyDeviceToHost, s));
      JT_CUDA(cudaMemcpyAsync(c->h_candlam, c->d_candlam, ncand * sizeof(double), cudaMemcpyDeviceToHost, s));
      JT_CUDA(cudaStreamSynchronize(s));
      JT_CUDA(c->prof.harvest());
      stt.n_resid_matvec += ncand;
      c->work[K_RESID] += (double)ncand * mv_units;
      for (int q = 0; q < ncand; ++q) {
        const int i = c->h_cand[q];
        res[i] = c->h_res[q];
        rq[i] = c->h_candlam[q];
        conv[i] = res[i] < tol_ph;
      }
    } else if (ncand > 0) {  // true residuals ||A v_i - ev_i v_i|| of the candidates
      JT_CUDA(cudaMemcpyAsync(c->d_cand, c->h_cand, ncand * sizeof(int), cudaMemcpyHostToDevice, s));
      JT_CUDA(cudaMemcpyAsync(c->d_candlam, c->h_candlam, ncand * sizeof(double), cudaMemcpyHostToDevice, s));
      LAUNCH(K_RESID, launch_matvec<R>(ph.op, (const C*)ph.Vtmp, nullptr, MV_RESID, ph.resid_part, c->d_cand,
                                       c->d_candlam, ncand, n, nullptr, s));
      c->work[K_RESID] += (double)ncand * mv_units;
      LAUNCH(K_OTHER, launch_reduce_norms(ph.resid_part, ph.mv_nblk, ncand, c->d_res, s));
      JT_CUDA(cudaMemcpyAsync(c->h_res, c->d_res, ncand * sizeof(double), cudaMemcpyDeviceToHost, s));
      JT_CUDA(cudaStreamSynchronize(s));
      JT_CUDA(c->prof.harvest());
      stt.n_resid_matvec += ncand;
      for (int q = 0; q < ncand; ++q) {
        const int i = c->h_cand[q];
        res[i] = c->h_res[q];
        conv[i] = res[i] < tol_ph;
      }
    }
    // converged pairs to the top (stable), identity beyond nev
    int w = 0;
    for (int i = 0; i < nev; ++i) if (conv[i]) perm[w++] = i;
    icnv = w;
    for (int i = 0; i < nev; ++i) if (!conv[i]) perm[w++] = i;
    for (int i = nev; i < m; ++i) perm[i] = i;
    std::vector<double> ev2(nev), res2(nev), lam2(m), arrow2(m), rq2(nev);
    for (int i = 0; i < kk; ++i) { lam2[i] = lamv[perm[i]]; arrow2[i] = arrow[perm[i]]; }
    for (int i = 0; i < nev; ++i) { ev2[i] = ev[perm[i]]; res2[i] = res[perm[i]]; rq2[i] = rq[perm[i]]; }
    ev = ev2; res = res2; lamv = lam2; arrow = arrow2; rq = rq2;
    for (int i = 0; i < icnv; ++i) arrow[i] = 0.0;   // decouple the converged subspace
    locked_ev.assign(ev.begin(), ev.begin() + icnv);
    locked_res.assign(res.begin(), res.begin() + icnv);
    locked_rq.assign(rq.begin(), rq.begin() + icnv);
    *icnv_out = icnv;
    if (icnv == nev && ph.certify) ev = rq;   // eigenvalues of A, not of B = p(A)
    if (icnv == nev) {
      for (int i = 0; i < m; ++i) c->h_perm[i] = perm[i];
      JT_CUDA(cudaMemcpyAsync(c->d_perm, c->h_perm, m * sizeof(int), cudaMemcpyHostToDevice, s));
      if (ph.df)
        LAUNCH(K_SHRINK, launch_shrink_df(ph.V, ph.Vtmp, n, c->d_perm, nev, m, s));
      else
        LAUNCH(K_SHRINK, launch_shrink<R>(ph.V, ph.Vtmp, n, c->d_perm, nev, m, s));
      JT_CUDA(cudaStreamSynchronize(s));
      JT_CUDA(c->prof.harvest());
      break;
    }
    // ---- shrink to k + 1 (eq. (29)); T-bar = diag(lambda_1..k) with the arrow in row k+1
    k = std::min(icnv + c->mwin, m - 1);
    JT_TRY(rotate_cols(nev, k - nev));   // the kept columns beyond the candidates
    std::memset(c->h_T, 0, (size_t)ldt * ldt * sizeof(double));
    double tm = 0.0;
    for (int i = 0; i < k; ++i) {
      c->h_T[(size_t)i * ldt + i] = lamv[i];
      c->h_T[(size_t)k * ldt + i] = arrow[i];
      c->h_T[(size_t)i * ldt + k] = arrow[i];
      tm = std::max(tm, std::max(std::fabs(lamv[i]), std::fabs(arrow[i])));
    }
    c->h_misc[0] = tm;
    for (int i = 0; i < m; ++i) c->h_perm[i] = perm[i];
    JT_CUDA(cudaMemcpyAsync(c->T, c->h_T, (size_t)ldt * ldt * sizeof(double), cudaMemcpyHostToDevice, s));
    JT_CUDA(cudaMemcpyAsync(&c->st->tmax, c->h_misc, sizeof(double), cudaMemcpyHostToDevice, s));
    JT_CUDA(cudaMemcpyAsync(c->d_perm, c->h_perm, m * sizeof(int), cudaMemcpyHostToDevice, s));
    if (ph.df)
      LAUNCH(K_SHRINK, launch_shrink_df(ph.V, ph.Vtmp, n, c->d_perm, k, m, s));  // and v_{k+1} = v_{m+1}
    else
      LAUNCH(K_SHRINK, launch_shrink<R>(ph.V, ph.Vtmp, n, c->d_perm, k, m, s));
  }
  // carry the device counters of this phase into the next one
  c->work_base[0] = c->work[K_GS_FIRST];
  c->work_base[1] = c->work[K_GS_DOT];
  c->work_base[2] = c->work[K_GS_UPDATE];
  c->fallback_base = stt.n_ritz_fallbacks;
  c->gs_pass_base = 0;
  if (icnv != nev) return fail(JTRLAN_ENOCONV, "max_restarts reached before nev pairs converged");
  return JTRLAN_OK;
}

// Spectral bounds from `steps` unrestarted Lanczos steps on A (see jtrlan_bounds).
jtrlan_status bounds_impl(jtrlan_ctx* c, int steps, double* lo, double* hi) {
  if (steps < 2 || steps > c->m) return fail(JTRLAN_EINVAL, "need 2 <= steps <= m");
  const bool fp32 = c->prm.precision == JTRLAN_MIXED;
  Phase& ph = fp32 ? c->p32 : c->mixed ? c->pdf : c->p64;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const int ldt = c->m + 1;
  c->prof.used = 0;
  for (int t = 0; t < K_NTAGS; ++t) { c->prof.ms[t] = 0; c->nl[t] = 0; c->work[t] = 0; }
  JT_CUDA(cudaMemsetAsync(c->st, 0, sizeof(StepState), s));
  JT_CUDA(cudaMemsetAsync(c->T, 0, (size_t)ldt * ldt * sizeof(double), s));
  const uint64_t seed = 0xb07d5ull;
  if (ph.df) {
    LAUNCH(K_OTHER, launch_fill_random<double>(ph.x, n, seed, s));
    LAUNCH(K_OTHER, launch_normalize_col<double>(ph.x, n, c->part_nrm, c->gs_nblk, s));
    LAUNCH(K_OTHER, launch_df_from_fp64(ph.x, ph.V, n, s));
  } else if (fp32) {
    LAUNCH(K_OTHER, launch_fill_random<float>(ph.V, n, seed, s));
    LAUNCH(K_OTHER, launch_normalize_col<float>(ph.V, n, c->part_nrm, c->gs_nblk, s));
  } else {
    LAUNCH(K_OTHER, launch_fill_random<double>(ph.V, n, seed, s));
    LAUNCH(K_OTHER, launch_normalize_col<double>(ph.V, n, c->part_nrm, c->gs_nblk, s));
  }
  GSArgs a{};
  a.V = ph.V; a.n = n; a.h = c->h; a.y = ph.y; a.part_dot = c->part_dot; a.part_nrm = c->part_nrm;
  a.coef = c->coef; a.st = c->st; a.T = c->T; a.ldt = ldt; a.m = c->m; a.nblk = c->gs_nblk;
  a.rows_per_block = c->gs_rpb;
  a.no_w = c->prm.plain_trlan ? 1 : 0;
  if (fp32) JT_TRY(lanczos_steps<float>(c, ph, a, 0, steps, false));
  else JT_TRY(lanczos_steps<double>(c, ph, a, 0, steps, false));
  LAUNCH(K_RITZ, launch_ritz(c->T, ldt, steps, 0, steps, JTRLAN_SMALLEST, c->lam, c->Z, c->ritz_flags, s));
  LAUNCH(K_RITZ_FALLBACK, launch_ritz_fallback(c->T, ldt, steps, JTRLAN_SMALLEST, c->lam, c->Z, c->work_ritz(),
                                               c->ritz_flags, &c->st->n_ritz_fallbacks, s));
  LAUNCH(K_OTHER, launch_report(c->lam, c->Z, steps, c->T, ldt, c->st, c->d_rep, s));
  JT_CUDA(cudaMemcpyAsync(c->h_rep, c->d_rep, (size_t)(2 * steps + 8) * sizeof(double), cudaMemcpyDeviceToHost, s));
  JT_CUDA(cudaStreamSynchronize(s));
  JT_CUDA(c->prof.harvest());
  if (c->h_rep[2 * steps + 1] != 0.0) return fail(JTRLAN_EBREAKDOWN, "Lanczos breakdown while estimating bounds");
  const double beta = std::fabs(c->h_rep[2 * steps]);
  *lo = c->h_rep[0] - beta * std::fabs(c->h_rep[steps]);   // theta_min - |beta z_{steps,1}|
  *hi = c->h_rep[steps - 1] + beta;
  return JTRLAN_OK;
}

jtrlan_status solve_impl(jtrlan_ctx* c, jtrlan_stats* stats_out) {
  const auto t0 = std::chrono::steady_clock::now();
  c->solved = false;
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  jtrlan_stats stt{};
  c->prof.on = c->prm.profile != 0;
  c->prof.used = 0;
  for (int t = 0; t < K_NTAGS; ++t) { c->prof.ms[t] = 0; c->nl[t] = 0; c->work[t] = 0; }
  for (int t = 0; t < 3; ++t) c->work_base[t] = 0;
  c->fallback_base = 0;
  c->cg_matvecs = c->cg_iters = 0;
  c->gs_pass_base = 0;
  std::vector<double> ev, res;
  int icnv = 0;
  jtrlan_status st = JTRLAN_OK;
  if (c->prm.precision == JTRLAN_MIXED) {
    // FP32 phase: matvec, Gram-Schmidt and rotation in FP32, alpha/beta and Ritz in FP64, to the
    // tolerance max(tol, 1e-5 max|t|) that FP32 vectors can certify.
    Phase& ph = c->p32;
    if (c->prm.v1) {
      JT_CUDA(cudaMemcpyAsync(c->pdf.y, c->prm.v1, (size_t)n * sizeof(double2), cudaMemcpyDefault, s));
      LAUNCH(K_OTHER, launch_c128_to_c64(c->pdf.y, ph.V, n, s));
    } else {
      LAUNCH(K_OTHER, launch_fill_ones<float>(ph.V, n, s));
    }
    LAUNCH(K_OTHER, launch_normalize_col<float>(ph.V, n, c->part_nrm, c->gs_nblk, s));
    c->nl[K_OTHER] += 1;
    jtrlan_stats s32{};
    st = run_phase<float>(c, ph, c->prm.tol, 1e-5, c->max_restarts, s32, ev, res, &icnv);
    if (st != JTRLAN_OK && st != JTRLAN_ENOCONV) return st;
    stt.n_matvec_fp32 = s32.n_matvec;
    stt.n_matvec += s32.n_matvec;
    stt.n_resid_matvec += s32.n_resid_matvec;
    stt.n_gs_passes += s32.n_gs_passes;
    stt.n_restarts_fp32 = s32.n_restarts;
    stt.n_restarts += s32.n_restarts;
    // the double-float phase starts from the normalised sum of the FP32 Ritz vectors (promoted)
    LAUNCH(K_OTHER, launch_sum_columns(ph.V, n, std::max(icnv, 1), c->pdf.x, s));
  } else if (c->mixed) {
    if (c->prm.v1)
      JT_CUDA(cudaMemcpyAsync(c->pdf.x, c->prm.v1, (size_t)n * sizeof(double2), cudaMemcpyDefault, s));
    else
      LAUNCH(K_OTHER, launch_fill_ones<double>(c->pdf.x, n, s));
  } else {
    if (c->prm.v1) {
      JT_CUDA(cudaMemcpyAsync(c->p64.V, c->prm.v1, (size_t)n * sizeof(double2), cudaMemcpyDefault, s));
      LAUNCH(K_OTHER, launch_normalize_col<double>(c->p64.V, n, c->part_nrm, c->gs_nblk, s));
      c->nl[K_OTHER] += 1;  // two kernels
    } else {
      LAUNCH(K_OTHER, launch_fill_ones<double>(c->p64.V, n, s));  // v_1 = 1 / ||1||
    }
  }
  if (c->mixed) {  // normalise the FP64 start and store it split into the (hi, lo) basis
    LAUNCH(K_OTHER, launch_normalize_col<double>(c->pdf.x, n, c->part_nrm, c->gs_nblk, s));
    c->nl[K_OTHER] += 1;
    LAUNCH(K_OTHER, launch_df_from_fp64(c->pdf.x, c->pdf.V, n, s));
  }
  jtrlan_stats s64{};
  st = run_phase<double>(c, c->mixed ? c->pdf : c->p64, c->prm.tol, 0.0, c->max_restarts, s64, ev, res, &icnv);
  stt.n_matvec += s64.n_matvec;
  stt.n_resid_matvec += s64.n_resid_matvec;
  stt.n_gs_passes += s64.n_gs_passes;
  stt.n_restarts += s64.n_restarts;
  stt.n_ritz_fallbacks = s64.n_ritz_fallbacks;
  stt.icnv = icnv;
  stt.n_matvec_inner = c->cg_matvecs;
  stt.n_cg_iters = c->cg_iters;
  for (int t = 0; t < K_NTAGS; ++t) stt.n_launches += c->nl[t];
  stt.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  c->stats = stt;
  if (stats_out) *stats_out = stt;
  if (st != JTRLAN_OK) return st;
  c->ev = ev;
  c->res = res;
  c->solved = true;
  return JTRLAN_OK;
}

}  // namespace

extern "C" {

jtrlan_status jtrlan_create(const jtrlan_operator* op, const jtrlan_params* params, void* cuda_stream,
                            jtrlan_ctx** out) {
  if (!out) return fail(JTRLAN_EINVAL, "null out pointer");
  *out = nullptr;
  jtrlan_ctx* c = nullptr;
  jtrlan_status s = create_impl(op, params, cuda_stream, &c);
  if (s != JTRLAN_OK) {
    delete c;
    return s;
  }
  *out = c;
  g_last_error.clear();
  return JTRLAN_OK;
}

jtrlan_status jtrlan_apply(jtrlan_ctx* c, const void* x, void* y) {
  if (!c || !x || !y) return fail(JTRLAN_EINVAL, "null argument");
  if (c->mixed)
    JT_CUDA(launch_matvec<float>(c->p32.op, (const float2*)x, (float2*)y, MV_PLAIN, nullptr, nullptr, nullptr, 0, 0,
                                 nullptr, c->stream));
  else
    JT_CUDA(launch_matvec<double>(c->p64.op, (const double2*)x, (double2*)y, MV_PLAIN, nullptr, nullptr, nullptr, 0,
                                  0, nullptr, c->stream));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_solve(jtrlan_ctx* c, jtrlan_stats* stats) {
  if (!c) return fail(JTRLAN_EINVAL, "null context");
  return solve_impl(c, stats);
}

jtrlan_status jtrlan_pairs(jtrlan_ctx* c, int with_partners, double* evals, void* evecs, double* res) {
  if (!c) return fail(JTRLAN_EINVAL, "null context");
  if (!c->solved) return fail(JTRLAN_ESTATE, "no successful solve to report");
  const int nev = c->nev;
  std::vector<int> order(nev);
  for (int i = 0; i < nev; ++i) order[i] = i;
  const bool largest = c->prm.which == JTRLAN_LARGEST;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return largest ? c->ev[a] > c->ev[b] : c->ev[a] < c->ev[b];
  });
  for (int i = 0; i < nev; ++i) {
    if (evals) evals[i] = c->ev[order[i]];
    if (res) res[i] = c->res[order[i]];
  }
  if (evecs) {
    for (int i = 0; i < nev; ++i) c->h_order[i] = order[i];
    JT_CUDA(cudaMemcpyAsync(c->d_order, c->h_order, nev * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    const int ncols = with_partners ? 2 * nev : nev;
    const size_t bytes = (size_t)c->n * ncols * sizeof(double2);
    cudaPointerAttributes attr{};
    const bool dev = cudaPointerGetAttributes(&attr, evecs) == cudaSuccess &&
                     (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) {
      if (c->mixed)
        JT_CUDA(launch_gather_pairs_df(c->pdf.V, c->n, c->d_order, nev, with_partners, evecs, c->stream));
      else
        JT_CUDA(launch_gather_pairs<double>(c->p64.V, c->n, c->d_order, nev, with_partners, evecs, c->stream));
    } else {
      void* tmp = nullptr;
      JT_CUDA(cudaMallocAsync(&tmp, bytes, c->stream));
      if (c->mixed)
        JT_CUDA(launch_gather_pairs_df(c->pdf.V, c->n, c->d_order, nev, with_partners, tmp, c->stream));
      else
        JT_CUDA(launch_gather_pairs<double>(c->p64.V, c->n, c->d_order, nev, with_partners, tmp, c->stream));
      JT_CUDA(cudaMemcpyAsync(evecs, tmp, bytes, cudaMemcpyDeviceToHost, c->stream));
      JT_CUDA(cudaFreeAsync(tmp, c->stream));
    }
  }
  JT_CUDA(cudaStreamSynchronize(c->stream));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_get_profile(jtrlan_ctx* c, jtrlan_profile* out) {
  if (!c || !out) return fail(JTRLAN_EINVAL, "null argument");
  std::memset(out, 0, sizeof(*out));
  out->n_classes = K_NTAGS;
  for (int t = 0; t < K_NTAGS; ++t) {
    out->names[t] = kTagNames[t];
    out->ms[t] = c->prof.ms[t];
    out->launches[t] = c->nl[t];
    out->work[t] = c->work[t];
  }
  return JTRLAN_OK;
}

jtrlan_status jtrlan_apply_filter(jtrlan_ctx* c, const void* x, void* y) {
  if (!c || !x || !y) return fail(JTRLAN_EINVAL, "null argument");
  cudaStream_t s = c->stream;
  if (c->p32.filtered) {
    JT_TRY(filter_apply<float>(c, c->p32, x, y, nullptr));
    return JTRLAN_OK;
  }
  Phase& ph = c->mixed ? c->pdf : c->p64;
  if (!ph.certify) return fail(JTRLAN_EINVAL, "the context has no filter");
  if (ph.dfmv) LAUNCH(K_RESID, launch_df_from_fp64(x, ph.fbuf[3], c->n, s));
  JT_TRY(filter_apply_cert_io(c, ph, x, ph.fbuf[3], y));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_bounds(jtrlan_ctx* c, int steps, double* lo, double* hi) {
  if (!c || !lo || !hi) return fail(JTRLAN_EINVAL, "null argument");
  return bounds_impl(c, steps, lo, hi);
}

jtrlan_status jtrlan_damped_step(const double* tau, int count, int degree, float* out, void* cuda_stream) {
  if (count < 0 || degree < 0 || degree > 1024) return fail(JTRLAN_EINVAL, "need count >= 0 and 0 <= degree <= 1024");
  if (count > 0 && (!tau || !out)) return fail(JTRLAN_EINVAL, "null argument");
  JT_CUDA(launch_damped_step(tau, count, degree, out, (cudaStream_t)cuda_stream));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_rotate_df(const void* V, int64_t n, int m, const double* Z, int kk, void* out, int path,
                               void* cuda_stream) {
  if (!V || !Z || !out) return fail(JTRLAN_EINVAL, "null argument");
  if (n < 1 || m < 1 || kk < 1) return fail(JTRLAN_EINVAL, "need n, m, kk >= 1");
  if (path < 0 || path > 2) return fail(JTRLAN_EINVAL, "path must be 0 (tensor cores), 1 (CUDA cores) or 2 (self-test)");
  if (path != 1 && m > tc_rotate_max_m())
    return fail(JTRLAN_EINVAL, "tensor-core rotation needs m <= " + std::to_string(tc_rotate_max_m()));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (path == 1) {
    JT_CUDA(launch_rotate_df(V, n, m, Z, kk, out, s));
    JT_CUDA(cudaStreamSynchronize(s));
    return JTRLAN_OK;
  }
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, tc_rotate_bytes(n, m, kk));
  if (e != cudaSuccess) return fail(JTRLAN_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  TcWork w = tc_rotate_carve(base, n, m, kk);
  int herr = 0;
  e = cudaMemsetAsync(w.err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_rotate_tc(V, n, m, Z, kk, out, w, true, s, path == 2 ? 1 : 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(base);
  if (e != cudaSuccess) return fail(JTRLAN_ECUDA, std::string("tensor-core rotation: ") + cudaGetErrorString(e));
  if (herr != 0)
    return fail(JTRLAN_ETIMEOUT, "tensor-core rotation: a bounded wait ran out (code " + std::to_string(herr) + ")");
  return JTRLAN_OK;
}

jtrlan_status jtrlan_set_filter(jtrlan_ctx* c, int degree, const double* coeffs, double lo, double hi) {
  if (!c || !coeffs) return fail(JTRLAN_EINVAL, "null argument");
  if (degree < 1 || degree > 1024) return fail(JTRLAN_EINVAL, "need 1 <= degree <= 1024");
  if (!(lo < hi)) return fail(JTRLAN_EINVAL, "need lo < hi");
  if (c->invert) return fail(JTRLAN_EINVAL, "invert mode takes no filter");
  for (int k = 0; k <= degree; ++k)
    if (!std::isfinite(coeffs[k])) return fail(JTRLAN_EINVAL, "filter coefficients must be finite");
  JT_TRY(setup_certify(c, coeffs, degree));
  c->prm.filter_final_degree = degree;
  c->prm.filter_final_coeffs = nullptr;   // the caller's array is not kept
  c->prm.filter_lo = lo;
  c->prm.filter_hi = hi;
  c->fc = 0.5 * (lo + hi);
  c->fe = 0.5 * (hi - lo);
  c->solved = false;
  return JTRLAN_OK;
}

void jtrlan_destroy(jtrlan_ctx* c) { delete c; }

const char* jtrlan_status_string(jtrlan_status s) {
  switch (s) {
    case JTRLAN_OK: return "ok";
    case JTRLAN_EINVAL: return "invalid argument";
    case JTRLAN_ENOMEM: return "out of memory";
    case JTRLAN_ECUDA: return "CUDA error";
    case JTRLAN_ENOTJSYM: return "operator is not Hermitian J-symmetric (Lemma 1 check)";
    case JTRLAN_EBREAKDOWN: return "Lanczos breakdown";
    case JTRLAN_ENOCONV: return "not converged within max_restarts";
    case JTRLAN_ETIMEOUT: return "device wait timed out";
    case JTRLAN_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* jtrlan_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
