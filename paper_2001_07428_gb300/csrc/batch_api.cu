// batch_api.cu -- the C ABI of the batched dense solver (include/jtrlan.h, jtrlan_batch_*): packing
// of many dense Hermitian J-symmetric operators of uneven order, the launch shape (occupancy, the
// autotuner), the CUDA graph that holds the persistent launch, and the result read-back.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "../../include/jtrlan.h"

using namespace jtr;

namespace {

jtrlan_status bfail(jtrlan_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

#define JB_CUDA(expr)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return bfail(e_ == cudaErrorMemoryAllocation ? JTRLAN_ENOMEM : JTRLAN_ECUDA,                 \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

#define JB_TRY(expr)                \
  do {                              \
    jtrlan_status s_ = (expr);      \
    if (s_ != JTRLAN_OK) return s_; \
  } while (0)

}  // namespace

struct jtrlan_batch {
  cudaStream_t user = nullptr;  // the caller's stream (ordering only)
  cudaStream_t own = nullptr;   // the library's stream: capturable whatever the caller passed
  cudaEvent_t e0 = nullptr, e1 = nullptr, ej = nullptr;
  int count = 0, nev = 0, m = 0, mwin = 0, kk = 0, which = 0, gs_passes = 3, max_restarts = 1000;
  double tol = 0.0;
  bool df = false;
  int64_t nmax = 0;
  std::vector<int64_t> h, a_off, vec_off;
  std::vector<int> order;
  void* A11 = nullptr;
  void* A12 = nullptr;
  int* d_order = nullptr;
  int64_t* d_h = nullptr;
  int64_t* d_aoff = nullptr;
  int64_t* d_voff = nullptr;
  void* slots_v = nullptr;
  void* slots_t = nullptr;
  int slots_grid = 0;
  double* out_ev = nullptr;
  double* out_res = nullptr;
  int* out_stats = nullptr;
  long long* prof = nullptr;    // per-instance phase cycles (params.profile)
  void* out_vec = nullptr;
  int* queue = nullptr;
  int n_sm = 0;
  int threads = 256;
  int ctas_per_sm = 0;          // 0: as many as fit
  cudaGraphExec_t exec = nullptr;
  int exec_grid = 0, exec_threads = 0;
  int mv_rows = 0;              // tile shape (0 until set: the form's default, see tiles_of)
  int gs_groups = 0;            // 0: as many update groups as fit
  int exec_mv_rows = -1, exec_gs_groups = -1;
  bool solved = false;
  std::vector<void*> allocs;

  jtrlan_status dalloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    JB_CUDA(cudaMalloc(p, bytes));
    allocs.push_back(*p);
    return JTRLAN_OK;
  }
  void release(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) allocs.erase(it);
    cudaFree(p);
  }
  ~jtrlan_batch() {
    if (own) cudaStreamSynchronize(own);
    if (exec) cudaGraphExecDestroy(exec);
    for (void* p : allocs) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ej) cudaEventDestroy(ej);
    if (own) cudaStreamDestroy(own);
  }
};

namespace {

jtrlan_status validate_batch(int count, const jtrlan_operator* ops, const jtrlan_params* p) {
  if (count <= 0 || !ops || !p) return bfail(JTRLAN_EINVAL, "need count >= 1, operators and params");
  if (p->nev <= 0 || p->m <= p->nev) return bfail(JTRLAN_EINVAL, "need 0 < nev < m");
  if (p->m > kBatchMaxM) return bfail(JTRLAN_EINVAL, "the batched solver supports m <= 64");
  if (p->nev > kBatchMaxNev) return bfail(JTRLAN_EINVAL, "the batched solver supports nev <= 32");
  if (p->mwin < 0) return bfail(JTRLAN_EINVAL, "need mwin >= 0");
  if (!(p->tol > 0.0)) return bfail(JTRLAN_EINVAL, "need tol > 0");
  if (p->which != JTRLAN_SMALLEST && p->which != JTRLAN_LARGEST) return bfail(JTRLAN_EINVAL, "unknown which");
  if (p->precision != JTRLAN_FP64 && p->precision != JTRLAN_MIXED_REORTH)
    return bfail(JTRLAN_EINVAL, "the batched solver runs JTRLAN_FP64 or JTRLAN_MIXED_REORTH");
  if (p->gs_max_passes < 0 || p->gs_max_passes > 7) return bfail(JTRLAN_EINVAL, "gs_max_passes must be 0..7");
  if (p->max_restarts < 0) return bfail(JTRLAN_EINVAL, "max_restarts must be >= 0");
  if (p->v1) return bfail(JTRLAN_EINVAL, "the batched solver starts every instance from (1, ..., 1)");
  if (p->check_jsym) return bfail(JTRLAN_EINVAL, "check_jsym is not offered by the batched solver");
  for (int i = 0; i < count; ++i) {
    const jtrlan_operator& o = ops[i];
    if (o.kind != JTRLAN_DENSE) return bfail(JTRLAN_EINVAL, "the batched solver takes dense operators only");
    if (o.n <= 0 || (o.n & 1)) return bfail(JTRLAN_EINVAL, "n must be positive and even");
    if (o.dtype != JTRLAN_C128 && o.dtype != JTRLAN_C64) return bfail(JTRLAN_EINVAL, "unknown dtype");
    if (!o.a11 || !o.a12) return bfail(JTRLAN_EINVAL, "null dense block");
    if ((int64_t)p->m >= o.n / 2) return bfail(JTRLAN_EINVAL, "need m < n/2 for every instance");
  }
  return JTRLAN_OK;
}

jtrlan_status upload_block(jtrlan_batch* b, const void* src, int dtype, int64_t count, double2* dst, void* tmp) {
  if (dtype == JTRLAN_C128) {
    JB_CUDA(cudaMemcpyAsync(dst, src, (size_t)count * sizeof(double2), cudaMemcpyDefault, b->own));
  } else {
    JB_CUDA(cudaMemcpyAsync(tmp, src, (size_t)count * sizeof(float2), cudaMemcpyDefault, b->own));
    JB_CUDA(launch_c64_to_c128(tmp, dst, count, b->own));
  }
  return JTRLAN_OK;
}

jtrlan_status create_batch(int count, const jtrlan_operator* ops, const jtrlan_params* p, void* stream,
                           jtrlan_batch* b) {
  JB_TRY(validate_batch(count, ops, p));
  b->user = (cudaStream_t)stream;
  JB_CUDA(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
  JB_CUDA(cudaEventCreate(&b->e0));
  JB_CUDA(cudaEventCreate(&b->e1));
  JB_CUDA(cudaEventCreateWithFlags(&b->ej, cudaEventDisableTiming));
  int dev = 0;
  JB_CUDA(cudaGetDevice(&dev));
  JB_CUDA(cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev));
  b->count = count;
  b->nev = p->nev;
  b->m = p->m;
  b->mwin = p->mwin;
  // Ritz pairs needed per restart: the nev candidates and the kept columns of eq. (29)
  b->kk = std::max(p->nev, std::min(p->nev - 1 + p->mwin, p->m - 1));
  b->which = p->which;
  b->tol = p->tol;
  b->gs_passes = p->gs_max_passes ? p->gs_max_passes : 3;
  b->max_restarts = p->max_restarts ? p->max_restarts : 1000;
  b->df = p->precision == JTRLAN_MIXED_REORTH;
  b->h.resize(count);
  b->a_off.resize(count);
  b->vec_off.resize(count);
  int64_t a_total = 0, v_total = 0;
  for (int i = 0; i < count; ++i) {
    b->h[i] = ops[i].n / 2;
    b->a_off[i] = a_total;
    b->vec_off[i] = v_total;
    a_total += b->h[i] * b->h[i];
    v_total += ops[i].n * (int64_t)p->nev;
    b->nmax = std::max<int64_t>(b->nmax, ops[i].n);
  }
  // largest first: the queue hands the long instances out before the short ones
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return b->h[x] > b->h[y]; });
  void* vp = nullptr;
  JB_TRY(b->dalloc(&b->A11, (size_t)a_total * 16));
  JB_TRY(b->dalloc(&b->A12, (size_t)a_total * 16));
  JB_TRY(b->dalloc(&vp, count * sizeof(int)));
  b->d_order = (int*)vp;
  JB_TRY(b->dalloc(&vp, count * sizeof(int64_t)));
  b->d_h = (int64_t*)vp;
  JB_TRY(b->dalloc(&vp, count * sizeof(int64_t)));
  b->d_aoff = (int64_t*)vp;
  JB_TRY(b->dalloc(&vp, count * sizeof(int64_t)));
  b->d_voff = (int64_t*)vp;
  JB_TRY(b->dalloc(&vp, (size_t)count * p->nev * sizeof(double)));
  b->out_ev = (double*)vp;
  JB_TRY(b->dalloc(&vp, (size_t)count * p->nev * sizeof(double)));
  b->out_res = (double*)vp;
  JB_TRY(b->dalloc(&vp, (size_t)count * kBatchStats * sizeof(int)));
  b->out_stats = (int*)vp;
  if (p->profile) {
    JB_TRY(b->dalloc(&vp, (size_t)count * kBatchPhases * sizeof(long long)));
    b->prof = (long long*)vp;
  }
  JB_TRY(b->dalloc(&b->out_vec, (size_t)v_total * sizeof(double2)));
  JB_TRY(b->dalloc(&vp, sizeof(int)));
  b->queue = (int*)vp;
  JB_CUDA(cudaMemcpyAsync(b->d_order, b->order.data(), count * sizeof(int), cudaMemcpyHostToDevice, b->own));
  JB_CUDA(cudaMemcpyAsync(b->d_h, b->h.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, b->own));
  JB_CUDA(cudaMemcpyAsync(b->d_aoff, b->a_off.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, b->own));
  JB_CUDA(cudaMemcpyAsync(b->d_voff, b->vec_off.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, b->own));
  // the caller's blocks may be on the caller's stream: order the copies after it
  JB_CUDA(cudaEventRecord(b->ej, b->user));
  JB_CUDA(cudaStreamWaitEvent(b->own, b->ej, 0));
  void* tmp = nullptr;
  JB_TRY(b->dalloc(&tmp, (size_t)(b->nmax / 2) * (b->nmax / 2) * sizeof(float2)));
  for (int i = 0; i < count; ++i) {
    const int64_t hh = b->h[i] * b->h[i];
    JB_TRY(upload_block(b, ops[i].a11, ops[i].dtype, hh, (double2*)b->A11 + b->a_off[i], tmp));
    JB_TRY(upload_block(b, ops[i].a12, ops[i].dtype, hh, (double2*)b->A12 + b->a_off[i], tmp));
  }
  if (b->df) {
    JB_CUDA(launch_split_df_inplace(b->A11, a_total, b->own));
    JB_CUDA(launch_split_df_inplace(b->A12, a_total, b->own));
  }
  JB_CUDA(cudaStreamSynchronize(b->own));  // the caller may free its blocks after this call
  b->release(tmp);
  return JTRLAN_OK;
}

// Launch shape for (threads, ctas_per_sm): one resident wave of CTAs, no more than there are instances.
BatchArgs args_of(const jtrlan_batch* b);

jtrlan_status shape(jtrlan_batch* b, int threads, int ctas_per_sm, int* grid) {
  const size_t sm = batch_smem_bytes(b->nmax, b->m, b->kk, threads);
  int dev = 0, optin = 0;
  JB_CUDA(cudaGetDevice(&dev));
  JB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (sm + 8192 > (size_t)optin)
    return bfail(JTRLAN_EINVAL, "the largest instance needs more shared memory per CTA than the device has");
  int fit = 0;
  JB_CUDA(batch_occupancy(b->df, args_of(b).mv_rows, threads, sm, &fit));
  if (fit < 1) return bfail(JTRLAN_EINVAL, "the batched kernel does not fit on an SM at this size");
  const int per = ctas_per_sm > 0 ? std::min(ctas_per_sm, fit) : fit;
  *grid = std::max(1, std::min(b->count, per * b->n_sm));
  if (*grid > b->slots_grid) {  // per-CTA V and rotation slots
    b->release(b->slots_v);
    b->release(b->slots_t);
    b->slots_v = b->slots_t = nullptr;
    b->slots_grid = 0;
    JB_TRY(b->dalloc(&b->slots_v, (size_t)*grid * b->nmax * (b->m + 1) * 16));
    JB_TRY(b->dalloc(&b->slots_t, (size_t)*grid * b->nmax * b->kk * sizeof(double2)));
    b->slots_grid = *grid;
  }
  return JTRLAN_OK;
}

BatchArgs args_of(const jtrlan_batch* b) {
  BatchArgs a{};
  a.count = b->count;
  a.order = b->d_order;
  a.h = b->d_h;
  a.a_off = b->d_aoff;
  a.A11 = b->A11;
  a.A12 = b->A12;
  a.Vslots = b->slots_v;
  a.Tslots = b->slots_t;
  a.nmax = b->nmax;
  a.m = b->m;
  a.nev = b->nev;
  a.mwin = b->mwin;
  a.kk = b->kk;
  a.which = b->which;
  a.gs_passes = b->gs_passes;
  a.max_restarts = b->max_restarts;
  a.tol = b->tol;
  a.out_ev = b->out_ev;
  a.out_res = b->out_res;
  a.out_stats = b->out_stats;
  a.out_vec = b->out_vec;
  a.vec_off = b->d_voff;
  a.prof = b->prof;
  a.queue = b->queue;
  // default tile: two product rows per warp in the compensated form, one in FP64 (measured best
  // before the tile search existed); the autotuner may change both
  a.mv_rows = b->mv_rows > 0 ? b->mv_rows : (b->df ? 2 : 1);
  a.gs_groups = b->gs_groups;
  return a;
}

// One solve of the whole batch on the library stream, timed with events; *ms receives the time.
jtrlan_status run_once(jtrlan_batch* b, int threads, int ctas_per_sm, bool graph, float* ms) {
  int grid = 0;
  JB_TRY(shape(b, threads, ctas_per_sm, &grid));
  const BatchArgs a = args_of(b);
  if (graph && (!b->exec || b->exec_grid != grid || b->exec_threads != threads || b->exec_mv_rows != a.mv_rows ||
                b->exec_gs_groups != a.gs_groups)) {
    if (b->exec) {
      JB_CUDA(cudaGraphExecDestroy(b->exec));
      b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    JB_CUDA(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->queue, 0, sizeof(int), b->own);
    cudaError_t e2 = launch_batch(b->df, a, grid, threads, b->own);
    cudaError_t e3 = cudaStreamEndCapture(b->own, &g);
    JB_CUDA(e1);
    JB_CUDA(e2);
    JB_CUDA(e3);
    cudaError_t e4 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    JB_CUDA(e4);
    b->exec_grid = grid;
    b->exec_threads = threads;
    b->exec_mv_rows = a.mv_rows;
    b->exec_gs_groups = a.gs_groups;
  }
  JB_CUDA(cudaEventRecord(b->ej, b->user));
  JB_CUDA(cudaStreamWaitEvent(b->own, b->ej, 0));
  JB_CUDA(cudaEventRecord(b->e0, b->own));
  if (graph) {
    JB_CUDA(cudaGraphLaunch(b->exec, b->own));
  } else {
    JB_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(int), b->own));
    JB_CUDA(launch_batch(b->df, a, grid, threads, b->own));
  }
  JB_CUDA(cudaEventRecord(b->e1, b->own));
  JB_CUDA(cudaEventSynchronize(b->e1));
  JB_CUDA(cudaEventElapsedTime(ms, b->e0, b->e1));
  JB_CUDA(cudaEventRecord(b->ej, b->own));
  JB_CUDA(cudaStreamWaitEvent(b->user, b->ej, 0));
  return JTRLAN_OK;
}

}  // namespace

extern "C" {

jtrlan_status jtrlan_batch_create(int count, const jtrlan_operator* ops, const jtrlan_params* params,
                                  void* cuda_stream, jtrlan_batch** out) {
  if (!out) return bfail(JTRLAN_EINVAL, "null out pointer");
  *out = nullptr;
  jtrlan_batch* b = new (std::nothrow) jtrlan_batch();
  if (!b) return bfail(JTRLAN_ENOMEM, "host allocation failed");
  jtrlan_status s = create_batch(count, ops, params, cuda_stream, b);
  if (s != JTRLAN_OK) {
    delete b;
    return s;
  }
  *out = b;
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_set_shape(jtrlan_batch* b, int threads, int ctas_per_sm) {
  if (!b) return bfail(JTRLAN_EINVAL, "null batch");
  if (threads < 64 || threads > kBatchMaxThreads || threads % 32)
    return bfail(JTRLAN_EINVAL, "threads must be a multiple of 32 in [64, 512]");
  if (ctas_per_sm < 0) return bfail(JTRLAN_EINVAL, "ctas_per_sm must be >= 0");
  int grid = 0;
  JB_TRY(shape(b, threads, ctas_per_sm, &grid));
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_tune(jtrlan_batch* b, int* threads_out, int* ctas_per_sm_out, double* best_ms) {
  if (!b) return bfail(JTRLAN_EINVAL, "null batch");
  float ms = 0.f;
  JB_TRY(run_once(b, b->threads, b->ctas_per_sm, false, &ms));  // warm-up (module load, caches)
  const int cand_threads[] = {128, 256, 512};
  int best_t = b->threads, best_c = b->ctas_per_sm;
  float best = 3.4e38f;
  for (int t : cand_threads) {
    int fit = 0;
    JB_CUDA(batch_occupancy(b->df, args_of(b).mv_rows, t, batch_smem_bytes(b->nmax, b->m, b->kk, t), &fit));
    for (int c = 1; c <= fit; ++c) {
      if ((c - 1) * b->n_sm >= b->count) break;  // the grid is capped at the instance count
      JB_TRY(run_once(b, t, c, false, &ms));
      if (ms < best) {
        best = ms;
        best_t = t;
        best_c = c;
      }
    }
  }
  b->threads = best_t;
  b->ctas_per_sm = best_c;
  // tile shapes at the chosen launch shape: rows of the product per warp, and (compensated form) the
  // number of thread groups that split the columns of the Gram-Schmidt update
  const int cand_rows[] = {1, 2};
  const int cand_groups_df[] = {0, 1, 2, 4};
  const int cand_groups_64[] = {0};
  const int* groups = b->df ? cand_groups_df : cand_groups_64;
  const int ngroups = b->df ? 4 : 1;
  int best_r = b->df ? 2 : 1, best_g = 0;
  for (int r : cand_rows)
    for (int q = 0; q < ngroups; ++q) {
      b->mv_rows = r;
      b->gs_groups = groups[q];
      JB_TRY(run_once(b, best_t, best_c, false, &ms));
      if (ms < best) {
        best = ms;
        best_r = r;
        best_g = groups[q];
      }
    }
  b->mv_rows = best_r;
  b->gs_groups = best_g;
  if (threads_out) *threads_out = best_t;
  if (ctas_per_sm_out) *ctas_per_sm_out = best_c;
  if (best_ms) *best_ms = best;
  b->solved = true;
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_set_tiles(jtrlan_batch* b, int mv_rows, int gs_groups) {
  if (!b) return bfail(JTRLAN_EINVAL, "null batch");
  if (mv_rows != 1 && mv_rows != 2) return bfail(JTRLAN_EINVAL, "mv_rows must be 1 or 2");
  if (gs_groups < 0 || gs_groups > 16) return bfail(JTRLAN_EINVAL, "gs_groups must be 0..16");
  b->mv_rows = mv_rows;
  b->gs_groups = gs_groups;
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_get_tiles(jtrlan_batch* b, int* mv_rows, int* gs_groups) {
  if (!b) return bfail(JTRLAN_EINVAL, "null batch");
  const BatchArgs a = args_of(b);
  if (mv_rows) *mv_rows = a.mv_rows;
  if (gs_groups) *gs_groups = a.gs_groups;
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_solve(jtrlan_batch* b, jtrlan_batch_stats* stats) {
  if (!b) return bfail(JTRLAN_EINVAL, "null batch");
  float ms = 0.f;
  JB_TRY(run_once(b, b->threads, b->ctas_per_sm, true, &ms));
  b->solved = true;
  std::vector<int> st((size_t)b->count * kBatchStats);
  JB_CUDA(cudaMemcpy(st.data(), b->out_stats, st.size() * sizeof(int), cudaMemcpyDeviceToHost));
  int n_ok = 0, max_rs = 0;
  int64_t mv = 0, rmv = 0, fb = 0, gs = 0;
  jtrlan_status worst = JTRLAN_OK;
  for (int i = 0; i < b->count; ++i) {
    const int* o = &st[(size_t)kBatchStats * i];
    mv += o[0];
    max_rs = std::max(max_rs, o[1]);
    rmv += o[3];
    fb += o[4];
    gs += o[5];
    if (o[2] == JTRLAN_OK) ++n_ok;
    else if (worst == JTRLAN_OK) worst = (jtrlan_status)o[2];
  }
  double phase[kBatchPhases] = {};
  if (b->prof) {
    std::vector<long long> pr((size_t)b->count * kBatchPhases);
    JB_CUDA(cudaMemcpy(pr.data(), b->prof, pr.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    double tot = 0.0;
    for (size_t q = 0; q < pr.size(); ++q) {
      phase[q % kBatchPhases] += (double)pr[q];
      tot += (double)pr[q];
    }
    for (int q = 0; q < kBatchPhases; ++q) phase[q] = tot > 0 ? phase[q] / tot : 0.0;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->count = b->count;
    stats->n_ok = n_ok;
    stats->n_matvec = mv;
    stats->n_resid_matvec = rmv;
    stats->max_restarts = max_rs;
    stats->solve_ms = ms;
    stats->grid = b->exec_grid;
    stats->threads = b->exec_threads;
    stats->graph = 1;
    stats->n_ritz_fallbacks = fb;
    stats->n_gs_passes = gs;
    for (int q = 0; q < kBatchPhases; ++q) stats->phase_frac[q] = phase[q];
  }
  if (worst != JTRLAN_OK) return bfail(worst, "at least one instance did not converge (see per-instance status)");
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_results(jtrlan_batch* b, double* evals, double* res, int* istats) {
  if (!b) return bfail(JTRLAN_EINVAL, "null batch");
  if (!b->solved) return bfail(JTRLAN_ESTATE, "no solve to report");
  const size_t ne = (size_t)b->count * b->nev;
  if (evals) JB_CUDA(cudaMemcpy(evals, b->out_ev, ne * sizeof(double), cudaMemcpyDeviceToHost));
  if (res) JB_CUDA(cudaMemcpy(res, b->out_res, ne * sizeof(double), cudaMemcpyDeviceToHost));
  if (istats)
    JB_CUDA(cudaMemcpy(istats, b->out_stats, (size_t)b->count * kBatchStats * sizeof(int), cudaMemcpyDeviceToHost));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_batch_vectors(jtrlan_batch* b, int i, void* evecs) {
  if (!b || !evecs) return bfail(JTRLAN_EINVAL, "null argument");
  if (i < 0 || i >= b->count) return bfail(JTRLAN_EINVAL, "instance index out of range");
  if (!b->solved) return bfail(JTRLAN_ESTATE, "no solve to report");
  int st[kBatchStats];
  JB_CUDA(cudaMemcpy(st, b->out_stats + (size_t)kBatchStats * i, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[2] != JTRLAN_OK) return bfail(JTRLAN_ESTATE, "instance did not converge");
  const size_t bytes = (size_t)(2 * b->h[i]) * b->nev * sizeof(double2);
  JB_CUDA(cudaMemcpy(evecs, (double2*)b->out_vec + b->vec_off[i], bytes, cudaMemcpyDefault));
  return JTRLAN_OK;
}

void jtrlan_batch_destroy(jtrlan_batch* b) { delete b; }

}  // extern "C"
