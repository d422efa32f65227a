// mlp.cu -- the 3-layer perceptron that maps cheap spectral features to the coefficients of the
// polynomial filter (the paper has no counterpart): forward pass, loss, back-propagation and Adam
// in FP32 CUDA kernels, with the full-batch training step held in a CUDA graph.
//
//   A1 = tanh(X W1^T + b1), A2 = tanh(A1 W2^T + b2), Y = A2 W3^T + b3
//   L  = mean over samples and outputs of (Y - T)^2
//   Adam: Kingma and Ba, "Adam: a method for stochastic optimization", ICLR 2015 (b1 = 0.9,
//   b2 = 0.999, eps = 1e-8).
// Packed parameters: W1 (H x F, row-major), b1, W2 (H x H), b2, W3 (O x H), b3.
// Every reduction runs in a fixed order, so results do not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "../../include/jtrlan.h"

using namespace jtr;

namespace {

constexpr int kT = 16;   // tile edge of the FP32 GEMM kernels

// Y[n][m] = act(sum_k X[n][k] W[m][k] + b[m]); act: 0 identity, 1 tanh.
__global__ void linear_fwd_kernel(const float* __restrict__ X, int N, int K, const float* __restrict__ W,
                                  const float* __restrict__ b, float* __restrict__ Y, int M, int act) {
  __shared__ float xs[kT][kT + 1], ws[kT][kT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int n = blockIdx.y * kT + ty, m = blockIdx.x * kT + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += kT) {
    const int nn = blockIdx.y * kT + ty, kk = k0 + tx;
    xs[ty][tx] = (nn < N && kk < K) ? X[(size_t)nn * K + kk] : 0.f;
    const int mm = blockIdx.x * kT + ty;
    ws[ty][tx] = (mm < M && kk < K) ? W[(size_t)mm * K + kk] : 0.f;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kT; ++q) acc = fmaf(xs[ty][q], ws[tx][q], acc);
    __syncthreads();
  }
  if (n < N && m < M) {
    const float z = acc + b[m];
    Y[(size_t)n * M + m] = act ? tanhf(z) : z;
  }
}

// D = 2 (Y - T) / (N O); per-block partial sums of (Y - T)^2 in FP64.
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T, int64_t count, float scale,
                            float* __restrict__ D, double* __restrict__ part) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256) {
    const float d = Y[i] - T[i];
    D[i] = scale * d;
    acc += (double)d * (double)d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += red[q];
    part[blockIdx.x] = s;
  }
}

// loss = sum(part) / count into *loss and, if hist, hist[*step] (step < cap).
__global__ void loss_final_kernel(const double* __restrict__ part, int nblk, int64_t count, double* loss,
                                  float* hist, const int* step, int cap) {
  double s = 0.0;
  for (int q = 0; q < nblk; ++q) s += part[q];
  s /= (double)count;
  *loss = s;
  if (hist && step && *step < cap) hist[*step] = (float)s;
}

// dW[m][k] = sum_n G[n][m] A[n][k] (and db[m] = sum_n G[n][m] from the blocks of column tile 0).
__global__ void grad_w_kernel(const float* __restrict__ G, const float* __restrict__ A, int N, int M, int K,
                              float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float gs[kT][kT + 1], as[kT][kT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m = blockIdx.y * kT + ty, k = blockIdx.x * kT + tx;
  float acc = 0.f, accb = 0.f;
  for (int n0 = 0; n0 < N; n0 += kT) {
    const int nn = n0 + ty;
    const int mm = blockIdx.y * kT + tx;
    gs[ty][tx] = (nn < N && mm < M) ? G[(size_t)nn * M + mm] : 0.f;   // gs[n][m]
    as[ty][tx] = (nn < N && k < K) ? A[(size_t)nn * K + k] : 0.f;     // as[n][k]
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kT; ++q) {
      acc = fmaf(gs[q][ty], as[q][tx], acc);
      accb += gs[q][ty];
    }
    __syncthreads();
  }
  if (m < M && k < K) dW[(size_t)m * K + k] = acc;
  if (blockIdx.x == 0 && tx == 0 && m < M) db[m] = accb;
}

// dZ[n][k] = (sum_m G[n][m] W[m][k]) (1 - A[n][k]^2): back through a linear layer and a tanh.
__global__ void grad_data_kernel(const float* __restrict__ G, const float* __restrict__ W, const float* __restrict__ A,
                                 int N, int M, int K, float* __restrict__ dZ) {
  __shared__ float gs[kT][kT + 1], ws[kT][kT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int n = blockIdx.y * kT + ty, k = blockIdx.x * kT + tx;
  float acc = 0.f;
  for (int m0 = 0; m0 < M; m0 += kT) {
    const int mm = m0 + tx;
    gs[ty][tx] = (n < N && mm < M) ? G[(size_t)n * M + mm] : 0.f;             // gs[n][m]
    const int mr = m0 + ty;
    ws[ty][tx] = (mr < M && k < K) ? W[(size_t)mr * K + k] : 0.f;             // ws[m][k]
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kT; ++q) acc = fmaf(gs[ty][q], ws[q][tx], acc);
    __syncthreads();
  }
  if (n < N && k < K) {
    const float a = A[(size_t)n * K + k];
    dZ[(size_t)n * K + k] = acc * (1.f - a * a);
  }
}

// Adam bias corrections for the next step: ++step; bc[0] = 1 - b1^t, bc[1] = 1 - b2^t.
__global__ void adam_prep_kernel(int* step, float* bc, float b1, float b2) {
  const int t = ++(*step);
  bc[0] = 1.f - powf(b1, (float)t);
  bc[1] = 1.f - powf(b2, (float)t);
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t P, const float* __restrict__ lr, const float* __restrict__ bc,
                            float b1, float b2, float eps) {
  const float l = *lr, c1 = bc[0], c2 = bc[1];
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < P; i += (int64_t)gridDim.x * 256) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= l * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Glorot-uniform weights from splitmix64 (Steele, Lea and Flood, OOPSLA 2014) on the parameter
// index; zero biases.
__global__ void init_kernel(float* th, int F, int H, int O, uint64_t seed) {
  const int64_t P = (int64_t)H * F + H + (int64_t)H * H + H + (int64_t)O * H + O;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < P; i += (int64_t)gridDim.x * 256) {
    int64_t r = i;
    int fan_in = 0, fan_out = 0;
    bool bias = false;
    if (r < (int64_t)H * F) { fan_in = F; fan_out = H; }
    else if ((r -= (int64_t)H * F) < H) bias = true;
    else if ((r -= H) < (int64_t)H * H) { fan_in = H; fan_out = H; }
    else if ((r -= (int64_t)H * H) < H) bias = true;
    else if ((r -= H) < (int64_t)O * H) { fan_in = H; fan_out = O; }
    else bias = true;
    if (bias) {
      th[i] = 0.f;
    } else {
      const double u = u01_sym(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));   // in [-1, 1)
      th[i] = (float)(u * sqrt(6.0 / (double)(fan_in + fan_out)));
    }
  }
}

jtrlan_status mfail(jtrlan_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

#define JM_CUDA(expr)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return mfail(e_ == cudaErrorMemoryAllocation ? JTRLAN_ENOMEM : JTRLAN_ECUDA,                 \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

#define JM_TRY(expr)                \
  do {                              \
    jtrlan_status s_ = (expr);      \
    if (s_ != JTRLAN_OK) return s_; \
  } while (0)

}  // namespace

struct jtrlan_mlp {
  int F = 0, H = 0, O = 0;
  int64_t P = 0;
  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ej = nullptr;
  float* theta = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* lr = nullptr;     // device scalar (so the graph needs no recapture for a new rate)
  float* bc = nullptr;     // Adam bias corrections
  int* step = nullptr;     // Adam step counter
  double* loss = nullptr;
  double* loss_part = nullptr;
  int loss_nblk = 0;
  int cap = 0;             // batch capacity of the workspaces
  float *A1 = nullptr, *A2 = nullptr, *Y = nullptr, *D = nullptr, *G2 = nullptr, *G1 = nullptr;
  float* hist = nullptr;
  int hist_cap = 0;
  cudaGraphExec_t exec = nullptr;
  const float* gX = nullptr;
  const float* gT = nullptr;
  int gN = 0;
  std::vector<void*> allocs;

  jtrlan_status dalloc(void** p, size_t bytes) {
    JM_CUDA(cudaMalloc(p, bytes ? bytes : 16));
    allocs.push_back(*p);
    return JTRLAN_OK;
  }
  void release(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) allocs.erase(it);
    cudaFree(p);
  }
  ~jtrlan_mlp() {
    if (own) cudaStreamSynchronize(own);
    if (exec) cudaGraphExecDestroy(exec);
    for (void* p : allocs) cudaFree(p);
    if (ej) cudaEventDestroy(ej);
    if (own) cudaStreamDestroy(own);
  }
};

namespace {

float* sub(float* th, const jtrlan_mlp* p, int which) {   // 0 W1, 1 b1, 2 W2, 3 b2, 4 W3, 5 b3
  const int64_t sz[6] = {(int64_t)p->H * p->F, p->H, (int64_t)p->H * p->H, p->H, (int64_t)p->O * p->H, p->O};
  int64_t off = 0;
  for (int q = 0; q < which; ++q) off += sz[q];
  return th + off;
}

jtrlan_status ensure_cap(jtrlan_mlp* p, int N) {
  if (N <= p->cap) return JTRLAN_OK;
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  for (float** b : {&p->A1, &p->A2, &p->Y, &p->D, &p->G2, &p->G1}) {
    p->release(*b);
    *b = nullptr;
  }
  p->release(p->loss_part);
  void* q = nullptr;
  JM_TRY(p->dalloc(&q, (size_t)N * p->H * sizeof(float))); p->A1 = (float*)q;
  JM_TRY(p->dalloc(&q, (size_t)N * p->H * sizeof(float))); p->A2 = (float*)q;
  JM_TRY(p->dalloc(&q, (size_t)N * p->O * sizeof(float))); p->Y = (float*)q;
  JM_TRY(p->dalloc(&q, (size_t)N * p->O * sizeof(float))); p->D = (float*)q;
  JM_TRY(p->dalloc(&q, (size_t)N * p->H * sizeof(float))); p->G2 = (float*)q;
  JM_TRY(p->dalloc(&q, (size_t)N * p->H * sizeof(float))); p->G1 = (float*)q;
  p->loss_nblk = (int)std::min<int64_t>(1024, ((int64_t)N * p->O + 255) / 256);
  JM_TRY(p->dalloc(&q, (size_t)p->loss_nblk * sizeof(double))); p->loss_part = (double*)q;
  p->cap = N;
  return JTRLAN_OK;
}

dim3 tiles(int cols, int rows) { return dim3((cols + kT - 1) / kT, (rows + kT - 1) / kT); }

cudaError_t enqueue_forward(jtrlan_mlp* p, const float* X, int N, float* Y, cudaStream_t s) {
  const dim3 b(kT, kT);
  linear_fwd_kernel<<<tiles(p->H, N), b, 0, s>>>(X, N, p->F, sub(p->theta, p, 0), sub(p->theta, p, 1), p->A1, p->H, 1);
  linear_fwd_kernel<<<tiles(p->H, N), b, 0, s>>>(p->A1, N, p->H, sub(p->theta, p, 2), sub(p->theta, p, 3), p->A2, p->H, 1);
  linear_fwd_kernel<<<tiles(p->O, N), b, 0, s>>>(p->A2, N, p->H, sub(p->theta, p, 4), sub(p->theta, p, 5), Y, p->O, 0);
  return cudaGetLastError();
}

// Loss and gradient of the batch into p->grad (forward pass included).
cudaError_t enqueue_gradient(jtrlan_mlp* p, const float* X, const float* T, int N, float* hist, int hist_cap,
                             cudaStream_t s) {
  const dim3 b(kT, kT);
  cudaError_t e = enqueue_forward(p, X, N, p->Y, s);
  if (e != cudaSuccess) return e;
  const int64_t cnt = (int64_t)N * p->O;
  loss_kernel<<<p->loss_nblk, 256, 0, s>>>(p->Y, T, cnt, 2.f / (float)cnt, p->D, p->loss_part);
  loss_final_kernel<<<1, 1, 0, s>>>(p->loss_part, p->loss_nblk, cnt, p->loss, hist, p->step, hist_cap);
  float* g = p->grad;
  grad_w_kernel<<<tiles(p->H, p->O), b, 0, s>>>(p->D, p->A2, N, p->O, p->H, sub(g, p, 4), sub(g, p, 5));
  grad_data_kernel<<<tiles(p->H, N), b, 0, s>>>(p->D, sub(p->theta, p, 4), p->A2, N, p->O, p->H, p->G2);
  grad_w_kernel<<<tiles(p->H, p->H), b, 0, s>>>(p->G2, p->A1, N, p->H, p->H, sub(g, p, 2), sub(g, p, 3));
  grad_data_kernel<<<tiles(p->H, N), b, 0, s>>>(p->G2, sub(p->theta, p, 2), p->A1, N, p->H, p->H, p->G1);
  grad_w_kernel<<<tiles(p->F, p->H), b, 0, s>>>(p->G1, X, N, p->H, p->F, sub(g, p, 0), sub(g, p, 1));
  return cudaGetLastError();
}

jtrlan_status order_after_user(jtrlan_mlp* p) {
  JM_CUDA(cudaEventRecord(p->ej, p->user));
  JM_CUDA(cudaStreamWaitEvent(p->own, p->ej, 0));
  return JTRLAN_OK;
}
jtrlan_status order_user_after(jtrlan_mlp* p) {
  JM_CUDA(cudaEventRecord(p->ej, p->own));
  JM_CUDA(cudaStreamWaitEvent(p->user, p->ej, 0));
  return JTRLAN_OK;
}

}  // namespace

extern "C" {

int64_t jtrlan_mlp_param_count(int n_in, int width, int n_out) {
  return (int64_t)width * n_in + width + (int64_t)width * width + width + (int64_t)n_out * width + n_out;
}

jtrlan_status jtrlan_mlp_create(int n_in, int width, int n_out, uint64_t seed, void* cuda_stream, jtrlan_mlp** out) {
  if (!out) return mfail(JTRLAN_EINVAL, "null out pointer");
  *out = nullptr;
  if (n_in < 1 || width < 1 || n_out < 1 || n_in > 4096 || width > 4096 || n_out > 4096)
    return mfail(JTRLAN_EINVAL, "layer sizes must be in 1..4096");
  jtrlan_mlp* p = new (std::nothrow) jtrlan_mlp();
  if (!p) return mfail(JTRLAN_ENOMEM, "host allocation failed");
  auto body = [&]() -> jtrlan_status {
    p->F = n_in;
    p->H = width;
    p->O = n_out;
    p->P = jtrlan_mlp_param_count(n_in, width, n_out);
    p->user = (cudaStream_t)cuda_stream;
    JM_CUDA(cudaStreamCreateWithFlags(&p->own, cudaStreamNonBlocking));
    JM_CUDA(cudaEventCreateWithFlags(&p->ej, cudaEventDisableTiming));
    void* q = nullptr;
    JM_TRY(p->dalloc(&q, (size_t)p->P * sizeof(float))); p->theta = (float*)q;
    JM_TRY(p->dalloc(&q, (size_t)p->P * sizeof(float))); p->grad = (float*)q;
    JM_TRY(p->dalloc(&q, (size_t)p->P * sizeof(float))); p->m = (float*)q;
    JM_TRY(p->dalloc(&q, (size_t)p->P * sizeof(float))); p->v = (float*)q;
    JM_TRY(p->dalloc(&q, 4 * sizeof(float))); p->lr = (float*)q;
    JM_TRY(p->dalloc(&q, 4 * sizeof(float))); p->bc = (float*)q;
    JM_TRY(p->dalloc(&q, 4 * sizeof(int))); p->step = (int*)q;
    JM_TRY(p->dalloc(&q, 2 * sizeof(double))); p->loss = (double*)q;
    JM_TRY(order_after_user(p));
    JM_CUDA(cudaMemsetAsync(p->m, 0, (size_t)p->P * sizeof(float), p->own));
    JM_CUDA(cudaMemsetAsync(p->v, 0, (size_t)p->P * sizeof(float), p->own));
    JM_CUDA(cudaMemsetAsync(p->step, 0, sizeof(int), p->own));
    init_kernel<<<(int)std::min<int64_t>(1024, (p->P + 255) / 256), 256, 0, p->own>>>(p->theta, n_in, width, n_out, seed);
    JM_CUDA(cudaGetLastError());
    JM_CUDA(cudaStreamSynchronize(p->own));
    return JTRLAN_OK;
  };
  jtrlan_status s = body();
  if (s != JTRLAN_OK) {
    delete p;
    return s;
  }
  *out = p;
  return JTRLAN_OK;
}

jtrlan_status jtrlan_mlp_get_params(jtrlan_mlp* p, float* theta) {
  if (!p || !theta) return mfail(JTRLAN_EINVAL, "null argument");
  JM_CUDA(cudaStreamSynchronize(p->own));
  JM_CUDA(cudaMemcpy(theta, p->theta, (size_t)p->P * sizeof(float), cudaMemcpyDefault));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_mlp_set_params(jtrlan_mlp* p, const float* theta) {
  if (!p || !theta) return mfail(JTRLAN_EINVAL, "null argument");
  JM_CUDA(cudaStreamSynchronize(p->own));
  JM_CUDA(cudaMemcpy(p->theta, theta, (size_t)p->P * sizeof(float), cudaMemcpyDefault));
  JM_CUDA(cudaMemset(p->m, 0, (size_t)p->P * sizeof(float)));
  JM_CUDA(cudaMemset(p->v, 0, (size_t)p->P * sizeof(float)));
  JM_CUDA(cudaMemset(p->step, 0, sizeof(int)));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_mlp_forward(jtrlan_mlp* p, const float* X, int N, float* Y) {
  if (!p || !X || !Y || N < 1) return mfail(JTRLAN_EINVAL, "null argument or N < 1");
  JM_TRY(ensure_cap(p, N));
  JM_TRY(order_after_user(p));
  JM_CUDA(enqueue_forward(p, X, N, Y, p->own));
  JM_TRY(order_user_after(p));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_mlp_gradient(jtrlan_mlp* p, const float* X, const float* T, int N, float* grad, double* loss) {
  if (!p || !X || !T || N < 1) return mfail(JTRLAN_EINVAL, "null argument or N < 1");
  JM_TRY(ensure_cap(p, N));
  JM_TRY(order_after_user(p));
  JM_CUDA(enqueue_gradient(p, X, T, N, nullptr, 0, p->own));
  JM_CUDA(cudaStreamSynchronize(p->own));
  if (grad) JM_CUDA(cudaMemcpy(grad, p->grad, (size_t)p->P * sizeof(float), cudaMemcpyDefault));
  if (loss) JM_CUDA(cudaMemcpy(loss, p->loss, sizeof(double), cudaMemcpyDeviceToHost));
  return JTRLAN_OK;
}

jtrlan_status jtrlan_mlp_train(jtrlan_mlp* p, const float* X, const float* T, int N, int steps, float lr,
                               float* loss_hist) {
  if (!p || !X || !T || N < 1 || steps < 0) return mfail(JTRLAN_EINVAL, "null argument, N < 1 or steps < 0");
  if (!(lr > 0.f)) return mfail(JTRLAN_EINVAL, "need lr > 0");
  JM_TRY(ensure_cap(p, N));
  // the step counter indexes the loss history, so the history must cover every step taken so far
  int done = 0;
  JM_CUDA(cudaMemcpy(&done, p->step, sizeof(int), cudaMemcpyDeviceToHost));
  const int need = done + steps;
  if (need > p->hist_cap) {
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    p->release(p->hist);
    void* q = nullptr;
    const int cap = std::max(need, 2 * p->hist_cap);
    JM_TRY(p->dalloc(&q, (size_t)cap * sizeof(float)));
    p->hist = (float*)q;
    p->hist_cap = cap;
  }
  if (!p->exec || p->gX != X || p->gT != T || p->gN != N) {   // one graph per (X, T, N)
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    JM_CUDA(cudaStreamBeginCapture(p->own, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = enqueue_gradient(p, X, T, N, p->hist, p->hist_cap, p->own);
    adam_prep_kernel<<<1, 1, 0, p->own>>>(p->step, p->bc, 0.9f, 0.999f);
    adam_kernel<<<(int)std::min<int64_t>(1024, (p->P + 255) / 256), 256, 0, p->own>>>(
        p->theta, p->grad, p->m, p->v, p->P, p->lr, p->bc, 0.9f, 0.999f, 1e-8f);
    cudaError_t e2 = cudaGetLastError();
    cudaError_t e3 = cudaStreamEndCapture(p->own, &g);
    JM_CUDA(e1);
    JM_CUDA(e2);
    JM_CUDA(e3);
    cudaError_t e4 = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    JM_CUDA(e4);
    p->gX = X;
    p->gT = T;
    p->gN = N;
  }
  JM_TRY(order_after_user(p));
  JM_CUDA(cudaMemcpyAsync(p->lr, &lr, sizeof(float), cudaMemcpyHostToDevice, p->own));
  JM_CUDA(cudaStreamSynchronize(p->own));   // lr is a stack value
  for (int i = 0; i < steps; ++i) JM_CUDA(cudaGraphLaunch(p->exec, p->own));
  JM_CUDA(cudaStreamSynchronize(p->own));
  if (loss_hist && steps > 0)
    JM_CUDA(cudaMemcpy(loss_hist, p->hist + done, (size_t)steps * sizeof(float), cudaMemcpyDeviceToHost));
  JM_TRY(order_user_after(p));
  return JTRLAN_OK;
}

void jtrlan_mlp_destroy(jtrlan_mlp* p) { delete p; }

}  // extern "C"
