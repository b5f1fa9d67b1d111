// Learned tile proposer: a 3-layer ReLU MLP that scores every configuration
// of the GEMM autotuner's single-pass class for a shape (features: log2 M,
// log2 N, log2 K and a one-hot dtype), trained on the GPU by this file's
// kernels on the autotuner's own measurements (target: TFLOP/s of the config
// over the best TFLOP/s of the shape). The proposal is the arg-max config;
// the exhaustive autotuner over the same class stays the fallback for low
// scores and shapes outside the trained range. Every config of that class
// computes each C element as one K-ordered accumulation by one program, so
// whichever config the proposal or its fallback picks, C is bit-identical:
// the proposal never changes numerics. Split-K configs, which round
// differently, are outside the class and never proposed.
//
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3
//   L  = sum V (y - T)^2 / max(1, sum V)      (V masks invalid configs)
//   Adam with bias correction.
// Parameters are one contiguous fp32 buffer [W1, b1, W2, b2, W3, b3] (row-
// major [out, in] matrices). Every reduction runs in a fixed order, so
// training is deterministic.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "tp_internal.h"

struct tp_mlp {
  tp_ctx* ctx = nullptr;
  int32_t in = 0, hidden = 0, out = 0, max_batch = 0;
  int64_t nparams = 0;
  int64_t step = 0;
  float* params = nullptr;  // device
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* z1 = nullptr;      // [B, H] pre-activations
  float* z2 = nullptr;
  float* y = nullptr;       // [B, C]
  float* dy = nullptr;
  float* dz1 = nullptr;
  float* dz2 = nullptr;
  float* xbuf = nullptr;    // [B, in] features (propose)
};

namespace tp {
namespace {

struct Off {
  int64_t w1, b1, w2, b2, w3, b3, n;
};

__host__ __device__ inline Off offsets(int F, int H, int C) {
  Off o;
  o.w1 = 0;
  o.b1 = o.w1 + (int64_t)H * F;
  o.w2 = o.b1 + H;
  o.b2 = o.w2 + (int64_t)H * H;
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + (int64_t)C * H;
  o.n = o.b3 + C;
  return o;
}

// One block per row; thread j computes hidden unit j (blockDim >= max(H, C)).
__global__ void forward_kernel(const float* __restrict__ P, const float* __restrict__ X, int B, int F, int H, int C,
                               float* z1, float* z2, float* Y) {
  extern __shared__ float sh[];
  float* h1 = sh;
  float* h2 = sh + H;
  const Off o = offsets(F, H, C);
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  const float* x = X + (int64_t)b * F;
  if (j < H) {
    float s = P[o.b1 + j];
    for (int f = 0; f < F; ++f) s = fmaf(P[o.w1 + (int64_t)j * F + f], x[f], s);
    z1[(int64_t)b * H + j] = s;
    h1[j] = fmaxf(s, 0.f);
  }
  __syncthreads();
  if (j < H) {
    float s = P[o.b2 + j];
    for (int i = 0; i < H; ++i) s = fmaf(P[o.w2 + (int64_t)j * H + i], h1[i], s);
    z2[(int64_t)b * H + j] = s;
    h2[j] = fmaxf(s, 0.f);
  }
  __syncthreads();
  if (j < C) {
    float s = P[o.b3 + j];
    for (int i = 0; i < H; ++i) s = fmaf(P[o.w3 + (int64_t)j * H + i], h2[i], s);
    Y[(int64_t)b * C + j] = s;
  }
}

// dY = 2 V (Y - T) / max(1, sum V) and the loss, by one block (fixed order).
__global__ void loss_kernel(const float* Y, const float* T, const float* V, int64_t n, float* dY, float* loss) {
  __shared__ float red[2][32];
  float sv = 0.f, se = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = Y[i] - T[i];
    sv += V[i];
    se = fmaf(V[i] * d, d, se);
  }
  for (int off = 16; off > 0; off >>= 1) {
    sv += __shfl_xor_sync(0xffffffffu, sv, off);
    se += __shfl_xor_sync(0xffffffffu, se, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x / 32] = sv;
    red[1][threadIdx.x / 32] = se;
  }
  __syncthreads();
  float tv = 0.f, te = 0.f;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
    tv += red[0][w];
    te += red[1][w];
  }
  const float den = fmaxf(1.f, tv);
  if (threadIdx.x == 0 && loss) *loss = te / den;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dY[i] = 2.f * V[i] * (Y[i] - T[i]) / den;
}

// Per row: dz2 = (dY W3) * (z2 > 0), dz1 = (dz2 W2) * (z1 > 0).
__global__ void backprop_rows_kernel(const float* __restrict__ P, int B, int F, int H, int C, const float* dY,
                                     const float* z1, const float* z2, float* dz1, float* dz2) {
  extern __shared__ float sh[];
  const Off o = offsets(F, H, C);
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  float* d2 = sh;
  if (j < H) {
    float s = 0.f;
    for (int c = 0; c < C; ++c) s = fmaf(dY[(int64_t)b * C + c], P[o.w3 + (int64_t)c * H + j], s);
    const float g = z2[(int64_t)b * H + j] > 0.f ? s : 0.f;
    dz2[(int64_t)b * H + j] = g;
    d2[j] = g;
  }
  __syncthreads();
  if (j < H) {
    float s = 0.f;
    for (int i = 0; i < H; ++i) s = fmaf(d2[i], P[o.w2 + (int64_t)i * H + j], s);
    dz1[(int64_t)b * H + j] = z1[(int64_t)b * H + j] > 0.f ? s : 0.f;
  }
}

// One thread per parameter: its gradient summed over the batch in row order.
__global__ void param_grad_kernel(int B, int F, int H, int C, const float* X, const float* z1, const float* z2,
                                  const float* dY, const float* dz1, const float* dz2, float* G) {
  const Off o = offsets(F, H, C);
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= o.n) return;
  float s = 0.f;
  if (p < o.b1) {  // W1[j][f] = sum dz1[b][j] x[b][f]
    const int64_t j = p / F, f = p % F;
    for (int b = 0; b < B; ++b) s = fmaf(dz1[(int64_t)b * H + j], X[(int64_t)b * F + f], s);
  } else if (p < o.w2) {
    const int64_t j = p - o.b1;
    for (int b = 0; b < B; ++b) s += dz1[(int64_t)b * H + j];
  } else if (p < o.b2) {  // W2[j][i] = sum dz2[b][j] relu(z1[b][i])
    const int64_t q = p - o.w2, j = q / H, i = q % H;
    for (int b = 0; b < B; ++b) s = fmaf(dz2[(int64_t)b * H + j], fmaxf(z1[(int64_t)b * H + i], 0.f), s);
  } else if (p < o.w3) {
    const int64_t j = p - o.b2;
    for (int b = 0; b < B; ++b) s += dz2[(int64_t)b * H + j];
  } else if (p < o.b3) {  // W3[c][i] = sum dY[b][c] relu(z2[b][i])
    const int64_t q = p - o.w3, c = q / H, i = q % H;
    for (int b = 0; b < B; ++b) s = fmaf(dY[(int64_t)b * C + c], fmaxf(z2[(int64_t)b * H + i], 0.f), s);
  } else {
    const int64_t c = p - o.b3;
    for (int b = 0; b < B; ++b) s += dY[(int64_t)b * C + c];
  }
  G[p] = s;
}

__global__ void adam_kernel(float* P, const float* G, float* M, float* V, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

tp_status launch_forward(tp_mlp* n, const float* X, int B, cudaStream_t st) {
  const int threads = ((std::max(n->hidden, n->out) + 31) / 32) * 32;
  forward_kernel<<<B, threads, 2 * n->hidden * sizeof(float), st>>>(n->params, X, B, n->in, n->hidden, n->out,
                                                                    n->z1, n->z2, n->y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "mlp forward");
}

tp_status launch_loss_grad(tp_mlp* n, const float* X, const float* T, const float* V, int B, float* loss,
                           cudaStream_t st) {
  tp_status s = launch_forward(n, X, B, st);
  if (s != TP_OK) return s;
  loss_kernel<<<1, 1024, 0, st>>>(n->y, T, V, (int64_t)B * n->out, n->dy, loss);
  const int threads = ((n->hidden + 31) / 32) * 32;
  backprop_rows_kernel<<<B, threads, n->hidden * sizeof(float), st>>>(n->params, B, n->in, n->hidden, n->out, n->dy,
                                                                     n->z1, n->z2, n->dz1, n->dz2);
  param_grad_kernel<<<(unsigned)((n->nparams + 255) / 256), 256, 0, st>>>(B, n->in, n->hidden, n->out, X, n->z1,
                                                                          n->z2, n->dy, n->dz1, n->dz2, n->grads);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "mlp backward");
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

tp_status tp_mlp_create(tp_ctx* ctx, int32_t in, int32_t hidden, int32_t out, int32_t max_batch,
                        const float* init_params, tp_mlp** mlp) {
  if (!ctx || !mlp || !init_params) return fail(TP_ERR_INVALID, "null argument");
  *mlp = nullptr;
  DeviceGuard guard(ctx);
  if (in < 1 || hidden < 1 || out < 1 || hidden > 1024 || out > 1024 || max_batch < 1)
    return fail(TP_ERR_INVALID, "need 1 <= in, 1 <= hidden, out <= 1024, max_batch >= 1");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->capturing) return fail(TP_ERR_CAPTURE, "creating an MLP allocates device memory");
  }
  auto* n = new tp_mlp();
  n->ctx = ctx;
  n->in = in;
  n->hidden = hidden;
  n->out = out;
  n->max_batch = max_batch;
  n->nparams = offsets(in, hidden, out).n;
  const size_t P = n->nparams * sizeof(float), BH = (size_t)max_batch * hidden * sizeof(float),
               BC = (size_t)max_batch * out * sizeof(float);
  cudaError_t e = cudaSuccess;
  for (auto pr : {std::make_pair(&n->params, P), std::make_pair(&n->grads, P), std::make_pair(&n->m, P),
                  std::make_pair(&n->v, P), std::make_pair(&n->z1, BH), std::make_pair(&n->z2, BH),
                  std::make_pair(&n->y, BC), std::make_pair(&n->dy, BC), std::make_pair(&n->dz1, BH),
                  std::make_pair(&n->dz2, BH), std::make_pair(&n->xbuf, (size_t)max_batch * in * sizeof(float))})
    if (e == cudaSuccess) e = cudaMalloc(pr.first, pr.second);
  if (e == cudaSuccess) e = cudaMemcpy(n->params, init_params, P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, P);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, P);
  if (e != cudaSuccess) {
    for (float* p : {n->params, n->grads, n->m, n->v, n->z1, n->z2, n->y, n->dy, n->dz1, n->dz2, n->xbuf}) cudaFree(p);
    delete n;
    return cuda_fail(e, "allocating the MLP");
  }
  *mlp = n;
  return TP_OK;
}

tp_status tp_mlp_destroy(tp_mlp* n) {
  if (!n) return fail(TP_ERR_INVALID, "null mlp");
  for (float* p : {n->params, n->grads, n->m, n->v, n->z1, n->z2, n->y, n->dy, n->dz1, n->dz2, n->xbuf}) cudaFree(p);
  delete n;
  return TP_OK;
}

tp_status tp_mlp_num_params(const tp_mlp* n, int64_t* count) {
  if (!n || !count) return fail(TP_ERR_INVALID, "null argument");
  *count = n->nparams;
  return TP_OK;
}

tp_status tp_mlp_get_params(const tp_mlp* n, float* host_out) {
  if (!n || !host_out) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  cudaError_t e = cudaMemcpy(host_out, n->params, n->nparams * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "reading MLP parameters");
}

tp_status tp_mlp_set_params(tp_mlp* n, const float* host_in) {
  if (!n || !host_in) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  cudaError_t e = cudaMemcpy(n->params, host_in, n->nparams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, n->nparams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, n->nparams * sizeof(float));
  n->step = 0;
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "writing MLP parameters");
}

tp_status tp_mlp_forward(tp_mlp* n, const float* X, int32_t batch, float* Y, const tp_exec* ex) {
  if (!n || !X || !Y || !ex) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  if (batch < 1 || batch > n->max_batch) return fail(TP_ERR_SHAPE, "batch must be 1..max_batch");
  cudaStream_t st = static_cast<cudaStream_t>(ex->stream);
  tp_status s = launch_forward(n, X, batch, st);
  if (s != TP_OK) return s;
  cudaError_t e = cudaMemcpyAsync(Y, n->y, (size_t)batch * n->out * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && ex->mode == TP_SYNC) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "mlp forward output");
}

tp_status tp_mlp_loss_grad(tp_mlp* n, const float* X, const float* T, const float* V, int32_t batch, float* loss,
                           float* grads, const tp_exec* ex) {
  if (!n || !X || !T || !V || !ex) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  if (batch < 1 || batch > n->max_batch) return fail(TP_ERR_SHAPE, "batch must be 1..max_batch");
  cudaStream_t st = static_cast<cudaStream_t>(ex->stream);
  tp_status s = launch_loss_grad(n, X, T, V, batch, loss, st);
  if (s != TP_OK) return s;
  cudaError_t e = cudaSuccess;
  if (grads) e = cudaMemcpyAsync(grads, n->grads, n->nparams * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && ex->mode == TP_SYNC) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "mlp gradients");
}

tp_status tp_mlp_train_step(tp_mlp* n, const float* X, const float* T, const float* V, int32_t batch, float lr,
                            float* loss, const tp_exec* ex) {
  if (!n || !X || !T || !V || !ex) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  if (batch < 1 || batch > n->max_batch) return fail(TP_ERR_SHAPE, "batch must be 1..max_batch");
  cudaStream_t st = static_cast<cudaStream_t>(ex->stream);
  tp_status s = launch_loss_grad(n, X, T, V, batch, loss, st);
  if (s != TP_OK) return s;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow(0.9, (double)n->step), c2 = 1.f - (float)std::pow(0.999, (double)n->step);
  adam_kernel<<<(unsigned)((n->nparams + 255) / 256), 256, 0, st>>>(n->params, n->grads, n->m, n->v, n->nparams, lr,
                                                                  b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && ex->mode == TP_SYNC) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? TP_OK : cuda_fail(e, "mlp train step");
}

tp_status tp_mlp_save(const tp_mlp* n, const char* path) {
  if (!n || !path) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  std::vector<float> h(n->nparams);
  tp_status s = tp_mlp_get_params(n, h.data());
  if (s != TP_OK) return s;
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(TP_ERR_INVALID, std::string("cannot write ") + path);
  std::fprintf(f, "tp-mlp v1 %d %d %d\n", n->in, n->hidden, n->out);
  for (float v : h) std::fprintf(f, "%.9g\n", v);
  std::fclose(f);
  return TP_OK;
}

tp_status tp_mlp_load(tp_mlp* n, const char* path) {
  if (!n || !path) return fail(TP_ERR_INVALID, "null argument");
  DeviceGuard guard(n->ctx);
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(TP_ERR_INVALID, std::string("cannot read ") + path);
  int a = 0, b = 0, c = 0;
  if (std::fscanf(f, "tp-mlp v1 %d %d %d", &a, &b, &c) != 3 || a != n->in || b != n->hidden || c != n->out) {
    std::fclose(f);
    return fail(TP_ERR_SHAPE, "MLP file does not match this network");
  }
  std::vector<float> h(n->nparams);
  for (auto& v : h)
    if (std::fscanf(f, "%f", &v) != 1) {
      std::fclose(f);
      return fail(TP_ERR_INVALID, "truncated MLP file");
    }
  std::fclose(f);
  return tp_mlp_set_params(n, h.data());
}

tp_status tp_mlp_features(int64_t M, int64_t N, int64_t K, int32_t dtype, float* out) {
  if (!out) return fail(TP_ERR_INVALID, "null output");
  if (M < 1 || N < 1 || K < 1) return fail(TP_ERR_SHAPE, "dimensions must be >= 1");
  if (dtype != TP_BF16 && dtype != TP_F8E4M3) return fail(TP_ERR_UNSUPPORTED, "dtype must be BF16 or F8E4M3");
  out[0] = (float)std::log2((double)M);
  out[1] = (float)std::log2((double)N);
  out[2] = (float)std::log2((double)K);
  out[3] = dtype == TP_BF16 ? 1.f : 0.f;
  out[4] = dtype == TP_BF16 ? 0.f : 1.f;
  return TP_OK;
}

tp_status tp_mlp_targets(const float* tflops, int32_t count, float* target, float* mask) {
  if (!tflops || !target || !mask || count < 1) return fail(TP_ERR_INVALID, "null argument or empty table");
  float best = 0.f;
  for (int i = 0; i < count; ++i) best = std::max(best, tflops[i]);
  // a config that did not run on the shape is its worst proposal: target 0,
  // still trained (an untrained output could otherwise win the arg-max)
  for (int i = 0; i < count; ++i) {
    mask[i] = best > 0.f ? 1.f : 0.f;
    target[i] = best > 0.f ? std::max(tflops[i], 0.f) / best : 0.f;
  }
  return TP_OK;
}

tp_status tp_propose(tp_ctx* ctx, tp_mlp* n, int64_t M, int64_t N, int64_t K, int32_t dtype, float min_score,
                     tp_gemm_config* out, float* score, int32_t* used_fallback) {
  if (!ctx || !n || !out) return fail(TP_ERR_INVALID, "null argument");
  if (n->in != 5) return fail(TP_ERR_SHAPE, "the proposer takes 5 features");
  int32_t count = 0;
  tp_status s = tp_autotune_space(dtype, 0, nullptr, 0, &count);
  if (s != TP_OK) return s;
  if (count != n->out) return fail(TP_ERR_SHAPE, "MLP outputs differ from the autotuner's single-pass config count");
  std::vector<tp_gemm_config> cfgs(count);
  tp_autotune_space(dtype, 0, cfgs.data(), count, &count);
  float x[5];
  s = tp_mlp_features(M, N, K, dtype, x);
  if (s != TP_OK) return s;
  cudaError_t e = cudaMemcpy(n->xbuf, x, sizeof(x), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "proposer features");
  s = launch_forward(n, n->xbuf, 1, nullptr);
  if (s != TP_OK) return s;
  std::vector<float> y(count);
  e = cudaMemcpy(y.data(), n->y, count * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "proposer scores");
  // arg-max over the single-pass configs the autotuner would try on this
  // shape (ties keep the lower index)
  int best = -1;
  for (int i = 0; i < count; ++i)
    if (autotune_config_runs(ctx, M, N, K, dtype, cfgs[i]) && (best < 0 || y[i] > y[best])) best = i;
  if (best < 0) return fail(TP_ERR_UNSUPPORTED, "no config of the space runs on this shape");
  const bool in_range = M <= 16384 && N <= 16384 && K <= 16384;
  if (score) *score = y[best];
  if (y[best] >= min_score && in_range) {
    *out = cfgs[best];
    if (used_fallback) *used_fallback = 0;
    return TP_OK;
  }
  if (used_fallback) *used_fallback = 1;
  int32_t found = 0;
  s = tp_autotune_lookup(ctx, M, N, K, dtype, 0, out, &found);
  if (s != TP_OK || found) return s;
  return tp_autotune(ctx, M, N, K, dtype, 0, 0, out, nullptr, nullptr);
}

}  // extern "C"
