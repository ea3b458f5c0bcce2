// Learned cost model: a multilayer perceptron 8 -> 64 -> 64 -> 64 -> 1 (ReLU
// hidden layers, linear output) that predicts the log latency of one operator
// of a micro-batch from eight batch features.  The paper's cost model is
// analytic (Eqs. 5-9); this network is trained on the engine's own timings and
// replaces Eq. 5's bytes / AvgThPut term in Alg. 1 when installed.
//
// Numerics: master weights in FP32; the forward and backward passes use the
// weights rounded to bf16 (round to nearest even) and accumulate in FP32.
// Loss = mean over the batch of (prediction - target)^2.  Training is Adam
// (beta1 0.9, beta2 0.999, eps 1e-8) on the master weights.
//
// Kernels (plain FMA: at most 4096 samples x 8.8K multiply-adds per step, far
// too little work for tensor cores to matter):
//   k_mlp_forward      one thread per sample, weights staged in shared memory;
//   k_mlp_grad_partial one thread per sample for forward + backward, then the
//                      CTA's 64 samples reduce into one partial gradient;
//   k_mlp_reduce_adam  sums the partial gradients in a fixed order
//                      (deterministic) and applies Adam, refreshing the bf16
//                      copy.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lmstream.h"

namespace {

constexpr int kIn = LMS_MLP_INPUTS, kH = LMS_MLP_HIDDEN;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + kH,
              kP = ob4 + 1;
static_assert(kP == LMS_MLP_PARAMS, "parameter layout");
constexpr int kSamplesPerCta = 64;  // training kernel
constexpr int kPad = kH + 1;        // shared-memory row pitch (conflict-free columns)

__device__ __forceinline__ void stage_weights(const __nv_bfloat16* __restrict__ wb, float* w) {
  for (int i = threadIdx.x; i < kP; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  __syncthreads();
}

__global__ void __launch_bounds__(128) k_mlp_forward(const __nv_bfloat16* __restrict__ wb,
                                                     const float* __restrict__ x, int n,
                                                     float* __restrict__ y) {
  extern __shared__ float w[];
  stage_weights(wb, w);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xi[kIn], h1[kH], h2[kH];
#pragma unroll
  for (int k = 0; k < kIn; ++k) xi[k] = x[i * kIn + k];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float a = w[ob1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(w[oW1 + j * kIn + k], xi[k], a);
    h1[j] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float a = w[ob2 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) a = fmaf(w[oW2 + j * kH + k], h1[k], a);
    h2[j] = fmaxf(a, 0.f);
  }
  float out = w[ob4];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float a = w[ob3 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) a = fmaf(w[oW3 + j * kH + k], h2[k], a);
    out = fmaf(w[oW4 + j], fmaxf(a, 0.f), out);
  }
  y[i] = out;
}

// Shared memory of the training kernel: weights, then per-sample rows of the
// input, the three hidden activations and the three hidden deltas.
constexpr size_t kTrainSmem =
    sizeof(float) * (kP + kSamplesPerCta * (kIn + 6 * kPad) + kSamplesPerCta);

__global__ void __launch_bounds__(kSamplesPerCta)
    k_mlp_grad_partial(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ x,
                       const float* __restrict__ t, int n, float* __restrict__ part,
                       float* __restrict__ loss_part) {
  extern __shared__ float sm[];
  float* w = sm;
  float* X = w + kP;                         // [64][8]
  float* A1 = X + kSamplesPerCta * kIn;      // [64][65] post-ReLU
  float* A2 = A1 + kSamplesPerCta * kPad;
  float* A3 = A2 + kSamplesPerCta * kPad;
  float* D1 = A3 + kSamplesPerCta * kPad;    // dL/d(pre-activation)
  float* D2 = D1 + kSamplesPerCta * kPad;
  float* D3 = D2 + kSamplesPerCta * kPad;
  float* DY = D3 + kSamplesPerCta * kPad;    // [64] dL/dy
  stage_weights(wb, w);
  const int s = threadIdx.x;
  const int i = blockIdx.x * kSamplesPerCta + s;
  const bool valid = i < n;
  float err = 0.f;
  // forward (invalid samples run on zeros and get a zero delta)
#pragma unroll
  for (int k = 0; k < kIn; ++k) X[s * kIn + k] = valid ? x[i * kIn + k] : 0.f;
  for (int j = 0; j < kH; ++j) {
    float a = w[ob1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(w[oW1 + j * kIn + k], X[s * kIn + k], a);
    A1[s * kPad + j] = fmaxf(a, 0.f);
  }
  for (int j = 0; j < kH; ++j) {
    float a = w[ob2 + j];
#pragma unroll 16
    for (int k = 0; k < kH; ++k) a = fmaf(w[oW2 + j * kH + k], A1[s * kPad + k], a);
    A2[s * kPad + j] = fmaxf(a, 0.f);
  }
  float yhat = w[ob4];
  for (int j = 0; j < kH; ++j) {
    float a = w[ob3 + j];
#pragma unroll 16
    for (int k = 0; k < kH; ++k) a = fmaf(w[oW3 + j * kH + k], A2[s * kPad + k], a);
    const float h = fmaxf(a, 0.f);
    A3[s * kPad + j] = h;
    yhat = fmaf(w[oW4 + j], h, yhat);
  }
  // backward: dL/dy = 2 (yhat - t) / n
  float dy = 0.f;
  if (valid) {
    err = yhat - t[i];
    dy = 2.f * err / (float)n;
  }
  DY[s] = dy;
  for (int j = 0; j < kH; ++j)
    D3[s * kPad + j] = A3[s * kPad + j] > 0.f ? dy * w[oW4 + j] : 0.f;
  for (int k = 0; k < kH; ++k) {
    float a = 0.f;
#pragma unroll 16
    for (int j = 0; j < kH; ++j) a = fmaf(w[oW3 + j * kH + k], D3[s * kPad + j], a);
    D2[s * kPad + k] = A2[s * kPad + k] > 0.f ? a : 0.f;
  }
  for (int k = 0; k < kH; ++k) {
    float a = 0.f;
#pragma unroll 16
    for (int j = 0; j < kH; ++j) a = fmaf(w[oW2 + j * kH + k], D2[s * kPad + j], a);
    D1[s * kPad + k] = A1[s * kPad + k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // the CTA's partial gradient: thread s owns output row j = s of every layer
  float* g = part + (size_t)blockIdx.x * kP;
  const int j = s;
  {
    float gb = 0.f, gw[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) gw[k] = 0.f;
    for (int r = 0; r < kSamplesPerCta; ++r) {
      const float d = D1[r * kPad + j];
      gb += d;
#pragma unroll
      for (int k = 0; k < kIn; ++k) gw[k] = fmaf(d, X[r * kIn + k], gw[k]);
    }
    g[ob1 + j] = gb;
#pragma unroll
    for (int k = 0; k < kIn; ++k) g[oW1 + j * kIn + k] = gw[k];
  }
  const float* Ds[2] = {D2, D3};
  const float* As[2] = {A1, A2};
  const int oW[2] = {oW2, oW3}, ob[2] = {ob2, ob3};
  for (int l = 0; l < 2; ++l) {
    const float* D = Ds[l];
    const float* A = As[l];
    float gb = 0.f;
    for (int k0 = 0; k0 < kH; k0 += 16) {
      float acc[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) acc[kk] = 0.f;
      for (int r = 0; r < kSamplesPerCta; ++r) {
        const float d = D[r * kPad + j];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc[kk] = fmaf(d, A[r * kPad + k0 + kk], acc[kk]);
      }
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) g[oW[l] + j * kH + k0 + kk] = acc[kk];
    }
    for (int r = 0; r < kSamplesPerCta; ++r) gb += D[r * kPad + j];
    g[ob[l] + j] = gb;
  }
  {
    float gw = 0.f;
    for (int r = 0; r < kSamplesPerCta; ++r) gw = fmaf(DY[r], A3[r * kPad + j], gw);
    g[oW4 + j] = gw;
  }
  if (s == 0) {
    float gb = 0.f;
    for (int r = 0; r < kSamplesPerCta; ++r) gb += DY[r];
    g[ob4] = gb;
  }
  // squared error of the CTA's samples (fixed-order sum)
  __syncthreads();
  DY[s] = err * err;
  __syncthreads();
  if (s == 0) {
    float acc = 0.f;
    for (int r = 0; r < kSamplesPerCta; ++r) acc += DY[r];
    loss_part[blockIdx.x] = acc;
  }
}

struct AdamArgs {
  float lr, b1, b2, omb1, omb2, eps, c1, c2;  // omb = 1 - b; c1 = 1 - b1^t, c2 = 1 - b2^t
  int apply;
};

__global__ void __launch_bounds__(256) k_mlp_reduce_adam(const float* __restrict__ part, int nblk,
                                                         float* __restrict__ grad,
                                                         float* __restrict__ master,
                                                         float* __restrict__ m, float* __restrict__ v,
                                                         __nv_bfloat16* __restrict__ wb,
                                                         AdamArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kP) return;
  float gsum = 0.f;
  for (int b = 0; b < nblk; ++b) gsum += part[(size_t)b * kP + p];
  grad[p] = gsum;
  if (!a.apply) return;
  const float mi = a.b1 * m[p] + a.omb1 * gsum;
  const float vi = a.b2 * v[p] + a.omb2 * gsum * gsum;
  m[p] = mi;
  v[p] = vi;
  const float mhat = mi / a.c1, vhat = vi / a.c2;
  const float w = master[p] - a.lr * mhat / (sqrtf(vhat) + a.eps);
  master[p] = w;
  wb[p] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_round(const float* __restrict__ master, __nv_bfloat16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kP) wb[p] = __float2bfloat16_rn(master[p]);
}

}  // namespace

struct lms_mlp {
  int dev = 0;
  cudaStream_t st = nullptr;
  std::mutex mu;
  float* master = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wb = nullptr;
  float* part = nullptr;      // [max_cta][kP]
  float* loss_part = nullptr; // [max_cta]
  float* x = nullptr;
  float* t = nullptr;
  float* y = nullptr;
  int cap = 0;                // samples the device buffers hold
  long long step = 0;         // Adam steps taken
  float* h_io = nullptr;      // pinned staging
};

namespace {

void mlp_free(lms_mlp* p) {
  cudaFree(p->part);
  cudaFree(p->loss_part);
  cudaFree(p->x);
  cudaFree(p->t);
  cudaFree(p->y);
  cudaFreeHost(p->h_io);
  p->part = p->loss_part = p->x = p->t = p->y = p->h_io = nullptr;
  p->cap = 0;
}

lms_status ensure_cap(lms_mlp* p, int n) {
  if (n <= p->cap) return LMS_OK;
  mlp_free(p);
  int c = 256;
  while (c < n) c <<= 1;
  const int nblk = (c + kSamplesPerCta - 1) / kSamplesPerCta;
  if (cudaMalloc(&p->part, sizeof(float) * kP * nblk) != cudaSuccess ||
      cudaMalloc(&p->loss_part, sizeof(float) * nblk) != cudaSuccess ||
      cudaMalloc(&p->x, sizeof(float) * kIn * c) != cudaSuccess ||
      cudaMalloc(&p->t, sizeof(float) * c) != cudaSuccess ||
      cudaMalloc(&p->y, sizeof(float) * c) != cudaSuccess ||
      cudaHostAlloc(&p->h_io, sizeof(float) * (kIn + 2) * c + sizeof(float) * (kP + nblk),
                    cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    mlp_free(p);
    return LMS_ENOMEM;
  }
  p->cap = c;
  return LMS_OK;
}

bool train_smem_ok() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] {
    ok = cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kTrainSmem) == cudaSuccess;
  });
  return ok;
}

// Enqueues forward+backward over the n samples at p->x / p->t and the reduce
// (and Adam step if apply).
lms_status enqueue_step(lms_mlp* p, int n, int apply, float lr) {
  const int nblk = (n + kSamplesPerCta - 1) / kSamplesPerCta;
  if (!train_smem_ok()) return LMS_ECUDA;
  k_mlp_grad_partial<<<nblk, kSamplesPerCta, kTrainSmem, p->st>>>(p->wb, p->x, p->t, n, p->part,
                                                                   p->loss_part);
  AdamArgs a{};
  a.lr = lr;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.omb1 = (float)(1.0 - 0.9);
  a.omb2 = (float)(1.0 - 0.999);
  a.eps = 1e-8f;
  a.apply = apply;
  if (apply) {
    p->step += 1;
    a.c1 = (float)(1.0 - std::pow(0.9, (double)p->step));
    a.c2 = (float)(1.0 - std::pow(0.999, (double)p->step));
  }
  k_mlp_reduce_adam<<<(kP + 255) / 256, 256, 0, p->st>>>(p->part, nblk, p->grad, p->master, p->m,
                                                         p->v, p->wb, a);
  return cudaGetLastError() == cudaSuccess ? LMS_OK : LMS_ECUDA;
}

}  // namespace

extern "C" {

lms_mlp* lms_mlp_create(int32_t device, const float* params) {
  lms_mlp* p = new lms_mlp();
  p->dev = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&p->master, sizeof(float) * kP) != cudaSuccess ||
      cudaMalloc(&p->m, sizeof(float) * kP) != cudaSuccess ||
      cudaMalloc(&p->v, sizeof(float) * kP) != cudaSuccess ||
      cudaMalloc(&p->grad, sizeof(float) * kP) != cudaSuccess ||
      cudaMalloc(&p->wb, sizeof(__nv_bfloat16) * kP) != cudaSuccess) {
    cudaGetLastError();
    lms_mlp_destroy(p);
    return nullptr;
  }
  if (lms_mlp_set_params(p, params) != LMS_OK) {
    lms_mlp_destroy(p);
    return nullptr;
  }
  return p;
}

void lms_mlp_destroy(lms_mlp* p) {
  if (!p) return;
  cudaSetDevice(p->dev);
  if (p->st) cudaStreamSynchronize(p->st);
  mlp_free(p);
  cudaFree(p->master);
  cudaFree(p->m);
  cudaFree(p->v);
  cudaFree(p->grad);
  cudaFree(p->wb);
  if (p->st) cudaStreamDestroy(p->st);
  delete p;
}

lms_status lms_mlp_set_params(lms_mlp* p, const float* params) {
  if (!p || !params) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (cudaSetDevice(p->dev) != cudaSuccess ||
      cudaMemcpyAsync(p->master, params, sizeof(float) * kP, cudaMemcpyHostToDevice, p->st) !=
          cudaSuccess ||
      cudaMemsetAsync(p->m, 0, sizeof(float) * kP, p->st) != cudaSuccess ||
      cudaMemsetAsync(p->v, 0, sizeof(float) * kP, p->st) != cudaSuccess)
    return LMS_ECUDA;
  k_mlp_round<<<(kP + 255) / 256, 256, 0, p->st>>>(p->master, p->wb);
  p->step = 0;
  return cudaStreamSynchronize(p->st) == cudaSuccess ? LMS_OK : LMS_ECUDA;
}

lms_status lms_mlp_get_params(lms_mlp* p, float* params) {
  if (!p || !params) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (cudaSetDevice(p->dev) != cudaSuccess ||
      cudaMemcpyAsync(params, p->master, sizeof(float) * kP, cudaMemcpyDeviceToHost, p->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(p->st) != cudaSuccess)
    return LMS_ECUDA;
  return LMS_OK;
}

lms_status lms_mlp_forward(lms_mlp* p, const float* x, int32_t n, float* y) {
  if (!p || n < 0 || (n > 0 && (!x || !y))) return LMS_EINVAL;
  if (n == 0) return LMS_OK;
  std::lock_guard<std::mutex> lk(p->mu);
  if (cudaSetDevice(p->dev) != cudaSuccess) return LMS_ECUDA;
  lms_status r = ensure_cap(p, n);
  if (r != LMS_OK) return r;
  std::memcpy(p->h_io, x, sizeof(float) * kIn * n);
  float* hy = p->h_io + (size_t)kIn * p->cap;
  if (cudaMemcpyAsync(p->x, p->h_io, sizeof(float) * kIn * n, cudaMemcpyHostToDevice, p->st) !=
      cudaSuccess)
    return LMS_ECUDA;
  k_mlp_forward<<<(n + 127) / 128, 128, sizeof(float) * kP, p->st>>>(p->wb, p->x, n, p->y);
  if (cudaMemcpyAsync(hy, p->y, sizeof(float) * n, cudaMemcpyDeviceToHost, p->st) != cudaSuccess ||
      cudaStreamSynchronize(p->st) != cudaSuccess)
    return LMS_ECUDA;
  std::memcpy(y, hy, sizeof(float) * n);
  return LMS_OK;
}

lms_status lms_mlp_train(lms_mlp* p, const float* x, const float* t, int32_t n, int32_t steps,
                         float lr, float* grad_out, float* loss_out) {
  if (!p || n < 1 || n > LMS_MLP_MAX_BATCH || steps < 0 || (!x || !t)) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (cudaSetDevice(p->dev) != cudaSuccess) return LMS_ECUDA;
  lms_status r = ensure_cap(p, n);
  if (r != LMS_OK) return r;
  std::memcpy(p->h_io, x, sizeof(float) * kIn * n);
  std::memcpy(p->h_io + (size_t)kIn * p->cap, t, sizeof(float) * n);
  if (cudaMemcpyAsync(p->x, p->h_io, sizeof(float) * kIn * n, cudaMemcpyHostToDevice, p->st) !=
          cudaSuccess ||
      cudaMemcpyAsync(p->t, p->h_io + (size_t)kIn * p->cap, sizeof(float) * n,
                      cudaMemcpyHostToDevice, p->st) != cudaSuccess)
    return LMS_ECUDA;
  // steps == 0: gradient and loss at the current weights only
  const int reps = steps == 0 ? 1 : steps;
  for (int s = 0; s < reps; ++s)
    if ((r = enqueue_step(p, n, steps == 0 ? 0 : 1, lr)) != LMS_OK) return r;
  const int nblk = (n + kSamplesPerCta - 1) / kSamplesPerCta;
  float* hg = p->h_io + (size_t)(kIn + 2) * p->cap;
  float* hl = hg + kP;
  if ((grad_out &&
       cudaMemcpyAsync(hg, p->grad, sizeof(float) * kP, cudaMemcpyDeviceToHost, p->st) !=
           cudaSuccess) ||
      cudaMemcpyAsync(hl, p->loss_part, sizeof(float) * nblk, cudaMemcpyDeviceToHost, p->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(p->st) != cudaSuccess)
    return LMS_ECUDA;
  if (grad_out) std::memcpy(grad_out, hg, sizeof(float) * kP);
  if (loss_out) {
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += hl[b];
    *loss_out = (float)(acc / n);
  }
  return LMS_OK;
}

}  // extern "C"
