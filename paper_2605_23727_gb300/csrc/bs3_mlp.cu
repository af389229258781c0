// Learned step-size proposer: dataset from step histories, training of the
// 6-32-32-1 tanh MLP on the GPU (per-sample forward/backward, Adam), and the
// full-batch gradient used to check training against the CPU oracle.
//
// Parameter layout (1313 binary32): W1 [32][6] row-major, b1 [32], W2 [32][32],
// b2 [32], W3 [32], b3.  A "model" is those 1313 values followed by the input
// standardisation: mean[6], std[6] (1325 binary32).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/bs3.h"
#include "bs3_mlp.cuh"

using namespace bs3;

namespace {

// One thread per sample: forward, squared-error backward, gradients summed in
// shared memory (then one atomic per parameter per block into grad).
__global__ void mlp_grad_kernel(const float* __restrict__ p, const float* __restrict__ X,
                                const float* __restrict__ y, const int* __restrict__ idx, int n, float inv_n,
                                float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float sp[kMlpParams];
  __shared__ float sg[kMlpParams];
  __shared__ float sl;
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) {
    sp[k] = p[k];
    sg[k] = 0.f;
  }
  if (threadIdx.x == 0) sl = 0.f;
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    const int row = idx ? idx[s] : s;
    const float* W1 = sp;
    const float* b1 = W1 + kMlpH * kMlpIn;
    const float* W2 = b1 + kMlpH;
    const float* b2 = W2 + kMlpH * kMlpH;
    const float* W3 = b2 + kMlpH;
    const float b3 = W3[kMlpH];
    float x[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = X[(size_t)row * kMlpIn + k];
    float h1[kMlpH], h2[kMlpH];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
      float a = b1[j];
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) a = fmaf(W1[j * kMlpIn + k], x[k], a);
      h1[j] = tanhf(a);
    }
    float out = b3;
#pragma unroll 4
    for (int j = 0; j < kMlpH; ++j) {
      float a = b2[j];
#pragma unroll
      for (int k = 0; k < kMlpH; ++k) a = fmaf(W2[j * kMlpH + k], h1[k], a);
      h2[j] = tanhf(a);
      out = fmaf(W3[j], h2[j], out);
    }
    const float r = out - y[row];
    atomicAdd(&sl, 0.5f * r * r * inv_n);
    const float go = r * inv_n;
    float* gW1 = sg;
    float* gb1 = gW1 + kMlpH * kMlpIn;
    float* gW2 = gb1 + kMlpH;
    float* gb2 = gW2 + kMlpH * kMlpH;
    float* gW3 = gb2 + kMlpH;
    atomicAdd(&gW3[kMlpH], go);
    float gh1[kMlpH];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) gh1[k] = 0.f;
#pragma unroll 4
    for (int j = 0; j < kMlpH; ++j) {
      atomicAdd(&gW3[j], go * h2[j]);
      const float ga2 = go * W3[j] * (1.f - h2[j] * h2[j]);
      atomicAdd(&gb2[j], ga2);
#pragma unroll
      for (int k = 0; k < kMlpH; ++k) {
        atomicAdd(&gW2[j * kMlpH + k], ga2 * h1[k]);
        gh1[k] = fmaf(ga2, W2[j * kMlpH + k], gh1[k]);
      }
    }
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
      const float ga1 = gh1[j] * (1.f - h1[j] * h1[j]);
      atomicAdd(&gb1[j], ga1);
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) atomicAdd(&gW1[j * kMlpIn + k], ga1 * x[k]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) atomicAdd(&grad[k], sg[k]);
  if (threadIdx.x == 0) atomicAdd(loss, sl);
}

// Adam (Kingma & Ba 2015), one thread per parameter; t counts from 1.
__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int t, float lr, float b1, float b2, float eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  const float mk = b1 * m[k] + (1.f - b1) * g[k];
  const float vk = b2 * v[k] + (1.f - b2) * g[k] * g[k];
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / (1.f - powf(b1, (float)t));
  const float vh = vk / (1.f - powf(b2, (float)t));
  p[k] -= lr * mh / (sqrtf(vh) + eps);
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

#define ML_CUDA(call)                               \
  do {                                              \
    if ((call) != cudaSuccess) { rc = BS3_ERR_CUDA; goto done; } \
  } while (0)

}  // namespace

extern "C" int bs3_mlp_dataset(const double* hist, int64_t n_rec, double rtol, float* X, float* y,
                               int64_t* n_out) {
  if (!hist || !X || !y || !n_out || n_rec < 0 || !(rtol > 0.0)) return BS3_ERR_INVALID_ARG;
  std::vector<int64_t> acc;
  for (int64_t r = 0; r < n_rec; ++r)
    if (hist[r * 8 + 3] > 0.5) acc.push_back(r);
  std::vector<double> errs;
  int64_t n = 0;
  for (size_t a = 0; a + 1 < acc.size(); ++a) {
    const double* cur = hist + acc[a] * 8;
    const double* nxt = hist + acc[a + 1] * 8;
    errs.push_back(cur[2]);
    double f[kMlpIn];
    mlp_features(errs.data(), (int)errs.size(), cur[1], rtol, f);
    const double r_next = std::min(std::max(nxt[2] / rtol, kMlpRClamp), 1.0 / kMlpRClamp);
    const double h_star = nxt[1] * std::cbrt(kMlpTheta / r_next);
    for (int k = 0; k < kMlpIn; ++k) X[n * kMlpIn + k] = (float)f[k];
    y[n] = (float)std::log(h_star / cur[1]);
    ++n;
  }
  *n_out = n;
  return BS3_OK;
}

extern "C" int bs3_mlp_grad(const float* params, const float* X, const float* y, int64_t n, float* grad_out,
                            float* loss_out) {
  if (!params || !X || !y || !grad_out || !loss_out || n < 1 || n > (1ll << 30)) return BS3_ERR_INVALID_ARG;
  int rc = BS3_OK;
  float *dp = nullptr, *dX = nullptr, *dy = nullptr, *dg = nullptr, *dl = nullptr;
  ML_CUDA(cudaMalloc(&dp, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMalloc(&dX, n * kMlpIn * sizeof(float)));
  ML_CUDA(cudaMalloc(&dy, n * sizeof(float)));
  ML_CUDA(cudaMalloc(&dg, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMalloc(&dl, sizeof(float)));
  ML_CUDA(cudaMemcpy(dp, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice));
  ML_CUDA(cudaMemcpy(dX, X, n * kMlpIn * sizeof(float), cudaMemcpyHostToDevice));
  ML_CUDA(cudaMemcpy(dy, y, n * sizeof(float), cudaMemcpyHostToDevice));
  ML_CUDA(cudaMemset(dg, 0, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMemset(dl, 0, sizeof(float)));
  mlp_grad_kernel<<<(unsigned)((n + 127) / 128), 128>>>(dp, dX, dy, nullptr, (int)n, 1.f / (float)n, dg, dl);
  ML_CUDA(cudaGetLastError());
  ML_CUDA(cudaMemcpy(grad_out, dg, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  ML_CUDA(cudaMemcpy(loss_out, dl, sizeof(float), cudaMemcpyDeviceToHost));
done:
  cudaFree(dp); cudaFree(dX); cudaFree(dy); cudaFree(dg); cudaFree(dl);
  return rc;
}

extern "C" int bs3_mlp_train(const float* X_raw, const float* y, int64_t n, const float* params_init, int epochs,
                             int batch, float lr, uint64_t seed, float* model_out, float* loss_hist) {
  if (!X_raw || !y || !params_init || !model_out || n < 2 || epochs < 1 || batch < 1 || !(lr > 0.f))
    return BS3_ERR_INVALID_ARG;
  // input standardisation (mean, std per feature, binary64 sums)
  float mean[kMlpIn], stdv[kMlpIn];
  for (int k = 0; k < kMlpIn; ++k) {
    double s = 0.0, s2 = 0.0;
    for (int64_t r = 0; r < n; ++r) s += X_raw[r * kMlpIn + k];
    const double mu = s / (double)n;
    for (int64_t r = 0; r < n; ++r) {
      const double d = X_raw[r * kMlpIn + k] - mu;
      s2 += d * d;
    }
    const double sd = std::sqrt(s2 / (double)n);
    mean[k] = (float)mu;
    stdv[k] = (float)(sd > 1e-6 ? sd : 1.0);
  }
  std::vector<float> Xs((size_t)n * kMlpIn);
  for (int64_t r = 0; r < n; ++r)
    for (int k = 0; k < kMlpIn; ++k) Xs[r * kMlpIn + k] = (X_raw[r * kMlpIn + k] - mean[k]) / stdv[k];
  int rc = BS3_OK;
  float *dp = nullptr, *dX = nullptr, *dy = nullptr, *dg = nullptr, *dl = nullptr, *dm = nullptr, *dv = nullptr;
  int* didx = nullptr;
  std::vector<int> perm(n);
  uint64_t st = seed;
  int t = 0;
  ML_CUDA(cudaMalloc(&dp, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMalloc(&dg, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMalloc(&dm, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMalloc(&dv, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMalloc(&dl, sizeof(float)));
  ML_CUDA(cudaMalloc(&dX, n * kMlpIn * sizeof(float)));
  ML_CUDA(cudaMalloc(&dy, n * sizeof(float)));
  ML_CUDA(cudaMalloc(&didx, n * sizeof(int)));
  ML_CUDA(cudaMemcpy(dp, params_init, kMlpParams * sizeof(float), cudaMemcpyHostToDevice));
  ML_CUDA(cudaMemcpy(dX, Xs.data(), n * kMlpIn * sizeof(float), cudaMemcpyHostToDevice));
  ML_CUDA(cudaMemcpy(dy, y, n * sizeof(float), cudaMemcpyHostToDevice));
  ML_CUDA(cudaMemset(dm, 0, kMlpParams * sizeof(float)));
  ML_CUDA(cudaMemset(dv, 0, kMlpParams * sizeof(float)));
  for (int64_t r = 0; r < n; ++r) perm[r] = (int)r;
  for (int e = 0; e < epochs; ++e) {
    for (int64_t r = n - 1; r > 0; --r) std::swap(perm[r], perm[splitmix64(st) % (uint64_t)(r + 1)]);
    ML_CUDA(cudaMemcpy(didx, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    ML_CUDA(cudaMemset(dl, 0, sizeof(float)));
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int nb = (int)std::min<int64_t>(batch, n - b0);
      ML_CUDA(cudaMemsetAsync(dg, 0, kMlpParams * sizeof(float)));
      mlp_grad_kernel<<<(unsigned)((nb + 127) / 128), 128>>>(dp, dX, dy, didx + b0, nb, 1.f / (float)nb, dg,
                                                              dl);
      mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256>>>(dp, dg, dm, dv, ++t, lr, 0.9f, 0.999f, 1e-8f);
    }
    ML_CUDA(cudaGetLastError());
    if (loss_hist) {
      float l = 0.f;
      ML_CUDA(cudaMemcpy(&l, dl, sizeof(float), cudaMemcpyDeviceToHost));
      loss_hist[e] = l * (float)batch / (float)n;   // mean of the minibatch losses
    }
  }
  ML_CUDA(cudaMemcpy(model_out, dp, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  std::memcpy(model_out + kMlpParams, mean, sizeof(mean));
  std::memcpy(model_out + kMlpParams + kMlpIn, stdv, sizeof(stdv));
done:
  cudaFree(dp); cudaFree(dg); cudaFree(dm); cudaFree(dv); cudaFree(dl); cudaFree(dX); cudaFree(dy); cudaFree(didx);
  return rc;
}
