// Learned step-size proposer shared by the trainer (bs3_mlp.cu) and the
// solver's controller (bs3_solver.cuh): sizes, features and the warp-level
// bfloat16 inference.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace bs3 {

constexpr int kMlpIn = 6, kMlpH = 32;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;   // 1313
constexpr int kMlpModel = kMlpParams + 2 * kMlpIn;                                        // + mean, std
constexpr double kMlpTheta = 0.75;       // target E / Rel of the training targets
constexpr double kMlpRClamp = 1e-8;      // E / Rel clamped to [1e-8, 1e8] before the log
constexpr double kMlpDMin = -1.6094379124341003;   // log(0.2)
constexpr double kMlpDMax = 1.6094379124341003;    // log(5)

// Features of an accepted step from the errors of the last accepted steps
// (errs[0..n-1], chronological, n >= 1; only the last 4 are used and missing
// ones repeat the oldest): [log r x4, log h, log Rel], r = clamp(E / Rel).
__host__ __device__ inline void mlp_features(const double* errs, int n, double h, double rtol, double* f) {
  double r[4];
  const int m = n < 4 ? n : 4;
  for (int k = 0; k < m; ++k) {
    double q = errs[n - m + k] / rtol;
    q = q < kMlpRClamp ? kMlpRClamp : (q > 1.0 / kMlpRClamp ? 1.0 / kMlpRClamp : q);
    r[4 - m + k] = q;
  }
  for (int k = 0; k < 4 - m; ++k) r[k] = r[4 - m];
  for (int k = 0; k < 4; ++k) f[k] = log(r[k]);
  f[4] = log(h);
  f[5] = log(rtol);
}

// Forward pass by one warp (lane j = hidden unit j); w holds the bfloat16-
// rounded parameters as binary32 in the layout W1, b1, W2, b2, W3, b3.
// Returns the output on every lane.
__device__ __forceinline__ float mlp_warp_forward(const float* w, const float* x, int lane) {
  const float* W1 = w;
  const float* b1 = W1 + kMlpH * kMlpIn;
  const float* W2 = b1 + kMlpH;
  const float* b2 = W2 + kMlpH * kMlpH;
  const float* W3 = b2 + kMlpH;
  float a = b1[lane];
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) a = fmaf(W1[lane * kMlpIn + k], x[k], a);
  const float h1 = tanhf(a);
  float a2 = b2[lane];
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) a2 = fmaf(W2[lane * kMlpH + k], __shfl_sync(0xffffffffu, h1, k), a2);
  const float h2 = tanhf(a2);
  float o = W3[lane] * h2;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
  return o + W3[kMlpH];
}

}  // namespace bs3
