// Host side of the C ABI declared in include/bs3.h: system lifecycle,
// quantisation of the coupling weights, launches of the persistent solver
// and the wall-clock watchdog of Sec. 2.2.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <chrono>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/bs3.h"
#include "bs3_device.cuh"
#include "bs3_ensemble.h"
#include "bs3_kernels.h"
#include "bs3_mlp.cuh"
#include "bs3_solver.cuh"

using namespace bs3;

struct bs3_system {
  int device = 0;
  cudaStream_t stream = nullptr;
  int kind = 0, d = 1;
  int64_t N = 0, ld = 0;
  int store = -1;
  // per-agent parameters
  double* par = nullptr;
  double* theta_h = nullptr;
  double* rowsum = nullptr;
  float* bias = nullptr;       // row_bias of sum_j |q_ij| per row
  double g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // stored weights
  void* q = nullptr;
  float* scale = nullptr;
  // state and stage buffers
  double* X = nullptr;
  double* Xn = nullptr;
  double* Kb[4] = {nullptr, nullptr, nullptr, nullptr};
  float* jv32 = nullptr;
  double* jv64 = nullptr;
  Control* ctrl = nullptr;
  // host-mapped watchdog words
  int* cancel_h = nullptr;
  int* cancel_d = nullptr;
  double* progress_h = nullptr;
  double* progress_d = nullptr;
  // staging for host input/output
  double* stage_in = nullptr;
  size_t stage_in_n = 0;
  double* stage_out = nullptr;
  size_t stage_out_n = 0;
  double* hist = nullptr;
  int64_t hist_cap = 0;
  int64_t hist_n = 0;
  int grid = 0;
  int rc = 0;
  size_t smem = 0;
  int slab = 0;
  bool allow_resident = false;   // see BS3_TUNE_RESIDENT_WEIGHTS
  int l2_keep = 1;
  int tune_ctas = 0;           // 0 = one CTA per SM
  int method = BS3_METHOD_BS32;
  float* mlp = nullptr;        // learned proposer (kMlpModel binary32, weights bf16-rounded)
  bool mlp_on = false;
  int mlp_off = 0;
  int grid_store = -1;
  double* bstate = nullptr;    // [6][d][N] state slots of the system in a batch (bs3_solve_batch), on first use
};

namespace {

size_t store_bytes(int st) {
  switch (st) {
    case ST_F64: return 8;
    case ST_F32: return 4;
    case ST_BF16:
    case ST_F16: return 2;
    default: return 1;
  }
}

#define BS3_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return BS3_ERR_CUDA; \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

const void* kernel_for(int kind, int st) { return kernel_lookup(kind, st); }

// ---------------------------------------------------------------- quantise
// Row maxima of |fp32(K_ij)| (one CTA per row).
template <typename Src>
__global__ void row_amax_kernel(const Src* __restrict__ K, int64_t N, float* __restrict__ amax) {
  const int64_t i = blockIdx.x;
  float m = 0.f;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) m = fmaxf(m, fabsf((float)K[i * N + j]));
  __shared__ float sm[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, sm[w]);
    amax[i] = r;
  }
}

__global__ void scale_kernel(const float* __restrict__ amax, int64_t N, int st, float* __restrict__ s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float m = amax[i];
  float r = 1.f;
  if (m > 0.f && isfinite(m)) {
    if (st == ST_F16) {
      int k;
      frexpf(m, &k);                       // m = f 2^k, f in [0.5, 1)
      r = ldexpf(1.f, max(k - 1 - 14, -126));
    } else if (st == ST_FP8) {
      r = __fdiv_rn(m, 448.0f);
    }
  }
  s[i] = r;
}

// q_ij = round_store(fp32(K_ij) / s_i) into the padded [N][ld] layout.
template <typename Src>
__global__ void quantize_kernel(const Src* __restrict__ K, int64_t N, int64_t ld, int st, int src_is_f64,
                                const float* __restrict__ s, void* __restrict__ q) {
  const int64_t total = N * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ld, j = e - i * ld;
    const bool in = j < N;
    switch (st) {
      case ST_F64: {
        double v = 0.0;
        if (in) v = src_is_f64 ? (double)K[i * N + j] : (double)(float)K[i * N + j];
        ((double*)q)[e] = v;
        break;
      }
      case ST_F32:
        ((float*)q)[e] = in ? (float)K[i * N + j] : 0.f;
        break;
      case ST_BF16:
        ((__nv_bfloat16*)q)[e] = __float2bfloat16_rn(in ? (float)K[i * N + j] : 0.f);
        break;
      case ST_F16:
        ((__half*)q)[e] = __float2half_rn(in ? __fdiv_rn((float)K[i * N + j], s[i]) : 0.f);
        break;
      default:
        ((__nv_fp8_storage_t*)q)[e] =
            __nv_cvt_float_to_fp8(in ? __fdiv_rn((float)K[i * N + j], s[i]) : 0.f, __NV_SATFINITE, __NV_E4M3);
        break;
    }
  }
}

// rowsum_i = s_i * sum_j q_ij in binary64 (paper-form oscillators) and
// bias_i = row_bias(sum_j |q_ij|) (the start of the packed float-float sums).
__global__ void rowsum_kernel(const void* __restrict__ q, int st, int64_t N, int64_t ld,
                              const float* __restrict__ s, double* __restrict__ out, float* __restrict__ bias) {
  const int64_t i = blockIdx.x;
  double acc = 0.0, aacc = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    double v;
    const int64_t e = i * ld + j;
    switch (st) {
      case ST_F64: v = ((const double*)q)[e]; break;
      case ST_F32: v = ((const float*)q)[e]; break;
      case ST_BF16: v = __bfloat162float(((const __nv_bfloat16*)q)[e]); break;
      case ST_F16: v = __half2float(((const __half*)q)[e]); break;
      default: {
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(((const __nv_fp8_storage_t*)q)[e], __NV_E4M3);
        v = __half2float(__half(hr));
      }
    }
    acc += v;
    aacc += fabs(v);
  }
  __shared__ double sm[32], sa[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, off);
    aacc += __shfl_xor_sync(0xffffffffu, aacc, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = acc;
    sa[threadIdx.x >> 5] = aacc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, ra = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      r += sm[w];
      ra += sa[w];
    }
    out[i] = (double)s[i] * r;
    bias[i] = row_bias(ra);
  }
}

int ensure_stage(double** buf, size_t* cap, size_t n) {
  if (*cap >= n && *buf) return BS3_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  BS3_CUDA(cudaMalloc(buf, std::max<size_t>(n, 1) * sizeof(double)));
  *cap = n;
  return BS3_OK;
}

// One CTA per SM (at most one per row block of agents).  Each CTA keeps the
// state of ceil(N / grid) agents in shared memory.
int n_slots(int method) { return method == BS3_METHOD_DP54 ? 9 : 6; }

int pick_grid(bs3_system* s) {
  if (s->grid_store == s->store && s->grid > 0) return BS3_OK;
  const void* k = kernel_for(s->kind, s->store);
  int sms = 0;
  BS3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
  const int rb = rows_per_tile(s->kind);
  const int64_t cap = s->tune_ctas > 0 ? std::min(s->tune_ctas, sms) : sms;
  const int64_t grid = std::min<int64_t>(cap, std::max<int64_t>(1, (s->N + rb - 1) / rb));
  const int rc = (int)((s->N + grid - 1) / grid);
  const size_t state = (state_smem_bytes(s->d, rc, n_slots(s->method)) + 15) / 16 * 16;
  const size_t mlp = s->mlp_on ? (size_t)kMlpModel * sizeof(float) : 0;
  if (state + mlp > (size_t)200 * 1024) return BS3_ERR_INVALID_ARG;
  // keep each CTA's weight rows resident in shared memory when they fit
  // (streaming kinds only; the pairwise arctangent kernel is ALU-bound)
  const size_t slab = ((size_t)rc * s->ld * store_bytes(s->store) + 127) / 128 * 128;
  const size_t budget = (size_t)224 * 1024;
  const bool resident = s->kind != BS3_CIRCADIAN && s->allow_resident && slab + state + mlp <= budget;
  const size_t smem = (resident ? slab : 0) + state + mlp;
  s->mlp_off = (int)((resident ? slab : 0) + state);
  BS3_CUDA(allow_max_smem(k, s->device));
  int nb = 0;
  BS3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBlock, smem));
  if (nb < 1) return BS3_ERR_CUDA;
  int l2 = 0;
  BS3_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, s->device));
  s->l2_keep = ((double)s->N * s->ld * store_bytes(s->store) <= 0.6 * (double)l2) ? 1 : 0;
  s->grid = (int)grid;
  s->rc = rc;
  s->smem = smem;
  s->slab = resident ? (int)slab : 0;
  s->grid_store = s->store;
  return BS3_OK;
}

// Launch plan of a ragged batch (systems sorted by decreasing N).  Cost of a
// system on one CTA, per attempt: a fixed part (barriers and binary64
// latency, ~15 us measured) plus three evaluations streaming N^2 weights at
// the rate one SM reaches (~30 GB/s measured on GB300).  A system above the
// mean cost per CTA would keep one SM busy long after the others finish, so
// such systems go to teams of `team` CTAs, team = ceil(largest cost / mean
// cost) (at most the SM count, and at least 64 rows per CTA); the teams get
// the CTAs in proportion to the big systems' share of the cost.
constexpr int kMaxTeams = 256;
constexpr double kAttemptFixedUs = 15.0;
constexpr double kCtaStreamBytesPerUs = 30e3;

struct BatchPlan {
  int grid, n_big, team, n_teams;
};

BatchPlan plan_batch(const std::vector<int64_t>& sortedN, int sms, size_t weight_bytes) {
  const int64_t S = (int64_t)sortedN.size();
  BatchPlan p{(int)std::min<int64_t>(sms, S), 0, 1, 0};
  auto cost = [&](int64_t n) {
    return kAttemptFixedUs + 3.0 * (double)n * (double)n * (double)weight_bytes / kCtaStreamBytesPerUs;
  };
  double total = 0.0;
  for (int64_t n : sortedN) total += cost(n);
  if (sms < 4 || S < 1) return p;
  const double share = total / sms;
  int team = (int)std::ceil(cost(sortedN[0]) / share);
  team = std::min<int>(team, sms);
  team = std::min<int64_t>(team, std::max<int64_t>(1, sortedN[0] / 64));
  if (team < 2) return p;
  int n_big = 0;
  double big = 0.0;
  while (n_big < S && cost(sortedN[n_big]) > share) big += cost(sortedN[n_big++]);
  int ctas = (int)std::lround(sms * big / total);
  ctas = std::max(ctas, team);
  ctas = std::min(ctas, n_big < S ? sms - 1 : sms);
  const int n_teams = std::min<int>(std::min(ctas / team, n_big), kMaxTeams);
  if (n_teams < 1) return p;
  p.grid = sms;
  p.n_big = n_big;
  p.team = team;
  p.n_teams = n_teams;
  return p;
}

void fill_args(const bs3_system* s, Args& a) {
  std::memset(&a, 0, sizeof(a));
  a.N = (int)s->N;
  a.ld = (int)s->ld;
  a.q = s->q;
  a.scale = s->scale;
  a.rowsum = s->rowsum;
  a.bias = s->bias;
  a.par = s->par;
  a.theta_h = s->theta_h;
  for (int k = 0; k < 8; ++k) a.g[k] = s->g[k];
  a.X = s->X;
  a.Xn = s->Xn;
  for (int k = 0; k < 4; ++k) a.Kb[k] = s->Kb[k];
  a.jv32 = s->jv32;
  a.jv64 = s->jv64;
  a.ctrl = s->ctrl;
  a.cancel = s->cancel_d;
  a.progress = s->progress_d;
  a.spin_limit = (long long)1 << 26;
  a.max_attempts = 100000;
  a.max_rejects = 85000;
  a.rtol = 1.0;
  a.atol = 1.0;
  a.method = s->method;
  a.n_slots = n_slots(s->method);
}

int launch(bs3_system* s, Args& a) {
  int rc = pick_grid(s);
  if (rc != BS3_OK) return rc;
  a.rc = s->rc;
  a.slab_bytes = s->slab;
  a.mlp = s->mlp_on ? s->mlp : nullptr;
  a.smem_mlp_off = s->mlp_off;
  a.l2_keep = s->l2_keep;
  BS3_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(Control), s->stream));
  void* params[] = {&a};
  BS3_CUDA(cudaLaunchCooperativeKernel(kernel_for(s->kind, s->store), dim3(s->grid), dim3(kBlock), params,
                                       s->smem, s->stream));
  return BS3_OK;
}

// Waits for the stream, enforcing the wall-clock failure conditions through
// the host-mapped cancel flag that the device polls once per attempt.
int wait_with_watchdog(bs3_system* s, const bs3_limits& lim, double t0, double t1) {
  const auto start = std::chrono::steady_clock::now();
  int spins = 0;
  while (true) {
    const cudaError_t q = cudaStreamQuery(s->stream);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return BS3_ERR_CUDA;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
    const double done = (*(volatile double*)s->progress_h - t0) / (t1 - t0);
    if (el > lim.wall_limit_s || (el > lim.slow_limit_s && done < lim.slow_fraction))
      *(volatile int*)s->cancel_h = 1;
    if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return BS3_OK;
}

}  // namespace

extern "C" {

void bs3_default_limits(bs3_limits* lim) {
  if (!lim) return;
  lim->max_attempts = 100000;
  lim->max_rejects = 85000;
  lim->hmin_factor = 100.0;
  lim->wall_limit_s = 1.5 * 3600.0;
  lim->slow_limit_s = 45.0 * 60.0;
  lim->slow_fraction = 0.1;
  lim->spin_limit = (int64_t)1 << 26;
}

const char* bs3_status_string(int status) {
  switch (status) {
    case BS3_OK: return "BS3_OK";
    case BS3_ERR_INVALID_ARG: return "BS3_ERR_INVALID_ARG";
    case BS3_ERR_CUDA: return "BS3_ERR_CUDA";
    case BS3_ERR_MAX_STEPS: return "BS3_ERR_MAX_STEPS";
    case BS3_ERR_MAX_REJECTS: return "BS3_ERR_MAX_REJECTS";
    case BS3_ERR_STEP_TOO_SMALL: return "BS3_ERR_STEP_TOO_SMALL";
    case BS3_ERR_TIMEOUT: return "BS3_ERR_TIMEOUT";
    case BS3_ERR_DEVICE_WAIT: return "BS3_ERR_DEVICE_WAIT";
    case BS3_ERR_NONFINITE: return "BS3_ERR_NONFINITE";
    default: return "BS3_UNKNOWN_STATUS";
  }
}

int bs3_create_system(int kind, int64_t N, const double* params, int64_t n_params, int device, void* stream,
                      bs3_system_t* out) {
  if (!out) return BS3_ERR_INVALID_ARG;
  *out = nullptr;
  if (kind < BS3_LCO_CFG || kind > BS3_CIRCADIAN || N < 1 || N > (int64_t)1 << 30) return BS3_ERR_INVALID_ARG;
  const int64_t need = (kind == BS3_LCO_PAPER) ? 0 : (kind == BS3_CIRCADIAN ? N + 8 : N);
  if (n_params != need || (need > 0 && !params)) return BS3_ERR_INVALID_ARG;
  if (kind == BS3_CIRCADIAN) {
    const double k0 = params[N];
    for (int64_t i = 0; i < N; ++i)
      if (!(params[i] < k0) || !(params[i] > 0.0)) return BS3_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return BS3_ERR_CUDA;
  DeviceGuard guard(device);
  bs3_system* s = new bs3_system();
  s->device = device;
  s->stream = (cudaStream_t)stream;
  s->kind = kind;
  s->d = (kind == BS3_KURAMOTO) ? 1 : (kind == BS3_CIRCADIAN ? 4 : 2);
  s->N = N;
  s->ld = (N + 15) / 16 * 16;
  const size_t dN = (size_t)s->d * N;
  auto fail = [&](int rc) {
    bs3_destroy_system(s);
    return rc;
  };
  if (cudaMalloc(&s->par, N * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMemset(s->par, 0, N * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (kind == BS3_LCO_CFG || kind == BS3_KURAMOTO || kind == BS3_CIRCADIAN) {
    if (cudaMemcpy(s->par, params, N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(BS3_ERR_CUDA);
  }
  if (kind == BS3_CIRCADIAN) {
    for (int k = 0; k < 8; ++k) s->g[k] = params[N + k];
    std::vector<double> th(N);
    for (int64_t i = 0; i < N; ++i) th[i] = params[i] / (s->g[0] - params[i]);
    if (cudaMalloc(&s->theta_h, N * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
    if (cudaMemcpy(s->theta_h, th.data(), N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(BS3_ERR_CUDA);
  }
  if (cudaMalloc(&s->rowsum, N * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->bias, N * sizeof(float)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->scale, N * sizeof(float)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->X, dN * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->Xn, dN * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  for (int k = 0; k < 4; ++k)
    if (cudaMalloc(&s->Kb[k], dN * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->jv32, 6 * s->ld * sizeof(float)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->jv64, 6 * s->ld * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMemset(s->jv32, 0, 6 * s->ld * sizeof(float)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMemset(s->jv64, 0, 6 * s->ld * sizeof(double)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaMalloc(&s->ctrl, sizeof(Control)) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaHostAlloc(&s->cancel_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaHostAlloc(&s->progress_h, sizeof(double), cudaHostAllocMapped) != cudaSuccess)
    return fail(BS3_ERR_CUDA);
  if (cudaHostGetDevicePointer((void**)&s->cancel_d, s->cancel_h, 0) != cudaSuccess) return fail(BS3_ERR_CUDA);
  if (cudaHostGetDevicePointer((void**)&s->progress_d, s->progress_h, 0) != cudaSuccess)
    return fail(BS3_ERR_CUDA);
  *s->cancel_h = 0;
  *s->progress_h = 0.0;
  *out = s;
  return BS3_OK;
}

int bs3_batch_solve(int kind, int64_t S, const int64_t* Ns, const double* params, const float* K, int store,
                    const double* y0, const double* t0, const double* t1, double rtol, double atol, int variant,
                    int accum, double* y_final, bs3_stats* stats, double* kernel_ms, int device, void* stream_) {
  if (kind < BS3_LCO_CFG || kind > BS3_CIRCADIAN || S < 1 || S > (1 << 24) || !Ns || !K || !y0 || !t0 || !t1 ||
      !y_final)
    return BS3_ERR_INVALID_ARG;
  if (store < BS3_F64 || store > BS3_FP8E4M3 || !(rtol > 0.0) || !(atol >= 0.0)) return BS3_ERR_INVALID_ARG;
  if (variant < BS3_SINGLE || variant > BS3_DOUBLE || accum < BS3_ACC_F32 || accum > BS3_ACC_F64)
    return BS3_ERR_INVALID_ARG;
  if (kind != BS3_LCO_PAPER && !params) return BS3_ERR_INVALID_ARG;
  const int d = (kind == BS3_KURAMOTO) ? 1 : (kind == BS3_CIRCADIAN ? 4 : 2);
  const int per_agent = (kind == BS3_LCO_PAPER) ? 0 : 1;
  std::vector<int64_t> offN(S + 1, 0), offK(S + 1, 0), offQ(S + 1, 0), offL(S + 1, 0);
  for (int64_t k = 0; k < S; ++k) {
    if (Ns[k] < 1 || Ns[k] > (1 << 20) || !(t1[k] > t0[k])) return BS3_ERR_INVALID_ARG;
    const int64_t ld = (Ns[k] + 15) / 16 * 16;
    offN[k + 1] = offN[k] + Ns[k];
    offK[k + 1] = offK[k] + Ns[k] * Ns[k];
    offQ[k + 1] = offQ[k] + Ns[k] * ld;
    offL[k + 1] = offL[k] + ld;
  }
  const int64_t TN = offN[S];
  // circadian: 8 constants after each system's k1 values (params concat: N_k + 8 per system)
  std::vector<int64_t> offP(S + 1, 0);
  for (int64_t k = 0; k < S; ++k) offP[k + 1] = offP[k] + (kind == BS3_CIRCADIAN ? Ns[k] + 8 : per_agent * Ns[k]);
  DeviceGuard guard(device);
  cudaStream_t st = (cudaStream_t)stream_;
  int rc = BS3_OK;
  unsigned char* arena = nullptr;
  float* kdev = nullptr;
  float* amax = nullptr;
  // arena layout
  const size_t eb = store_bytes(store);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oQ = take((size_t)offQ[S] * eb), oScale = take(TN * 4), oRow = take(TN * 8), oBias = take(TN * 4), oPar = take(TN * 8),
               oTh = take(TN * 8), oY0 = take((size_t)d * TN * 8), oYF = take((size_t)d * TN * 8),
               oState = take((size_t)6 * d * TN * 8), oJ32 = take((size_t)6 * offL[S] * 4),
               oJ64 = take((size_t)6 * offL[S] * 8), oCtl = take((size_t)S * sizeof(Control)),
               oDesc = take((size_t)S * sizeof(SysDesc)), oNext = take(sizeof(int)), oBigNext = take(sizeof(int)),
               oTeamJob = take(kMaxTeams * sizeof(int)), oTeamBar = take(kMaxTeams * sizeof(unsigned long long)),
               oTeamStatus = take(kMaxTeams * sizeof(int));
  std::vector<SysDesc> desc(S);
  std::vector<int64_t> order(S);
  std::vector<double> par_h(TN), th_h(TN);
  std::vector<Control> ctl(S);
  int64_t maxNN = 0, maxN = 0;
  for (int64_t k = 0; k < S; ++k) {
    maxNN = std::max(maxNN, Ns[k] * Ns[k]);
    maxN = std::max(maxN, Ns[k]);
  }
  if (cudaMalloc(&arena, off) != cudaSuccess) return BS3_ERR_CUDA;
  if (cudaMalloc(&kdev, (size_t)maxNN * 4) != cudaSuccess) { cudaFree(arena); return BS3_ERR_CUDA; }
  if (cudaMalloc(&amax, (size_t)maxN * 4) != cudaSuccess) {
    cudaFree(arena); cudaFree(kdev); return BS3_ERR_CUDA;
  }
  do {
    if (cudaMemsetAsync(arena + oJ32, 0, (size_t)6 * offL[S] * 4, st) != cudaSuccess ||
        cudaMemsetAsync(arena + oJ64, 0, (size_t)6 * offL[S] * 8, st) != cudaSuccess ||
        cudaMemsetAsync(arena + oCtl, 0, (size_t)S * sizeof(Control), st) != cudaSuccess ||
        cudaMemsetAsync(arena + oNext, 0, oTeamStatus + kMaxTeams * sizeof(int) - oNext, st) != cudaSuccess) {
      rc = BS3_ERR_CUDA; break;
    }
    // per-agent parameters (and k1/(k0-k1) for the circadian kind)
    double g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = 0; k < S; ++k) {
      for (int64_t i = 0; i < Ns[k]; ++i) {
        const double pv = per_agent ? params[offP[k] + i] : 0.0;
        par_h[offN[k] + i] = pv;
        if (kind == BS3_CIRCADIAN) {
          for (int q = 0; q < 8; ++q) g[q] = params[offP[k] + Ns[k] + q];
          th_h[offN[k] + i] = pv / (g[0] - pv);
        } else {
          th_h[offN[k] + i] = 0.0;
        }
      }
    }
    if (cudaMemcpyAsync(arena + oPar, par_h.data(), TN * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(arena + oTh, th_h.data(), TN * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(arena + oY0, y0, (size_t)d * TN * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = BS3_ERR_CUDA; break;
    }
    // quantise each system's weights into its slice of the arena
    for (int64_t k = 0; k < S && rc == BS3_OK; ++k) {
      const int64_t N = Ns[k], ld = (N + 15) / 16 * 16;
      float* sc = (float*)(arena + oScale) + offN[k];
      void* q = arena + oQ + (size_t)offQ[k] * eb;
      if (cudaMemcpyAsync(kdev, K + offK[k], (size_t)N * N * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = BS3_ERR_CUDA; break;
      }
      const int blocks = (int)std::min<int64_t>((N * ld + 255) / 256, 152 * 64);
      row_amax_kernel<float><<<(unsigned)N, 256, 0, st>>>(kdev, N, amax);
      scale_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(amax, N, store, sc);
      quantize_kernel<float><<<blocks, 256, 0, st>>>(kdev, N, ld, store, 0, sc, q);
      rowsum_kernel<<<(unsigned)N, 256, 0, st>>>(q, store, N, ld, sc, (double*)(arena + oRow) + offN[k],
                                                 (float*)(arena + oBias) + offN[k]);
      if (cudaGetLastError() != cudaSuccess) rc = BS3_ERR_CUDA;
    }
    if (rc != BS3_OK) break;
    // descriptors, largest systems first (longest-processing-time order)
    for (int64_t k = 0; k < S; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return Ns[x] > Ns[y]; });
    for (int64_t r = 0; r < S; ++r) {
      const int64_t k = order[r];
      SysDesc& D = desc[r];
      D.N = (int)Ns[k];
      D.ld = (int)((Ns[k] + 15) / 16 * 16);
      D.q = arena + oQ + (size_t)offQ[k] * eb;
      D.scale = (const float*)(arena + oScale) + offN[k];
      D.rowsum = (const double*)(arena + oRow) + offN[k];
      D.bias = (const float*)(arena + oBias) + offN[k];
      D.par = (const double*)(arena + oPar) + offN[k];
      D.theta_h = (kind == BS3_CIRCADIAN) ? (const double*)(arena + oTh) + offN[k] : nullptr;
      D.y0 = (const double*)(arena + oY0) + (size_t)d * offN[k];
      D.y_final = (double*)(arena + oYF) + (size_t)d * offN[k];
      D.state = (double*)(arena + oState) + (size_t)6 * d * offN[k];
      D.jv32 = (float*)(arena + oJ32) + (size_t)6 * offL[k];
      D.jv64 = (double*)(arena + oJ64) + (size_t)6 * offL[k];
      D.ctrl = (Control*)(arena + oCtl) + k;
      D.t0 = t0[k];
      D.t1 = t1[k];
      D.rtol = rtol;
      D.atol = atol;
    }
    if (cudaMemcpyAsync(arena + oDesc, desc.data(), S * sizeof(SysDesc), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    BatchArgs ba;
    std::memset(&ba, 0, sizeof(ba));
    Args& a = ba.common;
    a.variant = variant;
    a.accum = accum;
    a.rtol = rtol;
    a.atol = atol;
    a.hmin = 100.0 * (variant == BS3_SINGLE ? (double)FLT_EPSILON : DBL_EPSILON);
    a.max_attempts = 100000;
    a.max_rejects = 85000;
    a.l2_keep = 0;
    a.method = M_BS32;
    a.n_slots = 6;
    if (kind == BS3_CIRCADIAN)
      for (int q = 0; q < 8; ++q) a.g[q] = params[offP[0] + Ns[0] + q];   // constants shared by the batch
    ba.sys = (const SysDesc*)(arena + oDesc);
    ba.S = (int)S;
    ba.next = (int*)(arena + oNext);
    ba.big_next = (int*)(arena + oBigNext);
    ba.team_job = (int*)(arena + oTeamJob);
    ba.team_bar = (unsigned long long*)(arena + oTeamBar);
    ba.team_status = (int*)(arena + oTeamStatus);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    // teams of CTAs for the systems too large for one SM's share of the batch
    // (cost ~ N^2: the weight bytes each evaluation streams)
    std::vector<int64_t> sortedN(S);
    for (int64_t k = 0; k < S; ++k) sortedN[k] = Ns[order[k]];
    const BatchPlan plan = plan_batch(sortedN, sms, eb);
    ba.n_big = plan.n_big;
    ba.team = plan.team;
    ba.n_teams = plan.n_teams;
    a.spin_limit = (long long)1 << 26;
    const unsigned grid = (unsigned)plan.grid;
    void* kargs[] = {&ba};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (kernel_ms && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess ||
                      cudaEventRecord(ev0, st) != cudaSuccess)) { rc = BS3_ERR_CUDA; break; }
    // cooperative: the CTAs of a team wait on one another
    if (cudaLaunchCooperativeKernel(batch_kernel_lookup(kind, store), dim3(grid), dim3(kBlock), kargs, 0, st) !=
        cudaSuccess) {
      rc = BS3_ERR_CUDA; break;
    }
    if (kernel_ms) {
      float ms = 0.f;
      if (cudaEventRecord(ev1, st) != cudaSuccess || cudaEventSynchronize(ev1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      *kernel_ms = ms;
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
    }
    std::vector<int> team_status(kMaxTeams, 0);
    if (cudaMemcpyAsync(team_status.data(), arena + oTeamStatus, kMaxTeams * sizeof(int), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    if (cudaMemcpyAsync(y_final, arena + oYF, (size_t)d * TN * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(ctl.data(), arena + oCtl, S * sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    int worst = BS3_OK;
    for (int64_t k = 0; k < S; ++k) {
      if (stats) {
        stats[k].n_accepted = ctl[k].n_acc;
        stats[k].n_rejected = ctl[k].n_rej;
        stats[k].n_rhs_evals = ctl[k].n_rhs;
        stats[k].t_reached = ctl[k].t;
        stats[k].h_last = ctl[k].h;
        stats[k].status = ctl[k].status;
        stats[k].n_out_written = 0;
      }
      if (ctl[k].status != BS3_OK && worst == BS3_OK) worst = ctl[k].status;
    }
    for (int t = 0; t < kMaxTeams; ++t)
      if (team_status[t] != 0 && worst == BS3_OK) worst = BS3_ERR_DEVICE_WAIT;
    rc = worst;
  } while (0);
  cudaFree(arena);
  cudaFree(kdev);
  cudaFree(amax);
  return rc;
}

int bs3_set_proposer(bs3_system_t s, const float* model) {
  if (!s) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  s->grid_store = -1;   // the shared-memory plan changes
  if (!model) {
    s->mlp_on = false;
    return BS3_OK;
  }
  float h[kMlpModel];
  for (int k = 0; k < kMlpModel; ++k) {
    if (!std::isfinite(model[k])) return BS3_ERR_INVALID_ARG;
    h[k] = model[k];
  }
  for (int k = kMlpModel - kMlpIn; k < kMlpModel; ++k)
    if (!(h[k] > 0.f)) return BS3_ERR_INVALID_ARG;   // standard deviations
  // inference weights in bfloat16 (round to nearest even), kept as binary32
  for (int k = 0; k < kMlpParams; ++k) {
    uint32_t u;
    std::memcpy(&u, &h[k], 4);
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    std::memcpy(&h[k], &u, 4);
  }
  if (!s->mlp) BS3_CUDA(cudaMalloc(&s->mlp, kMlpModel * sizeof(float)));
  BS3_CUDA(cudaMemcpy(s->mlp, h, kMlpModel * sizeof(float), cudaMemcpyHostToDevice));
  s->mlp_on = true;
  return BS3_OK;
}

int bs3_set_method(bs3_system_t s, int method) {
  if (!s || (method != BS3_METHOD_BS32 && method != BS3_METHOD_DP54)) return BS3_ERR_INVALID_ARG;
  s->method = method;
  s->grid_store = -1;   // the state slots change the launch plan
  return BS3_OK;
}

int bs3_set_tuning(bs3_system_t s, int key, int64_t value) {
  if (!s) return BS3_ERR_INVALID_ARG;
  if (key == BS3_TUNE_RESIDENT_WEIGHTS) {
    if (value != 0 && value != 1) return BS3_ERR_INVALID_ARG;
    s->allow_resident = value != 0;
    s->grid_store = -1;   // re-plan the launch
    return BS3_OK;
  }
  if (key == BS3_TUNE_CTAS) {
    if (value < 0 || value > 65536) return BS3_ERR_INVALID_ARG;
    s->tune_ctas = (int)value;
    s->grid_store = -1;
    return BS3_OK;
  }
  return BS3_ERR_INVALID_ARG;
}

int bs3_autotune(bs3_system_t s, const double* y0, double t0, double t1, double rtol, int variant, int accum,
                 int attempts, int64_t* choice_out, double* us_out) {
  if (!s || !y0 || attempts < 4 || s->store < 0) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  int sms = 0;
  BS3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
  const bool res0 = s->allow_resident;
  const int ctas0 = s->tune_ctas;
  double best = 1e300;
  int best_res = res0 ? 1 : 0, best_ctas = ctas0;
  bs3_limits lim;
  bs3_default_limits(&lim);
  lim.max_attempts = attempts;
  cudaEvent_t e0, e1;
  BS3_CUDA(cudaEventCreate(&e0));
  BS3_CUDA(cudaEventCreate(&e1));
  const int cand_ctas[3] = {sms, sms / 2, sms / 4};
  int rc = BS3_OK;
  for (int res = 0; res <= 1 && rc == BS3_OK; ++res) {
    for (int c = 0; c < 3 && rc == BS3_OK; ++c) {
      s->allow_resident = res != 0;
      s->tune_ctas = cand_ctas[c] > 0 ? cand_ctas[c] : 1;
      s->grid_store = -1;
      if (pick_grid(s) != BS3_OK) continue;
      if (res && s->slab == 0) continue;   // resident plan does not fit: same as streamed
      bs3_stats st;
      for (int rep = 0; rep < 2; ++rep) {   // first run warms up
        if (cudaEventRecord(e0, s->stream) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
        const int r = bs3_solve(s, t0, t1, y0, rtol, rtol, variant, accum, nullptr, 0, nullptr, nullptr, 0, &st, &lim);
        if (r != BS3_OK && r != BS3_ERR_MAX_STEPS) { rc = r; break; }
        if (cudaEventRecord(e1, s->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          rc = BS3_ERR_CUDA;
          break;
        }
      }
      if (rc != BS3_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double us = 1000.0 * ms / (double)std::max<int64_t>(1, st.n_accepted + st.n_rejected);
      if (us < best) {
        best = us;
        best_res = res;
        best_ctas = s->tune_ctas;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->allow_resident = rc == BS3_OK ? best_res != 0 : res0;
  s->tune_ctas = rc == BS3_OK ? best_ctas : ctas0;
  s->grid_store = -1;
  if (rc != BS3_OK) return rc;
  if (choice_out) {
    choice_out[0] = best_res;
    choice_out[1] = best_ctas;
  }
  if (us_out) *us_out = best;
  return BS3_OK;
}

int bs3_set_history(bs3_system_t s, int64_t capacity) {
  if (!s || capacity < 0) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  if (s->hist) cudaFree(s->hist);
  s->hist = nullptr;
  s->hist_cap = 0;
  s->hist_n = 0;
  if (capacity == 0) return BS3_OK;
  BS3_CUDA(cudaMalloc(&s->hist, (size_t)capacity * kHistDoubles * sizeof(double)));
  s->hist_cap = capacity;
  return BS3_OK;
}

int bs3_get_history(bs3_system_t s, double* out, int64_t* n_records) {
  if (!s || !n_records) return BS3_ERR_INVALID_ARG;
  *n_records = s->hist_n;
  if (s->hist_n > 0) {
    if (!out) return BS3_ERR_INVALID_ARG;
    DeviceGuard guard(s->device);
    BS3_CUDA(cudaMemcpy(out, s->hist, (size_t)s->hist_n * kHistDoubles * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return BS3_OK;
}

int bs3_destroy_system(bs3_system_t s) {
  if (!s) return BS3_OK;
  DeviceGuard guard(s->device);
  cudaFree(s->par);
  cudaFree(s->theta_h);
  cudaFree(s->rowsum);
  cudaFree(s->bias);
  cudaFree(s->q);
  cudaFree(s->scale);
  cudaFree(s->X);
  cudaFree(s->Xn);
  for (int k = 0; k < 4; ++k) cudaFree(s->Kb[k]);
  cudaFree(s->jv32);
  cudaFree(s->jv64);
  cudaFree(s->ctrl);
  cudaFree(s->stage_in);
  cudaFree(s->stage_out);
  cudaFree(s->hist);
  cudaFree(s->mlp);
  cudaFree(s->bstate);
  if (s->cancel_h) cudaFreeHost(s->cancel_h);
  if (s->progress_h) cudaFreeHost(s->progress_h);
  delete s;
  return BS3_OK;
}

int bs3_set_coupling(bs3_system_t s, const void* K, int src, int store, int is_device_ptr) {
  if (!s || !K) return BS3_ERR_INVALID_ARG;
  if ((src != BS3_F64 && src != BS3_F32) || store < BS3_F64 || store > BS3_FP8E4M3) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  const int64_t N = s->N, ld = s->ld;
  const size_t sb = (src == BS3_F64) ? 8 : 4;
  const size_t nbytes = (size_t)N * N * sb;
  const void* dK = K;
  void* tmp = nullptr;
  if (!is_device_ptr) {
    BS3_CUDA(cudaMalloc(&tmp, nbytes));
    if (cudaMemcpyAsync(tmp, K, nbytes, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
      cudaFree(tmp);
      return BS3_ERR_CUDA;
    }
    dK = tmp;
  }
  if (s->q) {
    cudaFree(s->q);
    s->q = nullptr;
  }
  int rc = BS3_OK;
  float* amax = nullptr;
  do {
    if (cudaMalloc(&s->q, (size_t)N * ld * store_bytes(store)) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    if (cudaMalloc(&amax, N * sizeof(float)) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    const int blocks = (int)std::min<int64_t>((N * ld + 255) / 256, 152 * 64);
    if (src == BS3_F64) {
      row_amax_kernel<double><<<(unsigned)N, 256, 0, s->stream>>>((const double*)dK, N, amax);
      scale_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s->stream>>>(amax, N, store, s->scale);
      quantize_kernel<double><<<blocks, 256, 0, s->stream>>>((const double*)dK, N, ld, store, 1, s->scale, s->q);
    } else {
      row_amax_kernel<float><<<(unsigned)N, 256, 0, s->stream>>>((const float*)dK, N, amax);
      scale_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s->stream>>>(amax, N, store, s->scale);
      quantize_kernel<float><<<blocks, 256, 0, s->stream>>>((const float*)dK, N, ld, store, 0, s->scale, s->q);
    }
    rowsum_kernel<<<(unsigned)N, 256, 0, s->stream>>>(s->q, store, N, ld, s->scale, s->rowsum, s->bias);
    if (cudaGetLastError() != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
  } while (0);
  if (amax) cudaFree(amax);
  if (tmp) cudaFree(tmp);
  if (rc != BS3_OK) {
    if (s->q) cudaFree(s->q);
    s->q = nullptr;
    s->store = -1;
    return rc;
  }
  s->store = store;
  return BS3_OK;
}

int bs3_get_coupling(bs3_system_t s, void* q_out, float* scales_out) {
  if (!s || s->store < 0) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  const size_t eb = store_bytes(s->store);
  if (q_out)
    BS3_CUDA(cudaMemcpy2DAsync(q_out, s->N * eb, s->q, s->ld * eb, s->N * eb, s->N, cudaMemcpyDeviceToHost,
                               s->stream));
  if (scales_out)
    BS3_CUDA(cudaMemcpyAsync(scales_out, s->scale, s->N * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
  BS3_CUDA(cudaStreamSynchronize(s->stream));
  return BS3_OK;
}

int bs3_rhs(bs3_system_t s, double t, const double* y, int f_prec, int sigma_prec, int g_prec, int accum,
            double* out) {
  (void)t;  // the benchmark systems are autonomous
  if (!s || !y || !out || s->store < 0) return BS3_ERR_INVALID_ARG;
  if ((f_prec | sigma_prec | g_prec) & ~1 || accum < BS3_ACC_F32 || accum > BS3_ACC_F64) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  const size_t dN = (size_t)s->d * s->N;
  BS3_CUDA(cudaMemcpyAsync(s->X, y, dN * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  Args a;
  fill_args(s, a);
  a.job = JOB_RHS;
  a.accum = accum;
  a.rhs_f = f_prec;
  a.rhs_s = sigma_prec;
  a.rhs_g = g_prec;
  a.out0 = out;
  int rc = launch(s, a);
  if (rc != BS3_OK) return rc;
  BS3_CUDA(cudaStreamSynchronize(s->stream));
  int st = 0;
  BS3_CUDA(cudaMemcpy(&st, &s->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost));
  return st == 0 ? BS3_OK : st;
}

int bs3_attempt(bs3_system_t s, double t, double h, const double* x, const double* k1, double rtol, double atol,
                int variant, int accum, double* xn_out, double* k4_out, double* err_out) {
  if (!s || !x || !k1 || !xn_out || !k4_out || !err_out || s->store < 0) return BS3_ERR_INVALID_ARG;
  if (s->method != BS3_METHOD_BS32) return BS3_ERR_INVALID_ARG;   // one attempt: Bogacki-Shampine only
  if (variant < BS3_SINGLE || variant > BS3_DOUBLE || accum < BS3_ACC_F32 || accum > BS3_ACC_F64)
    return BS3_ERR_INVALID_ARG;
  if (!(h > 0.0) || !(rtol > 0.0) || !(atol >= 0.0)) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  const size_t dN = (size_t)s->d * s->N;
  BS3_CUDA(cudaMemcpyAsync(s->X, x, dN * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  BS3_CUDA(cudaMemcpyAsync(s->Kb[0], k1, dN * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  Args a;
  fill_args(s, a);
  a.job = JOB_ATTEMPT;
  a.variant = variant;
  a.accum = accum;
  a.t0 = t;
  a.t1 = t + h;
  a.h_given = h;
  a.rtol = rtol;
  a.atol = atol;
  a.out0 = xn_out;
  a.out1 = k4_out;
  int rc = launch(s, a);
  if (rc != BS3_OK) return rc;
  BS3_CUDA(cudaStreamSynchronize(s->stream));
  Control c;
  BS3_CUDA(cudaMemcpy(&c, s->ctrl, sizeof(Control), cudaMemcpyDeviceToHost));
  uint64_t bits = c.emax[0];
  std::memcpy(err_out, &bits, sizeof(double));
  return c.status == 0 ? BS3_OK : c.status;
}

int bs3_solve(bs3_system_t s, double t0, double t1, const double* y0, double rtol, double atol, int variant,
              int accum, const double* t_out, int64_t n_out, double* y_out, double* final_y, int flags,
              bs3_stats* stats, const bs3_limits* lim_in) {
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->status = BS3_ERR_INVALID_ARG;
  }
  if (!s || !y0 || s->store < 0) return BS3_ERR_INVALID_ARG;
  if (!(t1 > t0) || !std::isfinite(t0) || !std::isfinite(t1)) return BS3_ERR_INVALID_ARG;
  if (!(rtol > 0.0) || !(atol >= 0.0)) return BS3_ERR_INVALID_ARG;
  if (variant < BS3_SINGLE || variant > BS3_DOUBLE || accum < BS3_ACC_F32 || accum > BS3_ACC_F64)
    return BS3_ERR_INVALID_ARG;
  if (n_out < 0 || (n_out > 0 && (!t_out || !y_out))) return BS3_ERR_INVALID_ARG;
  const bool host_io = (flags & BS3_HOST_IO) != 0;
  if (host_io && n_out > 0) {
    for (int64_t k = 0; k < n_out; ++k) {
      if (!(t_out[k] >= t0 && t_out[k] <= t1)) return BS3_ERR_INVALID_ARG;
      if (k > 0 && t_out[k] < t_out[k - 1]) return BS3_ERR_INVALID_ARG;
    }
  }
  bs3_limits lim;
  if (lim_in) lim = *lim_in;
  else bs3_default_limits(&lim);
  if (lim.max_attempts < 0 || lim.max_rejects < 0 || lim.spin_limit < 1) return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(s->device);
  const size_t dN = (size_t)s->d * s->N;
  int rc;
  // inputs
  const double* d_tout = t_out;
  double* d_yout = y_out;
  double* d_final = final_y;
  if (host_io) {
    rc = ensure_stage(&s->stage_in, &s->stage_in_n, (size_t)std::max<int64_t>(n_out, 1));
    if (rc) return rc;
    rc = ensure_stage(&s->stage_out, &s->stage_out_n, (size_t)n_out * dN + dN);
    if (rc) return rc;
    BS3_CUDA(cudaMemcpyAsync(s->X, y0, dN * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    if (n_out > 0)
      BS3_CUDA(cudaMemcpyAsync(s->stage_in, t_out, n_out * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    d_tout = s->stage_in;
    d_yout = s->stage_out;
    d_final = final_y ? s->stage_out + (size_t)n_out * dN : nullptr;
  } else {
    BS3_CUDA(cudaMemcpyAsync(s->X, y0, dN * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  }
  *(volatile int*)s->cancel_h = 0;
  *(volatile double*)s->progress_h = t0;
  Args a;
  fill_args(s, a);
  a.job = JOB_SOLVE;
  a.variant = variant;
  a.accum = accum;
  a.t0 = t0;
  a.t1 = t1;
  a.rtol = rtol;
  a.atol = atol;
  a.hmin = lim.hmin_factor * (variant == BS3_SINGLE ? (double)FLT_EPSILON : DBL_EPSILON);
  a.hmax = 0.1 * std::fabs(t1 - t0);
  a.h_given = 0.0;
  a.t_out = d_tout;
  a.n_out = n_out;
  a.y_out = d_yout;
  a.final_y = d_final;
  a.max_attempts = lim.max_attempts;
  a.max_rejects = lim.max_rejects;
  a.spin_limit = lim.spin_limit;
  a.hist = s->hist;
  a.hist_cap = s->hist_cap;
  rc = launch(s, a);
  if (rc != BS3_OK) return rc;
  rc = wait_with_watchdog(s, lim, t0, t1);
  if (rc != BS3_OK) return rc;
  Control c;
  BS3_CUDA(cudaMemcpy(&c, s->ctrl, sizeof(Control), cudaMemcpyDeviceToHost));
  if (host_io) {
    if (n_out > 0)
      BS3_CUDA(cudaMemcpy(y_out, s->stage_out, (size_t)n_out * dN * sizeof(double), cudaMemcpyDeviceToHost));
    if (final_y)
      BS3_CUDA(cudaMemcpy(final_y, s->stage_out + (size_t)n_out * dN, dN * sizeof(double),
                          cudaMemcpyDeviceToHost));
  }
  s->hist_n = std::min<int64_t>(s->hist_cap, c.n_acc + c.n_rej);
  if (stats) {
    stats->n_accepted = c.n_acc;
    stats->n_rejected = c.n_rej;
    stats->n_rhs_evals = c.n_rhs;
    stats->t_reached = c.t;
    stats->h_last = c.h;
    stats->status = c.status;
    stats->n_out_written = (int32_t)c.n_out;
  }
  return c.status;
}

int bs3_solve_batch(bs3_batch_item* items, int64_t n_items, int variant, int accum, int flags,
                    bs3_ensemble_group* group, int device, void* stream_, double* kernel_ms) {
  if (n_items < 0 || (n_items > 0 && !items) || (n_items == 0 && !group) || n_items > (1 << 24))
    return BS3_ERR_INVALID_ARG;
  if (variant < BS3_SINGLE || variant > BS3_DOUBLE || accum < BS3_ACC_F32 || accum > BS3_ACC_F64)
    return BS3_ERR_INVALID_ARG;
  const bool host_io = (flags & BS3_HOST_IO) != 0;
  for (int64_t k = 0; k < n_items; ++k) {
    bs3_batch_item& it = items[k];
    std::memset(&it.stats, 0, sizeof(it.stats));
    it.stats.status = BS3_ERR_INVALID_ARG;
  }
  // the items: one kind, one stored type, one device, the 3(2) pair, shared circadian constants
  const bs3_system* s0 = n_items > 0 ? items[0].sys : nullptr;
  for (int64_t k = 0; k < n_items; ++k) {
    const bs3_batch_item& it = items[k];
    const bs3_system* s = it.sys;
    if (!s || s->store < 0 || !it.y0 || !it.y_final || !(it.t1 > it.t0) || !std::isfinite(it.t0) ||
        !std::isfinite(it.t1) || !(it.rtol > 0.0) || !(it.atol >= 0.0))
      return BS3_ERR_INVALID_ARG;
    if (s->kind != s0->kind || s->store != s0->store || s->device != device || s->method != BS3_METHOD_BS32)
      return BS3_ERR_INVALID_ARG;
    if (s->kind == BS3_CIRCADIAN)
      for (int q = 0; q < 8; ++q)
        if (s->g[q] != s0->g[q]) return BS3_ERR_INVALID_ARG;
  }
  {
    // an item's system buffers hold its state during the solve: one system per item
    std::vector<const bs3_system*> seen(n_items);
    for (int64_t k = 0; k < n_items; ++k) seen[k] = items[k].sys;
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return BS3_ERR_INVALID_ARG;
  }
  if (group && (!group->K || !group->omega || !group->theta0 || !group->theta_out || group->ctas < 0))
    return BS3_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  const int64_t S = n_items;
  int sms = 0;
  BS3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  cudaStream_t st = (cudaStream_t)stream_, own = nullptr, side = nullptr, body = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  EnsembleRun* run = nullptr;
  unsigned char* arena = nullptr;
  int rc = BS3_OK;
  // CTA budgets: the group's stage products and the items' cooperative launch
  int g_ctas = 0, i_ctas = sms;
  std::vector<int64_t> order(S);
  std::vector<SysDesc> desc(S);
  std::vector<Control> ctl(S);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oDesc = take((size_t)std::max<int64_t>(S, 1) * sizeof(SysDesc)),
               oCtl = take((size_t)std::max<int64_t>(S, 1) * sizeof(Control)), oNext = take(sizeof(int)),
               oBigNext = take(sizeof(int)), oTeamJob = take(kMaxTeams * sizeof(int)),
               oTeamBar = take(kMaxTeams * sizeof(unsigned long long)), oTeamStatus = take(kMaxTeams * sizeof(int));
  BatchArgs ba;
  std::memset(&ba, 0, sizeof(ba));
  const void* bkern = S > 0 ? batch_kernel_lookup(s0->kind, s0->store) : nullptr;
  do {
    if (st == nullptr) {   // graphs cannot be captured on the legacy default stream
      if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess ||
          cudaDeviceSynchronize() != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      st = own;
    }
    if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    // group->ctas > 0 with items: the two run side by side on disjoint CTA
    // budgets; otherwise one after the other, each on the whole GPU (a solver
    // CTA holds all of an SM's registers, so the two never share an SM and a
    // split cannot finish sooner than the sum of the two parts)
    const bool side_by_side = group && S > 0 && group->ctas > 0;
    if (side_by_side) {
      g_ctas = std::max(1, std::min(group->ctas, sms - 1));
      i_ctas = sms - g_ctas;
    } else if (group) {
      g_ctas = group->ctas > 0 ? std::min(group->ctas, sms) : sms;
    }
    // ---- the items: initial states, descriptors (largest first), plan
    if (S > 0) {
      for (int64_t k = 0; k < S; ++k) {
        bs3_system* s = items[k].sys;
        const size_t dN = (size_t)s->d * s->N;
        if (!s->bstate && cudaMalloc(&s->bstate, 6 * dN * sizeof(double)) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
        if (cudaMemcpyAsync(s->X, items[k].y0, dN * sizeof(double),
                            host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
          rc = BS3_ERR_CUDA;
          break;
        }
      }
      if (rc != BS3_OK) break;
      if (cudaMalloc(&arena, off) != cudaSuccess || cudaMemsetAsync(arena, 0, off, st) != cudaSuccess) {
        rc = BS3_ERR_CUDA;
        break;
      }
      for (int64_t k = 0; k < S; ++k) order[k] = k;
      std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return items[x].sys->N > items[y].sys->N; });
      std::vector<int64_t> sortedN(S);
      for (int64_t r = 0; r < S; ++r) {
        const bs3_batch_item& it = items[order[r]];
        const bs3_system* s = it.sys;
        SysDesc& D = desc[r];
        D.N = (int)s->N;
        D.ld = (int)s->ld;
        D.q = s->q;
        D.scale = s->scale;
        D.rowsum = s->rowsum;
        D.bias = s->bias;
        D.par = s->par;
        D.theta_h = s->theta_h;
        D.y0 = s->X;
        D.y_final = s->Xn;
        D.state = s->bstate;
        D.jv32 = s->jv32;
        D.jv64 = s->jv64;
        D.ctrl = (Control*)(arena + oCtl) + order[r];
        D.t0 = it.t0;
        D.t1 = it.t1;
        D.rtol = it.rtol;
        D.atol = it.atol;
        sortedN[r] = s->N;
      }
      if (cudaMemcpyAsync(arena + oDesc, desc.data(), S * sizeof(SysDesc), cudaMemcpyHostToDevice, st) !=
          cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      Args& a = ba.common;
      a.variant = variant;
      a.accum = accum;
      a.rtol = 1.0;
      a.atol = 1.0;
      a.hmin = 100.0 * (variant == BS3_SINGLE ? (double)FLT_EPSILON : DBL_EPSILON);
      a.max_attempts = 100000;
      a.max_rejects = 85000;
      a.spin_limit = (long long)1 << 26;
      a.l2_keep = 0;
      a.method = M_BS32;
      a.n_slots = 6;
      for (int q = 0; q < 8; ++q) a.g[q] = s0->g[q];
      ba.sys = (const SysDesc*)(arena + oDesc);
      ba.S = (int)S;
      ba.next = (int*)(arena + oNext);
      ba.big_next = (int*)(arena + oBigNext);
      ba.team_job = (int*)(arena + oTeamJob);
      ba.team_bar = (unsigned long long*)(arena + oTeamBar);
      ba.team_status = (int*)(arena + oTeamStatus);
      const BatchPlan plan = plan_batch(sortedN, i_ctas, store_bytes(s0->store));
      ba.n_big = plan.n_big;
      ba.team = plan.team;
      ba.n_teams = plan.n_teams;
      i_ctas = plan.grid;
    }
    // ---- the group's buffers and initial state
    if (group) {
      const EnsembleSpec sp{group->K, group->N, group->T, group->omega, group->theta0, group->t0, group->t1,
                            group->rtol, group->atol, group->tile_n, 0, g_ctas, group->theta_out};
      rc = ensemble_create(sp, st, &run);
      if (rc != BS3_OK) break;
      if (cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    }
    // ---- one submission
    void* kargs[] = {&ba};
    cudaLaunchAttribute coop;
    coop.id = cudaLaunchAttributeCooperative;
    coop.val.cooperative = 1;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)i_ctas);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.attrs = &coop;
    cfg.numAttrs = 1;
    if (!group) {
      cfg.stream = st;
      if (cudaEventRecord(ev0, st) != cudaSuccess || cudaLaunchKernelExC(&cfg, bkern, kargs) != cudaSuccess ||
          cudaEventRecord(ev1, st) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    } else {
      if (side_by_side && (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)) {
        rc = BS3_ERR_CUDA;
        break;
      }
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      cudaError_t ce = cudaSuccess;
      if (side_by_side) {
        // the items' launch on a branch of its own
        ce = cudaEventRecord(fork, st);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(side, fork, 0);
        cfg.stream = side;
        if (ce == cudaSuccess) ce = cudaLaunchKernelExC(&cfg, bkern, kargs);
        if (ce == cudaSuccess) ce = cudaEventRecord(join, side);
      } else if (S > 0) {
        // the items' launch first, then the group, in the same graph
        cfg.stream = st;
        ce = cudaLaunchKernelExC(&cfg, bkern, kargs);
      }
      int crc = ce == cudaSuccess ? run->capture(st, body, nullptr, nullptr) : BS3_ERR_CUDA;
      if (side_by_side && crc == BS3_OK && cudaStreamWaitEvent(st, join, 0) != cudaSuccess) crc = BS3_ERR_CUDA;
      const cudaError_t ee = cudaStreamEndCapture(st, &graph);
      if (crc != BS3_OK || ee != cudaSuccess) { rc = crc != BS3_OK ? crc : BS3_ERR_CUDA; break; }
      if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess || cudaEventRecord(ev0, st) != cudaSuccess ||
          cudaGraphLaunch(exec, st) != cudaSuccess || cudaEventRecord(ev1, st) != cudaSuccess) {
        rc = BS3_ERR_CUDA;
        break;
      }
    }
    if (cudaEventSynchronize(ev1) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    if (kernel_ms) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      *kernel_ms = ms;
    }
    // ---- results
    int worst = BS3_OK;
    if (S > 0) {
      std::vector<int> team_status(kMaxTeams, 0);
      if (cudaMemcpyAsync(ctl.data(), arena + oCtl, S * sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(team_status.data(), arena + oTeamStatus, kMaxTeams * sizeof(int), cudaMemcpyDeviceToHost,
                          st) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      for (int64_t k = 0; k < S && rc == BS3_OK; ++k) {
        const bs3_system* s = items[k].sys;
        if (cudaMemcpyAsync(items[k].y_final, s->Xn, (size_t)s->d * s->N * sizeof(double),
                            host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          rc = BS3_ERR_CUDA;
      }
      if (rc != BS3_OK || cudaStreamSynchronize(st) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      for (int64_t k = 0; k < S; ++k) {
        bs3_stats& o = items[k].stats;
        o.n_accepted = ctl[k].n_acc;
        o.n_rejected = ctl[k].n_rej;
        o.n_rhs_evals = ctl[k].n_rhs;
        o.t_reached = ctl[k].t;
        o.h_last = ctl[k].h;
        o.status = ctl[k].status;
        o.n_out_written = 0;
        if (ctl[k].status != BS3_OK && worst == BS3_OK) worst = ctl[k].status;
      }
      for (int t = 0; t < kMaxTeams; ++t)
        if (team_status[t] != 0 && worst == BS3_OK) worst = BS3_ERR_DEVICE_WAIT;
    }
    if (group) {
      int64_t steps = 0;
      const int grc = run->finish(group->n_acc, group->n_rej, group->status, &steps);
      group->lockstep_attempts = steps;
      if (grc != BS3_OK && worst == BS3_OK) worst = grc;
    }
    rc = worst;
  } while (0);
  if (own) cudaStreamSynchronize(own);
  if (stream_) cudaStreamSynchronize((cudaStream_t)stream_);
  delete run;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (side) cudaStreamDestroy(side);
  if (body) cudaStreamDestroy(body);
  if (own) cudaStreamDestroy(own);
  cudaFree(arena);
  return rc;
}

}  // extern "C"
