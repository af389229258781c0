// bs3_solve_noalloc: the adaptive solve for callers that must not allocate
// device memory (for example code running under an allocator it does not own,
// inside a memory pool with a fixed budget, or in an environment where
// cudaMalloc is forbidden after start-up).  It runs the same persistent solver
// kernel as bs3_solve, but every scratch buffer lives in one file-scope
// __device__ array of fixed size instead of in a bs3 system.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/bs3.h"
#include "bs3_device.cuh"
#include "bs3_kernels.h"
#include "bs3_solver.cuh"

using namespace bs3;

namespace {

constexpr int64_t kNoAllocMaxN = 16384;   // BS3_NOALLOC_MAX_N of bs3.h
constexpr int64_t kLdMax = kNoAllocMaxN;  // already a multiple of 16

// Layout of the static scratch (byte offsets, each 256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffJv32 = align256(kOffCtrl + sizeof(Control));
constexpr size_t kOffJv64 = align256(kOffJv32 + 6 * kLdMax * sizeof(float));
constexpr size_t kOffScale = align256(kOffJv64 + 6 * kLdMax * sizeof(double));
constexpr size_t kOffRowsum = align256(kOffScale + kNoAllocMaxN * sizeof(float));
constexpr size_t kOffTheta = align256(kOffRowsum + kNoAllocMaxN * sizeof(double));
constexpr size_t kOffBias = align256(kOffTheta + kNoAllocMaxN * sizeof(double));
constexpr size_t kScratchBytes = align256(kOffBias + kNoAllocMaxN * sizeof(float));

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side device addresses of g_noalloc_scratch, one per device.  In host
// code the symbol itself is only a stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_addr[kMaxDevices];
std::mutex g_addr_mutex;

int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return BS3_ERR_INVALID_ARG;
  unsigned char* p = g_addr[device].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    p = g_addr[device].load(std::memory_order_relaxed);
    if (!p) {
      void* q = nullptr;
      if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) return BS3_ERR_CUDA;
      p = (unsigned char*)q;
      g_addr[device].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return BS3_OK;
}

// Per-call set-up of the scratch: row scales (1), row sums of the weights
// (paper-form oscillators), the rows' biases of the float-float sums
// (row_bias of sum_j |w_ij|), k1/(k0-k1) (circadian) and zeroed j-vectors (their
// padding columns multiply zero weights and must not hold stale NaN or Inf).
// A circadian k1_i outside (0, k0) sets the control block's status to
// S_INVALID (the check bs3_create_system makes on the host).
template <typename W>
__global__ void noalloc_setup(const W* __restrict__ w, int64_t N, int64_t ld, const double* __restrict__ par,
                              int kind, double k0, float* __restrict__ scale, double* __restrict__ rowsum,
                              float* __restrict__ bias, double* __restrict__ theta, float* __restrict__ jv32,
                              double* __restrict__ jv64, Control* __restrict__ ctrl) {
  const int64_t i = blockIdx.x;
  double acc = 0.0, aacc = 0.0;
  if (kind == BS3_LCO_PAPER || kind == BS3_KURAMOTO || kind == BS3_CIRCADIAN)
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
      const double v = (double)w[i * ld + j];
      if (kind == BS3_LCO_PAPER) acc += v;
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
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      r += sm[k];
      ra += sa[k];
    }
    rowsum[i] = r;
    bias[i] = row_bias(ra);
    scale[i] = 1.0f;
    theta[i] = (kind == BS3_CIRCADIAN) ? par[i] / (k0 - par[i]) : 0.0;
    if (kind == BS3_CIRCADIAN && !(par[i] > 0.0 && par[i] < k0)) atomicCAS(&ctrl->status, 0, (int)S_INVALID);
  }
  for (int64_t e = i * blockDim.x + threadIdx.x; e < 6 * ld; e += (int64_t)gridDim.x * blockDim.x) {
    jv32[e] = 0.0f;
    jv64[e] = 0.0;
  }
}

// A failed CUDA call ends the entry point with BS3_ERR_CUDA, also in the stats.
#define NA_CUDA(call)                           \
  do {                                          \
    if ((call) != cudaSuccess) {                \
      if (stats) stats->status = BS3_ERR_CUDA;  \
      return BS3_ERR_CUDA;                      \
    }                                           \
  } while (0)

}  // namespace

extern "C" int bs3_solve_noalloc(int kind, int64_t N, const double* par, const double* globals,
                                 const void* weights, int store, int64_t ld, double t0, double t1,
                                 const double* y0, double rtol, double atol, int variant, int accum,
                                 const double* t_out, int64_t n_out, double* y_out, double* final_y,
                                 bs3_stats* stats, void* stream_) {
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->status = BS3_ERR_INVALID_ARG;
  }
  if (kind < BS3_LCO_CFG || kind > BS3_CIRCADIAN) return BS3_ERR_INVALID_ARG;
  if (N < 1 || N > kNoAllocMaxN) return BS3_ERR_INVALID_ARG;   // beyond the static scratch
  // the j-vector regions of the scratch hold kLdMax columns
  if (ld < N || ld > kLdMax || ld % 16 != 0 || (store != BS3_F64 && store != BS3_F32) || !weights || !y0)
    return BS3_ERR_INVALID_ARG;
  if (((uintptr_t)weights & 15) != 0) return BS3_ERR_INVALID_ARG;
  if ((kind != BS3_LCO_PAPER && !par) || (kind == BS3_CIRCADIAN && !globals)) return BS3_ERR_INVALID_ARG;
  if (kind == BS3_CIRCADIAN && !(std::isfinite(globals[0]) && globals[0] > 0.0)) return BS3_ERR_INVALID_ARG;
  if (!(t1 > t0) || !std::isfinite(t0) || !std::isfinite(t1) || !(rtol > 0.0) || !(atol >= 0.0)) return BS3_ERR_INVALID_ARG;
  if (variant < BS3_SINGLE || variant > BS3_DOUBLE || accum < BS3_ACC_F32 || accum > BS3_ACC_F64) return BS3_ERR_INVALID_ARG;
  if (n_out < 0 || (n_out > 0 && (!t_out || !y_out))) return BS3_ERR_INVALID_ARG;
  if (stats) stats->status = BS3_OK;   // the arguments are valid; later failures are CUDA errors
  cudaStream_t stream = (cudaStream_t)stream_;
  int device = 0;
  NA_CUDA(cudaGetDevice(&device));
  unsigned char* base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc != BS3_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  Control* ctrl = (Control*)(base + kOffCtrl);
  float* jv32 = (float*)(base + kOffJv32);
  double* jv64 = (double*)(base + kOffJv64);
  float* scale = (float*)(base + kOffScale);
  double* rowsum = (double*)(base + kOffRowsum);
  double* theta = (double*)(base + kOffTheta);
  float* bias = (float*)(base + kOffBias);
  const int d = (kind == BS3_KURAMOTO) ? 1 : (kind == BS3_CIRCADIAN ? 4 : 2);
  const double k0 = (kind == BS3_CIRCADIAN) ? globals[0] : 0.0;
  // paper-form oscillators have no per-agent parameter: any readable array will do
  const double* par_k = par ? par : rowsum;

  NA_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Control), stream));
  if (store == BS3_F64)
    noalloc_setup<double><<<(unsigned)N, 128, 0, stream>>>((const double*)weights, N, ld, par_k, kind, k0, scale,
                                                           rowsum, bias, theta, jv32, jv64, ctrl);
  else
    noalloc_setup<float><<<(unsigned)N, 128, 0, stream>>>((const float*)weights, N, ld, par_k, kind, k0, scale,
                                                          rowsum, bias, theta, jv32, jv64, ctrl);
  NA_CUDA(cudaGetLastError());
  if (kind == BS3_CIRCADIAN) {
    // the per-cell check of k1 ran on the device: read its verdict first
    int bad = 0;
    NA_CUDA(cudaMemcpyAsync(&bad, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, stream));
    NA_CUDA(cudaStreamSynchronize(stream));
    if (bad != 0) {
      if (stats) stats->status = BS3_ERR_INVALID_ARG;
      return BS3_ERR_INVALID_ARG;
    }
  }

  // launch plan as for a system: one CTA per SM, weights kept in shared memory
  // when the rows of every CTA fit
  const void* kern = kernel_lookup(kind, store);
  int sms = 0;
  NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int rb = rows_per_tile(kind);
  const int64_t grid = std::min<int64_t>(sms, std::max<int64_t>(1, (N + rb - 1) / rb));
  const int rcap = (int)((N + grid - 1) / grid);
  const size_t state = state_smem_bytes(d, rcap);
  const size_t slab = ((size_t)rcap * ld * (store == BS3_F64 ? 8 : 4) + 127) / 128 * 128;
  const bool resident = kind != BS3_CIRCADIAN && slab + state <= (size_t)224 * 1024;
  const size_t smem = (resident ? slab : 0) + state;
  NA_CUDA(allow_max_smem(kern, device));

  Args a;
  std::memset(&a, 0, sizeof(a));
  a.N = (int)N;
  a.ld = (int)ld;
  a.q = weights;
  a.scale = scale;
  a.rowsum = rowsum;
  a.bias = bias;
  a.par = par_k;
  a.theta_h = theta;
  if (kind == BS3_CIRCADIAN)
    for (int k = 0; k < 8; ++k) a.g[k] = globals[k];
  a.X = const_cast<double*>(y0);   // read once, at the start of the launch
  a.jv32 = jv32;
  a.jv64 = jv64;
  a.ctrl = ctrl;
  a.job = JOB_SOLVE;
  a.variant = variant;
  a.accum = accum;
  a.t0 = t0;
  a.t1 = t1;
  a.rtol = rtol;
  a.atol = atol;
  a.hmin = 100.0 * (variant == BS3_SINGLE ? (double)FLT_EPSILON : DBL_EPSILON);
  a.hmax = 0.1 * std::fabs(t1 - t0);
  a.t_out = t_out;
  a.n_out = n_out;
  a.y_out = y_out;
  a.final_y = final_y;
  a.max_attempts = 100000;
  a.max_rejects = 85000;
  a.spin_limit = (long long)1 << 26;
  a.rc = rcap;
  a.slab_bytes = resident ? (int)slab : 0;
  a.method = M_BS32;
  a.n_slots = 6;
  int l2 = 0;
  NA_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device));
  a.l2_keep = ((double)N * ld * (store == BS3_F64 ? 8 : 4) <= 0.6 * (double)l2) ? 1 : 0;
  void* params[] = {&a};
  NA_CUDA(cudaLaunchCooperativeKernel(kern, dim3((unsigned)grid), dim3(kBlock), params, smem, stream));
  NA_CUDA(cudaStreamSynchronize(stream));
  Control c;
  NA_CUDA(cudaMemcpy(&c, ctrl, sizeof(Control), cudaMemcpyDeviceToHost));
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
