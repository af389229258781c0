// Lock-step ensembles of Kuramoto trajectories that share one coupling matrix
// (the build's batched extension of the paper's solver).  Every stage of every
// live trajectory is one tensor-core product
//   [S_b | C_b]_i = sum_j K_ij [sin Y_bj | cos Y_bj]      (b = trajectory)
// with K and the j-vectors split into bfloat16 pairs (bs3_tc.cuh), and the
// stage epilogue (agent term, i-side finish, stage combinations, next j-vector,
// error norm) fused into the tensor-memory readout.  Each trajectory keeps its
// own t, h and accept/reject decision (the controller of the single-trajectory
// solver), so the batch runs in lock step only at the level of attempts.
//
// Layout: states [T][N] (trajectory-major), j-vector operand [2T][N] with the
// rows of trajectory b at 2b (sine) and 2b+1 (cosine), so that a 256-column
// output tile holds both halves of 128 trajectories.  The operand is double
// buffered: a stage reads one copy while its epilogue writes the next stage's
// j-vector into the other (other CTAs of the launch may still be reading the
// first).  The binary32 sine and cosine of every stage argument are kept
// ([T][N] pairs) for the i-side finish of the next product, so the epilogue
// does not reduce the phase again: binary64 arithmetic is scarce on GB300 and
// the epilogue, not the tensor cores, bounds a stage (for the same reason the
// binary64 stage combinations use fused multiply-adds).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/bs3.h"
#include "bs3_device.cuh"
#include "bs3_tc.cuh"
#include "bs3_tc_host.h"
#include "bs3_ensemble.h"

namespace bs3 {
namespace ens {

enum EPhase { E_K1 = 0, E_F1 = 1, E_B2 = 2, E_B3 = 3, E_B4 = 4 };

struct Traj {
  double *t, *h, *h0, *c21, *c32, *hs;
  int *live, *xsel, *ksel, *last, *rej, *status;
  long long *n_acc, *n_rej, *n_rhs;
  unsigned long long *emax, *red0, *red1, *red2;
  int* any_live;
};

struct EArgs {
  int N, T, phase;
  const double* omega;   // [T][N]
  double* X;             // [2][T][N]
  double* K14;           // [2][T][N]: K1 and K4 slots
  double* K2;            // [T][N]
  double* E3;            // [T][N]: the error's terms through stage 3, e1 K1 + e2 K2 + e3 K3
  __nv_bfloat16* Vh;     // [2T][N] j-vector operand the epilogue writes (the copy not being read)
  __nv_bfloat16* Vl;     // [2T][N]
  float2* SC;            // [T][N] binary32 (sin, cos) of the current stage argument
  float2* SCX;           // [2][T][N] binary32 (sin, cos) of the states X (selected like X)
  Traj tr;
  double rtol, atol, t1, hmax, hmin;
  long long max_attempts, max_rejects;
};

// Conversions between binary32 and binary64 and the magnitude/maximum of
// binary64 values by integer operations on the IEEE 754 encodings: on GB300
// every binary64 instruction, conversions and fmax included, issues at the
// binary64 rate, integer operations at the full rate.  The conversions are
// exact (binary32 results rounded to nearest even, as the conversion
// instruction rounds) for normal binary32 values; zeros, subnormals,
// infinities and NaN, rare here, take the conversion instruction.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u >= 254u) return (double)f;
  // exponent rebiased by 1023 - 127; the 23 fraction bits lead the 52
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ float d2f(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  // normal binary32 results: binary64 exponents 897 .. 1150 (a carry out of
  // the top binade rounds to infinity, as it should)
  if (e - 897u > 253u) return (float)d;
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  // drop 29 fraction bits, rounding to nearest, ties to even
  const unsigned long long r = mag + 0x0fffffffull + ((mag >> 29) & 1ull);
  const unsigned fb = (unsigned)(r >> 29) - (896u << 23);
  return __uint_as_float(fb | ((unsigned)(b >> 32) & 0x80000000u));
}

__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffll);
}

// max of two non-negative binary64 values (their encodings order as integers;
// a NaN operand, whose encoding lies above +Inf, is returned)
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

// sin and cos of a binary64 phase in binary32: two-constant Cody-Waite
// reduction on 2 pi in binary64, the reduced phase converted by d2f, then the
// library sincosf (a few ulp; the bfloat16 split of the ensembles' operand
// keeps 16 bits, far above that)
__device__ __forceinline__ void sincos_phase(double th, float* s, float* c) {
  const double kInv2Pi = 0.15915494309189535;
  const double k2PiHi = 6.2831853069365025;             // 2 pi rounded to 33 bits
  const double k2PiLo = 2.430840202602477e-10;           // 2 pi - k2PiHi
  const double k = rint(th * kInv2Pi);
  double r = fma(-k, k2PiHi, th);
  r = fma(-k, k2PiLo, r);
  sincosf(d2f(r), s, c);
}

constexpr double kB1 = 2.0 / 9.0, kB2 = 1.0 / 3.0, kB3 = 4.0 / 9.0;
constexpr double kE1 = -5.0 / 72.0, kE2 = 1.0 / 12.0, kE3 = 1.0 / 9.0, kE4 = -1.0 / 8.0;

// j-vector entry (bf16 hi/lo of sin and cos) and the binary32 pair of a stage argument
__device__ __forceinline__ void put_sc(const EArgs& a, int b, int i, float s, float c) {
  a.SC[(size_t)b * a.N + i] = make_float2(s, c);
  const __nv_bfloat16 sh = __float2bfloat16_rn(s), ch = __float2bfloat16_rn(c);
  const size_t rs = (size_t)(2 * b) * a.N + i, rc = rs + a.N;
  a.Vh[rs] = sh;
  a.Vl[rs] = __float2bfloat16_rn(s - __bfloat162float(sh));
  a.Vh[rc] = ch;
  a.Vl[rc] = __float2bfloat16_rn(c - __bfloat162float(ch));
}

__device__ __forceinline__ void put_v(const EArgs& a, int b, int i, double y) {
  float s, c;
  sincos_phase(y, &s, &c);
  put_sc(a, b, i, s, c);
}

// Stage argument X + delta with small delta (h/2 K1, 3h/4 K2): sin and cos by
// angle addition from those of X, in binary32 (within ~2 ulp of the binary32
// rounding; binary64 is scarce on GB300 and the full reduction of a new phase
// costs five binary64 operations, this two).
__device__ __forceinline__ void put_v_shift(const EArgs& a, int b, int i, float2 scx, double delta) {
  float sd, cd;
  sincosf(d2f(delta), &sd, &cd);
  const float s = fmaf(scx.x, cd, scx.y * sd);
  const float c = fmaf(scx.y, cd, -(scx.x * sd));
  put_sc(a, b, i, s, c);
}

// Integer tests on the exponent field (binary64 compares issue at the binary64
// rate on GB300): not finite = exponent all ones; NaN = that and a nonzero
// fraction.
__device__ __forceinline__ bool finite_bits(double v) {
  return ((unsigned)__double2hiint(v) & 0x7ff00000u) != 0x7ff00000u;
}

__device__ __forceinline__ double warp_max(double v) {
  // |v| as bits; NaN keeps its (above +Inf) bits, canonicalised
  unsigned long long x = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  if (x > 0x7ff0000000000000ull) x = 0x7ff8000000000000ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, x, off);
    x = o > x ? o : x;
  }
  return __longlong_as_double((long long)x);
}

// n / d for the error ratio, n >= 0: a binary32 reciprocal refined by one
// Newton step in binary64 (relative error ~1e-14; three binary64 operations
// instead of a correctly rounded division).  Outside [1e-30, 1e30] it divides.
__device__ __forceinline__ double ratio(double n, double d) {
  const float df = d2f(d);
  if (!(df >= 1e-30f && df <= 1e30f)) return n / d;   // (the range test in binary32)
  const double r0 = f2d(__frcp_rn(df));
  return n * (r0 * fma(-d, r0, 2.0));
}

// The stage epilogue run on the accumulator rows of one 128-row tile, one
// instantiation per phase.  Each thread owns one row i and 16 trajectories
// per call; the inputs of four trajectories are loaded together (also for
// retired trajectories, whose buffers stay allocated) so that the loads
// overlap, and only live trajectories are written.
template <int PH>
struct Epilogue {
  EArgs a;
  __device__ __forceinline__ void operator()(int i, int col0, const float* v) const {
    constexpr int G = 4;
    const int lane = threadIdx.x & 31;
    const int N = a.N;
    const size_t slot = (size_t)a.T * N;
    const double thr = a.atol / a.rtol;
#pragma unroll
    for (int j0 = 0; j0 < 16; j0 += G) {
      int live[G], xs[G], ks[G];
      double x[G], om[G], k1[G], k2[G], e3[G], y[G];
      float2 sc[G], scx[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int b = col0 / 2 + j0 + g;
        const size_t o = (size_t)b * N + i;
        live[g] = a.tr.live[b];
        xs[g] = a.tr.xsel[b];
        ks[g] = a.tr.ksel[b];
        sc[g] = a.SC[o];   // sin, cos of this stage's argument (agent i)
        om[g] = a.omega[o];
        // stage 2 needs only the sin/cos of X (its next argument X + 3h/4 K2 by
        // angle addition); the others need X itself
        x[g] = (PH != E_B2) ? a.X[xs[g] * slot + o] : 0.0;
        scx[g] = (PH == E_B2) ? a.SCX[xs[g] * slot + o] : make_float2(0.f, 0.f);
        k1[g] = (PH == E_F1 || PH == E_B3) ? a.K14[ks[g] * slot + o] : 0.0;
        k2[g] = (PH == E_B3) ? a.K2[o] : 0.0;
        e3[g] = (PH == E_B4) ? a.E3[o] : 0.0;
        y[g] = (PH == E_B4) ? a.X[(1 - xs[g]) * slot + o] : 0.0;
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int j = j0 + g;
        const int b = col0 / 2 + j;
        if (!live[g]) continue;   // uniform over the warp
        const size_t o = (size_t)b * N + i;
        const float cpl = sc[g].y * v[2 * j] - sc[g].x * v[2 * j + 1];
        const double k = om[g] + f2d(cpl);
        if (PH == E_K1) {
          a.K14[ks[g] * slot + o] = k;
          const double s = a.rtol * fmax(fabs(x[g]), thr);
          const double m0 = warp_max(fabs(x[g]) / s), m1 = warp_max(fabs(k) / s);
          if (lane == 0) {
            atomicMax(&a.tr.red0[b], (unsigned long long)__double_as_longlong(m0));
            atomicMax(&a.tr.red1[b], (unsigned long long)__double_as_longlong(m1));
          }
        } else if (PH == E_F1) {
          const double s = a.rtol * fmax(fabs(x[g]), thr);
          const double m = warp_max(fabs(k - k1[g]) / s);
          if (lane == 0) atomicMax(&a.tr.red2[b], (unsigned long long)__double_as_longlong(m));
        } else if (PH == E_B2) {
          a.K2[o] = k;
          put_v_shift(a, b, i, scx[g], a.tr.c32[b] * k);
        } else if (PH == E_B3) {
          // stage 4 needs K1..K3 only in the error: their part of it, in the
          // order the full sum takes them (the same roundings)
          a.E3[o] = fma(kE3, k, fma(kE2, k2[g], kE1 * k1[g]));
          const double xn = fma(a.tr.hs[b], fma(kB3, k, fma(kB2, k2[g], kB1 * k1[g])), x[g]);
          a.X[(1 - xs[g]) * slot + o] = xn;
          float sn, cn;
          sincos_phase(xn, &sn, &cn);
          put_sc(a, b, i, sn, cn);
          a.SCX[(1 - xs[g]) * slot + o] = make_float2(sn, cn);   // X' (the state after acceptance)
        } else {
          a.K14[(1 - ks[g]) * slot + o] = k;
          const double dv = a.tr.hs[b] * fma(kE4, k, e3[g]);
          const double w = max_nonneg(max_nonneg(abs_bits(x[g]), abs_bits(y[g])), thr);
          double e = ratio(abs_bits(dv), w);
          if (!finite_bits(y[g]) || !finite_bits(k)) e = __longlong_as_double(0x7ff8000000000000ll);
          const double m = warp_max(e);
          if (lane == 0) atomicMax(&a.tr.emax[b], (unsigned long long)__double_as_longlong(m));
        }
      }
    }
  }
};

constexpr int kEpiWarps = 16;
constexpr int kEnsThreads = tc::threads_for(kEpiWarps);

// One stage product over all (N / 128) x (2T / BNT) tiles; persistent CTAs
// (at most one per SM) take the tiles in turn, each tile's epilogue
// overlapping the next tile's products.
template <int PH, int BNT>
__global__ void __launch_bounds__(kEnsThreads, 1)
    ens_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, EArgs a, int K,
                    int* err, long long spin) {
  const Epilogue<PH> epi{a};
  tc::gemm_persistent<kEpiWarps, BNT>(&mAh, &mAl, &mBh, &mBl, K / tc::BM, 2 * a.T / BNT, K, epi, err, spin);
}

// j-vector operand of the stage argument Y = X + c K1 (c = 0, h0 or h/2).
__global__ void ens_prologue(EArgs a, int which) {
  const size_t n = (size_t)a.T * a.N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / a.N), i = (int)(e % a.N);
    if (!a.tr.live[b]) continue;
    const size_t slot = (size_t)a.T * a.N;
    const int xs = a.tr.xsel[b];
    if (which == 2) {   // Y2 = X + h/2 K1 by angle addition from the sin/cos of X
      put_v_shift(a, b, i, a.SCX[xs * slot + e], a.tr.c21[b] * a.K14[a.tr.ksel[b] * slot + e]);
      continue;
    }
    const double x = a.X[xs * slot + e];
    if (which == 0) {
      float s0, c0;
      sincos_phase(x, &s0, &c0);
      put_sc(a, b, i, s0, c0);
      a.SCX[xs * slot + e] = make_float2(s0, c0);   // the initial state's pair
    } else {
      put_v(a, b, i, fma(a.tr.h0[b], a.K14[a.tr.ksel[b] * slot + e], x));
    }
  }
}

__device__ __forceinline__ double bits(unsigned long long u) { return __longlong_as_double((long long)u); }

// Sets up the next attempt of trajectory b (h clamp, last-step stretch,
// failure conditions of Sec. 2.2) or retires it.
__device__ __forceinline__ void next_attempt(const EArgs& a, int b) {
  const Traj& r = a.tr;
  if (!(r.t[b] < a.t1)) { r.live[b] = 0; return; }
  if (r.n_rej[b] > a.max_rejects) { r.status[b] = S_MAX_REJECTS; r.live[b] = 0; return; }
  if (r.n_acc[b] + r.n_rej[b] >= a.max_attempts) { r.status[b] = S_MAX_STEPS; r.live[b] = 0; return; }
  double h = fmin(r.h[b], a.hmax);
  if (h <= a.hmin) { r.status[b] = S_STEP_TOO_SMALL; r.live[b] = 0; return; }
  r.last[b] = (r.t[b] + 1.1 * h >= a.t1);
  if (r.last[b]) h = a.t1 - r.t[b];
  r.h[b] = h;
  r.hs[b] = h;
  r.c21[b] = 0.5 * h;
  r.c32[b] = 0.75 * h;
}

// stage: 0 after K1 (h0 from d0, d1), 1 after F1 (starting step), 2 after an attempt.
__global__ void ens_control(EArgs a, int stage) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  int live = 0;
  if (b < a.T) {
    const Traj& r = a.tr;
    if (r.live[b]) {
      if (stage == 0) {
        const double d0 = bits(r.red0[b]), d1 = bits(r.red1[b]);
        r.n_rhs[b] = 1;
        if (d0 != d0 || isinf(d0) || d1 != d1 || isinf(d1)) {
          r.status[b] = S_NONFINITE;
          r.live[b] = 0;
        } else {
          r.h0[b] = (d0 >= 1e-5 && d1 >= 1e-5) ? 0.01 * d0 / d1 : 1e-6;
        }
      } else if (stage == 1) {
        r.n_rhs[b] = 2;
        const double h0 = r.h0[b];
        const double d1 = bits(r.red1[b]), d2 = bits(r.red2[b]) / h0;
        const double m = fmax(d1, d2);
        const double h1 = (m > 1e-15) ? pow(0.01 / m, 1.0 / 3.0) : fmax(1e-6, h0 * 1e-3);
        r.h[b] = fmin(fmin(100.0 * h0, h1), a.hmax);
        next_attempt(a, b);
      } else {
        const double E = bits(r.emax[b]);
        r.emax[b] = 0ull;
        r.n_rhs[b] += 3;
        if (E != E || isinf(E)) {
          r.status[b] = S_NONFINITE;
          ++r.n_rej[b];
          r.live[b] = 0;
        } else {
          const double h = r.h[b];
          if (E <= a.rtol) {
            r.t[b] = r.last[b] ? a.t1 : r.t[b] + h;
            r.xsel[b] ^= 1;
            r.ksel[b] ^= 1;
            ++r.n_acc[b];
            double fac = (E == 0.0) ? 5.0 : fmin(5.0, 0.8 * cbrt_ratio(a.rtol, E));
            if (r.rej[b]) fac = fmin(1.0, fac);
            r.h[b] = h * fac;
            r.rej[b] = 0;
          } else {
            ++r.n_rej[b];
            r.h[b] = r.rej[b] ? h * 0.5 : h * fmax(0.5, 0.8 * cbrt_ratio(a.rtol, E));
            r.rej[b] = 1;
          }
          next_attempt(a, b);
        }
      }
      live = r.live[b];
    }
  }
  live = __syncthreads_or(live);
  if (threadIdx.x == 0 && live) atomicOr(a.tr.any_live, 1);
}

__global__ void ens_gather(EArgs a, double* out) {
  const size_t n = (size_t)a.T * a.N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / a.N);
    out[e] = a.X[(size_t)a.tr.xsel[b] * n + e];
  }
}

}  // namespace ens
}  // namespace bs3

namespace bs3 {
namespace ens {

// The attempt loop's condition: before the loop, whether any trajectory is
// live; after each lock-step attempt, whether any still is, no bounded wait
// ran out and the attempt bound is not reached.  One thread (concurrent
// updates of a graph condition are undefined).
__global__ void ens_loop_start(cudaGraphConditionalHandle h, const int* any_live, const int* err,
                               long long* iters) {
  *iters = 0;
  cudaGraphSetConditional(h, (*any_live != 0 && *err == 0) ? 1u : 0u);
}

__global__ void ens_loop_next(cudaGraphConditionalHandle h, const int* any_live, const int* err, long long* iters,
                              long long max_iters) {
  const long long it = *iters + 1;
  *iters = it;
  cudaGraphSetConditional(h, (*any_live != 0 && *err == 0 && it < max_iters) ? 1u : 0u);
}

}  // namespace ens

namespace {

using namespace ens;

template <int BNT>
class EnsembleRunT final : public EnsembleRun {
 public:
  ~EnsembleRunT() override {
    cudaFree(kh); cudaFree(kl); cudaFree(vh); cudaFree(vl); cudaFree(vh1); cudaFree(vl1); cudaFree(scb);
    cudaFree(scx); cudaFree(X); cudaFree(K14); cudaFree(K2); cudaFree(E3);
    cudaFree(dsc); cudaFree(isc); cudaFree(lsc); cudaFree(usc); cudaFree(derr); cudaFree(iters);
  }

  int init(const EnsembleSpec& sp, cudaStream_t st);
  int capture(cudaStream_t st, cudaStream_t body, cudaEvent_t loop_begin, cudaEvent_t loop_end) override;
  int finish(int64_t* n_acc, int64_t* n_rej, int32_t* status, int64_t* lockstep_attempts) override;
  double flop_per_attempt() const override { return 3.0 * 3.0 * 2.0 * (double)N * (double)N * (double)(2 * T); }

 private:
  using PT = tc::PTile<BNT>;
  int64_t N = 0, T = 0, max_lockstep = 0;
  double* theta_out = nullptr;
  void *kh = nullptr, *kl = nullptr, *vh = nullptr, *vl = nullptr, *vh1 = nullptr, *vl1 = nullptr, *scb = nullptr,
       *scx = nullptr;
  double *X = nullptr, *K14 = nullptr, *K2 = nullptr, *E3 = nullptr, *dsc = nullptr;
  int *isc = nullptr, *derr = nullptr;
  long long *lsc = nullptr, *iters = nullptr;
  unsigned long long* usc = nullptr;
  CUtensorMap mAh, mAl, mBh, mBl, mBh1, mBl1;
  EArgs a;
  dim3 ggrid;
  unsigned ctl_blocks = 1, ew_blocks = 1;
  cudaStream_t stream = nullptr;
};

#define EN_CUDA(call)                                         \
  do {                                                        \
    if ((call) != cudaSuccess) return BS3_ERR_CUDA;           \
  } while (0)
#define EN_RC(expr)              \
  do {                           \
    const int rc_ = (expr);      \
    if (rc_ != BS3_OK) return rc_; \
  } while (0)

template <int BNT>
int EnsembleRunT<BNT>::init(const EnsembleSpec& sp, cudaStream_t st) {
  N = sp.N;
  T = sp.T;
  max_lockstep = sp.max_lockstep;
  theta_out = sp.theta_out;
  stream = st;
  const size_t NN = (size_t)N * N, TN = (size_t)T * N;
  int dev = 0, sms = 0;
  EN_CUDA(cudaGetDevice(&dev));
  EN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t n_tiles = (N / tc::BM) * (2 * T / BNT);
  const int cap = sp.max_ctas > 0 ? std::min(sp.max_ctas, sms) : sms;
  ggrid = dim3((unsigned)std::min<int64_t>(n_tiles, cap));
  ctl_blocks = (unsigned)((T + 255) / 256);
  ew_blocks = (unsigned)std::min<size_t>((TN + 255) / 256, 152 * 16);
  EN_CUDA(cudaMalloc(&kh, NN * 2));
  EN_CUDA(cudaMalloc(&kl, NN * 2));
  EN_CUDA(cudaMalloc(&vh, 2 * TN * 2));
  EN_CUDA(cudaMalloc(&vl, 2 * TN * 2));
  EN_CUDA(cudaMalloc(&vh1, 2 * TN * 2));
  EN_CUDA(cudaMalloc(&vl1, 2 * TN * 2));
  EN_CUDA(cudaMalloc(&scb, TN * sizeof(float2)));
  EN_CUDA(cudaMalloc(&scx, 2 * TN * sizeof(float2)));
  EN_CUDA(cudaMalloc(&X, 2 * TN * sizeof(double)));
  EN_CUDA(cudaMalloc(&K14, 2 * TN * sizeof(double)));
  EN_CUDA(cudaMalloc(&K2, TN * sizeof(double)));
  EN_CUDA(cudaMalloc(&E3, TN * sizeof(double)));
  EN_CUDA(cudaMalloc(&dsc, 6 * T * sizeof(double)));
  EN_CUDA(cudaMalloc(&isc, (6 * T + 1) * sizeof(int)));
  EN_CUDA(cudaMalloc(&lsc, 3 * T * sizeof(long long)));
  EN_CUDA(cudaMalloc(&usc, 4 * T * sizeof(unsigned long long)));
  EN_CUDA(cudaMalloc(&derr, sizeof(int)));
  EN_CUDA(cudaMalloc(&iters, sizeof(long long)));
  EN_CUDA(cudaMemsetAsync(vh, 0, 2 * TN * 2, st));
  EN_CUDA(cudaMemsetAsync(vl, 0, 2 * TN * 2, st));
  EN_CUDA(cudaMemsetAsync(vh1, 0, 2 * TN * 2, st));
  EN_CUDA(cudaMemsetAsync(vl1, 0, 2 * TN * 2, st));
  EN_CUDA(cudaMemsetAsync(scb, 0, TN * sizeof(float2), st));
  EN_CUDA(cudaMemsetAsync(scx, 0, 2 * TN * sizeof(float2), st));
  EN_CUDA(cudaMemsetAsync(isc, 0, (6 * T + 1) * sizeof(int), st));
  EN_CUDA(cudaMemsetAsync(lsc, 0, 3 * T * sizeof(long long), st));
  EN_CUDA(cudaMemsetAsync(usc, 0, 4 * T * sizeof(unsigned long long), st));
  EN_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
  EN_CUDA(cudaMemsetAsync(iters, 0, sizeof(long long), st));
  EN_CUDA(cudaMemcpyAsync(X, sp.theta0, TN * sizeof(double), cudaMemcpyDeviceToDevice, st));
  EN_RC(tc_split(sp.K, NN, kh, kl, st));
  EN_RC(tc_encode_bf16_2d(&mAh, kh, N, N, tc::BM));
  EN_RC(tc_encode_bf16_2d(&mAl, kl, N, N, tc::BM));
  EN_RC(tc_encode_bf16_2d(&mBh, vh, 2 * T, N, BNT));
  EN_RC(tc_encode_bf16_2d(&mBl, vl, 2 * T, N, BNT));
  EN_RC(tc_encode_bf16_2d(&mBh1, vh1, 2 * T, N, BNT));
  EN_RC(tc_encode_bf16_2d(&mBl1, vl1, 2 * T, N, BNT));
  EN_CUDA(cudaFuncSetAttribute(ens_gemm_kernel<E_K1, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM_BYTES));
  EN_CUDA(cudaFuncSetAttribute(ens_gemm_kernel<E_F1, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM_BYTES));
  EN_CUDA(cudaFuncSetAttribute(ens_gemm_kernel<E_B2, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM_BYTES));
  EN_CUDA(cudaFuncSetAttribute(ens_gemm_kernel<E_B3, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM_BYTES));
  EN_CUDA(cudaFuncSetAttribute(ens_gemm_kernel<E_B4, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM_BYTES));
  std::memset(&a, 0, sizeof(a));
  a.N = (int)N;
  a.T = (int)T;
  a.omega = sp.omega;
  a.X = X;
  a.K14 = K14;
  a.K2 = K2;
  a.E3 = E3;
  a.Vh = (__nv_bfloat16*)vh;
  a.Vl = (__nv_bfloat16*)vl;
  a.SC = (float2*)scb;
  a.SCX = (float2*)scx;
  a.tr.t = dsc; a.tr.h = dsc + T; a.tr.h0 = dsc + 2 * T; a.tr.c21 = dsc + 3 * T; a.tr.c32 = dsc + 4 * T;
  a.tr.hs = dsc + 5 * T;
  a.tr.live = isc; a.tr.xsel = isc + T; a.tr.ksel = isc + 2 * T; a.tr.last = isc + 3 * T; a.tr.rej = isc + 4 * T;
  a.tr.status = isc + 5 * T; a.tr.any_live = isc + 6 * T;
  a.tr.n_acc = lsc; a.tr.n_rej = lsc + T; a.tr.n_rhs = lsc + 2 * T;
  a.tr.emax = usc; a.tr.red0 = usc + T; a.tr.red1 = usc + 2 * T; a.tr.red2 = usc + 3 * T;
  a.rtol = sp.rtol;
  a.atol = sp.atol;
  a.t1 = sp.t1;
  a.hmax = 0.1 * (sp.t1 - sp.t0);
  a.hmin = 100.0 * DBL_EPSILON;
  a.max_attempts = 100000;
  a.max_rejects = 85000;
  // t = t0 and every trajectory live
  std::vector<double> tt(T, sp.t0);
  std::vector<int> ones(T, 1);
  EN_CUDA(cudaMemcpyAsync(a.tr.t, tt.data(), T * sizeof(double), cudaMemcpyHostToDevice, st));
  EN_CUDA(cudaMemcpyAsync(a.tr.live, ones.data(), T * sizeof(int), cudaMemcpyHostToDevice, st));
  EN_CUDA(cudaStreamSynchronize(st));
  return BS3_OK;
}

// The whole solve, recorded into the capture in progress on st:
//   K1 = f(t0, y0) and the starting step (j-vector operand copy 0; these
//   epilogues write no j-vector), then the attempt loop (WHILE node): the
//   prologue (Y2 -> copy 0), stage 2 (reads copy 0, writes Y3 to copy 1),
//   stage 3 (reads copy 1, writes X' to copy 0), stage 4 (reads copy 0), the
//   per-trajectory control and the loop condition, all decided on the
//   device; then the gather of the final phases.
template <int BNT>
int EnsembleRunT<BNT>::capture(cudaStream_t st, cudaStream_t body, cudaEvent_t loop_begin, cudaEvent_t loop_end) {
  const long long spin = 1ll << 22;
  EArgs b = a;
  b.Vh = (__nv_bfloat16*)vh;
  b.Vl = (__nv_bfloat16*)vl;
  ens_prologue<<<ew_blocks, 256, 0, st>>>(b, 0);
  b.phase = E_K1;
  ens_gemm_kernel<E_K1, BNT><<<ggrid, kEnsThreads, PT::SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, b, (int)N, derr, spin);
  ens_control<<<ctl_blocks, 256, 0, st>>>(b, 0);
  ens_prologue<<<ew_blocks, 256, 0, st>>>(b, 1);
  b.phase = E_F1;
  ens_gemm_kernel<E_F1, BNT><<<ggrid, kEnsThreads, PT::SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, b, (int)N, derr, spin);
  EN_CUDA(cudaMemsetAsync(a.tr.any_live, 0, sizeof(int), st));
  ens_control<<<ctl_blocks, 256, 0, st>>>(b, 1);
  EN_CUDA(cudaGetLastError());
  // the loop condition, set on the device before the loop and after each attempt
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  EN_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
  if (cs != cudaStreamCaptureStatusActive) return BS3_ERR_CUDA;
  cudaGraphConditionalHandle h;
  EN_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
  ens_loop_start<<<1, 1, 0, st>>>(h, a.tr.any_live, derr, iters);
  if (loop_begin) EN_CUDA(cudaEventRecordWithFlags(loop_begin, st, cudaEventRecordExternal));
  EN_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  EN_CUDA(cudaGraphAddNode(&loop, graph, deps, nullptr, ndeps, &cp));
  EN_CUDA(cudaStreamUpdateCaptureDependencies(st, &loop, nullptr, 1, cudaStreamSetCaptureDependencies));
  // the loop body, captured on the second stream into the node's body graph
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  EN_CUDA(cudaStreamBeginCaptureToGraph(body, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    const long long max_iters = max_lockstep > 0 ? max_lockstep : a.max_attempts + 1;
    EArgs c = a;
    c.Vh = (__nv_bfloat16*)vh;
    c.Vl = (__nv_bfloat16*)vl;
    ens_prologue<<<ew_blocks, 256, 0, body>>>(c, 2);
    c.phase = E_B2;
    c.Vh = (__nv_bfloat16*)vh1;
    c.Vl = (__nv_bfloat16*)vl1;
    ens_gemm_kernel<E_B2, BNT><<<ggrid, kEnsThreads, PT::SMEM_BYTES, body>>>(mAh, mAl, mBh, mBl, c, (int)N, derr, spin);
    c.phase = E_B3;
    c.Vh = (__nv_bfloat16*)vh;
    c.Vl = (__nv_bfloat16*)vl;
    ens_gemm_kernel<E_B3, BNT><<<ggrid, kEnsThreads, PT::SMEM_BYTES, body>>>(mAh, mAl, mBh1, mBl1, c, (int)N, derr, spin);
    c.phase = E_B4;
    ens_gemm_kernel<E_B4, BNT><<<ggrid, kEnsThreads, PT::SMEM_BYTES, body>>>(mAh, mAl, mBh, mBl, c, (int)N, derr, spin);
    cudaMemsetAsync(a.tr.any_live, 0, sizeof(int), body);
    ens_control<<<ctl_blocks, 256, 0, body>>>(c, 2);
    ens_loop_next<<<1, 1, 0, body>>>(h, a.tr.any_live, derr, iters, max_iters);
  }
  const cudaError_t eb = cudaGetLastError();
  cudaGraph_t ended = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(body, &ended);
  if (eb != cudaSuccess || ee != cudaSuccess) return BS3_ERR_CUDA;
  if (loop_end) EN_CUDA(cudaEventRecordWithFlags(loop_end, st, cudaEventRecordExternal));
  ens_gather<<<ew_blocks, 256, 0, st>>>(a, theta_out);
  EN_CUDA(cudaGetLastError());
  return BS3_OK;
}

template <int BNT>
int EnsembleRunT<BNT>::finish(int64_t* n_acc, int64_t* n_rej, int32_t* status, int64_t* lockstep_attempts) {
  int herr = 0, any = 0;
  long long it = 0;
  EN_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, stream));
  EN_CUDA(cudaMemcpyAsync(&any, a.tr.any_live, sizeof(int), cudaMemcpyDeviceToHost, stream));
  EN_CUDA(cudaMemcpyAsync(&it, iters, sizeof(long long), cudaMemcpyDeviceToHost, stream));
  if (n_acc) EN_CUDA(cudaMemcpyAsync(n_acc, a.tr.n_acc, T * sizeof(long long), cudaMemcpyDeviceToHost, stream));
  if (n_rej) EN_CUDA(cudaMemcpyAsync(n_rej, a.tr.n_rej, T * sizeof(long long), cudaMemcpyDeviceToHost, stream));
  if (status) EN_CUDA(cudaMemcpyAsync(status, a.tr.status, T * sizeof(int), cudaMemcpyDeviceToHost, stream));
  EN_CUDA(cudaStreamSynchronize(stream));
  if (lockstep_attempts) *lockstep_attempts = it;
  if (herr) return BS3_ERR_DEVICE_WAIT;
  if (any && max_lockstep > 0 && it >= max_lockstep) return BS3_ERR_MAX_STEPS;
  return BS3_OK;
}

#undef EN_CUDA
#undef EN_RC

template <int BNT>
int create_t(const EnsembleSpec& sp, cudaStream_t st, EnsembleRun** out) {
  auto* r = new EnsembleRunT<BNT>();
  const int rc = r->init(sp, st);
  if (rc != BS3_OK) {
    delete r;
    return rc;
  }
  *out = r;
  return BS3_OK;
}

}  // namespace

int ensemble_create(const EnsembleSpec& sp, cudaStream_t st, EnsembleRun** out) {
  if (!out) return BS3_ERR_INVALID_ARG;
  *out = nullptr;
  const int tile = sp.tile_n == 0 ? 128 : sp.tile_n;
  if (!sp.K || !sp.omega || !sp.theta0 || !sp.theta_out || (tile != 128 && tile != 256)) return BS3_ERR_INVALID_ARG;
  if (sp.N < tc::BM || sp.N % tc::BM || sp.N % tc::BK || sp.T < tile / 2 || (2 * sp.T) % tile) return BS3_ERR_INVALID_ARG;
  if (sp.N > (1 << 20) || sp.T > (1 << 16) || sp.max_lockstep < 0 || sp.max_ctas < 0) return BS3_ERR_INVALID_ARG;
  if (!(sp.t1 > sp.t0) || !(sp.rtol > 0.0) || !(sp.atol >= 0.0)) return BS3_ERR_INVALID_ARG;
  return tile == 256 ? create_t<256>(sp, st, out) : create_t<128>(sp, st, out);
}

}  // namespace bs3

using namespace bs3;
using namespace bs3::ens;

namespace {

// A standalone ensemble solve: one graph (set-up stages, the attempt loop as a
// device-decided WHILE node, the gather), launched once; the host waits only
// for its end.  loop_ms (optional) receives the device time of the graph (the
// two set-up stage products, the attempt loop and the gather).
int ensemble_solve_graph(const EnsembleSpec& sp, int64_t* n_acc, int64_t* n_rej, int32_t* status,
                         int64_t* lockstep_attempts, cudaStream_t st_in, float* loop_ms) {
  cudaStream_t st = st_in, own = nullptr, body = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  EnsembleRun* run = nullptr;
  int rc = BS3_OK;
  do {
    if (st == nullptr) {   // graphs cannot be captured on the legacy default stream
      if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess ||
          cudaDeviceSynchronize() != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
      st = own;
    }
    if (cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    if (loop_ms && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess)) {
      rc = BS3_ERR_CUDA;
      break;
    }
    rc = ensemble_create(sp, st, &run);
    if (rc != BS3_OK) break;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    rc = run->capture(st, body, nullptr, nullptr);
    const cudaError_t ee = cudaStreamEndCapture(st, &graph);
    if (rc != BS3_OK) break;
    if (ee != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess ||
        (ev0 && cudaEventRecord(ev0, st) != cudaSuccess) || cudaGraphLaunch(exec, st) != cudaSuccess ||
        (ev1 && cudaEventRecord(ev1, st) != cudaSuccess)) { rc = BS3_ERR_CUDA; break; }
    rc = run->finish(n_acc, n_rej, status, lockstep_attempts);
    if (loop_ms && cudaEventElapsedTime(loop_ms, ev0, ev1) != cudaSuccess && rc == BS3_OK) rc = BS3_ERR_CUDA;
  } while (0);
  if (own) cudaStreamSynchronize(own);
  if (st_in) cudaStreamSynchronize(st_in);
  delete run;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (body) cudaStreamDestroy(body);
  if (own) cudaStreamDestroy(own);
  return rc;
}

}  // namespace

extern "C" int bs3_ensemble_solve_tiled(const float* K, int64_t N, int64_t T, const double* omega,
                                        const double* theta0, double t0, double t1, double rtol, double atol,
                                        int tile_n, int64_t max_lockstep, double* theta_out, int64_t* n_acc,
                                        int64_t* n_rej, int32_t* status, int64_t* lockstep_attempts, void* stream) {
  // narrow tiles by default: more tiles per persistent CTA, so more of each
  // binary64 epilogue overlaps the next tile's products
  const EnsembleSpec sp{K, N, T, omega, theta0, t0, t1, rtol, atol, tile_n == 0 ? 128 : tile_n, max_lockstep, 0,
                        theta_out};
  return ensemble_solve_graph(sp, n_acc, n_rej, status, lockstep_attempts, (cudaStream_t)stream, nullptr);
}

extern "C" int bs3_ensemble_solve(const float* K, int64_t N, int64_t T, const double* omega, const double* theta0,
                                  double t0, double t1, double rtol, double atol, double* theta_out,
                                  int64_t* n_acc, int64_t* n_rej, int32_t* status, int64_t* lockstep_attempts,
                                  void* stream) {
  return bs3_ensemble_solve_tiled(K, N, T, omega, theta0, t0, t1, rtol, atol, 0, 0, theta_out, n_acc, n_rej, status,
                                  lockstep_attempts, stream);
}

extern "C" int bs3_ensemble_autotune(const float* K, int64_t N, int64_t T, const double* omega, const double* theta0,
                                     double t0, double t1, double rtol, double atol, int64_t lockstep_attempts,
                                     double* scratch_theta, int* tile_out, double* us_out) {
  if (!K || !omega || !theta0 || !scratch_theta || !tile_out || lockstep_attempts < 8) return BS3_ERR_INVALID_ARG;
  int best = 0;
  double best_us = 0.0;
  for (const int tile : {256, 128}) {
    if ((2 * T) % tile != 0 || T < tile / 2) continue;
    double us = 0.0;
    // two bounded solves: the first warms up, the second's attempt loop is timed
    for (int rep = 0; rep < 2; ++rep) {
      int64_t steps = 0;
      float ms = 0.f;
      const EnsembleSpec sp{K, N, T, omega, theta0, t0, t1, rtol, atol, tile, lockstep_attempts, 0, scratch_theta};
      const int r = ensemble_solve_graph(sp, nullptr, nullptr, nullptr, &steps, nullptr, &ms);
      if (r != BS3_OK && r != BS3_ERR_MAX_STEPS) return r;
      us = 1e3 * ms / (double)std::max<int64_t>(1, steps);
    }
    if (best == 0 || us < best_us) {
      best = tile;
      best_us = us;
    }
  }
  if (best == 0) return BS3_ERR_INVALID_ARG;
  *tile_out = best;
  if (us_out) *us_out = best_us;
  return BS3_OK;
}
