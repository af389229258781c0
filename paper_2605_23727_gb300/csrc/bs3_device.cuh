// Device-side building blocks of the sm_103a BS3 solver: stored-weight
// loaders, accumulators for the Sigma precisions of Table MP-Distrib
// (Sec. 2.3), a bounded grid barrier and bit-pattern max reductions.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace bs3 {

enum Kind { K_LCO_CFG = 0, K_LCO_PAPER = 1, K_KURAMOTO = 2, K_CIRCADIAN = 3 };
enum Store { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_F16 = 3, ST_FP8 = 4 };
// Summation modes of one coupling evaluation:
//   SS   G = S, Sigma = S: binary32 products, binary32 sum (fmaf)
//   SD64 G = S, Sigma = D: binary32 products cast to binary64, binary64 sum
//   SD2  G = S, Sigma = D: binary32 products, compensated float-float sum
//   DD   G = D, Sigma = D: binary64 products and sum
enum Mode { M_SS = 0, M_SD64 = 1, M_SD2 = 2, M_DD = 3 };
enum Job { JOB_SOLVE = 0, JOB_RHS = 1, JOB_ATTEMPT = 2 };
enum Variant { V_SINGLE = 0, V_MIXED1 = 1, V_MIXED2 = 2, V_DOUBLE = 3 };
enum Accum { A_F32 = 0, A_FLOAT2 = 1, A_F64 = 2 };
enum Status {
  S_OK = 0, S_INVALID = 1, S_CUDA = 2, S_MAX_STEPS = 3, S_MAX_REJECTS = 4,
  S_STEP_TOO_SMALL = 5, S_TIMEOUT = 6, S_DEVICE_WAIT = 7, S_NONFINITE = 8
};

constexpr int kBlock = 512;          // threads per CTA of the persistent solver
constexpr int kGroupThreads = 128;   // a warp group: four warps share one row block
constexpr int kGroups = kBlock / kGroupThreads;
constexpr int kRBMax = 4;            // largest number of rows per row block
constexpr int kGrpSlots = (kBlock / 32) * kRBMax * 2;  // one set of per-warp partial sums of a row block

// Rows per row block: the streaming products share each j-vector chunk over 4
// rows; so does the ALU-bound pairwise arctangent pass, where four
// independent rows per thread hide the polynomial's latency (N=16384 bf16:
// 23.0 ms per solve against 26.1 ms with two rows).
__host__ __device__ constexpr int rows_per_tile(int) { return 4; }

// Persistent-solver control block (device memory, zeroed before each launch).
struct Control {
  unsigned long long bar;        // grid-barrier arrivals, monotonic
  unsigned long long emax[2];    // bit patterns of E (non-negative binary64), by attempt parity
  unsigned long long red[3];     // starting-step maxima d0, d1, d2
  int status;                    // first failure wins (atomicCAS from 0)
  int cancel_seen[2];            // host cancel flag latched by CTA 0, by attempt parity
  int pad;
  long long n_acc, n_rej, n_rhs, n_out;
  double t, h;
};

// One record per attempt of a solve (optional): t, h, E, accepted, then the
// device time (ns, %globaltimer) spent by CTA 0 from the start of the attempt
// to the end of each of its four barriers (A, B2, B3, B4).
constexpr int kHistDoubles = 8;

// ---------------------------------------------------------------------------
// Memory helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Streaming 16-byte load of weights that never change during a launch.
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

// 16-byte weight load with an L2 eviction-priority policy (createpolicy):
// evict_last keeps weights that fit in L2 resident across stages even after
// other traffic, evict_first keeps a weight stream larger than L2 from
// evicting the j-vectors.
__device__ __forceinline__ unsigned long long l2_policy(bool keep) {
  unsigned long long pol;
  if (keep) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint4 ld_stream16_pol(const void* p, unsigned long long pol) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p), "l"(pol));
  return r;
}

// (n / d)^(1/3) and (n / d)^(1/5) for n, d > 0 without a binary64 division
// (~210 ns of latency on GB300): a binary32 seed of the root of the binary32
// quotient, then one Newton step on y^k d = n in binary64 with a binary32
// estimate of 1 / (k y^(k-1) d); relative error ~1e-14.  The seed's quotient
// is clamped to [1e-30, 1e30]; at the clamps (and when d under- or
// overflows binary32) the step returns +Inf or the clamped root, beyond the
// controller's limits either way.
__device__ __forceinline__ double cbrt_ratio(double n, double d) {
  const float df = (float)d;
  const float yf = cbrtf(fminf(fmaxf(__fdividef((float)n, df), 1e-30f), 1e30f));
  const double y = (double)yf;
  const double r = (double)(1.0f / (3.0f * yf * yf * df));
  return fma(-fma((y * y) * y, d, -n), r, y);
}

__device__ __forceinline__ double root5_ratio(double n, double d) {
  const float df = (float)d;
  const float yf = exp2f(0.2f * log2f(fminf(fmaxf(__fdividef((float)n, df), 1e-30f), 1e30f)));
  const double y = (double)yf;
  const double y2 = y * y, y4 = y2 * y2;
  const double r = (double)(1.0f / (5.0f * (yf * yf) * (yf * yf) * df));
  return fma(-fma(y4 * y, d, -n), r, y);
}

// Grid barrier for a cooperative launch.  Every CTA adds one arrival to a
// monotonic counter (release) and polls it until it reaches its target.  The
// wait is bounded by spin_limit polls; a CTA that gives up sets the status to
// S_DEVICE_WAIT and adds kAbortBias to the counter, which every other waiter
// sees in the same poll.  Returns false when the launch must stop.
constexpr unsigned long long kAbortBias = 1ull << 48;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of nb co-resident CTAs on one monotonic counter (the whole grid,
// or a team of CTAs that solves one system of a batch).
__device__ __forceinline__ bool group_sync(unsigned long long* counter, int* status, unsigned long long& target,
                                           int nb, long long spin_limit, int* s_abort) {
  __syncthreads();
  target += nb;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" :: "l"(counter) : "memory");
    long long it = 0;
    int abort = 0;
    while (true) {
      const unsigned long long v = ld_acquire_u64(counter);
      if (v >= kAbortBias) { abort = 1; break; }
      if (v >= target) break;
      if (++it > spin_limit) {
        atomicCAS(status, 0, (int)S_DEVICE_WAIT);
        atomicAdd(counter, kAbortBias);
        abort = 1;
        break;
      }
      if (it > 256) __nanosleep(32);
    }
    *s_abort = abort;
  }
  __syncthreads();
  return !*s_abort;
}

__device__ __forceinline__ bool grid_sync(Control* c, unsigned long long& target, int nb,
                                          long long spin_limit, int* s_abort) {
  return group_sync(&c->bar, &c->status, target, nb, spin_limit, s_abort);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* slot, double v) {
  // non-negative binary64 (and NaN, whose bits compare above +Inf) order as u64
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Stored-weight loaders: one 16-byte chunk holds VEC elements.
// ---------------------------------------------------------------------------
template <int ST> struct KLoad;

template <> struct KLoad<ST_F64> {
  static constexpr int VEC = 2, BYTES = 8;
  __device__ static __forceinline__ float f(const uint4& r, int e) {
    return (float)get_d(r, e);
  }
  __device__ static __forceinline__ double get_d(const uint4& r, int e) {
    return e == 0 ? __hiloint2double((int)r.y, (int)r.x) : __hiloint2double((int)r.w, (int)r.z);
  }
};
template <> struct KLoad<ST_F32> {
  static constexpr int VEC = 4, BYTES = 4;
  __device__ static __forceinline__ float f(const uint4& r, int e) {
    const uint32_t w = e == 0 ? r.x : e == 1 ? r.y : e == 2 ? r.z : r.w;
    return __uint_as_float(w);
  }
  __device__ static __forceinline__ double get_d(const uint4& r, int e) { return (double)f(r, e); }
};
template <> struct KLoad<ST_BF16> {
  static constexpr int VEC = 8, BYTES = 2;
  __device__ static __forceinline__ float f(const uint4& r, int e) {
    const uint32_t w = (e >> 1) == 0 ? r.x : (e >> 1) == 1 ? r.y : (e >> 1) == 2 ? r.z : r.w;
    return __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
  }
  __device__ static __forceinline__ double get_d(const uint4& r, int e) { return (double)f(r, e); }
};
template <> struct KLoad<ST_F16> {
  static constexpr int VEC = 8, BYTES = 2;
  __device__ static __forceinline__ float f(const uint4& r, int e) {
    const uint32_t w = (e >> 1) == 0 ? r.x : (e >> 1) == 1 ? r.y : (e >> 1) == 2 ? r.z : r.w;
    const unsigned short hbits = (unsigned short)((e & 1) ? (w >> 16) : (w & 0xffffu));
    return __half2float(__ushort_as_half(hbits));
  }
  __device__ static __forceinline__ double get_d(const uint4& r, int e) { return (double)f(r, e); }
};
template <> struct KLoad<ST_FP8> {
  static constexpr int VEC = 16, BYTES = 1;
  __device__ static __forceinline__ float f(const uint4& r, int e) {
    const uint32_t w = (e >> 2) == 0 ? r.x : (e >> 2) == 1 ? r.y : (e >> 2) == 2 ? r.z : r.w;
    const __nv_fp8_storage_t b = (__nv_fp8_storage_t)((w >> (8 * (e & 3))) & 0xffu);
    const __half_raw h = __nv_cvt_fp8_to_halfraw(b, __NV_E4M3);
    return __half2float(__half(h));
  }
  __device__ static __forceinline__ double get_d(const uint4& r, int e) { return (double)f(r, e); }
};

// ---------------------------------------------------------------------------
// Accumulators
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int MODE> struct Acc;

template <> struct Acc<M_SS> {
  float s = 0.f;
  __device__ __forceinline__ void add_f(float k, float v) { s = fmaf(k, v, s); }
  __device__ __forceinline__ void add_d(double k, double v) { s = fmaf((float)k, (float)v, s); }
  __device__ __forceinline__ void xor_merge(int off) { s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off)); }
  __device__ __forceinline__ double value() const { return (double)s; }
};
template <> struct Acc<M_SD64> {
  double s = 0.0;
  __device__ __forceinline__ void add_f(float k, float v) { s = __dadd_rn(s, (double)__fmul_rn(k, v)); }
  __device__ __forceinline__ void add_d(double k, double v) { add_f((float)k, (float)v); }
  __device__ __forceinline__ void xor_merge(int off) { s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off)); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<M_SD2> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_f(float k, float v) {
    float s, e;
    two_sum(hi, __fmul_rn(k, v), s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_d(double k, double v) { add_f((float)k, (float)v); }
  __device__ __forceinline__ void xor_merge(int off) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
    float s, e;
    two_sum(hi, ohi, s, e);
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
  }
  __device__ __forceinline__ double value() const { return __dadd_rn((double)hi, (double)lo); }
};
template <> struct Acc<M_DD> {
  double s = 0.0;
  __device__ __forceinline__ void add_f(float k, float v) { s = fma((double)k, (double)v, s); }
  __device__ __forceinline__ void add_d(double k, double v) { s = fma(k, v, s); }
  __device__ __forceinline__ void xor_merge(int off) { s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off)); }
  __device__ __forceinline__ double value() const { return s; }
};

// sin and cos of a binary64 phase rounded to binary32 -- nearly always the
// correctly rounded values, with no systematic error.  The phase is reduced
// in binary64 to r = th - k pi/2, |r| <= pi/4 (two-constant Cody-Waite, pi/2
// split into a 33-bit head and a binary64 tail), r is split into binary32
// r_hi + r_lo, and the Taylor series of sin and cos (truncated where the next
// term is below 1e-11) are summed in binary32 with every part that reaches the
// last bit carried exactly: the leading r_hi of the sine, 1 - r_hi^2 / 2 of
// the cosine (exact square by FMA, then Fast2Sum), the r_lo terms, and the
// first coefficients -1/6 and 1/24 as binary32 pairs.  Before the final
// rounding only about 0.05 ulp of rounding noise from the small correction
// terms remains, so about 1 % of the results differ from the correct
// rounding, by one ulp, in either direction.  A library sincosf of the
// reduced phase is a few ulp off, and that error is a smooth function of the
// phase: oscillators with nearly equal phases share it, and in the coupling of
// a synchronised cluster it does not average out.
__device__ __forceinline__ void sincos_f_of_d(double th, float* s, float* c) {
  const double kTwoOverPi = 0.6366197723675814;
  const double kHalfPiHi = 1.5707963267341256;      // pi/2 rounded to 33 bits
  const double kHalfPiLo = 6.077100506506192e-11;   // pi/2 - kHalfPiHi
  const double k = rint(th * kTwoOverPi);
  double r = fma(-k, kHalfPiHi, th);
  r = fma(-k, kHalfPiLo, r);
  const float rh = __double2float_rn(r);
  const float rl = __double2float_rn(r - (double)rh);
  const float zh = __fmul_rn(rh, rh);
  const float zl = fmaf(rh, rh, -zh);                // rh^2 = zh + zl exactly
  // sin r = rh + [rl (1 - r^2/2) + r^3 (-1/6 + z/120 - z^2/5040 + z^3/362880 - z^4/39916800)]
  float p = -2.5052108385e-08f;
  p = fmaf(p, zh, 2.7557319224e-06f);
  p = fmaf(p, zh, -1.9841269841e-04f);
  p = fmaf(p, zh, 8.3333333333e-03f);
  const float r3 = __fmul_rn(zh, rh);
  const float u = fmaf(zh, p, 4.967053879312289e-09f);          // -1/6 - fp32(-1/6), then the series
  const float v = fmaf(r3, -0.1666666716337204f, __fmul_rn(r3, u));
  const float sr = __fadd_rn(rh, fmaf(rl, fmaf(-0.5f, zh, 1.0f), v));
  // cos r = (1 - zh/2) - zl/2 - rh rl + r^4 (1/24 - z/720 + z^2/40320 - z^3/3628800 + z^4/479001600)
  const float hz = __fmul_rn(0.5f, zh);
  const float t_hi = __fsub_rn(1.0f, hz);
  const float t_err = __fsub_rn(__fsub_rn(1.0f, t_hi), hz);     // exact: Fast2Sum with |1| >= |hz|
  float q = 2.0876756988e-09f;
  q = fmaf(q, zh, -2.7557319224e-07f);
  q = fmaf(q, zh, 2.4801587302e-05f);
  q = fmaf(q, zh, -1.3888888889e-03f);
  const float z2 = __fmul_rn(zh, zh);
  const float u2 = fmaf(zh, q, -1.2417634698280722e-09f);      // 1/24 - fp32(1/24), then the series
  const float v2 = fmaf(z2, 0.0416666679084301f, __fmul_rn(z2, u2));
  const float corr = __fadd_rn(__fsub_rn(__fsub_rn(t_err, __fmul_rn(0.5f, zl)), __fmul_rn(rh, rl)), v2);
  const float cr = __fadd_rn(t_hi, corr);
  switch ((int)((long long)k & 3)) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

// Arctangent in binary32 (the project's own): atan(x) = x P(x^2) on [0, 1]
// with P the degree-8 minimax polynomial fitted by csrc/fit_atan.py (Lawson's
// algorithm, relative error), and atan(x) = pi/2 - atan(1/x) above 1, 1/x by
// the hardware's approximate reciprocal (within 1 ulp; one instruction instead
// of a correctly rounded division).  Max error 1.8 ulp on [0, 1] and 2.9 ulp
// above 1 (fit script's grid, reciprocal off by one ulp either way).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float atan_f32(float x) {
  const float ax = fabsf(x);
  const bool big = ax > 1.0f;
  const float t = big ? rcp_approx(ax) : ax;
  const float z = t * t;
  float p = 2.849889454e-03f;
  p = fmaf(p, z, -1.606862806e-02f);
  p = fmaf(p, z, 4.269151762e-02f);
  p = fmaf(p, z, -7.504294813e-02f);
  p = fmaf(p, z, 1.064093411e-01f);
  p = fmaf(p, z, -1.420364380e-01f);
  p = fmaf(p, z, 1.999261975e-01f);
  p = fmaf(p, z, -3.333307207e-01f);
  p = fmaf(p, z, 1.000000000e+00f);
  float r = t * p;
  r = big ? (1.57079637f - r) : r;
  return copysignf(r, x);
}

// Packed binary32 pairs (Blackwell f32x2 instructions): each lane performs two
// IEEE operations per instruction, so the results equal the scalar ones.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Two arctangents at once: the same values as atan_f32 lane by lane
// (bit-identical results), with the polynomial in packed instructions.  The
// reduced argument min(|x|, 1/|x|) is one minimum instead of a test and a
// select (for |x| > 1 the approximate reciprocal is below 1 < |x|, for
// |x| <= 1 it is at least 1 >= |x|).
__device__ __forceinline__ void atan_f32x2(float x0, float x1, float& r0, float& r1) {
  const float a0 = fabsf(x0), a1 = fabsf(x1);
  const bool b0 = a0 > 1.0f, b1 = a1 > 1.0f;
  const unsigned long long t = pk2(fminf(a0, rcp_approx(a0)), fminf(a1, rcp_approx(a1)));
  const unsigned long long z = mul2(t, t);
  unsigned long long p = pk2(2.849889454e-03f, 2.849889454e-03f);
  p = fma2(p, z, pk2(-1.606862806e-02f, -1.606862806e-02f));
  p = fma2(p, z, pk2(4.269151762e-02f, 4.269151762e-02f));
  p = fma2(p, z, pk2(-7.504294813e-02f, -7.504294813e-02f));
  p = fma2(p, z, pk2(1.064093411e-01f, 1.064093411e-01f));
  p = fma2(p, z, pk2(-1.420364380e-01f, -1.420364380e-01f));
  p = fma2(p, z, pk2(1.999261975e-01f, 1.999261975e-01f));
  p = fma2(p, z, pk2(-3.333307207e-01f, -3.333307207e-01f));
  p = fma2(p, z, pk2(1.000000000e+00f, 1.000000000e+00f));
  float q0, q1;
  upk2(mul2(t, p), q0, q1);
  q0 = b0 ? (1.57079637f - q0) : q0;
  q1 = b1 ? (1.57079637f - q1) : q1;
  r0 = copysignf(q0, x0);
  r1 = copysignf(q1, x1);
}

}  // namespace bs3
