// Persistent cooperative BS3 solver kernel (one launch per solve).
//
// Per attempt (Eq. Stage-ODE23, Table Butcher-O23, Eq. ERROR-O23):
//   A : Y2 = X + (h/2) K1                         -> j-vector 0     | barrier
//   B2: K2 = f(Y2); Y3 = X + (3h/4) K2            -> j-vector 1     | barrier
//   B3: K3 = f(Y3); X' = X + h(2/9 K1+1/3 K2+4/9 K3) -> j-vector 2  | barrier
//   B4: K4 = f(X'); E = max_k |h sum e_l K_l| / W_k (grid max)      | barrier
//   every CTA then takes the same accept/reject decision from E.
// Each CTA owns a contiguous block of agents (rows) for the whole solve and
// keeps their state (X, X', K1..K4) and per-agent parameters in shared
// memory; only the j-vectors (G-precision values of the coupled component)
// cross CTAs, through global memory between grid barriers.  Inside a CTA,
// four groups of four warps take row blocks of RB agents; a group streams the
// RB rows of stored weights from HBM/L2 with 16-byte non-allocating loads,
// every thread reusing its j-vector chunk over the RB rows.
#pragma once

#include "bs3_device.cuh"
#include "bs3_mlp.cuh"

namespace bs3 {

struct Args {
  // system
  int N, ld;
  const void* q;            // [N][ld] stored weights, zero padded
  const float* scale;       // [N] row scales
  const double* rowsum;     // [N] sum_j s_i q_ij (paper-form oscillators)
  const float* bias;        // [N] row_bias(sum_j |q_ij|): start of the packed float-float sums
  const double* par;        // [N] omega_i or k1_i
  const double* theta_h;    // [N] k1/(k0-k1) (circadian)
  double g[8];              // circadian k0, k2, k3, a, b, c, eps, I0
  // device buffers owned by the system
  double* X;
  double* Xn;
  double* Kb[4];
  float* jv32;              // [3][2][ld]
  double* jv64;             // [3][2][ld]
  Control* ctrl;
  const volatile int* cancel;   // host-mapped cancel flag (may be null)
  volatile double* progress;    // host-mapped progress (may be null)
  // job
  int job, variant, accum;
  int rhs_f, rhs_s, rhs_g;
  double t0, t1, rtol, atol, hmin, hmax, h_given;
  const double* t_out;
  long long n_out;
  double* y_out;
  double* final_y;
  double* out0;
  double* out1;
  long long max_attempts, max_rejects, spin_limit;
  int rc;                   // rows per CTA capacity (ceil(N / grid))
  int slab_bytes;           // > 0: each CTA keeps its rc weight rows in shared memory
  int l2_keep;              // 1: weights fit in L2, load them evict_last; 0: evict_first
  double* hist;             // optional per-attempt records [hist_cap][kHistDoubles]
  long long hist_cap;
  const float* mlp;         // optional learned proposer: kMlpModel binary32 (bf16-rounded weights)
  int smem_mlp_off;         // byte offset of its shared-memory copy in the dynamic region
  int method;               // M_BS32 (Bogacki-Shampine 3(2)) or M_DP54 (Dormand-Prince 5(4))
  int n_slots;              // state slots per agent: 6 (BS3) or 9 (DP5)
};

enum Method { M_BS32 = 0, M_DP54 = 1 };

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Prec {
  int f, s, g;  // 0 = S (binary32), 1 = D (binary64)
};

// Table MP-Distrib (Sec. 2.3): (F, Sigma, G) of stages k2, k3, k4.
__device__ __forceinline__ Prec variant_prec(int v, int stage) {
  if (v == V_SINGLE) return Prec{0, 0, 0};
  if (v == V_MIXED1) return stage == 4 ? Prec{1, 1, 0} : Prec{0, 0, 0};
  if (v == V_MIXED2) return Prec{1, 1, 0};
  return Prec{1, 1, 1};
}

// Dormand-Prince 5(4) (the embedded pair of the extension to other explicit
// schemes, Sec. 4): a_lm (l = 2..7, m = 1..l-1; row 7 = b, the FSAL row) and
// e = b - b_hat, each the binary64 rounding of the published rational.
static __constant__ double kDpA[8][8] = {
    {0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0},
    {0, 1.0 / 5.0, 0, 0, 0, 0, 0, 0},
    {0, 3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0, 0},
    {0, 44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0, 0},
    {0, 19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0, 0},
    {0, 9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0, 0},
    {0, 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0},
};
static __constant__ double kDpE[8] = {0, 71.0 / 57600.0, 0.0, -71.0 / 16695.0, 71.0 / 1920.0,
                                      -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0};

// Table MP-Distrib carried to the seven stages: Mixed1 keeps every stage in
// binary32 except the last (FSAL) one, Mixed2 has F and Sigma in binary64.
__device__ __forceinline__ Prec variant_prec_dp(int v, int stage) {
  if (v == V_SINGLE) return Prec{0, 0, 0};
  if (v == V_MIXED1) return stage == 7 ? Prec{1, 1, 0} : Prec{0, 0, 0};
  if (v == V_MIXED2) return Prec{1, 1, 0};
  return Prec{1, 1, 1};
}

__device__ __forceinline__ int sum_mode(Prec p, int accum) {
  if (p.g == 1) return M_DD;
  if (p.s == 0) return M_SS;
  return accum == A_F64 ? M_SD64 : (accum == A_FLOAT2 ? M_SD2 : M_SS);
}

template <int KIND> struct Dim { static constexpr int d = (KIND == K_KURAMOTO) ? 1 : (KIND == K_CIRCADIAN ? 4 : 2); };

// ---------------------------------------------------------------------------
// j-vectors: the j-side value of agent i in G precision (component 0 of the
// stage argument; sin and cos of it for Kuramoto).
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void put_jv(const Args& a, int buf, int i, const double* Y, int g, bool single,
                                       float2* cache = nullptr) {
  const size_t o0 = (size_t)(buf * 2) * a.ld + i;
  const size_t o1 = o0 + a.ld;
  if (KIND == K_KURAMOTO) {
    if (g == 0) {
      float s, c;
      if (single) sincosf((float)Y[0], &s, &c);
      else sincos_f_of_d(Y[0], &s, &c);
      // binary32 j-vector of Kuramoto: interleaved (sin, cos) pairs
      reinterpret_cast<float2*>(a.jv32 + (size_t)(buf * 2) * a.ld)[i] = make_float2(s, c);
      if (cache) *cache = make_float2(s, c);   // the i-side finish of the next stage reads them
    } else {
      double s, c;
      sincos(Y[0], &s, &c);
      a.jv64[o0] = s;
      a.jv64[o1] = c;
    }
  } else {
    if (g == 0) a.jv32[o0] = (float)Y[0];
    else a.jv64[o0] = Y[0];
  }
}

// ---------------------------------------------------------------------------
// Accumulator transport between the warps of a group (packed in 64 bits).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long pack(const Acc<M_SS>& x) { return (unsigned long long)__float_as_uint(x.s); }
__device__ __forceinline__ unsigned long long pack(const Acc<M_SD64>& x) { return (unsigned long long)__double_as_longlong(x.s); }
__device__ __forceinline__ unsigned long long pack(const Acc<M_DD>& x) { return (unsigned long long)__double_as_longlong(x.s); }
__device__ __forceinline__ unsigned long long pack(const Acc<M_SD2>& x) {
  return ((unsigned long long)__float_as_uint(x.lo) << 32) | (unsigned long long)__float_as_uint(x.hi);
}
__device__ __forceinline__ void merge(Acc<M_SS>& x, unsigned long long b) { x.s = __fadd_rn(x.s, __uint_as_float((unsigned)b)); }
__device__ __forceinline__ void merge(Acc<M_SD64>& x, unsigned long long b) { x.s = __dadd_rn(x.s, __longlong_as_double((long long)b)); }
__device__ __forceinline__ void merge(Acc<M_DD>& x, unsigned long long b) { x.s = __dadd_rn(x.s, __longlong_as_double((long long)b)); }
__device__ __forceinline__ void merge(Acc<M_SD2>& x, unsigned long long b) {
  const float ohi = __uint_as_float((unsigned)(b & 0xffffffffu)), olo = __uint_as_float((unsigned)(b >> 32));
  float s, e;
  two_sum(x.hi, ohi, s, e);
  x.hi = s;
  x.lo = __fadd_rn(__fadd_rn(x.lo, olo), e);
}

// Synchronises the gt threads of warp group g (a single warp needs only a
// warp barrier; larger groups use named barrier 1 + g).
__device__ __forceinline__ void group_bar(int g, int gt) {
  if (gt == 32) __syncwarp();
  else asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(gt) : "memory");
}

// A thread's packed partial sums into its accumulator (hi and lo parts of
// the float-float sum; lo is zero for binary32 sums).
__device__ __forceinline__ void set_packed(Acc<M_SS>& x, float hi, float) { x.s = hi; }
__device__ __forceinline__ void set_packed(Acc<M_SD2>& x, float hi, float lo) { x.hi = hi; x.lo = lo; }
__device__ __forceinline__ void set_packed(Acc<M_SD64>&, float, float) {}
__device__ __forceinline__ void set_packed(Acc<M_DD>&, float, float) {}

// Bias of a row's packed float-float sums (see gemv_rows and cc_rows): the power of two
// B >= 2.5 s for s = sum_j |q_ij| (s computed in binary64; 2.5 covers its
// rounding and that of q to binary32).  Rows whose sum is not below 1e37 get
// B = 0, plain binary32 partial sums with approximate error terms.
__host__ __device__ inline float row_bias(double s) {
  if (!(s < 1e37)) return 0.0f;
  if (!(s > 0.0)) return 1.0f;
  int e = 0;
  frexp(2.5 * s, &e);   // 2.5 s = f 2^e, f in [0.5, 1)
  return ldexpf(1.0f, e < -126 ? -126 : e);
}

// The largest row_bias of rows rb .. rb+nr-1 (0, no bias, when one of them
// has none); every thread of the CTA calls it and gets the same value.
__device__ __forceinline__ float cta_bias(const float* bias, int rb, int nr) {
  __shared__ unsigned s_bits;
  if (threadIdx.x == 0) s_bits = 0u;
  __syncthreads();
  unsigned m = 0u;
  for (int li = threadIdx.x; li < nr; li += blockDim.x) {
    const float v = bias[rb + li];
    const unsigned u = (v > 0.0f) ? __float_as_uint(v) : 0x7f800000u;   // positive floats order as integers
    m = u > m ? u : m;
  }
  if (m) atomicMax(&s_bits, m);
  __syncthreads();
  const unsigned b = s_bits;
  __syncthreads();
  return b == 0x7f800000u ? 0.0f : (b ? __uint_as_float(b) : 1.0f);
}

// ---------------------------------------------------------------------------
// Coupling partial sums of one row block (rows row0 .. row0+nrows-1) for the
// columns of thread lt of a 128-thread group; then a warp-level reduction.
// ---------------------------------------------------------------------------
template <int ST, int MODE, int NV, int RB, bool RES>
__device__ __forceinline__ void gemv_rows(const Args& a, int buf, int row0, int lrow0, int nrows, int lt, int gt,
                                         const unsigned char* slab, float cbias, Acc<MODE> (&acc)[RB][NV]) {
  using L = KLoad<ST>;
  constexpr int VEC = L::VEC;
  constexpr bool DD = (MODE == M_DD);
  // weights come from the CTA's shared-memory slab (RES) or stream from HBM/L2
  const char* qb = RES ? (const char*)slab + (size_t)lrow0 * a.ld * L::BYTES
                       : (const char*)a.q + (size_t)row0 * a.ld * L::BYTES;
  const size_t rstride = (size_t)a.ld * L::BYTES;
  const float* v32 = a.jv32 + (size_t)(buf * 2) * a.ld;
  const double* v64 = a.jv64 + (size_t)(buf * 2) * a.ld;
  const unsigned long long pol = l2_policy(a.l2_keep != 0);
  // Kuramoto with binary32 sums (Sigma = S, or the float-float Sigma = D):
  // the sine and cosine sums of a row advance together in packed f32x2
  // instructions.  The float-float sums start from the CTA's bias B, a power
  // of two >= 2.5 sum_j |q_ij| for each of its rows: every product
  // |q_ij v_j| <= |q_ij| (|v_j| <= 1), so the running high part stays in
  // [B/2, 3B/2], above every product in magnitude, and Fast2Sum (Dekker) gives
  // each addition's rounding error exactly in three operations instead of
  // TwoSum's six; hi - B is exact (Sterbenz) at the end.
  constexpr bool PACKED = (NV == 2) && (MODE == M_SS || MODE == M_SD2);
  const float bias = (PACKED && MODE == M_SD2) ? cbias : 0.0f;
  unsigned long long acc2[RB], lo2[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    acc2[r] = pk2(bias, bias);
    lo2[r] = 0ull;
  }
#pragma unroll(VEC >= 16 ? 1 : 2)
  for (int col = lt * VEC; col < a.ld; col += gt * VEC) {
    uint4 raw[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const char* p = qb + (size_t)r * rstride + (size_t)col * L::BYTES;
      raw[r] = (r < nrows) ? (RES ? *reinterpret_cast<const uint4*>(p) : ld_stream16_pol(p, pol))
                           : make_uint4(0u, 0u, 0u, 0u);
    }
    if (!DD && NV == 2) {
      // interleaved (sin, cos) of the columns col .. col + VEC - 1
      const float4* src = reinterpret_cast<const float4*>(v32 + 2 * (size_t)col);
      unsigned long long sc[VEC];
#pragma unroll
      for (int q = 0; q < VEC / 2; ++q) {
        const float4 t = src[q];
        sc[2 * q] = pk2(t.x, t.y);
        sc[2 * q + 1] = pk2(t.z, t.w);
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const float k = L::f(raw[r], e);
          if (PACKED) {
            const unsigned long long k2 = pk2(k, k);
            if (MODE == M_SS) {
              acc2[r] = fma2(k2, sc[e], acc2[r]);
            } else {   // fast_two_sum of (hi, k v), then lo += e, for both sums at once
              const unsigned long long p = mul2(k2, sc[e]);
              const unsigned long long sm = add2(acc2[r], p);
              lo2[r] = add2(lo2[r], sub2(p, sub2(sm, acc2[r])));
              acc2[r] = sm;
            }
          } else {
            float sv0, sv1;
            upk2(sc[e], sv0, sv1);
            acc[r][0].add_f(k, sv0);
            acc[r][NV - 1].add_f(k, sv1);
          }
        }
    } else if (!DD) {
      float vv[NV][VEC];
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        const float* src = v32 + (size_t)n * a.ld + col;
        if (VEC >= 4) {
#pragma unroll
          for (int e = 0; e < VEC; e += 4) {
            const float4 t = *reinterpret_cast<const float4*>(src + e);
            vv[n][e] = t.x; vv[n][e + 1] = t.y; vv[n][e + 2] = t.z; vv[n][e + 3] = t.w;
          }
        } else {
          const float2 t = *reinterpret_cast<const float2*>(src);
          vv[n][0] = t.x; vv[n][VEC > 1 ? 1 : 0] = t.y;
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const float k = L::f(raw[r], e);
#pragma unroll
          for (int n = 0; n < NV; ++n) acc[r][n].add_f(k, vv[n][e]);
        }
    } else {
      double vv[NV][VEC];
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        const double* src = v64 + (size_t)n * a.ld + col;
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
          const double2 t = *reinterpret_cast<const double2*>(src + e);
          vv[n][e] = t.x; vv[n][e + 1] = t.y;
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const double k = L::get_d(raw[r], e);
#pragma unroll
          for (int n = 0; n < NV; ++n) acc[r][n].add_d(k, vv[n][e]);
        }
    }
  }
  if (PACKED) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      float a0, a1, l0, l1;
      upk2(acc2[r], a0, a1);
      upk2(lo2[r], l0, l1);
      if (MODE == M_SD2) {
        a0 = __fsub_rn(a0, bias);
        a1 = __fsub_rn(a1, bias);
      }
      set_packed(acc[r][0], a0, l0);
      set_packed(acc[r][NV - 1], a1, l1);
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int n = 0; n < NV; ++n)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[r][n].xor_merge(off);
}

// Circadian interaction: r_i = sum_j q_ij atan(x_j - x_i) (Eq. CC).
template <int ST, int MODE, int RB>
__device__ __forceinline__ void cc_rows(const Args& a, int buf, int row0, int nrows, int lt, int gt, float cbias,
                                       Acc<MODE> (&acc)[RB][1]) {
  using L = KLoad<ST>;
  constexpr int VEC = L::VEC;
  constexpr bool DD = (MODE == M_DD);
  const char* qb = (const char*)a.q;
  const size_t rstride = (size_t)a.ld * L::BYTES;
  const float* v32 = a.jv32 + (size_t)(buf * 2) * a.ld;
  const double* v64 = a.jv64 + (size_t)(buf * 2) * a.ld;
  const unsigned long long pol = l2_policy(a.l2_keep != 0);
  float xi32[RB];
  double xi64[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const int i = row0 + (r < nrows ? r : 0);
    xi32[r] = DD ? 0.f : v32[i];
    xi64[r] = DD ? v64[i] : 0.0;
  }
  // the weight chunks of the next iteration are loaded before the current
  // one's arctangents run, so the stream's latency hides behind them
  // the float-float sum of a Sigma = D stage runs as a packed Fast2Sum over
  // the even and odd columns of each row (two accumulators, merged after the
  // loop), both started from 2B for the CTA's bias B: |arctan| <= pi/2, so
  // 2B >= 5 sum_j |q_ij| keeps every high part above every product (as in
  // gemv_rows)
  constexpr bool PSD2 = (MODE == M_SD2 && VEC <= 8);
  const float bias = PSD2 ? 2.0f * cbias : 0.0f;
  unsigned long long hi2[RB], lo2[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    hi2[r] = pk2(bias, bias);
    lo2[r] = 0ull;
  }
  uint4 nxt[RB];
  {
    const int col = lt * VEC;
#pragma unroll
    for (int r = 0; r < RB; ++r)
      nxt[r] = (r < nrows && col < a.ld)
                   ? ld_stream16_pol(qb + (size_t)(row0 + r) * rstride + (size_t)col * L::BYTES, pol)
                   : make_uint4(0u, 0u, 0u, 0u);
  }
  for (int col = lt * VEC; col < a.ld; col += gt * VEC) {
    uint4 raw[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) raw[r] = nxt[r];
    const int ncol = col + gt * VEC;
#pragma unroll
    for (int r = 0; r < RB; ++r)
      nxt[r] = (r < nrows && ncol < a.ld)
                   ? ld_stream16_pol(qb + (size_t)(row0 + r) * rstride + (size_t)ncol * L::BYTES, pol)
                   : make_uint4(0u, 0u, 0u, 0u);
    if (!DD) {
      float xj[VEC];
#pragma unroll
      for (int e = 0; e < VEC; e += 4) {
        if (VEC >= 4) {
          const float4 t = *reinterpret_cast<const float4*>(v32 + col + e);
          xj[e] = t.x; xj[e + 1] = t.y; xj[e + 2] = t.z; xj[e + 3] = t.w;
        } else {
          const float2 t = *reinterpret_cast<const float2*>(v32 + col);
          xj[0] = t.x; xj[VEC > 1 ? 1 : 0] = t.y;
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
          float a0, a1;
          atan_f32x2(__fsub_rn(xj[e], xi32[r]), __fsub_rn(xj[e + 1], xi32[r]), a0, a1);
          if (PSD2) {
            const unsigned long long pr = mul2(pk2(L::f(raw[r], e), L::f(raw[r], e + 1)), pk2(a0, a1));
            const unsigned long long sm = add2(hi2[r], pr);
            lo2[r] = add2(lo2[r], sub2(pr, sub2(sm, hi2[r])));
            hi2[r] = sm;
          } else {
            acc[r][0].add_f(L::f(raw[r], e), a0);
            acc[r][0].add_f(L::f(raw[r], e + 1), a1);
          }
        }
    } else {
      double xj[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) xj[e] = v64[col + e];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; ++e)
          acc[r][0].add_d(L::get_d(raw[r], e), atan(__dsub_rn(xj[e], xi64[r])));
    }
  }
  if (PSD2) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      float e0, e1, l0, l1, s_, er;
      upk2(hi2[r], e0, e1);
      upk2(lo2[r], l0, l1);
      e0 = __fsub_rn(e0, bias);
      e1 = __fsub_rn(e1, bias);
      two_sum(e0, e1, s_, er);
      set_packed(acc[r][0], s_, __fadd_rn(__fadd_rn(l0, l1), er));
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[r][0].xor_merge(off);
}

// ---------------------------------------------------------------------------
// Agent term F and the i-side finish of the coupling: K_l of agent i.
// Y: stage argument of agent i (d values); s0, s1: coupling sums (binary32
// values when Sigma = S).  Operation order mirrors the definitions exactly.
// ---------------------------------------------------------------------------
struct RowPar {
  float scale;
  double par, th, rowsum;
};

template <int KIND>
__device__ __forceinline__ void finish(const Args& a, const RowPar& rp, const double* Y, double s0, double s1,
                                       Prec p, bool single, double* K, const float2* cached = nullptr,
                                       const double2* cached64 = nullptr) {
  if (KIND == K_KURAMOTO) {
    if (p.s == 0) {
      const float sc = rp.scale;
      const float S = (float)s0 * sc, C = (float)s1 * sc;
      float si, ci;
      if (cached) {   // the same values, from this row's j-vector of this stage argument
        si = cached->x;
        ci = cached->y;
      } else if (single) {
        sincosf((float)Y[0], &si, &ci);
      } else {
        sincos_f_of_d(Y[0], &si, &ci);
      }
      const float cpl = ci * S - si * C;
      K[0] = p.f == 0 ? (double)((float)rp.par + cpl) : rp.par + (double)cpl;
    } else {
      const double sc = (double)rp.scale;
      const double S = s0 * sc, C = s1 * sc;
      double si, ci;
      if (cached64) {   // the same values, computed while the previous barrier waited
        si = cached64->x;
        ci = cached64->y;
      } else {
        sincos(Y[0], &si, &ci);
      }
      const double cpl = ci * S - si * C;
      K[0] = p.f == 0 ? (double)((float)rp.par + (float)cpl) : rp.par + cpl;
    }
  } else if (KIND == K_LCO_CFG) {
    double ax;
    if (p.s == 0) ax = (double)((float)s0 * rp.scale);
    else ax = s0 * (double)rp.scale;
    if (p.f == 0) {
      const float w = (float)rp.par, x = (float)Y[0];
      K[0] = (double)(float)Y[1];
      K[1] = (double)((-(w * w) * x) + (float)ax);
    } else {
      const double w = rp.par;
      K[0] = Y[1];
      K[1] = (-(w * w) * Y[0]) + ax;
    }
  } else if (KIND == K_LCO_PAPER) {
    double cpl;
    if (p.s == 0) {
      const float mx = (float)s0 * rp.scale;
      cpl = (double)(mx - (float)rp.rowsum * (float)Y[0]);
    } else {
      const double mx = s0 * (double)rp.scale;
      cpl = mx - rp.rowsum * Y[0];
    }
    if (p.f == 0) {
      K[0] = (double)((float)Y[1] + (float)cpl);
      K[1] = (double)(-(float)Y[0]);
    } else {
      K[0] = Y[1] + cpl;
      K[1] = -Y[0];
    }
  } else {  // circadian
    double cpl;
    if (p.s == 0) {
      const float th = (float)rp.th;
      const float x2 = (float)Y[1], x2s = x2 * x2;
      const float pref = ((float)a.g[0] * th * (float)a.g[3]) / (th + x2s * x2s);
      cpl = (double)(pref * ((float)s0 * rp.scale));
    } else {
      const double th = rp.th;
      const double x2 = Y[1], x2s = x2 * x2;
      const double pref = (a.g[0] * th * a.g[3]) / (th + x2s * x2s);
      cpl = pref * (s0 * (double)rp.scale);
    }
    if (p.f == 0) {
      const float x1 = (float)Y[0], x2 = (float)Y[1], x3 = (float)Y[2], x4 = (float)Y[3];
      const float k0 = (float)a.g[0], k2 = (float)a.g[1], k3 = (float)a.g[2], aa = (float)a.g[3];
      const float b = (float)a.g[4], c = (float)a.g[5], eps = (float)a.g[6], I0 = (float)a.g[7];
      const float k1 = (float)rp.par, th = (float)rp.th;
      const float x2s = x2 * x2;
      const float hill = (k0 * th) / (th + x2s * x2s);
      const float F1 = hill * (aa * x1 * x1 + 1.f) - k1 * x1;
      K[0] = (double)(F1 + (float)cpl);
      K[1] = (double)(k2 * (x1 - x2));
      K[2] = (double)(x3 * (1.f - x3 * x3 / 3.f) - x4 + I0 * (1.f - (k3 * k3) / (k3 * k3 + x1 * x1)));
      K[3] = (double)(eps * (x3 + b - c * x4));
    } else {
      const double x1 = Y[0], x2 = Y[1], x3 = Y[2], x4 = Y[3];
      const double k0 = a.g[0], k2 = a.g[1], k3 = a.g[2], aa = a.g[3];
      const double b = a.g[4], c = a.g[5], eps = a.g[6], I0 = a.g[7];
      const double k1 = rp.par, th = rp.th;
      const double x2s = x2 * x2;
      const double hill = (k0 * th) / (th + x2s * x2s);
      const double F1 = hill * (aa * x1 * x1 + 1.0) - k1 * x1;
      K[0] = F1 + cpl;
      K[1] = k2 * (x1 - x2);
      K[2] = x3 * (1.0 - x3 * x3 / 3.0) - x4 + I0 * (1.0 - (k3 * k3) / (k3 * k3 + x1 * x1));
      K[3] = eps * (x3 + b - c * x4);
    }
  }
}

// ---------------------------------------------------------------------------
// Row epilogues of the phases.  One function with a runtime switch keeps the
// number of template instantiations of the coupling loops small.  The state
// of the CTA's agents lives in shared memory: six slots [d][rc] whose roles
// (X, X', K1..K4) rotate on accepted steps.
// ---------------------------------------------------------------------------
enum Phase { PH_RHS = 0, PH_K1 = 1, PH_F1 = 2, PH_B2 = 3, PH_B3 = 4, PH_B4 = 5, PH_D2 = 6 };
// Dormand-Prince stage l (2..7) is phase PH_D2 + l - 2.

struct Ctx {
  const unsigned char* slab;  // shared-memory copy of this CTA's weight rows (or null)
  int gt;                     // threads per warp group of the coupling pass
  double* S;          // shared state slots
  double* spar;       // shared per-agent omega_i / k1_i
  double* sth;        // shared k1/(k0-k1)
  double* srs;        // shared row sums
  float* sscale;      // shared row scales
  float cbias;        // bias of the float-float sums (Kuramoto, circadian): the largest row_bias of the CTA's rows
  float2* sisc;       // shared binary32 (sin, cos) of each row's last j-vector (Kuramoto), or null
  double2* sisc64;    // shared binary64 (sin, cos) of each row's stage argument (Kuramoto), or null
  bool have64;        // sisc64 holds this stage's values
  int rc, rb, nr;
  int rank, nb;      // this CTA's place in the group of CTAs that solves the system (nb = 1: alone)
  int iX, iXn, iK1, iK2, iK3, iK4;
  int iK7;           // Dormand-Prince: slot of K_7 (K_1 in iK1, K_2..K_6 fixed in slots 3..7)
  double c21, c32, hs, h0s, thr, rtol;
  Prec p;    // precision of the stage being evaluated
  Prec pn;   // G precision of the next j-vector
  bool single;
  double m0, m1;  // per-thread maxima (starting-step norms, error)
};

// BS3 coefficients (Table Butcher-O23); e = b - b~.
constexpr double kB1 = 2.0 / 9.0, kB2 = 1.0 / 3.0, kB3 = 4.0 / 9.0;
constexpr double kE1 = -5.0 / 72.0, kE2 = 1.0 / 12.0, kE3 = 1.0 / 9.0, kE4 = -1.0 / 8.0;

// stage combinations in the state precision (binary32 for Single)
__device__ __forceinline__ double axpy_state(double x, double c, double k, bool single) {
  if (single) return (double)((float)x + (float)c * (float)k);
  return x + c * k;
}

__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000ll); }
__device__ __forceinline__ double max_nan(double m, double v) { return (v != v || m != m) ? nan_d() : fmax(m, v); }

template <int KIND>
__device__ __forceinline__ double& sv(const Ctx& x, int slot, int c, int li) {
  return x.S[(slot * Dim<KIND>::d + c) * x.rc + li];
}

// Slot of Dormand-Prince stage value K_m: K_1 and K_7 swap on accepted steps
// (FSAL), K_2..K_6 stay in slots 3..7.
__device__ __forceinline__ int dp_slot(const Ctx& x, int m) {
  return m == 1 ? x.iK1 : (m == 7 ? x.iK7 : m + 1);
}

// Dormand-Prince stage argument Y_l = X + h (sum_{m<l} a_lm K_m), the sum
// over the nonzero a_lm in increasing m, in the state precision.
template <int KIND>
__device__ __forceinline__ double dp_arg(const Ctx& x, int l, int c, int li) {
  const double xo = sv<KIND>(x, x.iX, c, li);
  if (x.single) {
    float acc = 0.f;
    bool first = true;
    for (int m = 1; m < l; ++m) {
      const double am = kDpA[l][m];
      if (am == 0.0) continue;
      const float term = (float)am * (float)sv<KIND>(x, dp_slot(x, m), c, li);
      acc = first ? term : acc + term;
      first = false;
    }
    return (double)((float)xo + (float)x.hs * acc);
  }
  double acc = 0.0;
  bool first = true;
  for (int m = 1; m < l; ++m) {
    const double am = kDpA[l][m];
    if (am == 0.0) continue;
    const double term = am * sv<KIND>(x, dp_slot(x, m), c, li);
    acc = first ? term : acc + term;
    first = false;
  }
  return xo + x.hs * acc;
}

// Epilogue of Dormand-Prince stage l: K_l, then the next stage argument and
// its j-vector (Y_7 = X'), or after the last stage the error of Eq. ERROR-O23
// with e = b - b_hat.
template <int KIND>
__device__ __forceinline__ void epilogue_dp(const Args& a, Ctx& x, int l, int li, double s0, double s1) {
  constexpr int d = Dim<KIND>::d;
  const int i = x.rb + li;
  const RowPar rp{x.sscale[li], x.spar[li], x.sth[li], x.srs[li]};
  double Y[d], K[d];
#pragma unroll
  for (int c = 0; c < d; ++c) Y[c] = (l == 7) ? sv<KIND>(x, x.iXn, c, li) : dp_arg<KIND>(x, l, c, li);
  finish<KIND>(a, rp, Y, s0, s1, x.p, x.single, K, x.sisc ? x.sisc + li : nullptr);
#pragma unroll
  for (int c = 0; c < d; ++c) sv<KIND>(x, dp_slot(x, l), c, li) = K[c];
  if (l < 7) {
#pragma unroll
    for (int c = 0; c < d; ++c) {
      Y[c] = dp_arg<KIND>(x, l + 1, c, li);
      if (l + 1 == 7) sv<KIND>(x, x.iXn, c, li) = Y[c];
    }
    put_jv<KIND>(a, (l + 1) & 1, i, Y, x.pn.g, x.single, x.sisc ? x.sisc + li : nullptr);
    return;
  }
#pragma unroll
  for (int c = 0; c < d; ++c) {
    double dv;
    if (x.single) {
      float acc = 0.f;
      bool first = true;
      for (int m = 1; m <= 7; ++m) {
        const double em = kDpE[m];
        if (em == 0.0) continue;
        const float term = (float)em * (float)sv<KIND>(x, dp_slot(x, m), c, li);
        acc = first ? term : acc + term;
        first = false;
      }
      dv = (double)((float)x.hs * acc);
    } else {
      double acc = 0.0;
      bool first = true;
      for (int m = 1; m <= 7; ++m) {
        const double em = kDpE[m];
        if (em == 0.0) continue;
        const double term = em * sv<KIND>(x, dp_slot(x, m), c, li);
        acc = first ? term : acc + term;
        first = false;
      }
      dv = x.hs * acc;
    }
    const double w = fmax(fmax(fabs(sv<KIND>(x, x.iX, c, li)), fabs(Y[c])), x.thr);
    double v = fabs(dv) / w;
    if (!isfinite(Y[c]) || !isfinite(K[c])) v = nan_d();
    x.m1 = max_nan(x.m1, v);
  }
}

template <int KIND>
__device__ __forceinline__ void epilogue(const Args& a, Ctx& x, int phase, int li, double s0, double s1) {
  constexpr int d = Dim<KIND>::d;
  if (phase >= PH_D2) {
    epilogue_dp<KIND>(a, x, phase - PH_D2 + 2, li, s0, s1);
    return;
  }
  const int N = a.N;
  const int i = x.rb + li;
  const RowPar rp{x.sscale[li], x.spar[li], x.sth[li], x.srs[li]};
  double Y[d], K[d];
#pragma unroll
  for (int c = 0; c < d; ++c) {
    const double xo = sv<KIND>(x, x.iX, c, li);
    switch (phase) {
      case PH_F1: Y[c] = axpy_state(xo, x.h0s, sv<KIND>(x, x.iK1, c, li), x.single); break;
      case PH_B2: Y[c] = axpy_state(xo, x.c21, sv<KIND>(x, x.iK1, c, li), x.single); break;
      case PH_B3: Y[c] = axpy_state(xo, x.c32, sv<KIND>(x, x.iK2, c, li), x.single); break;
      case PH_B4: Y[c] = sv<KIND>(x, x.iXn, c, li); break;
      default: Y[c] = xo; break;   // PH_RHS, PH_K1
    }
  }
  finish<KIND>(a, rp, Y, s0, s1, x.p, x.single, K, x.sisc ? x.sisc + li : nullptr,
               x.have64 ? x.sisc64 + li : nullptr);
  switch (phase) {
    case PH_RHS:
#pragma unroll
      for (int c = 0; c < d; ++c) a.out0[c * N + i] = K[c];
      break;
    case PH_K1:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        sv<KIND>(x, x.iK1, c, li) = K[c];
        const double sc = x.rtol * fmax(fabs(Y[c]), x.thr);
        x.m0 = max_nan(x.m0, fabs(Y[c]) / sc);
        x.m1 = max_nan(x.m1, fabs(K[c]) / sc);
      }
      break;
    case PH_F1:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        const double sc = x.rtol * fmax(fabs(sv<KIND>(x, x.iX, c, li)), x.thr);
        x.m0 = max_nan(x.m0, fabs(K[c] - sv<KIND>(x, x.iK1, c, li)) / sc);
      }
      break;
    case PH_B2:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        sv<KIND>(x, x.iK2, c, li) = K[c];
        Y[c] = axpy_state(sv<KIND>(x, x.iX, c, li), x.c32, K[c], x.single);
      }
      put_jv<KIND>(a, 1, i, Y, x.pn.g, x.single, x.sisc ? x.sisc + li : nullptr);
      break;
    case PH_B3:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        sv<KIND>(x, x.iK3, c, li) = K[c];
        const double k1 = sv<KIND>(x, x.iK1, c, li), k2 = sv<KIND>(x, x.iK2, c, li), k3 = K[c];
        const double xo = sv<KIND>(x, x.iX, c, li);
        double xn;
        if (x.single) {
          const float cmb = ((float)kB1 * (float)k1 + (float)kB2 * (float)k2) + (float)kB3 * (float)k3;
          xn = (double)((float)xo + (float)x.hs * cmb);
        } else {
          xn = xo + x.hs * ((kB1 * k1 + kB2 * k2) + kB3 * k3);
        }
        sv<KIND>(x, x.iXn, c, li) = xn;
        Y[c] = xn;
      }
      put_jv<KIND>(a, 2, i, Y, x.pn.g, x.single, x.sisc ? x.sisc + li : nullptr);
      break;
    default:  // PH_B4: K4 and the error of Eq. ERROR-O23
#pragma unroll
      for (int c = 0; c < d; ++c) {
        sv<KIND>(x, x.iK4, c, li) = K[c];
        const double k1 = sv<KIND>(x, x.iK1, c, li), k2 = sv<KIND>(x, x.iK2, c, li);
        const double k3 = sv<KIND>(x, x.iK3, c, li), k4 = K[c];
        double dv;
        if (x.single) {
          const float cmb = (((float)kE1 * (float)k1 + (float)kE2 * (float)k2) + (float)kE3 * (float)k3) +
                            (float)kE4 * (float)k4;
          dv = (double)((float)x.hs * cmb);
        } else {
          dv = x.hs * (((kE1 * k1 + kE2 * k2) + kE3 * k3) + kE4 * k4);
        }
        const double w = fmax(fmax(fabs(sv<KIND>(x, x.iX, c, li)), fabs(Y[c])), x.thr);
        double v = fabs(dv) / w;
        if (!isfinite(Y[c]) || !isfinite(k4)) v = nan_d();
        x.m1 = max_nan(x.m1, v);
      }
      break;
  }
}

// ---------------------------------------------------------------------------
// One stage over the CTA's agents: row blocks of RB agents go to the four
// warp groups; each group reduces its partial sums through shared memory
// and the first RB threads of the group run the epilogues.
// ---------------------------------------------------------------------------
template <int KIND, int ST, int MODE, bool RES, int RB>
__device__ __forceinline__ void stage_m(const Args& a, Ctx& x, int phase, int buf, unsigned long long* red) {
  constexpr int NV = (KIND == K_KURAMOTO) ? 2 : 1;
  // warp groups of gt threads (4 x 128, 8 x 64 or 16 x 32) each take RB rows at
  // a time; the smallest groups that still cover the CTA's rows in one pass
  const int gt = x.gt, ng = kBlock / gt, wpg = gt >> 5;
  const int g = threadIdx.x / gt, lt = threadIdx.x % gt;
  const int wig = lt >> 5, lane = lt & 31;
  const int nrb = (x.nr + RB - 1) / RB;
  // two sets of partial-sum slots, used alternately: a group's warps write the
  // next row block's sums while its first threads still read this one's, so
  // one group barrier per row block suffices (the CTA-wide barrier that ends
  // every stage separates the last reads from the next stage's writes)
  unsigned long long* slots = red;
  for (int rbk = g; rbk < nrb; rbk += ng) {
    const int lrow0 = rbk * RB;
    const int nrows = min(RB, x.nr - lrow0);
    Acc<MODE> acc[RB][NV];
    if (KIND == K_CIRCADIAN) cc_rows<ST, MODE, RB>(a, buf, x.rb + lrow0, nrows, lt, gt, x.cbias, (Acc<MODE>(&)[RB][1])acc);
    else gemv_rows<ST, MODE, NV, RB, RES>(a, buf, x.rb + lrow0, lrow0, nrows, lt, gt, x.slab, x.cbias, acc);
    const int wbase = g * wpg;   // first warp of this group
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int n = 0; n < NV; ++n) slots[((wbase + wig) * kRBMax + r) * 2 + n] = pack(acc[r][n]);
    }
    group_bar(g, gt);
    if (lt < nrows) {
      double s[2] = {0.0, 0.0};
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        Acc<MODE> tot;
        for (int w = 0; w < wpg; ++w) merge(tot, slots[((wbase + w) * kRBMax + lt) * 2 + n]);
        s[n] = tot.value();
      }
      epilogue<KIND>(a, x, phase, lrow0 + lt, s[0], s[1]);
    }
    slots = (slots == red) ? red + kGrpSlots : red;
  }
}

template <int KIND, int ST, bool RES, int RB>
__device__ __forceinline__ void stage_r(const Args& a, Ctx& x, int phase, int buf, unsigned long long* red) {
  switch (sum_mode(x.p, a.accum)) {
    case M_SS: stage_m<KIND, ST, M_SS, RES, RB>(a, x, phase, buf, red); break;
    case M_SD64: stage_m<KIND, ST, M_SD64, RES, RB>(a, x, phase, buf, red); break;
    case M_SD2: stage_m<KIND, ST, M_SD2, RES, RB>(a, x, phase, buf, red); break;
    default: stage_m<KIND, ST, M_DD, RES, RB>(a, x, phase, buf, red); break;
  }
}

// The circadian interaction is ALU-bound and always streams its weights.
template <int KIND, int ST>
__device__ __forceinline__ void stage(const Args& a, Ctx& x, int phase, int buf, unsigned long long* red) {
  constexpr int RB = rows_per_tile(KIND);
  if (KIND != K_CIRCADIAN && x.slab != nullptr) stage_r<KIND, ST, (KIND != K_CIRCADIAN), RB>(a, x, phase, buf, red);
  else stage_r<KIND, ST, false, RB>(a, x, phase, buf, red);
}

// Block-wide max of non-negative binary64 values (bit patterns), then one
// atomic per CTA into slot.
__device__ __forceinline__ void block_max(double v, unsigned long long* slot, unsigned long long* s_buf) {
  unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
  if (v != v) b = 0x7ff8000000000000ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
    b = o > b ? o : b;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) s_buf[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_buf[w] > m ? s_buf[w] : m;
    atomicMax(slot, m);
  }
}

__device__ __forceinline__ double ld_bits(const unsigned long long* p) {
  return __longlong_as_double((long long)__ldcg(p));
}

// Shared-memory bytes of a launch: the state slots [slots][d][rc] (six for
// Bogacki-Shampine, nine for Dormand-Prince) plus per-agent
// parameters (three binary64 and one binary32 per agent), a binary32
// (sin, cos) pair and a binary64 (sin, cos) pair per agent.
__host__ __device__ constexpr size_t state_smem_bytes(int d, int rc, int slots = 6) {
  return (size_t)rc * (slots * d * 8 + 3 * 8 + 4 + 8 + 16) + 32;
}


// Scalar control of a solve, computed by thread 0 of every CTA (all CTAs
// compute identical values from identical inputs) and broadcast through
// shared memory: binary64 is scarce on this GPU, so no other thread repeats it.
constexpr int kThetaMax = 32;
struct Scal {
  double t, h, hs, c21, c32, E, hstep, tstep0;
  long long n_acc, n_rej, n_rhs, next_out, out_end;
  int status, last, stop, accepted, rejected, parity;
  int mlp_go, n_ehist;
  int cancel;               // the host's cancel flag as the last attempt saw it
  double ehist[4];          // errors of the last accepted steps (learned proposer)
  float feat[kMlpIn];
  double theta[kThetaMax];
};

// Smallest warp groups (>= 32 threads) whose row blocks cover rc rows in one pass.
template <int KIND>
__device__ __forceinline__ int group_threads(int rc) {
  constexpr int RBk = rows_per_tile(KIND);
  int gt = kBlock / 4;
  while (gt > 32 && (kBlock / gt) * RBk < rc) gt >>= 1;
  return gt;
}

// Barrier of the CTAs that solve the system: a CTA barrier when one CTA
// solves it alone, otherwise the group barrier on the system's counter.
__device__ __forceinline__ bool sync_all(const Ctx& x, Control* c, unsigned long long& target, long long spin_limit,
                                         int* s_abort) {
  if (x.nb == 1) {
    __syncthreads();
    return true;
  }
  return grid_sync(c, target, x.nb, spin_limit, s_abort);
}

// The same barrier, with work that the threads outside warp 0 do while thread
// 0 arrives and waits for the other CTAs (work(k, nk): share k of nk).
template <class W>
__device__ __forceinline__ bool sync_all_with(const Ctx& x, Control* c, unsigned long long& target,
                                              long long spin_limit, int* s_abort, W&& work) {
  if (x.nb == 1) {
    __syncthreads();
    work((int)threadIdx.x, (int)blockDim.x);
    __syncthreads();
    return true;
  }
  __syncthreads();
  target += x.nb;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" :: "l"(&c->bar) : "memory");
    long long it = 0;
    int abort = 0;
    while (true) {
      const unsigned long long v = ld_acquire_u64(&c->bar);
      if (v >= kAbortBias) { abort = 1; break; }
      if (v >= target) break;
      if (++it > spin_limit) {
        atomicCAS(&c->status, 0, (int)S_DEVICE_WAIT);
        atomicAdd(&c->bar, kAbortBias);
        abort = 1;
        break;
      }
      if (it > 256) __nanosleep(32);
    }
    *s_abort = abort;
  } else if (threadIdx.x >= 32) {
    work((int)threadIdx.x - 32, (int)blockDim.x - 32);
  }
  __syncthreads();
  return !*s_abort;
}

// A job (RHS, one attempt or a whole solve) on the agents [x.rb, x.rb + x.nr)
// whose state x already holds; the system's agents are spread over x.nb CTAs
// (the whole grid, a team of a batch, or this CTA alone).
template <int KIND, int ST>
__device__ __forceinline__ void run_job(const Args& a, Ctx& x, Scal& sc, int* s_abort, unsigned long long* s_red,
                                        unsigned long long* s_grp, const float* smlp) {
  constexpr int d = Dim<KIND>::d;
  const int N = a.N;
  const int b = x.rank;
  const int tid = threadIdx.x;
  const bool leader = (b == 0 && tid == 0);
  Control* ctrl = a.ctrl;
  unsigned long long bt = 0;
  const bool single = x.single;
  (void)b;
  if (a.job == JOB_RHS) {
    x.p = Prec{a.rhs_f, a.rhs_s, a.rhs_g};
    for (int li = tid; li < x.nr; li += blockDim.x) {
      double Y[d];
#pragma unroll
      for (int c = 0; c < d; ++c) Y[c] = sv<KIND>(x, x.iX, c, li);
      put_jv<KIND>(a, 0, x.rb + li, Y, x.p.g, single, x.sisc ? x.sisc + li : nullptr);
    }
    if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) return;
    stage<KIND, ST>(a, x, PH_RHS, 0, s_grp);
    return;
  }

  const Prec p2 = variant_prec(a.variant, 2);
  const Prec p3 = variant_prec(a.variant, 3);
  const Prec p4 = variant_prec(a.variant, 4);
  const bool dp = (a.method == M_DP54);
  const Prec plast = dp ? variant_prec_dp(a.variant, 7) : p4;   // row of the first K1 and the starting step
  const double rtol = a.rtol;

  if (tid == 0) {
    sc.t = a.t0; sc.h = a.h_given; sc.E = 0.0;
    sc.n_acc = 0; sc.n_rej = 0; sc.n_rhs = 0; sc.next_out = 0; sc.out_end = 0;
    sc.status = S_OK; sc.last = 0; sc.stop = 0; sc.accepted = 0; sc.rejected = 0; sc.parity = 0;
    sc.mlp_go = 0; sc.n_ehist = 0; sc.cancel = 0;
    if (a.job == JOB_SOLVE)
      while (sc.next_out < a.n_out && a.t_out[sc.next_out] <= a.t0) ++sc.next_out;
  }

  if (a.job == JOB_SOLVE) {
    for (int li = tid; li < x.nr; li += blockDim.x) {
      double Y[d];
#pragma unroll
      for (int c = 0; c < d; ++c) Y[c] = sv<KIND>(x, x.iX, c, li);
      put_jv<KIND>(a, 0, x.rb + li, Y, plast.g, single, x.sisc ? x.sisc + li : nullptr);
    }
  }
  if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) goto finish_up;

  if (a.job == JOB_SOLVE) {
    // ---- K1 = f(t0, y0) with the last stage's row; starting-step norms d0, d1
    x.p = plast;
    x.m0 = 0.0; x.m1 = 0.0;
    stage<KIND, ST>(a, x, PH_K1, 0, s_grp);
    block_max(x.m0, &ctrl->red[0], s_red);
    block_max(x.m1, &ctrl->red[1], s_red);
    if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) goto finish_up;
    if (tid == 0) {
      sc.n_rhs = 1;
      const double d0 = ld_bits(&ctrl->red[0]);
      const double d1 = ld_bits(&ctrl->red[1]);
      if (d0 != d0 || isinf(d0) || d1 != d1 || isinf(d1)) sc.status = S_NONFINITE;
      const double h0 = (d0 >= 1e-5 && d1 >= 1e-5) ? 0.01 * d0 / d1 : 1e-6;
      sc.hs = h0;
      sc.c21 = single ? (double)(float)h0 : h0;   // y1 = y0 + h0 f0 in the state precision
    }
    __syncthreads();
    if (sc.status != S_OK) goto finish_up;
    if (!(a.h_given > 0.0)) {
      x.h0s = sc.c21;
      for (int li = tid; li < x.nr; li += blockDim.x) {
        double Y[d];
#pragma unroll
        for (int c = 0; c < d; ++c)
          Y[c] = axpy_state(sv<KIND>(x, x.iX, c, li), x.h0s, sv<KIND>(x, x.iK1, c, li), single);
        put_jv<KIND>(a, 1, x.rb + li, Y, plast.g, single, x.sisc ? x.sisc + li : nullptr);
      }
      if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) goto finish_up;
      x.m0 = 0.0;
      stage<KIND, ST>(a, x, PH_F1, 1, s_grp);
      block_max(x.m0, &ctrl->red[2], s_red);
      if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) goto finish_up;
      if (tid == 0) {
        sc.n_rhs = 2;
        const double h0 = sc.hs;
        const double d1 = ld_bits(&ctrl->red[1]);
        const double d2 = ld_bits(&ctrl->red[2]) / h0;
        const double m = fmax(d1, d2);
        // exponent 1/(q+1), q the order of the embedded solution
        const double h1 = (m > 1e-15) ? pow(0.01 / m, dp ? 0.2 : 1.0 / 3.0) : fmax(1e-6, h0 * 1e-3);
        sc.h = fmin(fmin(100.0 * h0, h1), a.hmax);
      }
    }
  }

  while (true) {
    // ---- per-attempt scalars (thread 0), then A: Y2 -> j-vector 0
    __syncthreads();
    if (tid == 0) {
      const long long na = sc.n_acc + sc.n_rej;
      sc.stop = 0;
      if (a.job == JOB_SOLVE) {
        if (!(sc.t < a.t1)) sc.stop = 1;
        else if (sc.n_rej > a.max_rejects) { sc.status = S_MAX_REJECTS; sc.stop = 1; }
        else if (na >= a.max_attempts) { sc.status = S_MAX_STEPS; sc.stop = 1; }
        else if (na > 0 && sc.cancel) { sc.status = S_TIMEOUT; sc.stop = 1; }
        else {
          double h = fmin(sc.h, a.hmax);
          if (h <= a.hmin) { sc.status = S_STEP_TOO_SMALL; sc.stop = 1; }
          sc.last = (sc.t + 1.1 * h >= a.t1);
          if (sc.last) h = a.t1 - sc.t;
          sc.h = h;
        }
      } else if (na > 0) {
        sc.stop = 1;
      }
      const double h = sc.h;
      sc.hs = single ? (double)(float)h : h;
      sc.c21 = single ? (double)(0.5f * (float)h) : 0.5 * h;
      sc.c32 = single ? (double)(0.75f * (float)h) : 0.75 * h;
    }
    __syncthreads();
    if (sc.stop) break;
    const bool rec = (a.hist != nullptr) && leader && (sc.n_acc + sc.n_rej) < a.hist_cap;
    unsigned long long ts[5];
    if (rec) ts[0] = globaltimer_ns();
    x.hs = sc.hs;
    x.c21 = sc.c21;
    x.c32 = sc.c32;
    const int parity = sc.parity;
    bool aborted = false;
    if (dp) {
      // ---- Dormand-Prince: A: Y2 -> j-vector 0; stage l reads the j-vector
      // of Y_l (buffer l % 2) and writes that of Y_{l+1}
      for (int li = tid; li < x.nr; li += blockDim.x) {
        double Y[d];
#pragma unroll
        for (int c = 0; c < d; ++c) Y[c] = dp_arg<KIND>(x, 2, c, li);
        put_jv<KIND>(a, 0, x.rb + li, Y, variant_prec_dp(a.variant, 2).g, single, x.sisc ? x.sisc + li : nullptr);
      }
      if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) break;
      if (rec) ts[1] = globaltimer_ns();
      if (leader) ctrl->emax[parity ^ 1] = 0ull;
      // the host's cancel flag, read now and latched after the last stage
      // (the host-memory read overlaps the stages instead of delaying one)
      const int cancel_v = (leader && a.cancel) ? *a.cancel : 0;
      for (int l = 2; l <= 7; ++l) {
        x.p = variant_prec_dp(a.variant, l);
        x.pn = variant_prec_dp(a.variant, l < 7 ? l + 1 : 7);
        if (l == 7) x.m1 = 0.0;
        stage<KIND, ST>(a, x, PH_D2 + l - 2, l & 1, s_grp);
        if (l == 7 && leader) {
          ctrl->cancel_seen[parity] = cancel_v;
          if (a.progress) *a.progress = sc.t;
        }
        if (l == 7) block_max(x.m1, &ctrl->emax[parity], s_red);
        if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) { aborted = true; break; }
        if (rec && (l == 3 || l == 5)) ts[l == 3 ? 2 : 3] = globaltimer_ns();
      }
    } else {
      do {
        for (int li = tid; li < x.nr; li += blockDim.x) {
          double Y[d];
#pragma unroll
          for (int c = 0; c < d; ++c)
            Y[c] = axpy_state(sv<KIND>(x, x.iX, c, li), x.c21, sv<KIND>(x, x.iK1, c, li), single);
          put_jv<KIND>(a, 0, x.rb + li, Y, p2.g, single, x.sisc ? x.sisc + li : nullptr);
        }
        // binary64 sin/cos of a Sigma = D stage's argument for its i-side
        // finish, computed while the barrier before the stage waits
        const bool c2 = KIND == K_KURAMOTO && x.sisc64 != nullptr && p2.s == 1;
        const bool c3 = KIND == K_KURAMOTO && x.sisc64 != nullptr && p3.s == 1;
        const bool c4 = KIND == K_KURAMOTO && x.sisc64 != nullptr && p4.s == 1;
        if (!sync_all_with(x, ctrl, bt, a.spin_limit, s_abort, [&](int k, int nk) {
              if (c2)
                for (int li = k; li < x.nr; li += nk) {
                  double s, c;
                  sincos(axpy_state(sv<KIND>(x, x.iX, 0, li), x.c21, sv<KIND>(x, x.iK1, 0, li), single), &s, &c);
                  x.sisc64[li] = make_double2(s, c);
                }
            })) { aborted = true; break; }
        if (rec) ts[1] = globaltimer_ns();
        // the host's cancel flag, read now and latched after stage 4 (the
        // host-memory read overlaps stages 2 to 4 instead of delaying one)
        const int cancel_v = (leader && a.cancel) ? *a.cancel : 0;
        // ---- B2: K2 = f(Y2); Y3 -> j-vector 1
        if (leader) ctrl->emax[parity ^ 1] = 0ull;
        x.p = p2; x.pn = p3;
        x.have64 = c2;
        stage<KIND, ST>(a, x, PH_B2, 0, s_grp);
        if (!sync_all_with(x, ctrl, bt, a.spin_limit, s_abort, [&](int k, int nk) {
              if (c3)
                for (int li = k; li < x.nr; li += nk) {
                  double s, c;
                  sincos(axpy_state(sv<KIND>(x, x.iX, 0, li), x.c32, sv<KIND>(x, x.iK2, 0, li), single), &s, &c);
                  x.sisc64[li] = make_double2(s, c);
                }
            })) { aborted = true; break; }
        if (rec) ts[2] = globaltimer_ns();
        // ---- B3: K3 = f(Y3); X' -> j-vector 2
        x.p = p3; x.pn = p4;
        x.have64 = c3;
        stage<KIND, ST>(a, x, PH_B3, 1, s_grp);
        if (!sync_all_with(x, ctrl, bt, a.spin_limit, s_abort, [&](int k, int nk) {
              if (c4)
                for (int li = k; li < x.nr; li += nk) {
                  double s, c;
                  sincos(sv<KIND>(x, x.iXn, 0, li), &s, &c);
                  x.sisc64[li] = make_double2(s, c);
                }
            })) { aborted = true; break; }
        if (rec) ts[3] = globaltimer_ns();
        // ---- B4: K4 = f(X'); error norm
        x.p = p4;
        x.m1 = 0.0;
        x.have64 = c4;
        stage<KIND, ST>(a, x, PH_B4, 2, s_grp);
        x.have64 = false;
        if (leader) {
          ctrl->cancel_seen[parity] = cancel_v;
          if (a.progress) *a.progress = sc.t;
        }
        block_max(x.m1, &ctrl->emax[parity], s_red);
        if (!sync_all(x, ctrl, bt, a.spin_limit, s_abort)) { aborted = true; break; }
      } while (false);
    }
    if (aborted) break;
    // ---- decision (thread 0; warp 0 runs the learned proposer when installed)
    if (tid == 0) {
      const double E = ld_bits(&ctrl->emax[parity]);
      sc.cancel = __ldcg(&ctrl->cancel_seen[parity]);   // loaded beside E, off the path of the next attempt
      sc.E = E;
      sc.n_rhs += dp ? 6 : 3;
      if (rec) {
        ts[4] = globaltimer_ns();
        double* r = a.hist + (size_t)(sc.n_acc + sc.n_rej) * kHistDoubles;
        r[0] = sc.t; r[1] = sc.h; r[2] = E; r[3] = (E <= rtol) ? 1.0 : 0.0;
        for (int k = 1; k < 5; ++k) r[3 + k] = (double)(ts[k] - ts[0]);
      }
      sc.accepted = 0;
      if (a.job == JOB_ATTEMPT) {
        ++sc.n_acc;
      } else if (E != E || isinf(E)) {
        sc.status = S_NONFINITE;
        ++sc.n_rej;
      } else if (E <= rtol) {
        const double h = sc.h;
        const double t_new = sc.last ? a.t1 : sc.t + h;
        sc.hstep = h;
        sc.tstep0 = sc.t;
        long long e = sc.next_out;
        while (e < a.n_out && a.t_out[e] <= t_new && e - sc.next_out < kThetaMax) {
          sc.theta[e - sc.next_out] = (a.t_out[e] - sc.t) / h;
          ++e;
        }
        sc.out_end = e;
        double fac = (E == 0.0) ? 5.0 : fmin(5.0, 0.8 * (dp ? root5_ratio(rtol, E) : cbrt_ratio(rtol, E)));
        if (sc.rejected) fac = fmin(1.0, fac);
        sc.h = h * fac;
        sc.t = t_new;
        ++sc.n_acc;
        if (sc.n_ehist == 4) {
          for (int k = 0; k < 3; ++k) sc.ehist[k] = sc.ehist[k + 1];
          sc.ehist[3] = E;
        } else {
          sc.ehist[sc.n_ehist++] = E;
        }
        sc.mlp_go = (smlp != nullptr) && !sc.rejected;
        if (sc.mlp_go) {
          double f[kMlpIn];
          mlp_features(sc.ehist, sc.n_ehist, h, rtol, f);
          for (int k = 0; k < kMlpIn; ++k)
            sc.feat[k] = ((float)f[k] - smlp[kMlpParams + k]) / smlp[kMlpParams + kMlpIn + k];
        }
        sc.rejected = 0;
        sc.accepted = 1;
      } else {
        ++sc.n_rej;
        sc.h = sc.rejected ? sc.h * 0.5 : sc.h * fmax(0.5, 0.8 * (dp ? root5_ratio(rtol, E) : cbrt_ratio(rtol, E)));
        sc.rejected = 1;
        sc.mlp_go = 0;
      }
      sc.parity ^= 1;
    }
    if (smlp != nullptr && tid < 32) {
      __syncwarp();
      if (sc.accepted && sc.mlp_go) {
        // learned proposal of the next step (the error test still decides)
        const float dlt = mlp_warp_forward(smlp, sc.feat, tid);
        if (tid == 0) sc.h = sc.hstep * exp(fmin(fmax((double)dlt, kMlpDMin), kMlpDMax));
      }
    }
    __syncthreads();
    if (a.job == JOB_ATTEMPT) {
      for (int li = tid; li < x.nr; li += blockDim.x) {
#pragma unroll
        for (int c = 0; c < d; ++c) {
          a.out0[c * N + x.rb + li] = sv<KIND>(x, x.iXn, c, li);
          a.out1[c * N + x.rb + li] = sv<KIND>(x, x.iK4, c, li);
        }
      }
      break;
    }
    if (sc.status != S_OK) break;
    if (sc.accepted) {
      // dense output: cubic Hermite on (t_n, X, K1), (t_n + h, X', K4)
      while (true) {
        const long long k0 = sc.next_out, k1 = sc.out_end;
        if (k0 >= k1) break;
        const double hstep = sc.hstep;
        for (long long k = k0; k < k1; ++k) {
          const double th = sc.theta[k - k0];
          for (int li = tid; li < x.nr; li += blockDim.x) {
#pragma unroll
            for (int c = 0; c < d; ++c) {
              const double y0 = sv<KIND>(x, x.iX, c, li), y1 = sv<KIND>(x, x.iXn, c, li);
              const double f0 = sv<KIND>(x, x.iK1, c, li), f1 = sv<KIND>(x, dp ? x.iK7 : x.iK4, c, li);
              a.y_out[(size_t)k * d * N + c * N + x.rb + li] =
                  ((1.0 - th) * y0 + th * y1) +
                  (th * (th - 1.0)) * (((1.0 - 2.0 * th) * (y1 - y0) + ((th - 1.0) * hstep) * f0) + (th * hstep) * f1);
            }
          }
        }
        __syncthreads();
        if (tid == 0) {
          sc.next_out = k1;
          // more outputs inside this step than fit in one batch
          const double t_step0 = sc.tstep0;
          long long e = k1;
          while (e < a.n_out && a.t_out[e] <= sc.t && e - k1 < kThetaMax) {
            sc.theta[e - k1] = (a.t_out[e] - t_step0) / hstep;
            ++e;
          }
          sc.out_end = e;
        }
        __syncthreads();
      }
      int tmp = x.iX; x.iX = x.iXn; x.iXn = tmp;
      if (dp) {
        tmp = x.iK1; x.iK1 = x.iK7; x.iK7 = tmp;
      } else {
        tmp = x.iK1; x.iK1 = x.iK4; x.iK4 = tmp;
      }
    }
  }

finish_up:
  __syncthreads();
  if (a.job == JOB_SOLVE && a.final_y != nullptr && !*s_abort) {
    for (int li = tid; li < x.nr; li += blockDim.x) {
#pragma unroll
      for (int c = 0; c < d; ++c) a.final_y[c * N + x.rb + li] = sv<KIND>(x, x.iX, c, li);
    }
  }
  if (leader) {
    if (sc.status != S_OK) atomicCAS(&ctrl->status, 0, sc.status);
    ctrl->n_acc = sc.n_acc;
    ctrl->n_rej = sc.n_rej;
    ctrl->n_rhs = sc.n_rhs;
    ctrl->n_out = sc.next_out;
    ctrl->t = sc.t;
    ctrl->h = sc.h;
  }
}

template <int KIND, int ST>
__global__ void __launch_bounds__(kBlock, 1) bs3_kernel(Args a) {
  constexpr int d = Dim<KIND>::d;
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ int s_abort;
  __shared__ unsigned long long s_red[kBlock / 32];
  __shared__ unsigned long long s_grp[2 * kGrpSlots];
  __shared__ Scal sc;
  const int N = a.N;
  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) s_abort = 0;

  Ctx x;
  x.rc = a.rc;
  x.gt = group_threads<KIND>(a.rc);
  x.rb = (int)(((long long)b * N) / G);
  x.nr = (int)(((long long)(b + 1) * N) / G) - x.rb;
  x.rank = b;
  x.nb = G;
  x.slab = a.slab_bytes > 0 ? dyn : nullptr;
  x.S = (double*)(dyn + a.slab_bytes);
  x.spar = x.S + a.n_slots * d * x.rc;
  x.sth = x.spar + x.rc;
  x.srs = x.sth + x.rc;
  x.sscale = (float*)(x.srs + x.rc);
  x.sisc = (float2*)(((uintptr_t)(x.sscale + x.rc) + 7) & ~(uintptr_t)7);
  x.sisc64 = (double2*)(((uintptr_t)(x.sisc + x.rc) + 15) & ~(uintptr_t)15);
  x.have64 = false;
  x.iX = 0; x.iXn = 1; x.iK1 = 2; x.iK2 = 3; x.iK3 = 4; x.iK4 = 5;
  x.iK7 = 8;   // Dormand-Prince: K_l in slot l + 1 (nine slots)
  x.rtol = a.rtol;
  x.thr = a.atol / a.rtol;
  x.m0 = 0.0; x.m1 = 0.0;
  x.c21 = x.c32 = x.hs = x.h0s = 0.0;
  x.single = (a.job == JOB_RHS) ? (a.rhs_f == 0 && a.rhs_s == 0 && a.rhs_g == 0) : (a.variant == V_SINGLE);
  const bool single = x.single;

  // this CTA's weight rows into shared memory (contiguous in the [N][ld] layout)
  if (a.slab_bytes > 0) {
    const size_t eb = (size_t)KLoad<ST>::BYTES;
    const uint4* src = reinterpret_cast<const uint4*>((const char*)a.q + (size_t)x.rb * a.ld * eb);
    uint4* dst = reinterpret_cast<uint4*>(dyn);
    const int n16 = (int)((size_t)x.nr * a.ld * eb / 16);
    for (int e = tid; e < n16; e += blockDim.x) dst[e] = ld_stream16(src + e);
  }
  float* smlp = a.mlp ? (float*)(dyn + a.smem_mlp_off) : nullptr;
  if (a.mlp)
    for (int k = tid; k < kMlpModel; k += blockDim.x) smlp[k] = a.mlp[k];
  x.cbias = (KIND == K_KURAMOTO || KIND == K_CIRCADIAN) ? cta_bias(a.bias, x.rb, x.nr) : 0.0f;
  // per-agent parameters and the initial state of this CTA's agents
  for (int li = tid; li < x.nr; li += blockDim.x) {
    const int i = x.rb + li;
    x.spar[li] = a.par[i];
    x.sth[li] = a.theta_h ? a.theta_h[i] : 0.0;
    x.srs[li] = a.rowsum[i];
    x.sscale[li] = a.scale[i];
#pragma unroll
    for (int c = 0; c < d; ++c) {
      const double y = a.X[c * N + i];
      if (a.job == JOB_SOLVE)
        for (long long k = 0; k < a.n_out && a.t_out[k] <= a.t0; ++k) a.y_out[(size_t)k * d * N + c * N + i] = y;
      sv<KIND>(x, x.iX, c, li) = single ? (double)(float)y : y;
      if (a.job == JOB_ATTEMPT) {
        const double k1 = a.Kb[0][c * N + i];
        sv<KIND>(x, x.iK1, c, li) = single ? (double)(float)k1 : k1;
      }
    }
  }
  __syncthreads();

  run_job<KIND, ST>(a, x, sc, &s_abort, s_red, s_grp, smlp);
}

}  // namespace bs3

namespace bs3 {

// ---------------------------------------------------------------------------
// Ragged batches of independent systems in one cooperative launch.  The
// systems are sorted by decreasing N.  The first n_big of them (too large for
// one SM's share of the batch) are solved by teams of team CTAs: CTAs
// [0, n_teams * team) form the teams, each team takes systems from the team
// queue, splits their rows like the persistent solver and meets at the
// system's barrier counter.  Every other CTA, and a team CTA once the team
// queue is empty, takes whole systems from the single queue and solves them
// alone with CTA barriers.  The state lives in global memory (slots [6][d][N]
// per system).
// ---------------------------------------------------------------------------
struct SysDesc {
  int N, ld;
  const void* q;
  const float* scale;
  const double* rowsum;
  const float* bias;
  const double* par;
  const double* theta_h;
  const double* y0;
  double* y_final;
  double* state;     // [6][d][N]
  float* jv32;       // [3][2][ld]
  double* jv64;      // [3][2][ld]
  Control* ctrl;
  double t0, t1;
  double rtol, atol;   // this system's tolerances (Rel, Ab of Eq. ERROR-O23)
};

struct BatchArgs {
  Args common;       // variant, Sigma mode, tolerances, limits
  const SysDesc* sys;
  int S;
  int* next;         // single-queue counter (zero before the launch; systems n_big + next)
  int n_big;         // systems [0, n_big) go to teams
  int team;          // CTAs per team (1: no teams)
  int n_teams;
  int* big_next;     // team-queue counter (zero before the launch)
  int* team_job;     // [n_teams] the system a team is on
  unsigned long long* team_bar;   // [n_teams] team barrier counters (zero before the launch)
  int* team_status;  // [n_teams] status of a team barrier that ran out (zero before the launch)
};

// Solves system sidx on the rows [rb, rb + nr) of this CTA, one of nb CTAs.
template <int KIND, int ST>
__device__ __forceinline__ void batch_job(const BatchArgs& ba, int sidx, int rank, int nb, Scal& sc, int* s_abort,
                                          unsigned long long* s_red, unsigned long long* s_grp) {
  constexpr int d = Dim<KIND>::d;
  const int tid = threadIdx.x;
  const SysDesc D = ba.sys[sidx];
  Args a = ba.common;
  a.job = JOB_SOLVE;
  a.N = D.N;
  a.ld = D.ld;
  a.q = D.q;
  a.scale = D.scale;
  a.rowsum = D.rowsum;
  a.bias = D.bias;
  a.par = D.par;
  a.theta_h = D.theta_h;
  a.X = const_cast<double*>(D.y0);
  a.jv32 = D.jv32;
  a.jv64 = D.jv64;
  a.ctrl = D.ctrl;
  a.final_y = D.y_final;
  a.t0 = D.t0;
  a.t1 = D.t1;
  a.rtol = D.rtol;
  a.atol = D.atol;
  a.hmax = 0.1 * (D.t1 - D.t0);
  a.n_out = 0;
  a.slab_bytes = 0;
  a.hist = nullptr;
  a.mlp = nullptr;
  a.cancel = nullptr;
  a.progress = nullptr;
  Ctx x;
  x.rank = rank;
  x.nb = nb;
  x.rb = (int)(((long long)rank * D.N) / nb);
  x.nr = (int)(((long long)(rank + 1) * D.N) / nb) - x.rb;
  a.rc = (D.N + nb - 1) / nb;
  x.rc = D.N;   // slot stride of the global state; this CTA's rows start at rb
  x.gt = group_threads<KIND>(a.rc);
  x.slab = nullptr;
  x.S = D.state + x.rb;
  x.spar = const_cast<double*>(D.par) + x.rb;
  x.srs = const_cast<double*>(D.rowsum) + x.rb;
  x.sth = const_cast<double*>(D.theta_h ? D.theta_h : D.rowsum) + x.rb;   // read only by the circadian kind
  x.sscale = const_cast<float*>(D.scale) + x.rb;
  x.cbias = (KIND == K_KURAMOTO || KIND == K_CIRCADIAN) ? cta_bias(D.bias, x.rb, x.nr) : 0.0f;
  x.sisc = nullptr;
  x.sisc64 = nullptr;
  x.have64 = false;
  x.iX = 0; x.iXn = 1; x.iK1 = 2; x.iK2 = 3; x.iK3 = 4; x.iK4 = 5;
  x.rtol = a.rtol;
  x.thr = a.atol / a.rtol;
  x.m0 = 0.0; x.m1 = 0.0;
  x.c21 = x.c32 = x.hs = x.h0s = 0.0;
  x.single = (a.variant == V_SINGLE);
  for (int li = tid; li < x.nr; li += blockDim.x)
#pragma unroll
    for (int c = 0; c < d; ++c) {
      const double y = D.y0[c * D.N + x.rb + li];
      sv<KIND>(x, x.iX, c, li) = x.single ? (double)(float)y : y;
    }
  __syncthreads();
  run_job<KIND, ST>(a, x, sc, s_abort, s_red, s_grp, nullptr);
}

template <int KIND, int ST>
__global__ void __launch_bounds__(kBlock, 1) bs3_batch_kernel(BatchArgs ba) {
  __shared__ int s_abort, s_sys;
  __shared__ unsigned long long s_red[kBlock / 32];
  __shared__ unsigned long long s_grp[2 * kGrpSlots];
  __shared__ Scal sc;
  const int tid = threadIdx.x;
  if (ba.team > 1 && (int)blockIdx.x < ba.n_teams * ba.team) {
    const int team = blockIdx.x / ba.team, rank = blockIdx.x % ba.team;
    unsigned long long tt = 0;
    while (true) {
      __syncthreads();
      if (tid == 0) {
        s_abort = 0;
        if (rank == 0) {
          ba.team_job[team] = atomicAdd(ba.big_next, 1);
          __threadfence();
        }
      }
      // the team agrees on its next system (and, before that, every member
      // has left the previous one)
      if (!group_sync(&ba.team_bar[team], &ba.team_status[team], tt, ba.team, ba.common.spin_limit, &s_abort))
        return;
      if (tid == 0) s_sys = __ldcg(&ba.team_job[team]);
      __syncthreads();
      const int sidx = s_sys;
      if (sidx >= ba.n_big) break;
      batch_job<KIND, ST>(ba, sidx, rank, ba.team, sc, &s_abort, s_red, s_grp);
      if (!group_sync(&ba.team_bar[team], &ba.team_status[team], tt, ba.team, ba.common.spin_limit, &s_abort))
        return;
    }
  }
  while (true) {
    __syncthreads();
    if (tid == 0) {
      s_sys = ba.n_big + atomicAdd(ba.next, 1);
      s_abort = 0;
    }
    __syncthreads();
    const int sidx = s_sys;
    if (sidx >= ba.S) break;
    batch_job<KIND, ST>(ba, sidx, 0, 1, sc, &s_abort, s_red, s_grp);
  }
}

}  // namespace bs3
