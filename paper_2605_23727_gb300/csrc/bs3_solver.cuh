// Persistent cooperative BS3 solver kernel (one launch per solve).
//
// Per attempt (Eq. Stage-ODE23, Table Butcher-O23, Eq. ERROR-O23):
//   A : Y2 = X + (h/2) K1                         -> j-vector 0     | barrier
//   B2: K2 = f(Y2); Y3 = X + (3h/4) K2            -> j-vector 1     | barrier
//   B3: K3 = f(Y3); X' = X + h(2/9 K1+1/3 K2+4/9 K3) -> j-vector 2  | barrier
//   B4: K4 = f(X'); E = max_k |h sum e_l K_l| / W_k (grid max)      | barrier
//   every CTA then takes the same accept/reject decision from E.
// Each warp owns fixed tiles of RB rows (agents); lane r of the warp owns
// agent row0 + r for all row-local work (stage combinations, agent term,
// error, dense output), so only the j-vectors cross CTAs.  The coupling of a
// stage is an HBM/L2-streaming pass over the stored weights.
#pragma once

#include "bs3_device.cuh"

namespace bs3 {

struct Args {
  // system
  int N, ld;
  const void* q;            // [N][ld] stored weights, zero padded
  const float* scale;       // [N] row scales
  const double* rowsum;     // [N] sum_j s_i q_ij (paper-form oscillators)
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
};

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
__device__ __forceinline__ void put_jv(const Args& a, int buf, int i, const double* Y, int g, bool single) {
  const size_t o0 = (size_t)(buf * 2) * a.ld + i;
  const size_t o1 = o0 + a.ld;
  if (KIND == K_KURAMOTO) {
    if (g == 0) {
      float s, c;
      if (single) sincosf((float)Y[0], &s, &c);
      else sincos_f_of_d(Y[0], &s, &c);
      a.jv32[o0] = s;
      a.jv32[o1] = c;
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
// Coupling sums of one warp tile (rows row0 .. row0+RB-1).
// ---------------------------------------------------------------------------
template <int ST, int MODE, int NV, int RB>
__device__ __forceinline__ void gemv_tile(const Args& a, int buf, int row0, int lane, double (&res)[kRBMax][2]) {
  using L = KLoad<ST>;
  constexpr int VEC = L::VEC;
  constexpr bool DD = (MODE == M_DD);
  Acc<MODE> acc[RB][NV];
  const char* qb = (const char*)a.q;
  const size_t rstride = (size_t)a.ld * L::BYTES;
  const int nrows = min(RB, a.N - row0);
  const float* v32 = a.jv32 + (size_t)(buf * 2) * a.ld;
  const double* v64 = a.jv64 + (size_t)(buf * 2) * a.ld;
#pragma unroll(VEC >= 16 ? 1 : 2)
  for (int col = lane * VEC; col < a.ld; col += 32 * VEC) {
    uint4 raw[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
      raw[r] = (r < nrows) ? ld_stream16(qb + (size_t)(row0 + r) * rstride + (size_t)col * L::BYTES)
                           : make_uint4(0u, 0u, 0u, 0u);
    if (!DD) {
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
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int n = 0; n < NV; ++n) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[r][n].xor_merge(off);
      res[r][n] = acc[r][n].value();
    }
}

// Circadian interaction: r_i = sum_j q_ij atan(x_j - x_i) (Eq. CC).
template <int ST, int MODE, int RB>
__device__ __forceinline__ void cc_tile(const Args& a, int buf, int row0, int lane, double (&res)[kRBMax][2]) {
  using L = KLoad<ST>;
  constexpr int VEC = L::VEC;
  constexpr bool DD = (MODE == M_DD);
  Acc<MODE> acc[RB];
  const char* qb = (const char*)a.q;
  const size_t rstride = (size_t)a.ld * L::BYTES;
  const int nrows = min(RB, a.N - row0);
  const float* v32 = a.jv32 + (size_t)(buf * 2) * a.ld;
  const double* v64 = a.jv64 + (size_t)(buf * 2) * a.ld;
  float xi32[RB];
  double xi64[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const int i = row0 + (r < nrows ? r : 0);
    xi32[r] = DD ? 0.f : v32[i];
    xi64[r] = DD ? v64[i] : 0.0;
  }
  for (int col = lane * VEC; col < a.ld; col += 32 * VEC) {
    uint4 raw[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
      raw[r] = (r < nrows) ? ld_stream16(qb + (size_t)(row0 + r) * rstride + (size_t)col * L::BYTES)
                           : make_uint4(0u, 0u, 0u, 0u);
    if (!DD) {
      float xj[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) xj[e] = v32[col + e];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; ++e)
          acc[r].add_f(L::f(raw[r], e), atan_f32(__fsub_rn(xj[e], xi32[r])));
    } else {
      double xj[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) xj[e] = v64[col + e];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int e = 0; e < VEC; ++e)
          acc[r].add_d(L::get_d(raw[r], e), atan(__dsub_rn(xj[e], xi64[r])));
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[r].xor_merge(off);
    res[r][0] = acc[r].value();
    res[r][1] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Agent term F and the i-side finish of the coupling: K_l of agent i.
// Y: stage argument of agent i (d values); s0, s1: coupling sums (binary32
// values when Sigma = S).  Operation order mirrors the definitions exactly.
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void finish(const Args& a, int i, const double* Y, double s0, double s1,
                                       Prec p, bool single, double* K) {
  const int N = a.N;
  (void)N;
  if (KIND == K_KURAMOTO) {
    if (p.s == 0) {
      const float sc = a.scale[i];
      const float S = (float)s0 * sc, C = (float)s1 * sc;
      float si, ci;
      if (single) sincosf((float)Y[0], &si, &ci);
      else sincos_f_of_d(Y[0], &si, &ci);
      const float cpl = ci * S - si * C;
      K[0] = p.f == 0 ? (double)((float)a.par[i] + cpl) : a.par[i] + (double)cpl;
    } else {
      const double sc = (double)a.scale[i];
      const double S = s0 * sc, C = s1 * sc;
      double si, ci;
      sincos(Y[0], &si, &ci);
      const double cpl = ci * S - si * C;
      K[0] = p.f == 0 ? (double)((float)a.par[i] + (float)cpl) : a.par[i] + cpl;
    }
  } else if (KIND == K_LCO_CFG) {
    double ax;
    if (p.s == 0) ax = (double)((float)s0 * a.scale[i]);
    else ax = s0 * (double)a.scale[i];
    if (p.f == 0) {
      const float w = (float)a.par[i], x = (float)Y[0];
      K[0] = (double)(float)Y[1];
      K[1] = (double)((-(w * w) * x) + (float)ax);
    } else {
      const double w = a.par[i];
      K[0] = Y[1];
      K[1] = (-(w * w) * Y[0]) + ax;
    }
  } else if (KIND == K_LCO_PAPER) {
    double cpl;
    if (p.s == 0) {
      const float mx = (float)s0 * a.scale[i];
      cpl = (double)(mx - (float)a.rowsum[i] * (float)Y[0]);
    } else {
      const double mx = s0 * (double)a.scale[i];
      cpl = mx - a.rowsum[i] * Y[0];
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
      const float th = (float)a.theta_h[i];
      const float x2 = (float)Y[1], x2s = x2 * x2;
      const float pref = ((float)a.g[0] * th * (float)a.g[3]) / (th + x2s * x2s);
      cpl = (double)(pref * ((float)s0 * a.scale[i]));
    } else {
      const double th = a.theta_h[i];
      const double x2 = Y[1], x2s = x2 * x2;
      const double pref = (a.g[0] * th * a.g[3]) / (th + x2s * x2s);
      cpl = pref * (s0 * (double)a.scale[i]);
    }
    if (p.f == 0) {
      const float x1 = (float)Y[0], x2 = (float)Y[1], x3 = (float)Y[2], x4 = (float)Y[3];
      const float k0 = (float)a.g[0], k2 = (float)a.g[1], k3 = (float)a.g[2], aa = (float)a.g[3];
      const float b = (float)a.g[4], c = (float)a.g[5], eps = (float)a.g[6], I0 = (float)a.g[7];
      const float k1 = (float)a.par[i], th = (float)a.theta_h[i];
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
      const double k1 = a.par[i], th = a.theta_h[i];
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
// number of template instantiations of the coupling loops small.
// ---------------------------------------------------------------------------
enum Phase { PH_RHS = 0, PH_K1 = 1, PH_F1 = 2, PH_B2 = 3, PH_B3 = 4, PH_B4 = 5 };

struct Ctx {
  double* X;
  double* Xn;
  double* K1;
  double* K2;
  double* K3;
  double* K4;
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
__device__ __forceinline__ void epilogue(const Args& a, Ctx& x, int phase, int i, double s0, double s1) {
  constexpr int d = Dim<KIND>::d;
  const int N = a.N;
  double Y[d], K[d];
  // stage argument of this agent
#pragma unroll
  for (int c = 0; c < d; ++c) {
    const int o = c * N + i;
    switch (phase) {
      case PH_RHS: Y[c] = x.single ? (double)(float)x.X[o] : x.X[o]; break;
      case PH_K1: Y[c] = x.X[o]; break;
      case PH_F1: Y[c] = axpy_state(x.X[o], x.h0s, x.K1[o], x.single); break;
      case PH_B2: Y[c] = axpy_state(x.X[o], x.c21, x.K1[o], x.single); break;
      case PH_B3: Y[c] = axpy_state(x.X[o], x.c32, x.K2[o], x.single); break;
      default: Y[c] = x.Xn[o]; break;
    }
  }
  finish<KIND>(a, i, Y, s0, s1, x.p, x.single, K);
  switch (phase) {
    case PH_RHS:
#pragma unroll
      for (int c = 0; c < d; ++c) a.out0[c * N + i] = K[c];
      break;
    case PH_K1:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        x.K1[c * N + i] = K[c];
        const double sc = x.rtol * fmax(fabs(Y[c]), x.thr);
        x.m0 = max_nan(x.m0, fabs(Y[c]) / sc);
        x.m1 = max_nan(x.m1, fabs(K[c]) / sc);
      }
      break;
    case PH_F1:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        const double sc = x.rtol * fmax(fabs(x.X[c * N + i]), x.thr);
        x.m0 = max_nan(x.m0, fabs(K[c] - x.K1[c * N + i]) / sc);
      }
      break;
    case PH_B2:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        x.K2[c * N + i] = K[c];
        Y[c] = axpy_state(x.X[c * N + i], x.c32, K[c], x.single);
      }
      put_jv<KIND>(a, 1, i, Y, x.pn.g, x.single);
      break;
    case PH_B3:
#pragma unroll
      for (int c = 0; c < d; ++c) {
        const int o = c * N + i;
        x.K3[o] = K[c];
        const double k1 = x.K1[o], k2 = x.K2[o], k3 = K[c], xo = x.X[o];
        double xn;
        if (x.single) {
          const float cmb = ((float)kB1 * (float)k1 + (float)kB2 * (float)k2) + (float)kB3 * (float)k3;
          xn = (double)((float)xo + (float)x.hs * cmb);
        } else {
          xn = xo + x.hs * ((kB1 * k1 + kB2 * k2) + kB3 * k3);
        }
        x.Xn[o] = xn;
        Y[c] = xn;
      }
      put_jv<KIND>(a, 2, i, Y, x.pn.g, x.single);
      break;
    default:  // PH_B4: K4 and the error of Eq. ERROR-O23
#pragma unroll
      for (int c = 0; c < d; ++c) {
        const int o = c * N + i;
        x.K4[o] = K[c];
        const double k1 = x.K1[o], k2 = x.K2[o], k3 = x.K3[o], k4 = K[c];
        double dv;
        if (x.single) {
          const float cmb = (((float)kE1 * (float)k1 + (float)kE2 * (float)k2) + (float)kE3 * (float)k3) +
                            (float)kE4 * (float)k4;
          dv = (double)((float)x.hs * cmb);
        } else {
          dv = x.hs * (((kE1 * k1 + kE2 * k2) + kE3 * k3) + kE4 * k4);
        }
        const double w = fmax(fmax(fabs(x.X[o]), fabs(Y[c])), x.thr);
        double v = fabs(dv) / w;
        if (!isfinite(Y[c]) || !isfinite(k4)) v = nan_d();
        x.m1 = max_nan(x.m1, v);
      }
      break;
  }
}

// ---------------------------------------------------------------------------
// One stage: coupling sums of every tile of this warp, then the row epilogue.
// ---------------------------------------------------------------------------
template <int KIND, int ST, int MODE>
__device__ __forceinline__ void stage_m(const Args& a, Ctx& x, int phase, int buf, int gw, int tw, int lane) {
  constexpr int RB = rows_per_tile(KIND);
  const int ntiles = (a.N + RB - 1) / RB;
  for (int tile = gw; tile < ntiles; tile += tw) {
    const int row0 = tile * RB;
    double res[kRBMax][2];
    if (KIND == K_CIRCADIAN) cc_tile<ST, MODE, RB>(a, buf, row0, lane, res);
    else if (KIND == K_KURAMOTO) gemv_tile<ST, MODE, 2, RB>(a, buf, row0, lane, res);
    else gemv_tile<ST, MODE, 1, RB>(a, buf, row0, lane, res);
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (lane == r) { s0 = res[r][0]; s1 = (KIND == K_KURAMOTO) ? res[r][1] : 0.0; }
    const int i = row0 + lane;
    if (lane < RB && i < a.N) epilogue<KIND>(a, x, phase, i, s0, s1);
  }
}

template <int KIND, int ST>
__device__ __forceinline__ void stage(const Args& a, Ctx& x, int phase, int buf, int gw, int tw, int lane) {
  switch (sum_mode(x.p, a.accum)) {
    case M_SS: stage_m<KIND, ST, M_SS>(a, x, phase, buf, gw, tw, lane); break;
    case M_SD64: stage_m<KIND, ST, M_SD64>(a, x, phase, buf, gw, tw, lane); break;
    case M_SD2: stage_m<KIND, ST, M_SD2>(a, x, phase, buf, gw, tw, lane); break;
    default: stage_m<KIND, ST, M_DD>(a, x, phase, buf, gw, tw, lane); break;
  }
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

template <int KIND, int ST>
__global__ void __launch_bounds__(kBlock, 1) bs3_kernel(Args a) {
  constexpr int d = Dim<KIND>::d;
  constexpr int RB = rows_per_tile(KIND);
  __shared__ int s_abort;
  __shared__ unsigned long long s_red[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  // tile t belongs to CTA t % grid: consecutive tiles land on different SMs
  const int gw = warp * gridDim.x + blockIdx.x, tw = gridDim.x * nw;
  const int N = a.N;
  const int ntiles = (N + RB - 1) / RB;
  Control* ctrl = a.ctrl;
  unsigned long long bt = 0;
  if (threadIdx.x == 0) s_abort = 0;

  Ctx x;
  x.X = a.X; x.Xn = a.Xn;
  x.K1 = a.Kb[0]; x.K2 = a.Kb[1]; x.K3 = a.Kb[2]; x.K4 = a.Kb[3];
  x.rtol = a.rtol;
  x.thr = a.atol / a.rtol;
  x.m0 = 0.0; x.m1 = 0.0;
  x.c21 = x.c32 = x.hs = x.h0s = 0.0;

  // -------------------------------------------------------------------- RHS
  if (a.job == JOB_RHS) {
    x.p = Prec{a.rhs_f, a.rhs_s, a.rhs_g};
    x.single = (a.rhs_f == 0 && a.rhs_s == 0 && a.rhs_g == 0);
    for (int tile = gw; tile < ntiles; tile += tw) {
      const int i = tile * RB + lane;
      if (!(lane < RB && i < N)) continue;
      double Y[d];
#pragma unroll
      for (int c = 0; c < d; ++c) Y[c] = x.single ? (double)(float)x.X[c * N + i] : x.X[c * N + i];
      put_jv<KIND>(a, 0, i, Y, x.p.g, x.single);
    }
    if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) return;
    stage<KIND, ST>(a, x, PH_RHS, 0, gw, tw, lane);
    return;
  }

  x.single = (a.variant == V_SINGLE);
  const bool single = x.single;
  const Prec p2 = variant_prec(a.variant, 2);
  const Prec p3 = variant_prec(a.variant, 3);
  const Prec p4 = variant_prec(a.variant, 4);
  const double rtol = a.rtol;

  double t = a.t0, h = a.h_given;
  long long n_acc = 0, n_rej = 0, n_rhs = 0, next_out = 0;
  int status = S_OK;
  int parity = 0;
  bool rejected_this_step = false;

  // ------------------------------------------------------------ set-up rows
  for (int tile = gw; tile < ntiles; tile += tw) {
    const int i = tile * RB + lane;
    if (!(lane < RB && i < N)) continue;
    if (a.job == JOB_SOLVE) {
      for (long long k = 0; k < a.n_out && a.t_out[k] <= a.t0; ++k)
#pragma unroll
        for (int c = 0; c < d; ++c) a.y_out[(size_t)k * d * N + c * N + i] = x.X[c * N + i];
    }
    if (single) {
#pragma unroll
      for (int c = 0; c < d; ++c) {
        x.X[c * N + i] = (double)(float)x.X[c * N + i];
        if (a.job == JOB_ATTEMPT) x.K1[c * N + i] = (double)(float)x.K1[c * N + i];
      }
    }
    if (a.job == JOB_SOLVE) {
      double Y[d];
#pragma unroll
      for (int c = 0; c < d; ++c) Y[c] = x.X[c * N + i];
      put_jv<KIND>(a, 0, i, Y, p4.g, single);
    }
  }
  if (a.job == JOB_SOLVE)
    while (next_out < a.n_out && a.t_out[next_out] <= a.t0) ++next_out;

  if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) goto finish_up;

  if (a.job == JOB_SOLVE) {
    // ---- K1 = f(t0, y0) with the k4 row; starting-step norms d0, d1
    x.p = p4;
    x.m0 = 0.0; x.m1 = 0.0;
    stage<KIND, ST>(a, x, PH_K1, 0, gw, tw, lane);
    block_max(x.m0, &ctrl->red[0], s_red);
    block_max(x.m1, &ctrl->red[1], s_red);
    n_rhs = 1;
    if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) goto finish_up;
    {
      const double d0c = ld_bits(&ctrl->red[0]);
      const double d1c = ld_bits(&ctrl->red[1]);
      if (d0c != d0c || isinf(d0c) || d1c != d1c || isinf(d1c)) { status = S_NONFINITE; goto finish_up; }
    }
    if (!(a.h_given > 0.0)) {
      const double d0 = ld_bits(&ctrl->red[0]);
      const double d1 = ld_bits(&ctrl->red[1]);
      const double h0 = (d0 >= 1e-5 && d1 >= 1e-5) ? 0.01 * d0 / d1 : 1e-6;
      x.h0s = single ? (double)(float)h0 : h0;
      // y1 = y0 + h0 f0 -> j-vector 1
      for (int tile = gw; tile < ntiles; tile += tw) {
        const int i = tile * RB + lane;
        if (!(lane < RB && i < N)) continue;
        double Y[d];
#pragma unroll
        for (int c = 0; c < d; ++c) Y[c] = axpy_state(x.X[c * N + i], x.h0s, x.K1[c * N + i], single);
        put_jv<KIND>(a, 1, i, Y, p4.g, single);
      }
      if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) goto finish_up;
      x.m0 = 0.0;
      stage<KIND, ST>(a, x, PH_F1, 1, gw, tw, lane);
      block_max(x.m0, &ctrl->red[2], s_red);
      n_rhs = 2;
      if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) goto finish_up;
      const double d2 = ld_bits(&ctrl->red[2]) / h0;
      const double m = fmax(d1, d2);
      const double h1 = (m > 1e-15) ? pow(0.01 / m, 1.0 / 3.0) : fmax(1e-6, h0 * 1e-3);
      h = fmin(fmin(100.0 * h0, h1), a.hmax);
    }
  }

  while (true) {
    bool last = false;
    if (a.job == JOB_SOLVE) {
      if (!(t < a.t1)) break;
      if (n_rej > a.max_rejects) { status = S_MAX_REJECTS; break; }
      if (n_acc + n_rej >= a.max_attempts) { status = S_MAX_STEPS; break; }
      if (n_acc + n_rej > 0 && __ldcg(&ctrl->cancel_seen[parity ^ 1])) { status = S_TIMEOUT; break; }
      h = fmin(h, a.hmax);
      if (h <= a.hmin) { status = S_STEP_TOO_SMALL; break; }
      last = (t + 1.1 * h >= a.t1);
      if (last) h = a.t1 - t;
    }
    x.hs = single ? (double)(float)h : h;
    x.c21 = single ? (double)(0.5f * (float)h) : 0.5 * h;
    x.c32 = single ? (double)(0.75f * (float)h) : 0.75 * h;
    // ---- A: Y2 -> j-vector 0
    for (int tile = gw; tile < ntiles; tile += tw) {
      const int i = tile * RB + lane;
      if (!(lane < RB && i < N)) continue;
      double Y[d];
#pragma unroll
      for (int c = 0; c < d; ++c) Y[c] = axpy_state(x.X[c * N + i], x.c21, x.K1[c * N + i], single);
      put_jv<KIND>(a, 0, i, Y, p2.g, single);
    }
    if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) break;
    // ---- B2: K2 = f(Y2); Y3 -> j-vector 1
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->emax[parity ^ 1] = 0ull;
    x.p = p2; x.pn = p3;
    stage<KIND, ST>(a, x, PH_B2, 0, gw, tw, lane);
    if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) break;
    // ---- B3: K3 = f(Y3); X' -> j-vector 2
    x.p = p3; x.pn = p4;
    stage<KIND, ST>(a, x, PH_B3, 1, gw, tw, lane);
    if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) break;
    // ---- B4: K4 = f(X'); error norm
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctrl->cancel_seen[parity] = a.cancel ? *a.cancel : 0;
      if (a.progress) *a.progress = t;
    }
    x.p = p4;
    x.m1 = 0.0;
    stage<KIND, ST>(a, x, PH_B4, 2, gw, tw, lane);
    block_max(x.m1, &ctrl->emax[parity], s_red);
    if (!grid_sync(ctrl, bt, a.spin_limit, &s_abort)) break;
    n_rhs += 3;
    const double E = ld_bits(&ctrl->emax[parity]);
    if (a.job == JOB_ATTEMPT) {
      for (int tile = gw; tile < ntiles; tile += tw) {
        const int i = tile * RB + lane;
        if (!(lane < RB && i < N)) continue;
#pragma unroll
        for (int c = 0; c < d; ++c) {
          a.out0[c * N + i] = x.Xn[c * N + i];
          a.out1[c * N + i] = x.K4[c * N + i];
        }
      }
      break;
    }
    if (E != E || isinf(E)) { status = S_NONFINITE; ++n_rej; break; }
    if (E <= rtol) {
      const double t_new = last ? a.t1 : t + h;
      while (next_out < a.n_out && a.t_out[next_out] <= t_new) {
        const double th = (a.t_out[next_out] - t) / h;
        for (int tile = gw; tile < ntiles; tile += tw) {
          const int i = tile * RB + lane;
          if (!(lane < RB && i < N)) continue;
#pragma unroll
          for (int c = 0; c < d; ++c) {
            const int o = c * N + i;
            const double y0 = x.X[o], y1 = x.Xn[o], f0 = x.K1[o], f1 = x.K4[o];
            a.y_out[(size_t)next_out * d * N + o] =
                ((1.0 - th) * y0 + th * y1) +
                (th * (th - 1.0)) * (((1.0 - 2.0 * th) * (y1 - y0) + ((th - 1.0) * h) * f0) + (th * h) * f1);
          }
        }
        ++next_out;
      }
      double fac = (E == 0.0) ? 5.0 : fmin(5.0, 0.8 * pow(rtol / E, 1.0 / 3.0));
      if (rejected_this_step) fac = fmin(1.0, fac);
      const double h_new = h * fac;
      t = t_new;
      double* tmp = x.X; x.X = x.Xn; x.Xn = tmp;
      tmp = x.K1; x.K1 = x.K4; x.K4 = tmp;
      ++n_acc;
      rejected_this_step = false;
      h = h_new;
    } else {
      ++n_rej;
      if (!rejected_this_step) h = h * fmax(0.5, 0.8 * pow(rtol / E, 1.0 / 3.0));
      else h = h * 0.5;
      rejected_this_step = true;
    }
    parity ^= 1;
  }

finish_up:
  if (a.job == JOB_SOLVE && a.final_y != nullptr && !s_abort) {
    for (int tile = gw; tile < ntiles; tile += tw) {
      const int i = tile * RB + lane;
      if (!(lane < RB && i < N)) continue;
#pragma unroll
      for (int c = 0; c < d; ++c) a.final_y[c * N + i] = x.X[c * N + i];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (status != S_OK) atomicCAS(&ctrl->status, 0, status);
    ctrl->n_acc = n_acc;
    ctrl->n_rej = n_rej;
    ctrl->n_rhs = n_rhs;
    ctrl->n_out = next_out;
    ctrl->t = t;
    ctrl->h = h;
  }
}

}  // namespace bs3
