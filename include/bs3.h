/*
 * bs3.h -- C ABI of the GB300 (sm_103a) mixed-precision Bogacki-Shampine 3(2)
 * solver for large ODE systems with dense, all-pairs, heterogeneous coupling.
 *
 * Method (paper: "Mixed-Precision in adaptive Runge-Kutta method for large ODE
 * systems"):
 *   - general model X_i' = F_i(X_i) + sum_j M_ij (.) G_ij(X_i, X_j)
 *     (Sec. 2.1, Eq. General-Model) with three benchmark kinds (Eq. LCO,
 *     Eq. Kuramoto, Eq. CC) plus the second-order oscillator form;
 *   - the Bogacki-Shampine 3(2) pair with FSAL (Sec. 2.2, Table Butcher-O23,
 *     Eq. Stage-ODE23), the embedded max-norm error (Eq. ERROR-O23), the
 *     accept test E <= Rel and the failure conditions of Sec. 2.2;
 *   - the precision distribution Single / Mixed1 / Mixed2 / Double of
 *     Sec. 2.3, Table MP-Distrib, extended to bfloat16 / fp16 / fp8 storage of
 *     the coupling weights (Sec. 4 names these formats as the next step).
 *
 * Conventions for every entry point:
 *   - Return value: a bs3_status code (0 = BS3_OK).  Nothing throws; on error
 *     the outputs that could be produced are still written (see bs3_solve).
 *   - State vectors are binary64, structure-of-arrays: component k of agent i
 *     is y[k*N + i], length d*N with d = 2 (LCO_CFG, LCO_PAPER), 1 (KURAMOTO)
 *     or 4 (CIRCADIAN).
 *   - "Device pointer" means memory of the system's device (cudaMalloc or
 *     managed); "host pointer" means ordinary or pinned host memory.
 *   - The caller owns every pointer it passes; the library owns the system,
 *     its stored (quantised) weights and all of its scratch buffers.
 *   - Work is issued on the system's CUDA stream; bs3_solve and bs3_rhs
 *     return after their results are complete.
 *   - A system is not thread-safe: calls on one system must not overlap.
 */
#ifndef BS3_H
#define BS3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bs3_system* bs3_system_t;

/* Kinds of right-hand side (Sec. 2.1).
 * BS3_LCO_CFG   second-order oscillators: x' = v, v' = -omega_i^2 x + sum_j A_ij x_j.
 *               params[N] = omega_i.
 * BS3_LCO_PAPER Eq. LCO: x' = v + sum_j M_ij (x_j - x_i), v' = -x.  n_params = 0.
 * BS3_KURAMOTO  Eq. Kuramoto: theta' = omega_i + sum_j K_ij sin(theta_j - theta_i).
 *               params[N] = omega_i.
 * BS3_CIRCADIAN Eq. CC with Hill exponent 4, coupling on component 1:
 *               pref_i sum_j W_ij atan(x_j1 - x_i1), pref_i = k0 Th_i a/(Th_i + x_i2^4),
 *               Th_i = k1_i/(k0 - k1_i).  params[N + 8] = k1_i (N values), then
 *               k0, k2, k3, a, b, c, eps, I0.  The coupling coefficient K of
 *               the paper is folded into W. */
typedef enum { BS3_LCO_CFG = 0, BS3_LCO_PAPER = 1, BS3_KURAMOTO = 2, BS3_CIRCADIAN = 3 } bs3_kind;

/* Precision variants, Table MP-Distrib (Sec. 2.3): (F, Sigma, G) per stage.
 * SINGLE: all S, state and stage combinations in binary32 (t, h, E in binary64).
 * MIXED1: k2,k3 (S,S,S), k4 (D,D,S); MIXED2: k2..k4 (D,D,S); DOUBLE: all D. */
typedef enum { BS3_SINGLE = 0, BS3_MIXED1 = 1, BS3_MIXED2 = 2, BS3_DOUBLE = 3 } bs3_variant;

/* Element types of the coupling weights. */
typedef enum { BS3_F64 = 0, BS3_F32 = 1, BS3_BF16 = 2, BS3_F16 = 3, BS3_FP8E4M3 = 4 } bs3_dtype;

/* How a Sigma = D stage sums its binary32 products (G = S):
 * BS3_ACC_F64    each product cast to binary64 and added in binary64 (Sec. 2.3, literal);
 * BS3_ACC_FLOAT2 compensated float-float sum: the exact rounding error of every
 *                addition kept in a binary32 low part (TwoSum; the packed sums of the
 *                Kuramoto and circadian kinds start from a power-of-two bias
 *                >= 2.5 sum_j |q_ij| of every row of a CTA and take Fast2Sum);
 * BS3_ACC_F32    plain binary32 sum (departs from the table; for study only).
 * Sigma = S stages always sum in binary32; G = D stages in binary64. */
typedef enum { BS3_ACC_F32 = 0, BS3_ACC_FLOAT2 = 1, BS3_ACC_F64 = 2 } bs3_accum;

/* Status codes. */
enum {
    BS3_OK = 0,
    BS3_ERR_INVALID_ARG = 1,
    BS3_ERR_CUDA = 2,
    BS3_ERR_MAX_STEPS = 3,        /* accepted + failed attempts reached I_max (Sec. 2.2) */
    BS3_ERR_MAX_REJECTS = 4,      /* failed attempts above 0.85 I_max (Sec. 2.2) */
    BS3_ERR_STEP_TOO_SMALL = 5,   /* h <= h_min = 100 eps_m (Sec. 2.2) */
    BS3_ERR_TIMEOUT = 6,          /* wall-clock limits of Sec. 2.2 */
    BS3_ERR_DEVICE_WAIT = 7,      /* a bounded device-side wait ran out */
    BS3_ERR_NONFINITE = 8         /* NaN or Inf in the state, the stages or E */
};

/* Flags of bs3_solve. */
enum {
    BS3_HOST_IO = 1               /* y0, t_out and y_out are host pointers */
};

typedef struct {
    int64_t n_accepted;           /* accepted attempts */
    int64_t n_rejected;           /* failed attempts */
    int64_t n_rhs_evals;          /* right-hand-side evaluations (2 + 3 per attempt) */
    double  t_reached;            /* time of the last accepted state */
    double  h_last;               /* step size the controller would use next */
    int32_t status;               /* bs3_status of the solve */
    int32_t n_out_written;        /* dense outputs written (t_out <= t_reached) */
} bs3_stats;

/* Failure conditions of Sec. 2.2 and the device wait bound. */
typedef struct {
    int64_t max_attempts;         /* I_max, default 100000 */
    int64_t max_rejects;          /* default 85000 (0.85 I_max) */
    double  hmin_factor;          /* h_min = hmin_factor * eps_m, default 100 */
    double  wall_limit_s;         /* default 5400 (1.5 h) */
    double  slow_limit_s;         /* default 2700 (45 min) ... */
    double  slow_fraction;        /* ... with less than this fraction of [t0,t1] done, default 0.1 */
    int64_t spin_limit;           /* polls of one grid barrier before BS3_ERR_DEVICE_WAIT, default 2^26 */
} bs3_limits;

/* Fills *lim with the paper's defaults (Sec. 2.2). */
void bs3_default_limits(bs3_limits* lim);

/* Name of a status code ("BS3_OK", ...); never NULL. */
const char* bs3_status_string(int status);

/* Creates a system of N agents of the given kind on CUDA device `device`.
 * params: host array of n_params binary64 values, layout per bs3_kind above
 * (copied; NULL allowed when n_params == 0).  stream: a cudaStream_t or NULL
 * for the legacy default stream.  Allocates all per-system device buffers.
 * Errors: BS3_ERR_INVALID_ARG (bad kind, N < 1, wrong n_params, out == NULL),
 * BS3_ERR_CUDA (device selection or allocation failed). */
int bs3_create_system(int kind, int64_t N, const double* params, int64_t n_params,
                      int device, void* stream, bs3_system_t* out);

/* Stores the N x N coupling weights (Sec. 2.1: M_ij, with K, A or W folded in).
 * K: row-major N*N values of type src (BS3_F64 or BS3_F32), host or device
 * (is_device_ptr).  store: the element type kept on the device.  Quantisation
 * rounds to binary32 first, then to `store` (nearest even), with per-row scales
 * s_i: 1 for F64/F32/BF16; a power of two mapping each row's maximum into
 * [2^14, 2^15) for F16; fp32(rowmax/448) for FP8E4M3 (saturating).  An all-zero
 * row has s_i = 1.  Replaces any previous weights.  Must precede bs3_solve. */
int bs3_set_coupling(bs3_system_t sys, const void* K, int src, int store, int is_device_ptr);

/* Copies the stored weights back for inspection: q_out receives N*N values of
 * the stored type (host memory, row-major, no padding), scales_out N binary32
 * row scales (either may be NULL). */
int bs3_get_coupling(bs3_system_t sys, void* q_out, float* scales_out);

/* One right-hand-side evaluation out = f(t, y) (Eq. General-Model) with the
 * precision triple (f_prec, sigma_prec, g_prec), each 0 = S, 1 = D, and the
 * Sigma = D summation mode `accum`.  y, out: device pointers of d*N binary64.
 * With f_prec = sigma_prec = g_prec = S the input is first rounded to binary32
 * (the Single state) and the result holds binary32 values. */
int bs3_rhs(bs3_system_t sys, double t, const double* y, int f_prec, int sigma_prec,
            int g_prec, int accum, double* out);

/* One BS3 attempt of size h from (t, X, K1) (Eq. Stage-ODE23, Eq. ERROR-O23):
 * writes X^{n+1} to xn_out, K4 = f(t+h, X^{n+1}) to k4_out (device, d*N binary64)
 * and the error E to *err_out (host).  No controller, no counters. */
int bs3_attempt(bs3_system_t sys, double t, double h, const double* x, const double* k1,
                double rtol, double atol, int variant, int accum,
                double* xn_out, double* k4_out, double* err_out);

/* Adaptive solve of the system from t0 to t1 > t0 (Sec. 2.2-2.3), entirely on
 * the device in one persistent cooperative launch (no host round trip per step).
 * y0: d*N binary64 initial state.  rtol > 0, atol >= 0 (Rel, Ab of Eq. ERROR-O23).
 * variant: bs3_variant; accum: bs3_accum for Sigma = D stages.
 * t_out: n_out requested output times, ascending, within [t0, t1]; y_out receives
 * n_out * d*N values (dense output by cubic Hermite on each accepted step).
 * flags: BS3_HOST_IO if y0/t_out/y_out are host pointers, else device pointers.
 * final_y (optional, may be NULL): d*N state at t_reached, same memory kind as y_out.
 * stats (host, optional), lim (host, NULL = bs3_default_limits).
 * Returns the solve status (also in stats->status).  On a failure status the
 * outputs with t_out <= t_reached and final_y are still written. */
int bs3_solve(bs3_system_t sys, double t0, double t1, const double* y0, double rtol,
              double atol, int variant, int accum, const double* t_out, int64_t n_out,
              double* y_out, double* final_y, int flags, bs3_stats* stats,
              const bs3_limits* lim);

/* Tuning knobs (bs3_set_tuning keys). */
enum {
    /* 1: when the weight rows of every CTA fit in its shared memory (one CTA
     * per SM), load them once per solve and keep them on chip; 0 (default):
     * stream them from HBM/L2 at every stage.  Results are identical.  On
     * GB300 keeping them on chip leaves too little L1 for the j-vectors and
     * measured slower (Kuramoto N=4096, bf16: 64.5 vs 61.7 ms). */
    BS3_TUNE_RESIDENT_WEIGHTS = 1,
    /* CTAs of the persistent launch: 0 (default) = one per SM; otherwise at
     * most this many (fewer CTAs = cheaper grid barriers, more rows each). */
    BS3_TUNE_CTAS = 2
};

/* Embedded Runge-Kutta pair of bs3_solve (bs3_set_method). */
enum {
    /* Bogacki-Shampine 3(2), the paper's solver (default). */
    BS3_METHOD_BS32 = 0,
    /* Dormand-Prince 5(4), the extension of the precision variants to another
     * explicit FSAL pair (Sec. 4): seven stages (six evaluations per attempt),
     * error e = b - b_hat of the published pair in the norm of Eq.
     * ERROR-O23, controller exponent 1/5, Table MP-Distrib carried stage by
     * stage (Mixed1: stages 2..6 (S,S,S), stage 7 (D,D,S); Mixed2: all
     * (D,D,S)).  Dense output stays the cubic Hermite on X^n, K_1, X^{n+1},
     * K_7. */
    BS3_METHOD_DP54 = 1
};

/* Selects the embedded pair of later bs3_solve calls on this system.
 * bs3_attempt and bs3_batch_solve run Bogacki-Shampine 3(2) only (bs3_attempt
 * returns BS3_ERR_INVALID_ARG on a Dormand-Prince system).  Errors:
 * BS3_ERR_INVALID_ARG for an unknown method. */
int bs3_set_method(bs3_system_t sys, int method);

/* Sets a tuning knob of the system (takes effect at the next launch).
 * Errors: BS3_ERR_INVALID_ARG for an unknown key or value.  The paper has no
 * counterpart (it concerns only how this library maps the method on the GPU). */
int bs3_set_tuning(bs3_system_t sys, int key, int64_t value);

/* Autotuner: times bounded solves (at most `attempts` attempts each, from y0
 * on the device) of every candidate launch plan -- resident weights off/on x
 * CTAs = SMs, SMs/2, SMs/4 -- and applies the fastest per attempt to the
 * system.  choice_out[2] (host) receives (resident, ctas), us_out (host) the
 * chosen plan's microseconds per attempt.  The paper has no counterpart. */
int bs3_autotune(bs3_system_t sys, const double* y0, double t0, double t1, double rtol, int variant, int accum,
                 int attempts, int64_t* choice_out, double* us_out);

/* Step history (tracing, and the training data of a learned step-size
 * proposer): with capacity > 0, each later bs3_solve records its first
 * `capacity` attempts, 8 binary64 values each: t, h, E (Eq. ERROR-O23),
 * accepted (1/0), then the device time in ns from the start of the attempt
 * to the end of each of its four grid barriers (as seen by CTA 0).
 * capacity = 0 turns recording off and frees the buffer.  The paper has no
 * counterpart (its metrics are computed offline from MATLAB runs). */
int bs3_set_history(bs3_system_t sys, int64_t capacity);

/* Copies the records of the last solve to out (host, at least capacity*8
 * binary64) and their number to *n_records. */
int bs3_get_history(bs3_system_t sys, double* out, int64_t* n_records);

/* ------------------------------------------------------------------------
 * Learned step-size proposer (the paper has no learned component; this is the
 * build's extension).  A small MLP, 6 -> 32 -> 32 -> 1 with tanh, proposes the
 * next step size after an accepted step without rejections:
 *   features [log r_{n-3}, log r_{n-2}, log r_{n-1}, log r_n, log h_n, log Rel],
 *   r = clamp(E/Rel, 1e-8, 1e8) over the last accepted steps (missing ones
 *   repeat the oldest), standardised by the model's mean and std;
 *   h_{n+1} = h_n exp(clamp(out, log 0.2, log 5)).
 * The embedded error test (Eq. ERROR-O23) still accepts or rejects every
 * attempt, and a rejection falls back to the plain controller.
 * A model is 1325 binary32: 1313 parameters (W1[32][6] row-major, b1[32],
 * W2[32][32], b2[32], W3[32], b3) then mean[6], std[6].
 * ------------------------------------------------------------------------ */
#define BS3_MLP_PARAMS 1313
#define BS3_MLP_MODEL 1325

/* Training pairs from one solve's step history (bs3_get_history records):
 * for consecutive accepted steps n, n+1, X[n] = features of step n (raw, not
 * standardised; host, 6 binary32 each) and y[n] = log(h_star / h_n) with
 * h_star = h_{n+1} (0.75 / r_{n+1})^(1/3), the step that would have given
 * E = 0.75 Rel under E ~ h^3.  X and y need n_rec rows; *n_out receives the
 * number written.  Host computation. */
int bs3_mlp_dataset(const double* hist, int64_t n_rec, double rtol, float* X, float* y, int64_t* n_out);

/* Trains the MLP on the GPU (per-sample forward/backward kernels, Adam with
 * beta = (0.9, 0.999), eps 1e-8) on n raw samples (host X[n][6], y[n]),
 * minimising 0.5 mean((out - y)^2) from params_init (host, 1313) for `epochs`
 * shuffled passes of minibatches of `batch`.  Writes the model (host, 1325:
 * parameters, then the inputs' mean and std) and, if loss_hist is not NULL,
 * each epoch's mean minibatch loss. */
int bs3_mlp_train(const float* X, const float* y, int64_t n, const float* params_init, int epochs, int batch,
                  float lr, uint64_t seed, float* model_out, float* loss_hist);

/* Loss 0.5 mean((out - y)^2) and its gradient (host, 1313) at params (host,
 * 1313) over n standardised samples (host), computed by the training kernel. */
int bs3_mlp_grad(const float* params, const float* X, const float* y, int64_t n, float* grad_out,
                 float* loss_out);

/* Installs a trained model (host, 1325 binary32; weights rounded to bfloat16
 * for inference) in the system, or removes it (model = NULL).  Errors:
 * BS3_ERR_INVALID_ARG for non-finite values or a non-positive std. */
int bs3_set_proposer(bs3_system_t sys, const float* model);

/* Tensor-core product used by ensembles that share one coupling matrix
 * (the build's extension; the paper has no batching):
 *   C = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T,
 * A (M x K) and B (Nc x K) binary32 row-major, split into bfloat16 pairs
 * x_hi = bf16(x), x_lo = bf16(x - x_hi) (nearest even), products accumulated
 * in binary32 by tcgen05.mma in tensor memory; C (M x Nc) binary32 row-major.
 * All device pointers.  Requires M % 128 == 0, Nc % 256 == 0, K % 64 == 0.
 * Returns BS3_ERR_DEVICE_WAIT if a bounded pipeline wait ran out. */
int bs3_tc_gemm(int64_t M, int64_t Nc, int64_t K, const float* A, const float* B, float* C);

/* The same split product computed the way the ensembles' stage products run
 * (bs3_ensemble_solve): persistent CTAs, at most one per SM (and at most
 * max_ctas when max_ctas > 0), CTA b taking the 128 x tile_n output tiles b,
 * b + grid, ... (numbered row block by row block), with two accumulators in
 * tensor memory so that one tile's read-out overlaps the next tile's
 * products; 16 epilogue warps store the binary32 accumulators.  Arguments as
 * bs3_tc_gemm; tile_n = 128 or 256 with Nc % tile_n == 0.  Waits for
 * completion.  Returns BS3_ERR_DEVICE_WAIT if a bounded pipeline wait ran out.
 * The paper has no counterpart (the ensembles are the build's extension). */
int bs3_tc_gemm_persistent(int64_t M, int64_t Nc, int64_t K, const float* A, const float* B, float* C,
                           int tile_n, int max_ctas);

/* Lock-step ensemble of T Kuramoto trajectories sharing one coupling matrix
 * (the build's batched extension): theta_b' = omega_b + sum_j K_ij sin(theta_bj
 * - theta_bi), b = 0..T-1, each trajectory with its own adaptive h, t and
 * accept/reject decision (the controller and failure conditions of bs3_solve),
 * all stages of all live trajectories computed together on the tensor cores:
 * G = bfloat16 hi+lo split of K and of sin/cos (bs3_tc_gemm's three products),
 * Sigma = binary32 accumulation and i-side finish, F and the state, stage
 * combinations and error norm in binary64 (the oracle's "tensor" variant).
 * K: device, N x N binary32 row-major; omega, theta0, theta_out: device,
 * [T][N] binary64 (trajectory-major).  N % 128 == 0, T % 64 == 0 (the tile
 * width is chosen as bs3_ensemble_solve_tiled with tile_n = 0 does).
 * n_acc, n_rej, status (host arrays of T, may be NULL) receive each
 * trajectory's counts and status; *lockstep_attempts (host, may be NULL) the
 * number of lock-step attempts run.  Waits for completion.  Returns
 * BS3_ERR_DEVICE_WAIT if a bounded pipeline wait ran out. */
int bs3_ensemble_solve(const float* K, int64_t N, int64_t T, const double* omega, const double* theta0,
                       double t0, double t1, double rtol, double atol, double* theta_out, int64_t* n_acc,
                       int64_t* n_rej, int32_t* status, int64_t* lockstep_attempts, void* stream);

/* bs3_ensemble_solve with an explicit output tile width and an optional bound.
 * tile_n: 256 (128 x 256 accumulator tiles, 128 trajectories per tile; needs
 * T % 128 == 0), 128 (128 x 128 tiles, 64 trajectories; T % 64 == 0), or 0
 * (= 128).  Each stage product runs on at most one CTA per SM, each CTA taking
 * tiles in turn with two accumulators in tensor memory, so that one tile's
 * epilogue overlaps the next tile's products; the narrower tiles give every
 * CTA more tiles to overlap.  max_lockstep > 0 stops after that many
 * lock-step attempts (rounded up to the 8 of one graph launch) and returns
 * BS3_ERR_MAX_STEPS if trajectories are still running; 0 = no bound beyond
 * the per-trajectory limits.  The paper has no counterpart. */
int bs3_ensemble_solve_tiled(const float* K, int64_t N, int64_t T, const double* omega, const double* theta0,
                             double t0, double t1, double rtol, double atol, int tile_n, int64_t max_lockstep,
                             double* theta_out, int64_t* n_acc, int64_t* n_rej, int32_t* status,
                             int64_t* lockstep_attempts, void* stream);

/* Autotuner of the ensemble's tile width: runs bounded solves (lockstep_attempts
 * lock-step attempts, >= 8) with each valid width and returns the one with the
 * shortest device time per attempt in *tile_out (and that time in
 * microseconds in *us_out, may be NULL).  scratch_theta: device [T][N]
 * binary64 buffer the bounded solves write.  Arguments otherwise as
 * bs3_ensemble_solve.  The paper has no counterpart. */
int bs3_ensemble_autotune(const float* K, int64_t N, int64_t T, const double* omega, const double* theta0,
                          double t0, double t1, double rtol, double atol, int64_t lockstep_attempts,
                          double* scratch_theta, int* tile_out, double* us_out);

/* Ragged batch of S independent systems of one kind (sizes N_k may all
 * differ) solved in one launch (the build's batched extension): each CTA takes
 * whole systems from a work queue, largest first, and runs the solver of
 * bs3_solve on it with CTA barriers only; every system has its own adaptive
 * h, t1 and status.  All host arrays, concatenated over the systems in order:
 *   Ns[S]; params: the per-agent values of each system (N_k values; for
 *   BS3_CIRCADIAN N_k values then the 8 constants, which must agree across the
 *   batch; NULL for BS3_LCO_PAPER); K: each system's N_k x N_k binary32
 *   row-major weights; y0, y_final: each system's d*N_k state (SoA);
 *   t0[S], t1[S]; stats[S] (may be NULL); *kernel_ms (may be NULL) receives
 *   the device time of the solve launch alone (without quantisation and copies).
 * store, rtol, atol, variant, accum as bs3_set_coupling / bs3_solve (wall-clock
 * limits not enforced).  Returns the first non-OK system status, else BS3_OK. */
int bs3_batch_solve(int kind, int64_t S, const int64_t* Ns, const double* params, const float* K, int store,
                    const double* y0, const double* t0, const double* t1, double rtol, double atol, int variant,
                    int accum, double* y_final, bs3_stats* stats, double* kernel_ms, int device, void* stream);

/* One instance of bs3_solve_batch: a system made by bs3_create_system with
 * its weights stored (bs3_set_coupling), its initial state, span and
 * tolerances; stats receives its counts and status. */
typedef struct {
    bs3_system_t sys;
    const double* y0;             /* d*N initial state (memory kind per the call's flags) */
    double* y_final;              /* d*N state at t_reached (same memory kind) */
    double t0, t1;                /* t1 > t0 */
    double rtol, atol;            /* Rel > 0, Ab >= 0 of Eq. ERROR-O23 for this instance */
    bs3_stats stats;              /* out */
} bs3_batch_item;

/* A group of T Kuramoto trajectories that share one coupling matrix, solved
 * by bs3_solve_batch beside the items as bs3_ensemble_solve solves it.  All
 * pointers but the counts are device pointers: K N x N binary32 row-major,
 * omega, theta0, theta_out [T][N] binary64.  n_acc, n_rej, status: host
 * arrays of T (may be NULL).  ctas: 0 = the group's products use every SM,
 * after the items' launch; > 0 = the group runs beside the items with this
 * many CTAs per product (see bs3_solve_batch); tile_n as
 * bs3_ensemble_solve_tiled. */
typedef struct {
    const float* K;
    int64_t N, T;
    const double* omega;
    const double* theta0;
    double* theta_out;
    double t0, t1, rtol, atol;
    int tile_n;
    int ctas;
    int64_t* n_acc;
    int64_t* n_rej;
    int32_t* status;
    int64_t lockstep_attempts;    /* out: lock-step attempts run */
} bs3_ensemble_group;

/* Solves a batch in one submission (the build's batched extension; the paper
 * solves one system at a time): n_items independent systems, every one with
 * its own span, tolerances, adaptive h and decisions, plus optionally (group
 * != NULL) one shared-K trajectory group.  The items' systems must all be of
 * one kind and one stored weight type, on `device`, with the Bogacki-Shampine
 * pair (bs3_set_method), and circadian systems must share the eight
 * constants; a system appears in at most one item (its buffers hold the item's
 * state during the solve).  variant and accum apply to every item (the group runs the
 * tensor-core variant of bs3_ensemble_solve).  flags: BS3_HOST_IO if the
 * items' y0 and y_final are host pointers.
 *
 * The items run as bs3_batch_solve runs its systems: one cooperative launch,
 * largest systems first, systems too large for one SM's share solved by teams
 * of CTAs, the others whole by single CTAs, each CTA taking systems from a work
 * queue.  The group runs as bs3_ensemble_solve runs it, its attempt loop a
 * conditional graph node decided on the device.  With both, they form one
 * CUDA graph, launched once: by default the items' launch, then the group,
 * each on every SM (a solver CTA holds all of an SM's registers, so the two
 * cannot share SMs, and a split of the SMs cannot finish before the sum of the
 * two parts); with group->ctas > 0 the two run side by side, the group's
 * products on group->ctas CTAs and the items on the other SMs.  Items'
 * weights are the systems' stored copies; the call allocates a small
 * descriptor block and, once per system, a state buffer the system keeps.
 * Waits for completion; *kernel_ms (may be NULL) receives the device time of
 * the solve.  Returns the first non-OK item status, else the group's, else
 * BS3_OK; BS3_ERR_INVALID_ARG for mixed kinds, types or devices. */
int bs3_solve_batch(bs3_batch_item* items, int64_t n_items, int variant, int accum, int flags,
                    bs3_ensemble_group* group, int device, void* stream, double* kernel_ms);

/* Largest N accepted by bs3_solve_noalloc. */
#define BS3_NOALLOC_MAX_N 16384

/* bs3_solve without any device allocation, for callers that cannot allocate
 * device memory at solve time: code that runs under an allocator or memory
 * pool it does not own, a service with a fixed device-memory budget, or
 * any setting where cudaMalloc is not allowed once start-up is over.  (A
 * bs3 system allocates its buffers in bs3_create_system and bs3_set_coupling,
 * so such callers cannot use bs3_solve.)  The paper has no counterpart.
 *
 * Scratch: one file-scope __device__ array of about 1.5 MB (j-vectors, row
 * sums, row scales, k1/(k0-k1) and the control block for N <= 16384), which
 * every GPU that loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress)
 * with the device current.  All calls share the array and every call
 * overwrites it, so calls that overlap on the GPU (other streams, other host
 * threads) race: serialise them.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  The call is synchronous: it waits for the
 * solve and reads its control block back, so it cannot be called while the
 * stream is being captured into a CUDA graph.
 *
 * Arguments (all arrays are device pointers of the current device unless noted):
 *   kind, N       as bs3_create_system; 1 <= N <= BS3_NOALLOC_MAX_N;
 *   par           N per-agent values (omega_i or k1_i; NULL for BS3_LCO_PAPER);
 *   globals       host array of the 8 circadian constants k0, k2, k3, a, b, c,
 *                 eps, I0 (NULL for the other kinds); k0 finite and > 0, and
 *                 every k1_i in (0, k0), as bs3_create_system requires;
 *   weights, store, ld
 *                 the coupling weights already in their stored form: N rows of
 *                 ld values of type store (BS3_F32 or BS3_F64, row scale 1),
 *                 ld a multiple of 16 with N <= ld <= BS3_NOALLOC_MAX_N,
 *                 columns N..ld-1 equal to zero, 16-byte aligned;
 *   the rest      as bs3_solve with device pointers (t_out ascending within
 *                 [t0, t1]), stats on the host, stream a cudaStream_t or NULL.
 * The failure limits are bs3_default_limits() except the wall-clock ones,
 * which need host-mapped memory and are not enforced.  Returns the solve
 * status after the results are complete (also in stats->status);
 * BS3_ERR_INVALID_ARG for N or ld above BS3_NOALLOC_MAX_N or a malformed
 * argument, before anything is launched (the circadian k1 check runs on the
 * device and returns before the solve); BS3_ERR_CUDA if a CUDA call fails. */
int bs3_solve_noalloc(int kind, int64_t N, const double* par, const double* globals,
                      const void* weights, int store, int64_t ld, double t0, double t1,
                      const double* y0, double rtol, double atol, int variant, int accum,
                      const double* t_out, int64_t n_out, double* y_out, double* final_y,
                      bs3_stats* stats, void* stream);

/* Read-bandwidth probe (measurement only; the paper has no counterpart): one
 * untimed pass, then `reps` passes over `bytes` of device memory at buf
 * (16-byte aligned, bytes a multiple of 16) with the coupling pass's loads
 * (16-byte, non-allocating in L1, L2 evict_last), two 512-thread CTAs per SM
 * each reading a contiguous share; *gbs_out receives bytes * reps / time in
 * GB/s (CUDA events on the legacy default stream).  A buffer that fits in L2
 * gives the L2 read rate that bounds a coupling pass whose weights stay
 * there.  Errors: BS3_ERR_INVALID_ARG for a bad buffer, size or count. */
int bs3_read_bandwidth(const void* buf, int64_t bytes, int reps, double* gbs_out);

/* Frees the system and everything it owns.  NULL is allowed. */
int bs3_destroy_system(bs3_system_t sys);

#ifdef __cplusplus
}
#endif

#endif /* BS3_H */
