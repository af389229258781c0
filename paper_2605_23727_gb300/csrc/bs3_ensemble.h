// Host interface of one shared-K ensemble solve (bs3_ensemble.cu), used by the
// ensemble entry points and by bs3_solve_batch, which runs an ensemble beside
// a ragged batch of independent systems in one CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bs3 {

struct EnsembleSpec {
  const float* K;          // device, N x N binary32 row-major
  int64_t N, T;
  const double* omega;     // device [T][N]
  const double* theta0;    // device [T][N]
  double t0, t1, rtol, atol;
  int tile_n;              // 128 or 256 (0 = 128)
  int64_t max_lockstep;    // > 0: stop after that many lock-step attempts
  int max_ctas;            // > 0: at most this many CTAs per stage product (else one per SM)
  double* theta_out;       // device [T][N]
};

// One ensemble solve.  create() validates the arguments, allocates every
// buffer and sets up the initial state (waits for that set-up); capture()
// records every kernel of the solve into the capture in progress on `st`
// (set-up stages, the attempt loop as a conditional WHILE node whose body is
// captured on `body`, then the gather of the final phases; loop_begin and
// loop_end, when not null, become event-record nodes around the loop); after
// the graph has run, finish() reads the counts and returns the solve's
// status.
class EnsembleRun {
 public:
  virtual ~EnsembleRun() {}
  virtual int capture(cudaStream_t st, cudaStream_t body, cudaEvent_t loop_begin, cudaEvent_t loop_end) = 0;
  virtual int finish(int64_t* n_acc, int64_t* n_rej, int32_t* status, int64_t* lockstep_attempts) = 0;
  // tensor flop of the split products of one lock-step attempt
  virtual double flop_per_attempt() const = 0;
};

int ensemble_create(const EnsembleSpec& spec, cudaStream_t st, EnsembleRun** out);

}  // namespace bs3
