// Generated by gen_inst.py: solver kernels for circadian with fp8 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_circadian_fp8() { return (const void*)bs3_kernel<K_CIRCADIAN, ST_FP8>; }
const void* batch_kernel_circadian_fp8() {
  return (const void*)bs3_batch_kernel<K_CIRCADIAN, ST_FP8>;
}
}  // namespace bs3
