// Generated by gen_inst.py: solver kernels for circadian with f64 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_circadian_f64() { return (const void*)bs3_kernel<K_CIRCADIAN, ST_F64>; }
const void* batch_kernel_circadian_f64() {
  return (const void*)bs3_batch_kernel<K_CIRCADIAN, ST_F64>;
}
}  // namespace bs3
