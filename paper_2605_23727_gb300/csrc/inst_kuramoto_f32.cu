// Generated by gen_inst.py: solver kernels for kuramoto with f32 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_kuramoto_f32() { return (const void*)bs3_kernel<K_KURAMOTO, ST_F32>; }
const void* batch_kernel_kuramoto_f32() {
  return (const void*)bs3_batch_kernel<K_KURAMOTO, ST_F32>;
}
}  // namespace bs3
