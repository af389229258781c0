// Generated by gen_inst.py: solver kernels for kuramoto with bf16 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_kuramoto_bf16() { return (const void*)bs3_kernel<K_KURAMOTO, ST_BF16>; }
const void* batch_kernel_kuramoto_bf16() {
  return (const void*)bs3_batch_kernel<K_KURAMOTO, ST_BF16>;
}
}  // namespace bs3
