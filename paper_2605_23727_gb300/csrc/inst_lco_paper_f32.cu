// Generated by gen_inst.py: solver kernels for lco_paper with f32 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_lco_paper_f32() { return (const void*)bs3_kernel<K_LCO_PAPER, ST_F32>; }
const void* batch_kernel_lco_paper_f32() {
  return (const void*)bs3_batch_kernel<K_LCO_PAPER, ST_F32>;
}
}  // namespace bs3
