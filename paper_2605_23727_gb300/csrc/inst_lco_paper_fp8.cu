// Generated by gen_inst.py: solver kernels for lco_paper with fp8 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_lco_paper_fp8() { return (const void*)bs3_kernel<K_LCO_PAPER, ST_FP8>; }
const void* batch_kernel_lco_paper_fp8() {
  return (const void*)bs3_batch_kernel<K_LCO_PAPER, ST_FP8>;
}
}  // namespace bs3
