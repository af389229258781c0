// Generated by gen_inst.py: solver kernels for lco_cfg with bf16 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_lco_cfg_bf16() { return (const void*)bs3_kernel<K_LCO_CFG, ST_BF16>; }
const void* batch_kernel_lco_cfg_bf16() {
  return (const void*)bs3_batch_kernel<K_LCO_CFG, ST_BF16>;
}
}  // namespace bs3
