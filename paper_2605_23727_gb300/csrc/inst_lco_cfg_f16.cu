// Generated by gen_inst.py: solver kernels for lco_cfg with f16 weights.
#include "bs3_solver.cuh"

namespace bs3 {
const void* kernel_lco_cfg_f16() { return (const void*)bs3_kernel<K_LCO_CFG, ST_F16>; }
const void* batch_kernel_lco_cfg_f16() {
  return (const void*)bs3_batch_kernel<K_LCO_CFG, ST_F16>;
}
}  // namespace bs3
