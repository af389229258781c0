// Solver kernels for the two oscillator kinds (Eq. LCO and the second-order form).
#include "bs3_solver.cuh"
#include "bs3_kernels.h"

namespace bs3 {
const void* kernel_lco_cfg(int st) {
  switch (st) {
    case ST_F64: return (const void*)bs3_kernel<K_LCO_CFG, ST_F64>;
    case ST_F32: return (const void*)bs3_kernel<K_LCO_CFG, ST_F32>;
    case ST_BF16: return (const void*)bs3_kernel<K_LCO_CFG, ST_BF16>;
    case ST_F16: return (const void*)bs3_kernel<K_LCO_CFG, ST_F16>;
    default: return (const void*)bs3_kernel<K_LCO_CFG, ST_FP8>;
  }
}
const void* kernel_lco_paper(int st) {
  switch (st) {
    case ST_F64: return (const void*)bs3_kernel<K_LCO_PAPER, ST_F64>;
    case ST_F32: return (const void*)bs3_kernel<K_LCO_PAPER, ST_F32>;
    case ST_BF16: return (const void*)bs3_kernel<K_LCO_PAPER, ST_BF16>;
    case ST_F16: return (const void*)bs3_kernel<K_LCO_PAPER, ST_F16>;
    default: return (const void*)bs3_kernel<K_LCO_PAPER, ST_FP8>;
  }
}
}  // namespace bs3
