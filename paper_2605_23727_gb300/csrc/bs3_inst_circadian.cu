// Solver kernels for the circadian clock kind (Eq. CC).
#include "bs3_solver.cuh"
#include "bs3_kernels.h"

namespace bs3 {
const void* kernel_circadian(int st) {
  switch (st) {
    case ST_F64: return (const void*)bs3_kernel<K_CIRCADIAN, ST_F64>;
    case ST_F32: return (const void*)bs3_kernel<K_CIRCADIAN, ST_F32>;
    case ST_BF16: return (const void*)bs3_kernel<K_CIRCADIAN, ST_BF16>;
    case ST_F16: return (const void*)bs3_kernel<K_CIRCADIAN, ST_F16>;
    default: return (const void*)bs3_kernel<K_CIRCADIAN, ST_FP8>;
  }
}
}  // namespace bs3
