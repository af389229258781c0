// Read-bandwidth probe: the denominator of a roofline for a pass whose
// operand stays in L2 (the coupling weights of a system whose N x N matrix
// fits in the 126 MB L2).  It reads a device buffer with the same 16-byte
// non-allocating loads and L2 evict_last policy as the coupling pass, every
// CTA streaming a contiguous share, and times repeated passes with CUDA
// events.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/bs3.h"
#include "bs3_device.cuh"

namespace bs3 {

__global__ void __launch_bounds__(512) read_probe_kernel(const uint4* __restrict__ buf, int64_t n16, int reps,
                                                          unsigned* __restrict__ sink) {
  const unsigned long long pol = l2_policy(true);
  const int64_t per = (n16 + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per;
  const int64_t hi = min(n16, lo + per);
  unsigned x = 0;
  for (int r = 0; r < reps; ++r) {
#pragma unroll 4
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const uint4 v = ld_stream16_pol(buf + e, pol);
      x ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  // keeps the loads; the value is never 0xffffffff for a buffer of zeros
  if (x == 0xffffffffu) sink[blockIdx.x] = x;
}

}  // namespace bs3

extern "C" int bs3_read_bandwidth(const void* buf, int64_t bytes, int reps, double* gbs_out) {
  using namespace bs3;
  if (!buf || !gbs_out || bytes < 16 || bytes % 16 != 0 || reps < 1 || ((uintptr_t)buf & 15) != 0)
    return BS3_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return BS3_ERR_CUDA;
  const int64_t n16 = bytes / 16;
  const int grid = 2 * sms;   // two 512-thread CTAs per SM
  unsigned* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BS3_OK;
  float ms = 0.f;
  do {
    if (cudaMalloc(&sink, (size_t)grid * sizeof(unsigned)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    // one untimed pass brings the buffer into L2 when it fits there
    read_probe_kernel<<<grid, 512>>>((const uint4*)buf, n16, 1, sink);
    if (cudaEventRecord(e0) != cudaSuccess) { rc = BS3_ERR_CUDA; break; }
    read_probe_kernel<<<grid, 512>>>((const uint4*)buf, n16, reps, sink);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = BS3_ERR_CUDA;
      break;
    }
    *gbs_out = (double)bytes * reps / (ms * 1e-3) / 1e9;
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}
