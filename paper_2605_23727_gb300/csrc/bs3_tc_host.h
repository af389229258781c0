// Host helpers of the tensor-core product shared by its entry points.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace bs3 {
// 2D bf16 tensor map of a row-major [rows][cols] matrix, box tc::BK x box_rows,
// 128-byte swizzle.
int tc_encode_bf16_2d(CUtensorMap* map, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows);
// hi = bf16(x), lo = bf16(x - hi) for n binary32 values (device pointers).
int tc_split(const float* x, size_t n, void* hi, void* lo, cudaStream_t stream);
}  // namespace bs3
