// Generated by gen_inst.py: kernel lookup across translation units.
#pragma once

#include <cuda_runtime.h>

namespace bs3 {
const void* kernel_lco_cfg_f64();
const void* batch_kernel_lco_cfg_f64();
const void* kernel_lco_cfg_f32();
const void* batch_kernel_lco_cfg_f32();
const void* kernel_lco_cfg_bf16();
const void* batch_kernel_lco_cfg_bf16();
const void* kernel_lco_cfg_f16();
const void* batch_kernel_lco_cfg_f16();
const void* kernel_lco_cfg_fp8();
const void* batch_kernel_lco_cfg_fp8();
const void* kernel_lco_paper_f64();
const void* batch_kernel_lco_paper_f64();
const void* kernel_lco_paper_f32();
const void* batch_kernel_lco_paper_f32();
const void* kernel_lco_paper_bf16();
const void* batch_kernel_lco_paper_bf16();
const void* kernel_lco_paper_f16();
const void* batch_kernel_lco_paper_f16();
const void* kernel_lco_paper_fp8();
const void* batch_kernel_lco_paper_fp8();
const void* kernel_kuramoto_f64();
const void* batch_kernel_kuramoto_f64();
const void* kernel_kuramoto_f32();
const void* batch_kernel_kuramoto_f32();
const void* kernel_kuramoto_bf16();
const void* batch_kernel_kuramoto_bf16();
const void* kernel_kuramoto_f16();
const void* batch_kernel_kuramoto_f16();
const void* kernel_kuramoto_fp8();
const void* batch_kernel_kuramoto_fp8();
const void* kernel_circadian_f64();
const void* batch_kernel_circadian_f64();
const void* kernel_circadian_f32();
const void* batch_kernel_circadian_f32();
const void* kernel_circadian_bf16();
const void* batch_kernel_circadian_bf16();
const void* kernel_circadian_f16();
const void* batch_kernel_circadian_f16();
const void* kernel_circadian_fp8();
const void* batch_kernel_circadian_fp8();

inline const void* kernel_lookup(int kind, int store) {
  static const void* (*const table[4][5])() = {
      {kernel_lco_cfg_f64, kernel_lco_cfg_f32, kernel_lco_cfg_bf16, kernel_lco_cfg_f16, kernel_lco_cfg_fp8},
      {kernel_lco_paper_f64, kernel_lco_paper_f32, kernel_lco_paper_bf16, kernel_lco_paper_f16, kernel_lco_paper_fp8},
      {kernel_kuramoto_f64, kernel_kuramoto_f32, kernel_kuramoto_bf16, kernel_kuramoto_f16, kernel_kuramoto_fp8},
      {kernel_circadian_f64, kernel_circadian_f32, kernel_circadian_bf16, kernel_circadian_f16, kernel_circadian_fp8},
  };
  return table[kind][store]();
}

inline const void* batch_kernel_lookup(int kind, int store) {
  static const void* (*const table[4][5])() = {
      {batch_kernel_lco_cfg_f64, batch_kernel_lco_cfg_f32, batch_kernel_lco_cfg_bf16, batch_kernel_lco_cfg_f16, batch_kernel_lco_cfg_fp8},
      {batch_kernel_lco_paper_f64, batch_kernel_lco_paper_f32, batch_kernel_lco_paper_bf16, batch_kernel_lco_paper_f16, batch_kernel_lco_paper_fp8},
      {batch_kernel_kuramoto_f64, batch_kernel_kuramoto_f32, batch_kernel_kuramoto_bf16, batch_kernel_kuramoto_f16, batch_kernel_kuramoto_fp8},
      {batch_kernel_circadian_f64, batch_kernel_circadian_f32, batch_kernel_circadian_bf16, batch_kernel_circadian_f16, batch_kernel_circadian_fp8},
  };
  return table[kind][store]();
}

// Sets a kernel's dynamic shared-memory limit to the largest value the
// device allows.  The limit is an attribute of the kernel, shared by every
// caller in the process, so it only ever takes this one value: a smaller
// value set for one launch would make another launch of the same kernel
// with more shared memory fail.
inline cudaError_t allow_max_smem(const void* kern, int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}
}  // namespace bs3
