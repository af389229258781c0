"""Writes one translation unit per (kind, stored type) solver kernel so that
nvcc can compile them in parallel.  Run: python gen_inst.py"""

import os

HERE = os.path.dirname(os.path.abspath(__file__))
KINDS = [("lco_cfg", "K_LCO_CFG"), ("lco_paper", "K_LCO_PAPER"), ("kuramoto", "K_KURAMOTO"),
         ("circadian", "K_CIRCADIAN")]
STORES = [("f64", "ST_F64"), ("f32", "ST_F32"), ("bf16", "ST_BF16"), ("f16", "ST_F16"), ("fp8", "ST_FP8")]

for kname, kenum in KINDS:
    for sname, senum in STORES:
        with open(os.path.join(HERE, f"inst_{kname}_{sname}.cu"), "w") as fh:
            fh.write(f"// Generated by gen_inst.py: solver kernels for {kname} with {sname} weights.\n"
                     f'#include "bs3_solver.cuh"\n\n'
                     f"namespace bs3 {{\n"
                     f"const void* kernel_{kname}_{sname}() {{ return (const void*)bs3_kernel<{kenum}, {senum}>; }}\n"
                     f"const void* batch_kernel_{kname}_{sname}() {{\n"
                     f"  return (const void*)bs3_batch_kernel<{kenum}, {senum}>;\n}}\n"
                     f"}}  // namespace bs3\n")

with open(os.path.join(HERE, "bs3_kernels.h"), "w") as fh:
    fh.write("// Generated by gen_inst.py: kernel lookup across translation units.\n#pragma once\n\n"
             "#include <cuda_runtime.h>\n\n"
             "namespace bs3 {\n")
    for kname, _ in KINDS:
        for sname, _ in STORES:
            fh.write(f"const void* kernel_{kname}_{sname}();\n")
            fh.write(f"const void* batch_kernel_{kname}_{sname}();\n")
    fh.write("\ninline const void* kernel_lookup(int kind, int store) {\n"
             "  static const void* (*const table[4][5])() = {\n")
    for kname, _ in KINDS:
        fh.write("      {" + ", ".join(f"kernel_{kname}_{s}" for s, _ in STORES) + "},\n")
    fh.write("  };\n  return table[kind][store]();\n}\n\n")
    fh.write("inline const void* batch_kernel_lookup(int kind, int store) {\n"
             "  static const void* (*const table[4][5])() = {\n")
    for kname, _ in KINDS:
        fh.write("      {" + ", ".join(f"batch_kernel_{kname}_{s}" for s, _ in STORES) + "},\n")
    fh.write("  };\n  return table[kind][store]();\n}\n\n")
    fh.write("// Sets a kernel's dynamic shared-memory limit to the largest value the\n"
             "// device allows.  The limit is an attribute of the kernel, shared by every\n"
             "// caller in the process, so it only ever takes this one value: a smaller\n"
             "// value set for one launch would make another launch of the same kernel\n"
             "// with more shared memory fail.\n"
             "inline cudaError_t allow_max_smem(const void* kern, int device) {\n"
             "  int optin = 0;\n"
             "  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);\n"
             "  if (e != cudaSuccess) return e;\n"
             "  cudaFuncAttributes fa;\n"
             "  e = cudaFuncGetAttributes(&fa, kern);\n"
             "  if (e != cudaSuccess) return e;\n"
             "  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,\n"
             "                              optin - (int)fa.sharedSizeBytes);\n"
             "}\n"
             "}  // namespace bs3\n")
