// Kernel lookup across translation units (one unit per kind compiles in parallel).
#pragma once

namespace bs3 {
const void* kernel_lco_cfg(int store);
const void* kernel_lco_paper(int store);
const void* kernel_kuramoto(int store);
const void* kernel_circadian(int store);
}  // namespace bs3
