// limb_common.cuh -- tile geometry shared by the limb split and the limb GEMM.
#pragma once

#include <stdint.h>

namespace fm_limb {
constexpr int kBM = 128;                     // output rows per CTA (TMEM lanes)
constexpr int kBK = 64;                      // K per stage: one 128-byte swizzle row of f16
constexpr uint32_t kATileBytes = kBM * 128;  // 16 KB
}  // namespace fm_limb
