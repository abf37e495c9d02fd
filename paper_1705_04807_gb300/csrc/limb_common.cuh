// limb_common.cuh -- tile geometry shared by the limb split and the limb GEMM.
#pragma once

#include <stdint.h>

namespace fm_limb {
constexpr int kBM = 128;                     // output rows per CTA (TMEM lanes)
constexpr int kBK = 64;                      // K per stage: one 128-byte swizzle row of f16
constexpr uint32_t kATileBytes = kBM * 128;  // 16 KB

// Karatsuba planes: with w limbs, plane t < w holds digit t and plane w + u
// holds the digit sum d_i + d_j of pair u, pairs ordered (0,1), (0,2), (1,2),
// (0,3), (1,3), (2,3) (so the pairs of w limbs are the first w (w - 1) / 2).
constexpr int kMaxPlanes = 10;

__host__ __device__ __forceinline__ void karatsuba_pair(int u, int& i, int& j)
{
    j = u < 1 ? 1 : (u < 3 ? 2 : 3);
    i = u - j * (j - 1) / 2;
}
}  // namespace fm_limb
