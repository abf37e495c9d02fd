// fm_kernels.h -- launchers shared between the translation units of libfm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fm_sched.h"

enum { kArithNarrow = 0, kArithWide = 1, kArithDfma = 2 };

// Plain / DFMA base-case kernel over a work list (gemm_plain.cu). With a
// non-null queue (zeroed beforehand) the grid is persistent and CTAs pull
// items from it; otherwise CTA b processes item b.
int fm_plain_launch(int lt, int arith, const FmCallDesc* calls, const FmWorkItem* items,
                    const FmLPiece* lps, int64_t n_items, uint32_t p, int* queue, int grid,
                    int* status, cudaStream_t s);
int fm_plain_occupancy(int lt, int arith);

// Limb tensor-core form (limb_split.cu, limb_gemm.cu): split A and B into balanced 8-bit limb
// planes in the tensor-core tile layout, then the tcgen05 GEMM with the
// recombine / reduce / combine epilogue. workspace must hold
// fm_limb_workspace_bytes(...).
struct FmLimbPlan {
    int64_t M, N, K;
    int w;            // limbs per residue
    int n_planes;     // planes per operand: w, or 3 with Karatsuba (d0, d1, d0 + d1; w = 2)
    int n_products;   // limb products the GEMM runs
    int prod_a[16], prod_b[16];  // plane of A and of B multiplied by product k
    int prod_cs[16];             // 64-wide K stages per exact chunk of product k
    uint32_t prod_w[16];         // weight of product k, mod p
    int block_n;      // 128 or 256
    int fold;         // 1: residue folded into the fp32 accumulator (p < 2^16)
    int pair = 0;     // 1: CTA pairs (cta_group::2) on 256 x 256 tiles (fold form, BN 256)
    int gf2 = 0;      // 1: GF(2), one E4M3 plane per operand, 128 elements per K stage
    int MB, NB, KB;
    size_t a_plane_bytes, b_plane_bytes;  // bytes of ONE plane
};
int fm_limb_plan(int64_t M, int64_t N, int64_t K, uint32_t p, const fm_opts* opts,
                 FmLimbPlan* plan);
// GF(2) product on bit-packed operands: one E4M3 0/1 plane per operand (tiles of
// 128 rows x 128 k bytes), one product, parity folded over p = 2 (gf2.cu splits,
// limb_gemm.cu multiplies).
int fm_gf2_plan(int64_t M, int64_t N, int64_t K, bool pair, FmLimbPlan* plan);
size_t fm_limb_workspace_bytes(const FmLimbPlan& plan);
int fm_limb_run(const FmLimbPlan& plan, fm_sub C, fm_sub A, fm_sub B, uint32_t p, int op,
                void* workspace, int* status, cudaStream_t s);
int fm_limb_split_run(const FmLimbPlan& plan, fm_sub X, int role, uint32_t p, void* planes,
                      cudaStream_t s);
int fm_limb_gemm_run(const FmLimbPlan& plan, fm_sub C, const void* a_planes,
                     const void* b_planes, uint32_t p, int op, int* status, cudaStream_t s);

// Remembered autotune choice for a problem class (autotune.cu).
bool fm_tuned_choice(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out);
