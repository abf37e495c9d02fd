// fm_kernels.h -- launchers shared between the translation units of libfm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
    int max_ctas = 0; // > 0: at most this many GEMM CTAs resident (leaves SMs to other streams)
};
int fm_limb_plan(int64_t M, int64_t N, int64_t K, uint32_t p, const fm_opts* opts,
                 FmLimbPlan* plan);
// fm_limb_plan with the output tile width chosen from the shape when opts
// leave it open (for callers that split and multiply with the same plan).
int fm_limb_plan_shaped(int64_t M, int64_t N, int64_t K, uint32_t p, const fm_opts* opts,
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
// One operand of a batched split: X (rows x cols as used: M x K for A, K x N
// for B) -> its limb planes at out.
struct FmSplitDesc {
    const uint32_t* src;
    int lt;
    int KB;
    int64_t row0, col0, rows, cols;
    uint8_t* out;
    size_t plane_bytes;
};
// Splits tile jobs[b].y of operand descs[jobs[b].x], b < n_jobs, in one launch;
// q supplies the limb parameters (w, planes, block_n) shared by all operands.
int fm_limb_split_batch_run(const FmLimbPlan& q, int role, const FmSplitDesc* d_descs,
                            const int2* d_jobs, int64_t n_jobs, uint32_t p, cudaStream_t s);
int fm_limb_gemm_run(const FmLimbPlan& plan, fm_sub C, const void* a_planes,
                     const void* b_planes, uint32_t p, int op, int* status, cudaStream_t s);

// Batched limb form (limb_gemm.cu): every call's limb planes in one workspace;
// a run is two split launches and one persistent GEMM launch over the output
// tiles of every call. Calls with K = 0 are set aside (zero_calls): the caller
// runs them (only FM_OP_SET changes C).
struct FmLimbBatch;
int fm_limb_batch_create(const fm_gemm_call* calls, int64_t n, uint32_t p, const fm_opts* opts,
                         FmLimbBatch** out);
int fm_limb_batch_run(FmLimbBatch* b, int* status, cudaStream_t s);
int64_t fm_limb_batch_tiles(const FmLimbBatch* b);
int fm_limb_batch_launches(const FmLimbBatch* b);  // per run, excluding zero_calls
const std::vector<fm_gemm_call>& fm_limb_batch_zero_calls(const FmLimbBatch* b);
void fm_limb_batch_destroy(FmLimbBatch* b);
// Fused limb batches (limb_fused.cu): the two-limb Karatsuba fold form (plan q:
// w = 2, three products, block_n 128) in ONE launch that splits the operands
// on the fly; FM_EUNSUPPORTED when q or an operand does not allow it (T' < 8,
// a base not 16-byte aligned). Calls with K = 0 are skipped (the caller's).
struct FmFusedBatch;
int fm_fused_batch_create(const fm_gemm_call* calls, int64_t n, uint32_t p, const FmLimbPlan& q,
                          FmFusedBatch** out);
int fm_fused_batch_run(FmFusedBatch* b, int* status, cudaStream_t s);
int64_t fm_fused_batch_tiles(const FmFusedBatch* b);
void fm_fused_batch_destroy(FmFusedBatch* b);
// GF(2) batches (gf2.cu splits; limb_gemm.cu plans and multiplies): the same
// three launches on bit-packed operands (FmSplitDesc.lt carries log2_grid).
int fm_gf2_batch_create(const fm_gf2_call* calls, int64_t n, const fm_opts* opts, FmLimbBatch** out);
int fm_gf2_split_batch_run(int role, const FmSplitDesc* d_descs, const int2* d_jobs, int64_t n_jobs,
                           cudaStream_t s);
int fm_gf2_zero_sub(const fm_gf2_sub& C, cudaStream_t s);
int fm_gf2_check_call(const fm_gf2_call& g);  // argument checks of fm_gf2_gemm

// One-time per-device queries of the limb kernels (how many CTA pairs fit at
// once), made ahead of the first launch that needs them (limb_gemm.cu).
int fm_limb_prepare_device();

// The fixed scratch of fm_gemm_modp_noalloc (noalloc.cu): the device address of
// its status word on the current device (set up on first use), and a reader
// that copies that word to *out and clears it (FM_OK in *out when no call has
// used the array on this device).
int* fm_noalloc_status_word();
int fm_noalloc_take_status(cudaStream_t s, int* out);

// Remembered autotune choice for a problem class, and for a batch class (autotune.cu).
bool fm_tuned_choice(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out);
bool fm_tuned_batch_choice(const fm_gemm_call* calls, int64_t n, uint32_t p, fm_tune_result* out);
