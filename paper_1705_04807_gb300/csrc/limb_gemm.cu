// limb_gemm.cu -- the tensor-core form of C <- C op A*B mod p.
//
// With residues split into balanced signed 8-bit limbs (limb_split.cu),
//     A*B == sum_k weight_k * (A_{a(k)} * B_{b(k)})      (mod p)
// over the limb products k: (i, j) with weight 256^(i+j) mod p, or, for two
// limbs, the three Karatsuba products A0B0, (A0+A1)(B0+B1), A1B1 with weights
// (1-256), 256, (2^16-256) mod p. Every limb product is an integer GEMM whose
// entries are at most 2^14 (255^2 for the Karatsuba middle product) in
// magnitude. sm_103a's tcgen05 has no integer MMA kind, so the limbs are carried
// exactly as FP16 values through tcgen05.mma kind::f16 with FP32 accumulation in
// tensor memory. FP32 holds every integer of magnitude <= 2^24 exactly, so K is
// cut into chunks small enough that no partial sum can leave that range, and
// each chunk's accumulator is drained into exact integers.
//
// Persistent kernel, one CTA per SM walking 128 x BN output tiles: a producer
// warp (one 1-D bulk copy per operand per 64-wide K stage, only the rows and
// columns the tile uses), an MMA warp (tcgen05.mma into TMEM, two accumulators
// alternating between jobs = (limb product, K chunk), N = the tile's columns
// rounded to 16) and eight epilogue warps that drain each chunk with
// tcgen05.ld / st. Fold form (p < 2^16): the running residue is folded back into
// the FP32 accumulator, with an exact FP32 reduction between chunks of one
// product and a weight change at product boundaries, in packed FP32. Residue
// form (any p < 2^31): an exact int32 sum per product, folded into a residue
// region of TMEM once per product. The final residue is combined with C (set /
// add / subtract) in the Morton-hybrid layout; C's lines are prefetched into L2
// when the tile starts. The same kernel runs one call (fields in the kernel
// arguments) or a batch (a call table and a tile list), on f16 limb planes or on
// E4M3 0/1 planes for GF(2) (kind::f8f6f4, parity bits written to a bit-packed
// C). A CTA-pair variant (cta_group::2) computes 256 x 256 tiles.
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "fm_internal.cuh"
#include "fm_kernels.h"
#include "limb_common.cuh"
#include "limb_drain.cuh"

namespace {

using namespace fm_limb;
constexpr int kEpiWarps = 8;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // producer, MMA, epilogue warps

// Residue-form fold of one product's sum into the running residue:
// r + w * s mod p for an int32 sum s, a weight w < p and r in [0, p), p < 2^31,
// all in 32-bit integer arithmetic. w * |s| mod p by Shoup's method: with
// ws = floor(w 2^32 / p), q = floor(|s| ws / 2^32) falls short of w |s| / p by
// less than 2, so w |s| - q p (exact mod 2^32) lies in [0, 2p) and one
// conditional subtraction leaves y in [0, p). A negative s gives p - y, in
// [1, p]; r plus that is below 2p and is reduced once more.
__device__ __forceinline__ uint32_t umin_sub(uint32_t x, uint32_t p)
{
    return min(x, x - p);  // x - p when x >= p (otherwise x - p wraps above x)
}

__device__ __forceinline__ uint32_t fold_sum(int32_t s, uint32_t w, uint32_t ws, uint32_t r, uint32_t p)
{
    const uint32_t a = (uint32_t)abs(s);  // |s| < 2^31
    const uint32_t q = __umulhi(a, ws);
    const uint32_t y = umin_sub(a * w - q * p, p);
    return umin_sub(r + (s < 0 ? p - y : y), p);
}

// Per-call part of a limb GEMM: its limb planes, K stages and jobs, and its C
// sub-matrix.
struct LimbCall {
    const uint8_t* Ap;
    const uint8_t* Bp;
    uint64_t a_plane_bytes, b_plane_bytes;
    int MB, NB, KB, njobs;
    int first[17];  // first job of product k; first[n_products] = njobs
    uint32_t* C;
    int c_lt, op;
    int64_t c_row0, c_col0, M, N;
};

struct LimbGemmArgs {
    LimbCall call;          // one call (the batched kernel reads calls[] instead)
    const LimbCall* calls;  // batched: call table
    const int4* tiles;      // batched: (call, mb, nb) per output tile, longest first
    int n_tiles;            // batched: number of output tiles
    int n_products;
    int pa[16], pb[16];  // planes of A and B of product k
    int cs[16];          // 64-wide K stages per chunk of product k
    uint32_t p, mu32;
    uint32_t wt[16];  // weight of product k mod p
    uint32_t wts[16]; // residue form: floor(wt[k] * 2^32 / p), Shoup's constant for wt[k]
    uint32_t cn[16];  // fold form: cn[k * 4 + k2] = wt[k] * wt[k2]^-1 mod p
    float invp, pf;   // fold form: 1/p and p as float
    int* status;
};

// GF(2) output: the residues (0 or 1) of columns j0 .. j0+31 of row gi become
// one word of bits, combined into the bit-packed Morton-hybrid C (T' = 32: word
// Z(I, J) * 32 + u holds tile row u). SET replaces the bits, ADD and SUB flip
// them (+1 = -1 in GF(2)). A run not starting on a word boundary spans two
// words shared with the neighbouring runs, updated with atomics; a whole word
// belongs to this thread alone.
__device__ __forceinline__ void gf2_apply(uint32_t* w, uint32_t m, uint32_t x, int op)
{
    if (m == 0u) return;
    if (m == ~0u) {
        if (op == FM_OP_SET)
            *w = x;
        else
            *w ^= x;
        return;
    }
    if (op == FM_OP_SET) {
        atomicAnd(w, ~m);
        atomicOr(w, x & m);
    } else {
        atomicXor(w, x & m);
    }
}

__device__ __forceinline__ void write_gf2_run(const CView& c, int64_t gi, int64_t j0,
                                              const uint32_t (&r)[32])
{
    const int64_t nvalid = c.N - j0;
    if (nvalid <= 0) return;
    uint32_t bits = 0;
#pragma unroll
    for (int e = 0; e < 32; ++e) bits |= (r[e] & 1u) << e;
    const uint32_t vmask = nvalid >= 32 ? ~0u : ((1u << nvalid) - 1u);
    bits &= vmask;
    const uint64_t ci = (uint64_t)(c.c_row0 + gi);
    const uint64_t cj = (uint64_t)(c.c_col0 + j0);
    const uint32_t b = (uint32_t)(cj & 31);
    gf2_apply(c.C + (fm_encode(ci, cj, 5) >> 5), vmask << b, bits << b, c.op);
    if (b != 0) {
        const uint32_t m1 = vmask >> (32 - b);
        if (m1) gf2_apply(c.C + (fm_encode(ci, cj + (32 - b), 5) >> 5), m1, bits >> (32 - b), c.op);
    }
}

// TWO: two CTAs per SM (fold form, 128-wide tiles): each holds only its two
// 128-column accumulators (256 TMEM columns) and three 32 KB stages, so that
// two fit on one SM; for short K, where every tile is mostly epilogue, one
// CTA's drains and C update then overlap the other's MMAs, and the SM has
// twice the epilogue warps to hide their latency.
template <int BN, bool TWO = false>
struct GemmCfg {
    static constexpr int kStages = TWO ? 3 : (BN == 256 ? 4 : 6);
    static constexpr uint32_t kBTileBytes = BN * 128;
    static constexpr uint32_t kStageBytes = kATileBytes + kBTileBytes;
    static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024;  // + alignment slack
    static constexpr uint32_t kTmemCols = TWO ? 2 * BN : 512;
};

// Persistent: one CTA per SM walks the output tiles blockIdx.x, + gridDim.x, ...
// The producer and MMA warps run ahead into the next tile while the epilogue
// finishes the previous one; barrier phases and the two TMEM accumulators carry
// on across tiles (job counter T).
// KIND: kF16Res = f16 limb planes, residues written to a uint32 Morton-hybrid C;
// kE4M3Gf2 = E4M3 0/1 planes (GF(2)), parity bits written to a bit-packed C.
enum { kF16Res = 0, kE4M3Gf2 = 1 };

template <int BN, bool FOLD, int KIND, bool BATCH, bool TWO = false>
__global__ void __launch_bounds__(kGemmThreads, TWO ? 2 : 1)
    limb_gemm_kernel(const __grid_constant__ LimbGemmArgs args)
{
    static_assert(!TWO || (FOLD && BN == 128 && KIND == kF16Res), "two CTAs per SM: fold form, 128-wide tiles");
    using Cfg = GemmCfg<BN, TWO>;
    constexpr int S = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    __shared__ __align__(8) uint64_t full_bar[S];
    __shared__ __align__(8) uint64_t empty_bar[S];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    __shared__ uint32_t s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // row blocks holding rows of C (the A planes may carry one more, zero)
    const int mb_rows = (int)((args.call.M + kBM - 1) / kBM);
    const int n_tiles = BATCH ? args.n_tiles : mb_rows * args.call.NB;

    // tile -> its call and (mb, nb). One call: grouped raster for L2 reuse (a
    // wave of 152 tiles covers GROUP row blocks; 16 for 256-wide tiles, whose B
    // panels are twice as wide, makes the wave's panel bytes near minimal);
    // batched: the plan's tile list.
    auto tile_call = [&](int tile, int& mb, int& nb) -> const LimbCall& {
        if (BATCH) {
            const int4 e = args.tiles[tile];
            mb = e.y;
            nb = e.z;
            return args.calls[e.x];
        }
        const int GROUP = BN == 256 ? 16 : 8;
        const int per_group = GROUP * args.call.NB;
        const int first_mb = (tile / per_group) * GROUP;
        const int gsz = min(mb_rows - first_mb, GROUP);
        const int inner = tile % per_group;
        mb = first_mb + inner % gsz;
        nb = inner / gsz;
        return args.call;
    };
    // rows and columns of the tile inside C; the MMA runs on the valid columns
    // rounded up to 16 (its N granularity) and loads only the rows it needs
    auto tile_rows = [&](const LimbCall& cl, int mb) {
        return (int)min((int64_t)kBM, cl.M - (int64_t)mb * kBM);
    };
    auto tile_cols = [&](const LimbCall& cl, int nb) {
        return (int)min((int64_t)BN, cl.N - (int64_t)nb * BN);
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            fm_mbar_init(&full_bar[s], 1);
            fm_mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            fm_mbar_init(&accf_bar[b], 1);
            fm_mbar_init(&acce_bar[b], kEpiWarps);
        }
        fm_mbar_init(&done_bar, 1);
        fm_fence_mbar_init();
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 1) {
        fm_tmem_alloc(&tmem_slot, Cfg::kTmemCols);
        fm_tmem_relinquish();
    }
    fm_tc_fence_before();
    __syncthreads();
    fm_tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: one bulk copy per operand per stage ----
            uint32_t g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                int mb, nb;
                const LimbCall& cl = tile_call(tile, mb, nb);
                const int njobs = cl.njobs;
                const uint32_t a_bytes = (uint32_t)tile_rows(cl, mb) * 128u;
                const uint32_t b_bytes = (uint32_t)((tile_cols(cl, nb) + 15) & ~15) * 128u;
                int idx = 0;
                for (int t = 0; t < njobs && ok; ++t) {
                    while (t >= cl.first[idx + 1]) ++idx;
                    const int c = t - cl.first[idx];
                    const int kb0 = c * args.cs[idx], kb1 = min(cl.KB, kb0 + args.cs[idx]);
                    const uint8_t* a_src = cl.Ap + (size_t)args.pa[idx] * cl.a_plane_bytes +
                                           ((size_t)mb * cl.KB) * kATileBytes;
                    const uint8_t* b_src = cl.Bp + (size_t)args.pb[idx] * cl.b_plane_bytes +
                                           ((size_t)nb * cl.KB) * Cfg::kBTileBytes;
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int s = g % S;
                        const uint32_t ph = (g / S) & 1;
                        if (!fm_mbar_wait(&empty_bar[s], ph ^ 1, args.status, &s_abort)) {
                            ok = false;
                            break;
                        }
                        uint8_t* sa = smem + (size_t)s * Cfg::kStageBytes;
                        fm_mbar_arrive_expect_tx(&full_bar[s], a_bytes + b_bytes);
                        fm_bulk_g2s(sa, a_src + (size_t)kb * kATileBytes, a_bytes, &full_bar[s]);
                        fm_bulk_g2s(sa + kATileBytes, b_src + (size_t)kb * Cfg::kBTileBytes, b_bytes,
                                    &full_bar[s]);
                    }
                }
            }
            s_issued = g;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            uint32_t g = 0, T = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                int mb, nb;
                const LimbCall& cl = tile_call(tile, mb, nb);
                const int njobs = cl.njobs;
                const uint32_t idesc = fm_idesc_f16_f32(kBM, (tile_cols(cl, nb) + 15) & ~15);
                int idx = 0;
                for (int t = 0; t < njobs && ok; ++t, ++T) {
                    const int b = T & 1;
                    while (t >= cl.first[idx + 1]) ++idx;
                    const int c = t - cl.first[idx];
                    const int kb0 = c * args.cs[idx], kb1 = min(cl.KB, kb0 + args.cs[idx]);
                    if (T >= 2 &&
                        !fm_mbar_wait(&acce_bar[b], ((T >> 1) - 1) & 1, args.status, &s_abort)) {
                        ok = false;
                        break;
                    }
                    fm_tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)(b * BN);
                    bool first = true;
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int s = g % S;
                        const uint32_t ph = (g / S) & 1;
                        if (!fm_mbar_wait(&full_bar[s], ph, args.status, &s_abort)) {
                            ok = false;
                            break;
                        }
                        fm_tc_fence_after();
                        const uint32_t a_addr = fm_smem_u32(smem + (size_t)s * Cfg::kStageBytes);
                        const uint32_t b_addr = a_addr + kATileBytes;
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k) {
                            const uint64_t ad = fm_smem_desc_sw128(a_addr + k * 32);
                            const uint64_t bd = fm_smem_desc_sw128(b_addr + k * 32);
                            // fold form: from the third job of a tile on, each job
                            // accumulates onto the residue folded back by the epilogue
                            const uint32_t acc = ((FOLD && t >= 2) || !first || k > 0) ? 1u : 0u;
                            if (KIND == kE4M3Gf2)
                                fm_mma_e4m3(d_tmem, ad, bd, idesc, acc);
                            else
                                fm_mma_f16(d_tmem, ad, bd, idesc, acc);
                        }
                        fm_mma_commit(&empty_bar[s]);  // stage free once these MMAs have read it
                        first = false;
                    }
                    if (!ok) break;
                    fm_mma_commit(&accf_bar[b]);  // accumulator b complete for job T
                }
            }
            s_consumed = g;
            // every MMA issued by this thread has completed before TMEM is freed
            fm_mma_commit(&done_bar);
            fm_mbar_wait(&done_bar, 0, args.status, nullptr);
        }
    } else {
        // ---- epilogue: kEpiWarps warps. Warp w may only touch TMEM lanes
        // 32*(w%4) .. +31, so two warps share each lane quarter and split the BN
        // columns in halves; two warps per SM sub-partition hide each other's
        // TMEM load latency. ----
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;
        constexpr int kCols = BN / 2;  // columns handled by this warp
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const uint32_t col0 = (uint32_t)(half * kCols);
        const uint32_t p = args.p;
        
        uint32_t T = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            int mb, nb;
            const LimbCall& cl = tile_call(tile, mb, nb);
            const CView cv = c_view(cl);
            const int njobs = cl.njobs;
            // 32-column chunks of this warp inside C (none when its lane
            // quarter lies below the last row): the rest is never written
            const int live_cols = quarter * 32 < tile_rows(cl, mb) ? tile_cols(cl, nb) - (int)col0 : 0;
            const int n32 = max(0, min(kCols / 32, (live_cols + 31) / 32));
            // C of this tile is read at its end: start moving it into L2 now
            if (KIND != kE4M3Gf2 && cv.op != FM_OP_SET && live_cols > 0 &&
                (int64_t)mb * kBM + quarter * 32 + lane < cv.M)
                prefetch_c_row(cv, (int64_t)mb * kBM + quarter * 32 + lane, (int64_t)nb * BN + col0,
                               min(live_cols, kCols));
            int idx = 0;
            for (int t = 0; t < njobs; ++t, ++T) {
                const int b = T & 1;
                if (!fm_mbar_wait(&accf_bar[b], (T >> 1) & 1, args.status, &s_abort)) {
                    ok = false;
                    break;
                }
                fm_tc_fence_after();
                while (t >= cl.first[idx + 1]) ++idx;
                const int c = t - cl.first[idx];
                const int n_chunks = cl.first[idx + 1] - cl.first[idx];
                const bool last_on_buffer = (t + 2 >= njobs);
                // fold form: the job two steps later on this buffer continues the
                // same limb product (same weight) unless a product boundary lies between
                int idx2 = idx;
                if (!last_on_buffer)
                    while (t + 2 >= cl.first[idx2 + 1]) ++idx2;
                const bool same_next = !last_on_buffer && idx2 == idx;
                const uint32_t dbase = tmem + lane_base + (uint32_t)(b * BN) + col0;
                if constexpr (FOLD && TWO) {
                    // two CTAs per SM: one 32-column chunk at a time (register budget)
                    const uint32_t mul = last_on_buffer ? args.wt[idx] : args.cn[idx * 4 + idx2];
#pragma unroll 1
                    for (int g = 0; g < n32; ++g) {
                        uint32_t v0[32];
                        fm_tmem_ld32(dbase + g * 32, v0);
                        fm_tmem_wait_ld();
                        if (same_next)
                            fold_fp(v0, args.invp, args.pf);
                        else
                            fold_int(v0, mul, !last_on_buffer, p, args.invp, args.pf);
                        fm_tmem_st32(dbase + g * 32, v0);
                    }
                } else if constexpr (FOLD) {
                    const uint32_t mul = last_on_buffer ? args.wt[idx] : args.cn[idx * 4 + idx2];
#pragma unroll 1
                    for (int g = 0; g < (n32 + 1) / 2; ++g) {  // two 32-column chunks in flight
                        uint32_t v0[32], v1[32];
                        fm_tmem_ld32(dbase + g * 64, v0);
                        fm_tmem_ld32(dbase + g * 64 + 32, v1);
                        fm_tmem_wait_ld();
                        if (same_next) {
                            fold_fp(v0, args.invp, args.pf);
                            fold_fp(v1, args.invp, args.pf);
                        } else {
                            fold_int(v0, mul, !last_on_buffer, p, args.invp, args.pf);
                            fold_int(v1, mul, !last_on_buffer, p, args.invp, args.pf);
                        }
                        fm_tmem_st32(dbase + g * 64, v0);
                        fm_tmem_st32(dbase + g * 64 + 32, v1);
                    }
                } else {
                    // residue form: S (exact int32 sum of this product's chunks) is
                    // folded into R at the product's last chunk and every 120 chunks
                    const bool s_fresh = (c % 120) == 0;
                    const bool fold_now = (c == n_chunks - 1) || ((c % 120) == 119);
                    const bool r_fresh = (idx == 0 && c < 120);
                    const uint32_t sbase = tmem + lane_base + (uint32_t)(3 * BN) + col0;
                    const uint32_t rbase = tmem + lane_base + (uint32_t)(2 * BN) + col0;
#pragma unroll 1
                    for (int cc = 0; cc < n32; ++cc) {
                        uint32_t v[32], sv[32];
                        fm_tmem_ld32(dbase + cc * 32, v);
                        if (!s_fresh) fm_tmem_ld32(sbase + cc * 32, sv);
                        fm_tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int32_t d = __float2int_rn(__uint_as_float(v[e]));
                            sv[e] = (uint32_t)((s_fresh ? 0 : (int32_t)sv[e]) + d);
                        }
                        if (fold_now) {
                            if (!r_fresh) {
                                fm_tmem_ld32(rbase + cc * 32, v);
                                fm_tmem_wait_ld();
                            }
                            const uint32_t wt = args.wt[idx], wts = args.wts[idx];
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                v[e] = fold_sum((int32_t)sv[e], wt, wts, r_fresh ? 0u : v[e], p);
                            fm_tmem_st32(rbase + cc * 32, v);
                        } else {
                            fm_tmem_st32(sbase + cc * 32, sv);
                        }
                    }
                }
                fm_tmem_wait_st();
                fm_tc_fence_before();
                __syncwarp();
                // fold form: a buffer holding one of the tile's two final residues is
                // released only after the tile end below has read it
                if (!(FOLD && last_on_buffer) && lane == 0) fm_mbar_arrive(&acce_bar[b]);
            }
            if (!ok) break;

            // ---- tile end: final residue -> combine with C -> Morton-hybrid write
            const int64_t gi = (int64_t)mb * kBM + quarter * 32 + lane;
            uint32_t rsrc;  // TMEM column base of the final residue
            if (FOLD) {
                const int by = (T - 1) & 1;  // buffer of the tile's last job
                const int bx = by ^ 1;       // buffer of its second-to-last job
                rsrc = (uint32_t)(by * BN);
                if (njobs >= 2) {
                    // y <- x + y mod p, then x is free for the next tile's first job
                    const uint32_t xb = tmem + lane_base + (uint32_t)(bx * BN) + col0;
                    const uint32_t yb = tmem + lane_base + (uint32_t)(by * BN) + col0;
                    if constexpr (TWO) {
#pragma unroll 1
                        for (int cc = 0; cc < 2 * n32; ++cc) {
                            uint32_t xv[16], yv[16];
                            fm_tmem_ld16(xb + cc * 16, xv);
                            fm_tmem_ld16(yb + cc * 16, yv);
                            fm_tmem_wait_ld();
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const uint32_t x = xv[e] + yv[e];
                                yv[e] = x >= p ? x - p : x;
                            }
                            fm_tmem_st16(yb + cc * 16, yv);
                        }
                    } else {
#pragma unroll 1
                        for (int cc = 0; cc < n32; ++cc) {
                            uint32_t xv[32], yv[32];
                            fm_tmem_ld32(xb + cc * 32, xv);
                            fm_tmem_ld32(yb + cc * 32, yv);
                            fm_tmem_wait_ld();
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const uint32_t x = xv[e] + yv[e];
                                yv[e] = x >= p ? x - p : x;
                            }
                            fm_tmem_st32(yb + cc * 32, yv);
                        }
                    }
                    fm_tmem_wait_st();
                    fm_tc_fence_before();
                    __syncwarp();
                    if (lane == 0) fm_mbar_arrive(&acce_bar[bx]);
                }
            } else {
                rsrc = (uint32_t)(2 * BN);
            }
            if constexpr (TWO) {
#pragma unroll 1
                for (int cc = 0; cc < 2 * n32; ++cc) {
                    uint32_t sres[16];
                    const uint32_t col = col0 + cc * 16;
                    fm_tmem_ld16(tmem + lane_base + rsrc + col, sres);
                    fm_tmem_wait_ld();
                    if (gi < cv.M)
                        write_c_run<16>(cv, p, args.mu32, gi, (int64_t)nb * BN + col, (1ull << cv.c_lt) - 1,
                                        sres);
                }
            } else {
#pragma unroll 1
                for (int cc = 0; cc < n32; ++cc) {
                    uint32_t sres[32];
                    const uint32_t col = col0 + cc * 32;
                    fm_tmem_ld32(tmem + lane_base + rsrc + col, sres);
                    fm_tmem_wait_ld();
                    if (gi < cv.M) {
                        if (KIND == kE4M3Gf2)
                            write_gf2_run(cv, gi, (int64_t)nb * BN + col, sres);
                        else
                            write_c_run<32>(cv, p, args.mu32, gi, (int64_t)nb * BN + col, (1ull << cv.c_lt) - 1,
                                            sres);
                    }
                }
            }
            if (FOLD) {
                fm_tc_fence_before();
                __syncwarp();
                if (lane == 0) fm_mbar_arrive(&acce_bar[(T - 1) & 1]);
            }
        }
    }

    fm_tc_fence_before();
    __syncthreads();
    if (s_abort && tid == 0) {
        // let bulk copies still in flight land before the CTA exits
        for (uint32_t g = s_consumed; g < s_issued; ++g)
            fm_mbar_wait(&full_bar[g % S], (g / S) & 1, args.status, nullptr);
    }
    if (warp == 1) {
        fm_tc_fence_after();
        fm_tmem_dealloc(tmem, Cfg::kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// CTA-pair form: a cluster of two CTAs computes a 256 x BN output tile with
// tcgen05.mma.cta_group::2 (fold form: BN = 256; residue form: BN = 128, whose
// TMEM per CTA then holds the two accumulators, R and S as in the single-CTA
// kernel). CTA r of the pair stages A rows [128 r, 128 r + 128) and B rows (n)
// [BN/2 r, BN/2 r + BN/2) of the tile -- per 64-wide K stage 32 KB instead of
// 48 KB (BN = 256) or 24 KB instead of 32 KB (BN = 128), which is also the
// shared memory each MMA reads -- and holds D rows [128 r, 128 r + 128) in its
// tensor memory. The even CTA issues the MMAs; its commits are multicast to both
// CTAs. Each CTA's bulk copies complete on its own full barrier; a forwarder
// thread of the odd CTA then arrives on the even CTA's full barrier, and the odd
// CTA's epilogue warps arrive on the even CTA's accumulator-empty barriers.
template <int BN>
struct PairCfg {
    static constexpr uint32_t kBHalfBytes = (uint32_t)BN * 64;  // BN/2 rows of 128 bytes
    static constexpr uint32_t kStageBytes = kATileBytes + kBHalfBytes;
    static constexpr int kStages = BN == 256 ? 6 : 8;
    static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024;
};

template <int KIND, bool FOLD>
__global__ void __launch_bounds__(kGemmThreads, 1) limb_gemm_pair_kernel(const __grid_constant__ LimbGemmArgs args)
{
    constexpr int BN = FOLD ? 256 : 128;
    using Cfg = PairCfg<BN>;
    constexpr int S = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    __shared__ __align__(8) uint64_t full_bar[S];
    __shared__ __align__(8) uint64_t empty_bar[S];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    __shared__ uint32_t s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = fm_cluster_ctarank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const LimbCall& cl = args.call;
    const int MB2 = cl.MB >> 1;  // A planes are padded to an even number of row blocks
    const int n_tiles = MB2 * cl.NB;
    const int njobs = cl.njobs;

    // grouped raster: a wave of 76 pairs covers 8 pair rows x 9.5 pair
    // columns, near the fewest A and B panel bytes per wave
    auto coords = [&](int tile, int& mb2, int& nb) {
        const int GROUP = 8;
        const int per_group = GROUP * cl.NB;
        const int first = (tile / per_group) * GROUP;
        const int gsz = min(MB2 - first, GROUP);
        const int inner = tile % per_group;
        mb2 = first + inner % gsz;
        nb = inner / gsz;
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            fm_mbar_init(&full_bar[s], leader ? 2 : 1);
            fm_mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            fm_mbar_init(&accf_bar[b], 1);
            fm_mbar_init(&acce_bar[b], 2 * kEpiWarps);
        }
        fm_mbar_init(&done_bar, 1);
        fm_fence_mbar_init();
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 1) {
        fm_tmem_alloc_pair(&tmem_slot, 512);
        fm_tmem_relinquish_pair();
    }
    fm_tc_fence_before();
    __syncthreads();
    fm_cluster_sync();  // both CTAs' barriers exist before any cross-CTA arrive
    fm_tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer (both CTAs): this CTA's A half and B half per stage ----
            uint32_t g = 0;
            bool ok = true;
            for (int tile = pair; tile < n_tiles && ok; tile += npairs) {
                int mb2, nb;
                coords(tile, mb2, nb);
                int idx = 0;
                for (int t = 0; t < njobs && ok; ++t) {
                    while (t >= cl.first[idx + 1]) ++idx;
                    const int c = t - cl.first[idx];
                    const int kb0 = c * args.cs[idx], kb1 = min(cl.KB, kb0 + args.cs[idx]);
                    const uint8_t* a_src = cl.Ap + (size_t)args.pa[idx] * cl.a_plane_bytes +
                                           ((size_t)(2 * mb2 + rank) * cl.KB) * kATileBytes;
                    const uint8_t* b_src = cl.Bp + (size_t)args.pb[idx] * cl.b_plane_bytes +
                                           ((size_t)nb * cl.KB) * (2 * Cfg::kBHalfBytes) +
                                           (size_t)rank * Cfg::kBHalfBytes;
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int s = g % S;
                        const uint32_t ph = (g / S) & 1;
                        if (!fm_mbar_wait(&empty_bar[s], ph ^ 1, args.status, &s_abort)) {
                            ok = false;
                            break;
                        }
                        uint8_t* sa = smem + (size_t)s * Cfg::kStageBytes;
                        fm_mbar_arrive_expect_tx(&full_bar[s], Cfg::kStageBytes);
                        fm_bulk_g2s(sa, a_src + (size_t)kb * kATileBytes, kATileBytes, &full_bar[s]);
                        fm_bulk_g2s(sa + kATileBytes, b_src + (size_t)kb * (2 * Cfg::kBHalfBytes),
                                    Cfg::kBHalfBytes, &full_bar[s]);
                    }
                }
            }
            s_issued = g;
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---- MMA issuer (even CTA) ----
            const uint32_t idesc = fm_idesc_f16_f32(2 * kBM, BN);
            uint32_t g = 0, T = 0;
            bool ok = true;
            for (int tile = pair; tile < n_tiles && ok; tile += npairs) {
                int idx = 0;
                for (int t = 0; t < njobs && ok; ++t, ++T) {
                    const int b = T & 1;
                    while (t >= cl.first[idx + 1]) ++idx;
                    const int c = t - cl.first[idx];
                    const int kb0 = c * args.cs[idx], kb1 = min(cl.KB, kb0 + args.cs[idx]);
                    if (T >= 2 &&
                        !fm_mbar_wait(&acce_bar[b], ((T >> 1) - 1) & 1, args.status, &s_abort)) {
                        ok = false;
                        break;
                    }
                    fm_tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)(b * BN);
                    bool first = true;
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int s = g % S;
                        const uint32_t ph = (g / S) & 1;
                        if (!fm_mbar_wait(&full_bar[s], ph, args.status, &s_abort)) {
                            ok = false;
                            break;
                        }
                        fm_tc_fence_after();
                        const uint32_t a_addr = fm_smem_u32(smem + (size_t)s * Cfg::kStageBytes);
                        const uint32_t b_addr = a_addr + kATileBytes;
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k) {
                            const uint64_t ad = fm_smem_desc_sw128(a_addr + k * 32);
                            const uint64_t bd = fm_smem_desc_sw128(b_addr + k * 32);
                            // fold form: from the third job of a tile on, each job
                            // accumulates onto the residue folded back by the epilogue
                            const uint32_t acc = ((FOLD && t >= 2) || !first || k > 0) ? 1u : 0u;
                            if (KIND == kE4M3Gf2)
                                fm_mma_e4m3_pair(d_tmem, ad, bd, idesc, acc);
                            else
                                fm_mma_f16_pair(d_tmem, ad, bd, idesc, acc);
                        }
                        fm_mma_commit_pair(&empty_bar[s], 0x3);  // stage free in both CTAs
                        first = false;
                    }
                    if (!ok) break;
                    fm_mma_commit_pair(&accf_bar[b], 0x3);  // accumulator b complete in both CTAs
                }
            }
            s_consumed = g;
            fm_mma_commit_pair(&done_bar, 0x1);
            fm_mbar_wait(&done_bar, 0, args.status, nullptr);
        } else if (lane == 0) {
            // ---- forwarder (odd CTA): this CTA's stage landed -> even CTA's full barrier ----
            const uint32_t leader_full = fm_mapa(fm_smem_u32(&full_bar[0]), 0);
            uint32_t g = 0;
            bool ok = true;
            for (int tile = pair; tile < n_tiles && ok; tile += npairs) {
                int idx = 0;
                for (int t = 0; t < njobs && ok; ++t) {
                    while (t >= cl.first[idx + 1]) ++idx;
                    const int c = t - cl.first[idx];
                    const int kb0 = c * args.cs[idx], kb1 = min(cl.KB, kb0 + args.cs[idx]);
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int s = g % S;
                        if (!fm_mbar_wait(&full_bar[s], (g / S) & 1, args.status, &s_abort)) {
                            ok = false;
                            break;
                        }
                        fm_mbar_arrive_remote(leader_full + (uint32_t)(s * sizeof(uint64_t)));
                    }
                }
            }
            s_consumed = g;
        }
    } else {
        // ---- epilogue (both CTAs): as in the single-CTA kernel, for this CTA's 128 rows ----
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;
        constexpr int kCols = BN / 2;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const uint32_t col0 = (uint32_t)(half * kCols);
        const uint32_t p = args.p;
        const uint64_t cmask = (1ull << cl.c_lt) - 1;
        const uint32_t acce_leader = fm_mapa(fm_smem_u32(&acce_bar[0]), 0);
        uint32_t T = 0;
        bool ok = true;
        for (int tile = pair; tile < n_tiles && ok; tile += npairs) {
            int mb2, nb;
            coords(tile, mb2, nb);
            const int64_t gi = (int64_t)(2 * mb2 + rank) * kBM + quarter * 32 + lane;
            // C of this tile is read at its end: start moving it into L2 now
            const int64_t live_cols = min((int64_t)kCols, cl.N - (int64_t)nb * BN - (int64_t)col0);
            if (!FOLD && cl.op != FM_OP_SET && gi < cl.M && live_cols > 0)
                prefetch_c_row(cl, gi, (int64_t)nb * BN + col0, live_cols);
            int idx = 0;
            for (int t = 0; t < njobs; ++t, ++T) {
                const int b = T & 1;
                if (!fm_mbar_wait(&accf_bar[b], (T >> 1) & 1, args.status, &s_abort)) {
                    ok = false;
                    break;
                }
                fm_tc_fence_after();
                while (t >= cl.first[idx + 1]) ++idx;
                const bool last_on_buffer = (t + 2 >= njobs);
                const uint32_t dbase = tmem + lane_base + (uint32_t)(b * BN) + col0;
                if constexpr (FOLD) {
                    int idx2 = idx;
                    if (!last_on_buffer)
                        while (t + 2 >= cl.first[idx2 + 1]) ++idx2;
                    const bool same_next = !last_on_buffer && idx2 == idx;
                    const uint32_t mul = last_on_buffer ? args.wt[idx] : args.cn[idx * 4 + idx2];
#pragma unroll 1
                    for (int g = 0; g < kCols / 64; ++g) {
                        uint32_t v0[32], v1[32];
                        fm_tmem_ld32(dbase + g * 64, v0);
                        fm_tmem_ld32(dbase + g * 64 + 32, v1);
                        fm_tmem_wait_ld();
                        if (same_next) {
                            fold_fp(v0, args.invp, args.pf);
                            fold_fp(v1, args.invp, args.pf);
                        } else {
                            fold_int(v0, mul, !last_on_buffer, p, args.invp, args.pf);
                            fold_int(v1, mul, !last_on_buffer, p, args.invp, args.pf);
                        }
                        fm_tmem_st32(dbase + g * 64, v0);
                        fm_tmem_st32(dbase + g * 64 + 32, v1);
                    }
                } else {
                    // residue form: S (exact int32 sum of this product's chunks) is
                    // folded into R at the product's last chunk and every 120 chunks
                    const int c = t - cl.first[idx];
                    const int n_chunks = cl.first[idx + 1] - cl.first[idx];
                    const bool s_fresh = (c % 120) == 0;
                    const bool fold_now = (c == n_chunks - 1) || ((c % 120) == 119);
                    const bool r_fresh = (idx == 0 && c < 120);
                    const uint32_t sbase = tmem + lane_base + (uint32_t)(3 * BN) + col0;
                    const uint32_t rbase = tmem + lane_base + (uint32_t)(2 * BN) + col0;
#pragma unroll 1
                    for (int cc = 0; cc < kCols / 32; ++cc) {
                        uint32_t v[32], sv[32];
                        fm_tmem_ld32(dbase + cc * 32, v);
                        if (!s_fresh) fm_tmem_ld32(sbase + cc * 32, sv);
                        fm_tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int32_t d = __float2int_rn(__uint_as_float(v[e]));
                            sv[e] = (uint32_t)((s_fresh ? 0 : (int32_t)sv[e]) + d);
                        }
                        if (fold_now) {
                            if (!r_fresh) {
                                fm_tmem_ld32(rbase + cc * 32, v);
                                fm_tmem_wait_ld();
                            }
                            const uint32_t wt = args.wt[idx], wts = args.wts[idx];
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                v[e] = fold_sum((int32_t)sv[e], wt, wts, r_fresh ? 0u : v[e], p);
                            fm_tmem_st32(rbase + cc * 32, v);
                        } else {
                            fm_tmem_st32(sbase + cc * 32, sv);
                        }
                    }
                }
                fm_tmem_wait_st();
                fm_tc_fence_before();
                __syncwarp();
                // fold form: a buffer holding one of the tile's two final residues
                // is released only after the tile end below has read it
                if (!(FOLD && last_on_buffer) && lane == 0)
                    fm_mbar_arrive_remote(acce_leader + (uint32_t)(b * sizeof(uint64_t)));
            }
            if (!ok) break;
            // tile end: the final residue (fold form: the sum of the two buffers'
            // residues; residue form: R) -> combine with C -> Morton-hybrid write
            uint32_t rsrc = (uint32_t)(2 * BN);
            const int by = (T - 1) & 1, bx = by ^ 1;
            if (FOLD) {
                rsrc = (uint32_t)(by * BN);
                if (njobs >= 2) {
                    const uint32_t xb = tmem + lane_base + (uint32_t)(bx * BN) + col0;
                    const uint32_t yb = tmem + lane_base + (uint32_t)(by * BN) + col0;
#pragma unroll 1
                    for (int cc = 0; cc < kCols / 32; ++cc) {
                        uint32_t xv[32], yv[32];
                        fm_tmem_ld32(xb + cc * 32, xv);
                        fm_tmem_ld32(yb + cc * 32, yv);
                        fm_tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const uint32_t x = xv[e] + yv[e];
                            yv[e] = x >= p ? x - p : x;
                        }
                        fm_tmem_st32(yb + cc * 32, yv);
                    }
                    fm_tmem_wait_st();
                    fm_tc_fence_before();
                    __syncwarp();
                    if (lane == 0) fm_mbar_arrive_remote(acce_leader + (uint32_t)(bx * sizeof(uint64_t)));
                }
            }
#pragma unroll 1
            for (int cc = 0; cc < kCols / 32; ++cc) {
                uint32_t sres[32];
                const uint32_t col = col0 + cc * 32;
                fm_tmem_ld32(tmem + lane_base + rsrc + col, sres);
                fm_tmem_wait_ld();
                if (gi < cl.M) {
                    if (KIND == kE4M3Gf2)
                        write_gf2_run(c_view(cl), gi, (int64_t)nb * BN + col, sres);
                    else
                        write_c_run<32>(cl, p, args.mu32, gi, (int64_t)nb * BN + col, cmask, sres);
                }
            }
            if (FOLD) {
                fm_tc_fence_before();
                __syncwarp();
                if (lane == 0) fm_mbar_arrive_remote(acce_leader + (uint32_t)(by * sizeof(uint64_t)));
            }
        }
    }

    fm_tc_fence_before();
    __syncthreads();
    if (s_abort && tid == 0) {
        for (uint32_t g = s_consumed; g < s_issued; ++g)
            fm_mbar_wait(&full_bar[g % S], (g / S) & 1, args.status, nullptr);
    }
    fm_cluster_sync();  // the even CTA's MMAs are complete before either CTA frees TMEM
    if (warp == 1) {
        fm_tc_fence_after();
        fm_tmem_dealloc_pair(tmem, 512);
    }
}

uint32_t powmod(uint64_t b, uint64_t e, uint32_t p)
{
    uint64_t r = 1 % p;
    b %= p;
    while (e) {
        if (e & 1) r = r * b % p;
        b = b * b % p;
        e >>= 1;
    }
    return (uint32_t)r;
}

// Inverse of a mod m (gcd(a, m) = 1) by the extended Euclidean algorithm.
uint32_t invmod(uint32_t a, uint32_t m)
{
    int64_t t = 0, nt = 1, r = m, nr = a % m;
    while (nr != 0) {
        const int64_t q = r / nr;
        int64_t tmp = t - q * nt;
        t = nt;
        nt = tmp;
        tmp = r - q * nr;
        r = nr;
        nr = tmp;
    }
    if (t < 0) t += m;
    return (uint32_t)(t % m);
}

// Products with K up to this run the fold form's 128-wide tiles two CTAs per
// SM (measured 17-20 % ahead of one CTA per SM from K = 128 to 4096; beyond,
// three stages might not keep the MMAs fed, and the default there is 256-wide
// tiles anyway).
constexpr int64_t kTwoMaxK = 4096;

template <int BN, bool FOLD, int KIND = kF16Res, bool BATCH = false, bool TWO = false>
int launch_gemm(const LimbGemmArgs& a, int grid, cudaStream_t s)
{
    auto k = limb_gemm_kernel<BN, FOLD, KIND, BATCH, TWO>;
    const size_t smem = GemmCfg<BN, TWO>::kSmem;
    FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, kGemmThreads, smem, s>>>(a);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

// How many CTA pairs of limb_gemm_pair_kernel<KIND, FOLD> fit on the current
// device at once; queried once per device and variant.
template <int KIND, bool FOLD>
int pair_capacity(int* out)
{
    static std::mutex mu;
    static int max_pairs[64] = {0};
    int dev = 0;
    FM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && max_pairs[dev] > 0) {
        *out = max_pairs[dev];
        return FM_OK;
    }
    constexpr size_t smem = PairCfg<FOLD ? 256 : 128>::kSmem;
    auto k = limb_gemm_pair_kernel<KIND, FOLD>;
    FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * fm_sm_count());
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    FM_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, k, &cfg));
    n = n > 0 ? n : fm_sm_count() / 2;
    if (dev < 64) max_pairs[dev] = n;
    *out = n;
    return FM_OK;
}

// Clusters of two CTAs, one per pair tile up to the number of pairs that fit
// on the device at once (the kernel walks further tiles itself).
template <int KIND, bool FOLD>
int launch_gemm_pair(const LimbGemmArgs& a, int pair_tiles, cudaStream_t s)
{
    int cap = 0;
    FM_TRY((pair_capacity<KIND, FOLD>(&cap)));
    constexpr size_t smem = PairCfg<FOLD ? 256 : 128>::kSmem;
    auto k = limb_gemm_pair_kernel<KIND, FOLD>;
    FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int pairs = std::max(1, std::min(pair_tiles, cap));
    cfg.gridDim = dim3(2 * pairs);
    FM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, a));
    return FM_OK;
}

}  // namespace

namespace {
uint64_t gcd_u64(uint64_t a, uint64_t b)
{
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}
}  // namespace

int fm_limb_plan(int64_t M, int64_t N, int64_t K, uint32_t p, const fm_opts* opts,
                 FmLimbPlan* plan)
{
    constexpr int64_t kPairMinK = 1024;
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    FmLimbPlan q;
    q.M = M;
    q.N = N;
    q.K = K;
    int w = 1;
    while (w < 4 && (uint64_t)1 << (8 * w) < p) ++w;
    q.w = w;
    q.fold = (p < (1u << 16) && (w == 1 || (p & 1))) ? 1 : 0;
    int bn = q.fold ? 256 : 128;
    if (opts && opts->block_n) {
        if (opts->block_n != 128 && opts->block_n != 256) return FM_EINVAL;
        bn = opts->block_n;
    }
    if (!q.fold && bn != 128) return FM_EINVAL;  // residue and sum regions need TMEM slices 3, 4
    q.block_n = bn;
    // exactness: |chunk sum| + |folded residue| (at most 2p) must stay <= 2^24
    // with |limb product| <= 2^14 (2^16 for the Karatsuba product)
    const int64_t room = q.fold ? ((int64_t)1 << 24) - 2 * (int64_t)p : ((int64_t)1 << 24);
    int cs = (int)(room / (1 << 14) / kBK);
    if (opts && opts->k_chunk) {
        if (opts->k_chunk % kBK != 0 || opts->k_chunk / kBK > cs || opts->k_chunk <= 0)
            return FM_EINVAL;
        cs = opts->k_chunk / kBK;
    }
    if (cs < 1) return FM_EUNSUPPORTED;
    // Karatsuba on two limbs: A*B = (1-256) A0B0 + 256 (A0+A1)(B0+B1) + (2^16-256) A1B1,
    // three products instead of four; used when every weight is invertible mod p
    // (the fold form carries residues between products through weight ratios).
    const uint32_t wk[3] = {(uint32_t)((p + 1 - 256 % p) % p), 256u % p,
                            (uint32_t)(((uint64_t)65536 - 256) % p)};
    bool kara = w == 2 && q.fold && !(opts && opts->no_karatsuba == 1);
    for (int k = 0; kara && k < 3; ++k) kara = wk[k] != 0 && gcd_u64(wk[k], p) == 1;
    // Residue form (w >= 2, p >= 2^16 or even): Karatsuba over every pair of
    // limbs, A_i B_j + A_j B_i = (A_i + A_j)(B_i + B_j) - A_i B_i - A_j B_j, so
    //   A*B = sum_i w_ii A_i B_i + sum_{i<j} 256^(i+j) (A_i + A_j)(B_i + B_j)
    // with w_ii = 256^(2i) - sum_{j != i} 256^(i+j): w + w (w - 1) / 2 products
    // (6 for w = 3, 10 for w = 4) instead of w^2. The residue form reduces each
    // product on its own, so the weights need not be invertible. Digit sums lie
    // in [-256, 254]: a term of a pair product is at most 2^16 in magnitude.
    const bool kara_res = !q.fold && w >= 2 && !(opts && opts->no_karatsuba == 1);
    if (kara_res) {
        const int cs_m = std::max(1, std::min(cs, (int)(((int64_t)1 << 24) / (256 * 256) / kBK)));
        const int npairs = w * (w - 1) / 2;
        q.n_planes = w + npairs;
        q.n_products = w + npairs;
        for (int i = 0; i < w; ++i) {
            uint64_t wt = powmod(256, (uint64_t)(2 * i), p);
            for (int j = 0; j < w; ++j)
                if (j != i) wt = (wt + p - powmod(256, (uint64_t)(i + j), p)) % p;
            q.prod_a[i] = q.prod_b[i] = i;
            q.prod_cs[i] = cs;
            q.prod_w[i] = (uint32_t)wt;
        }
        for (int u = 0; u < npairs; ++u) {
            int i, j;
            karatsuba_pair(u, i, j);
            q.prod_a[w + u] = q.prod_b[w + u] = w + u;
            q.prod_cs[w + u] = cs_m;
            q.prod_w[w + u] = powmod(256, (uint64_t)(i + j), p);
        }
    } else if (kara) {
        // middle product: for p < 2^16 the representative is >= 32640 - p > -32896,
        // so d0 = d1 = -128 never occurs and |d0 + d1| <= 255; a term is at most
        // 255^2, and the value carried into a chunk is below p in magnitude (a
        // residue from a product change, or v - round(v/p) p within a product)
        const int64_t room_m = ((int64_t)1 << 24) - (int64_t)p;
        const int cs_m = std::max(1, std::min(cs, (int)(room_m / (255 * 255) / kBK)));
        q.n_planes = 3;
        q.n_products = 3;
        const int pa[3] = {0, 2, 1}, cks[3] = {cs, cs_m, cs};
        const uint32_t wts[3] = {wk[0], wk[1], wk[2]};
        for (int k = 0; k < 3; ++k) {
            q.prod_a[k] = q.prod_b[k] = pa[k];
            q.prod_cs[k] = cks[k];
            q.prod_w[k] = wts[k];
        }
    } else {
        q.n_planes = w;
        q.n_products = w * w;
        for (int k = 0; k < w * w; ++k) {
            const int i = k / w, j = k % w;
            q.prod_a[k] = i;
            q.prod_b[k] = j;
            q.prod_cs[k] = cs;
            q.prod_w[k] = powmod(256, (uint64_t)(i + j), p);
        }
        if (q.fold)
            for (int k = 0; k < w * w; ++k)
                if (gcd_u64(q.prod_w[k], p) != 1) return FM_EUNSUPPORTED;
    }
    // CTA pairs: 256 x 256 tiles in the fold form, 256 x 128 in the residue form
    if (opts && opts->cta_pair == 1 && bn != (q.fold ? 256 : 128)) return FM_EINVAL;
    // automatic: CTA pairs for the fold form on 256-wide tiles of a product
    // with several tiles in each direction and a K loop long enough to hide
    // the pair's two-epilogue coupling
    int pair = opts ? opts->cta_pair : 0;
    if (pair == 0) pair = (q.fold && bn == 256 && M > 256 && N > 256 && K >= kPairMinK) ? 1 : -1;
    q.pair = pair == 1 ? 1 : 0;
    q.MB = (int)((M + kBM - 1) / kBM);
    // an even number of A row blocks wherever a pair may run; the A plane
    // layout depends on the form and BN only
    if (bn == 256 || !q.fold) q.MB += q.MB & 1;
    q.NB = (int)((N + bn - 1) / bn);
    q.KB = (int)((K + kBK - 1) / kBK);
    q.a_plane_bytes = (size_t)q.MB * q.KB * kATileBytes;
    q.b_plane_bytes = (size_t)q.NB * q.KB * bn * 128;
    *plan = q;
    return FM_OK;
}

// fm_limb_plan with the output tile width chosen from the shape when the
// caller leaves it open (fold form; the residue form always takes 128). For
// K <= 1024 the tiles are 128 wide: every tile is then mostly epilogue, and
// 128-wide tiles run two CTAs per SM (measured ahead of 256-wide tiles on
// 384- to 11776-wide products). Beyond, the width whose tiles take fewer
// rounds of the persistent grid, a round of 128-wide tiles counting half of a
// 256-wide one times 1.5 (they run their MMAs slower): thin products -- a few
// hundred columns, or a single row block -- then take 128 as well, since a
// 256-wide tile over 128 valid columns leaves half the epilogue warps idle and
// more, smaller tiles reach more SMs. Only for paths that split and multiply
// with the same plan (the step-by-step limb API keeps fm_limb_plan).
int fm_limb_plan_shaped(int64_t M, int64_t N, int64_t K, uint32_t p, const fm_opts* opts, FmLimbPlan* plan)
{
    FM_TRY(fm_limb_plan(M, N, K, p, opts, plan));
    if (!plan->fold || (opts && (opts->block_n != 0 || opts->cta_pair == 1))) return FM_OK;
    const int64_t sms = fm_sm_count(), mb = (M + kBM - 1) / kBM;
    auto rounds = [&](int64_t bn) { return (mb * ((N + bn - 1) / bn) + sms - 1) / sms; };
    const double c256 = 2.0 * (double)rounds(256);
    const double c128 = (double)rounds(128) * 1.5;
    if (K > 1024 && c128 >= c256) return FM_OK;
    fm_opts o = opts ? *opts : fm_opts{};
    o.block_n = 128;
    return fm_limb_plan(M, N, K, p, &o, plan);
}

int fm_gf2_plan(int64_t M, int64_t N, int64_t K, bool pair, FmLimbPlan* plan)
{
    FmLimbPlan q;
    q.M = M;
    q.N = N;
    q.K = K;
    q.w = 1;
    q.n_planes = 1;
    q.n_products = 1;
    q.prod_a[0] = q.prod_b[0] = 0;
    q.prod_w[0] = 1;
    q.block_n = 256;
    q.fold = 1;
    q.gf2 = 1;
    q.pair = pair ? 1 : 0;
    q.MB = (int)((M + kBM - 1) / kBM);
    q.MB += q.MB & 1;
    q.NB = (int)((N + 255) / 256);
    q.KB = (int)((K + 127) / 128);  // 128 E4M3 elements per 128-byte stage row
    // 0/1 products: a chunk of c stages adds at most 128 c; with the carried
    // parity (|v| <= 1) every partial sum stays below 2^24
    q.prod_cs[0] = std::max(1, std::min(q.KB, (int)((((int64_t)1 << 24) - 2) / 128)));
    q.a_plane_bytes = (size_t)q.MB * q.KB * kATileBytes;
    q.b_plane_bytes = (size_t)q.NB * q.KB * 256 * 128;
    *plan = q;
    return FM_OK;
}

int fm_limb_prepare_device()
{
    int cap = 0;
    FM_TRY((pair_capacity<kF16Res, true>(&cap)));
    FM_TRY((pair_capacity<kF16Res, false>(&cap)));
    return pair_capacity<kE4M3Gf2, true>(&cap);
}

size_t fm_limb_workspace_bytes(const FmLimbPlan& q)
{
    return (size_t)q.n_planes * (q.a_plane_bytes + q.b_plane_bytes);
}

namespace {

// Fields shared by every call of a launch: the limb products and the modulus.
void fill_common(const FmLimbPlan& q, uint32_t p, int* status, LimbGemmArgs& a)
{
    std::memset(&a, 0, sizeof(a));
    a.n_products = q.n_products;
    a.p = p;
    a.mu32 = (uint32_t)(((uint64_t)1 << 32) / p);
    for (int k = 0; k < q.n_products; ++k) {
        a.pa[k] = q.prod_a[k];
        a.pb[k] = q.prod_b[k];
        a.cs[k] = q.prod_cs[k];
        a.wt[k] = q.prod_w[k];
    }
    if (q.fold) {
        for (int k = 0; k < q.n_products; ++k)
            for (int k2 = 0; k2 < q.n_products; ++k2) {
                const uint32_t inv = invmod(a.wt[k2], p);
                a.cn[k * 4 + k2] = (uint32_t)((uint64_t)a.wt[k] * inv % p);
            }
    }
    a.invp = 1.0f / (float)p;
    a.pf = (float)p;
    for (int k = 0; k < q.n_products; ++k) a.wts[k] = (uint32_t)(((uint64_t)a.wt[k] << 32) / p);
    a.status = status;
}

// One call: its planes, tile counts, jobs (chunks of every product) and C.
void fill_call(const FmLimbPlan& q, int MB, int NB, int KB, uint64_t a_plane_bytes,
               uint64_t b_plane_bytes, fm_sub C, const void* a_planes, const void* b_planes, int op,
               LimbCall& c)
{
    std::memset(&c, 0, sizeof(c));
    c.Ap = static_cast<const uint8_t*>(a_planes);
    c.Bp = static_cast<const uint8_t*>(b_planes);
    c.a_plane_bytes = a_plane_bytes;
    c.b_plane_bytes = b_plane_bytes;
    c.MB = MB;
    c.NB = NB;
    c.KB = KB;
    c.first[0] = 0;
    for (int k = 0; k < q.n_products; ++k) c.first[k + 1] = c.first[k] + (KB + q.prod_cs[k] - 1) / q.prod_cs[k];
    for (int k = q.n_products + 1; k <= 16; ++k) c.first[k] = c.first[q.n_products];
    c.njobs = c.first[q.n_products];
    c.C = C.m.base;
    c.c_lt = C.m.log2_T;
    c.op = op;
    c.c_row0 = C.row0;
    c.c_col0 = C.col0;
    c.M = C.rows;
    c.N = C.cols;
}

}  // namespace

int fm_limb_gemm_run(const FmLimbPlan& q, fm_sub C, const void* a_planes, const void* b_planes,
                     uint32_t p, int op, int* status, cudaStream_t s)
{
    if (q.M == 0 || q.N == 0 || q.K == 0) return FM_OK;
    LimbGemmArgs a;
    fill_common(q, p, status, a);
    fill_call(q, q.MB, q.NB, q.KB, q.a_plane_bytes, q.b_plane_bytes, C, a_planes, b_planes, op, a.call);
    a.call.M = q.M;
    a.call.N = q.N;
    if (q.gf2) {
        if (q.pair) return launch_gemm_pair<kE4M3Gf2, true>(a, q.MB / 2 * q.NB, s);
        return launch_gemm<256, true, kE4M3Gf2>(a, std::min(q.MB * q.NB, fm_sm_count()), s);
    }
    // q.max_ctas caps the resident CTAs (a persistent grid then walks more tiles each)
    auto cap = [&](int ctas) { return q.max_ctas > 0 ? std::max(1, std::min(ctas, q.max_ctas)) : ctas; };
    if (q.pair) {
        const int pt = std::min(q.MB / 2 * q.NB, q.max_ctas > 0 ? std::max(1, q.max_ctas / 2) : INT_MAX);
        if (q.fold) return launch_gemm_pair<kF16Res, true>(a, pt, s);
        return launch_gemm_pair<kF16Res, false>(a, pt, s);
    }
    const int grid = cap(std::min(q.MB * q.NB, fm_sm_count()));
    if (q.fold) {
        if (q.block_n == 256) return launch_gemm<256, true>(a, grid, s);
        if (q.K <= kTwoMaxK)
            return launch_gemm<128, true, kF16Res, false, true>(a, cap(std::min(q.MB * q.NB, 2 * fm_sm_count())), s);
        return launch_gemm<128, true>(a, grid, s);
    }
    return launch_gemm<128, false>(a, grid, s);
}

int fm_limb_run(const FmLimbPlan& q, fm_sub C, fm_sub A, fm_sub B, uint32_t p, int op,
                void* workspace, int* status, cudaStream_t s)
{
    if (q.M == 0 || q.N == 0) return FM_OK;
    uint8_t* Ap = static_cast<uint8_t*>(workspace);
    uint8_t* Bp = Ap + (size_t)q.n_planes * q.a_plane_bytes;
    FM_TRY(fm_limb_split_run(q, A, FM_LIMB_A, p, Ap, s));
    FM_TRY(fm_limb_split_run(q, B, FM_LIMB_B, p, Bp, s));
    return fm_limb_gemm_run(q, C, Ap, Bp, p, op, status, s);
}

// ---- batched limb form ------------------------------------------------------
// Every call of a batch gets its own limb planes in one workspace. Three
// launches run the whole batch: the A splits of every call, the B splits of
// every call, and one persistent GEMM over the output tiles of every call
// (longest first; each CTA walks tiles blockIdx.x, + gridDim.x, ...). On
// request (fm_opts.fused_batch) the batch runs as one fused launch instead
// (limb_fused.cu).
struct FmLimbBatch {
    FmLimbPlan q;  // limb parameters shared by every call (products, chunks, BN)
    uint32_t p = 0;
    void* ws = nullptr;
    FmSplitDesc* d_adesc = nullptr;
    FmSplitDesc* d_bdesc = nullptr;
    int2* d_ajobs = nullptr;
    int2* d_bjobs = nullptr;
    int64_t n_ajobs = 0, n_bjobs = 0;
    LimbCall* d_calls = nullptr;
    int4* d_tiles = nullptr;
    int n_tiles = 0;
    int max_kb = 0;                        // the longest call's 64-wide K stages
    bool gf2 = false;                      // bit-packed GF(2) operands
    FmFusedBatch* fused = nullptr;         // one launch, operands split on the fly
    std::vector<fm_gemm_call> zero_calls;  // K = 0: only FM_OP_SET changes C
    std::vector<fm_gf2_sub> zero_subs;     // GF(2), K = 0 under FM_OP_SET
};

namespace {
template <typename T>
int upload_vec(const std::vector<T>& v, T** out)
{
    *out = nullptr;
    if (v.empty()) return FM_OK;
    if (cudaMalloc(reinterpret_cast<void**>(out), v.size() * sizeof(T)) != cudaSuccess) return FM_ENOMEM;
    if (cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return FM_ECUDA;
    return FM_OK;
}
}  // namespace

void fm_limb_batch_destroy(FmLimbBatch* b)
{
    if (!b) return;
    fm_fused_batch_destroy(b->fused);
    cudaFree(b->ws);
    cudaFree(b->d_adesc);
    cudaFree(b->d_bdesc);
    cudaFree(b->d_ajobs);
    cudaFree(b->d_bjobs);
    cudaFree(b->d_calls);
    cudaFree(b->d_tiles);
    delete b;
}

namespace {

// One call of a batch before its planes are placed: shapes, the two operands
// (src, lt, row0, col0, rows, cols of its FmSplitDesc) and C.
struct BatchCall {
    int64_t M, N, K;
    FmSplitDesc a, b;
    fm_sub C;
    int op;
};

// Places every call's planes in one workspace (K tiles of kt elements, output
// tiles of 128 x bn) and uploads the split jobs, the call table and the tile
// list (longest first).
int build_batch(const std::vector<BatchCall>& in, int bn, int kt, FmLimbBatch* b)
{
    const FmLimbPlan& q = b->q;
    const uint64_t b_tile = (uint64_t)bn * 128;
    std::vector<uint64_t> a_off(in.size()), b_off(in.size());
    uint64_t total = 0;
    for (size_t c = 0; c < in.size(); ++c) {
        const int MB = (int)((in[c].M + kBM - 1) / kBM), NB = (int)((in[c].N + bn - 1) / bn);
        const int KB = (int)((in[c].K + kt - 1) / kt);
        a_off[c] = total;
        total += ((q.n_planes * (uint64_t)MB * KB * kATileBytes + 1023) / 1024) * 1024;
        b_off[c] = total;
        total += ((q.n_planes * (uint64_t)NB * KB * b_tile + 1023) / 1024) * 1024;
    }
    if (total > 0 && cudaMalloc(&b->ws, total) != cudaSuccess) return FM_ENOMEM;
    uint8_t* ws = static_cast<uint8_t*>(b->ws);
    std::vector<FmSplitDesc> ad, bd;
    std::vector<int2> aj, bj;
    std::vector<LimbCall> lc;
    std::vector<int4> tiles;
    std::vector<int64_t> cost;
    for (size_t c = 0; c < in.size(); ++c) {
        const BatchCall& g = in[c];
        const int MB = (int)((g.M + kBM - 1) / kBM), NB = (int)((g.N + bn - 1) / bn);
        const int KB = (int)((g.K + kt - 1) / kt);
        const uint64_t ab = (uint64_t)MB * KB * kATileBytes, bb = (uint64_t)NB * KB * b_tile;
        const int di = (int)ad.size();
        FmSplitDesc da = g.a, db = g.b;
        da.KB = db.KB = KB;
        da.out = ws + a_off[c];
        db.out = ws + b_off[c];
        da.plane_bytes = (size_t)ab;
        db.plane_bytes = (size_t)bb;
        ad.push_back(da);
        bd.push_back(db);
        for (int t = 0; t < MB * KB; ++t) aj.push_back(make_int2(di, t));
        for (int t = 0; t < NB * KB; ++t) bj.push_back(make_int2(di, t));
        LimbCall call;
        fill_call(q, MB, NB, KB, ab, bb, g.C, ws + a_off[c], ws + b_off[c], g.op, call);
        const int ci = (int)lc.size();
        lc.push_back(call);
        for (int mb = 0; mb < MB; ++mb)
            for (int nb = 0; nb < NB; ++nb) {
                tiles.push_back(make_int4(ci, mb, nb, 0));
                const int64_t rows = std::min<int64_t>(kBM, g.M - (int64_t)mb * kBM);
                const int64_t cols = std::min<int64_t>(bn, g.N - (int64_t)nb * bn);
                cost.push_back((int64_t)call.njobs * 4096 + (int64_t)KB * 64 + (rows * cols >> 10));
            }
    }
    // longest tiles first, so that the static walk of the persistent grid balances
    std::vector<size_t> order(tiles.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<int4> sorted(tiles.size());
    for (size_t t = 0; t < order.size(); ++t) sorted[t] = tiles[order[t]];
    if (sorted.size() > 0x7fffffff || aj.size() > 0x7fffffff || bj.size() > 0x7fffffff) return FM_EINVAL;
    FM_TRY(upload_vec(ad, &b->d_adesc));
    FM_TRY(upload_vec(bd, &b->d_bdesc));
    FM_TRY(upload_vec(aj, &b->d_ajobs));
    FM_TRY(upload_vec(bj, &b->d_bjobs));
    FM_TRY(upload_vec(lc, &b->d_calls));
    FM_TRY(upload_vec(sorted, &b->d_tiles));
    b->n_ajobs = (int64_t)aj.size();
    b->max_kb = 0;
    for (const LimbCall& c : lc) b->max_kb = std::max(b->max_kb, c.KB);
    b->n_bjobs = (int64_t)bj.size();
    b->n_tiles = (int)sorted.size();
    return FM_OK;
}

}  // namespace

int fm_limb_batch_create(const fm_gemm_call* calls, int64_t n, uint32_t p, const fm_opts* opts,
                         FmLimbBatch** out)
{
    *out = nullptr;
    if (opts && opts->cta_pair == 1) return FM_EUNSUPPORTED;
    // batches of small products waste less on 128-wide output tiles
    fm_opts o = opts ? *opts : fm_opts{};
    if (o.block_n == 0) o.block_n = 128;
    FmLimbPlan q;
    FM_TRY(fm_limb_plan(1, 1, 1, p, &o, &q));
    FmLimbBatch* b = new FmLimbBatch();
    b->q = q;
    b->p = p;
    std::vector<BatchCall> in;
    for (int64_t c = 0; c < n; ++c) {
        const fm_gemm_call& g = calls[c];
        if (g.C.rows == 0 || g.C.cols == 0) continue;
        if (g.A.cols == 0) {
            b->zero_calls.push_back(g);
            continue;
        }
        BatchCall bc;
        bc.M = g.C.rows;
        bc.N = g.C.cols;
        bc.K = g.A.cols;
        bc.a = FmSplitDesc{g.A.m.base, g.A.m.log2_T, 0, g.A.row0, g.A.col0, bc.M, bc.K, nullptr, 0};
        bc.b = FmSplitDesc{g.B.m.base, g.B.m.log2_T, 0, g.B.row0, g.B.col0, bc.K, bc.N, nullptr, 0};
        bc.C = g.C;
        bc.op = g.op;
        in.push_back(bc);
    }
    if (o.fused_batch) {
        const int rf = fm_fused_batch_create(calls, n, p, q, &b->fused);
        if (rf != FM_OK) {
            fm_limb_batch_destroy(b);
            return rf;
        }
        b->n_tiles = (int)fm_fused_batch_tiles(b->fused);
        *out = b;
        return FM_OK;
    }
    const int rc = build_batch(in, q.block_n, kBK, b);
    if (rc != FM_OK) {
        fm_limb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FM_OK;
}

int fm_gf2_batch_create(const fm_gf2_call* calls, int64_t n, const fm_opts* opts, FmLimbBatch** out)
{
    *out = nullptr;
    if (opts && opts->cta_pair == 1) return FM_EUNSUPPORTED;
    FmLimbPlan q;
    FM_TRY(fm_gf2_plan(1, 1, 1, false, &q));
    q.prod_cs[0] = (int)((((int64_t)1 << 24) - 2) / 128);  // one accumulation for any K < 2^24
    FmLimbBatch* b = new FmLimbBatch();
    b->q = q;
    b->p = 2;
    b->gf2 = true;
    std::vector<BatchCall> in;
    for (int64_t c = 0; c < n; ++c) {
        const fm_gf2_call& g = calls[c];
        if (g.C.rows == 0 || g.C.cols == 0) continue;
        if (g.A.cols == 0) {
            if (g.op == FM_OP_SET) b->zero_subs.push_back(g.C);
            continue;
        }
        BatchCall bc;
        bc.M = g.C.rows;
        bc.N = g.C.cols;
        bc.K = g.A.cols;
        bc.a = FmSplitDesc{g.A.m.base, g.A.m.log2_grid, 0, g.A.row0, g.A.col0, bc.M, bc.K, nullptr, 0};
        bc.b = FmSplitDesc{g.B.m.base, g.B.m.log2_grid, 0, g.B.row0, g.B.col0, bc.K, bc.N, nullptr, 0};
        fm_sub cs;
        cs.m.base = g.C.m.base;
        cs.m.log2_grid = g.C.m.log2_grid;
        cs.m.log2_T = 5;
        cs.row0 = g.C.row0;
        cs.col0 = g.C.col0;
        cs.rows = g.C.rows;
        cs.cols = g.C.cols;
        bc.C = cs;
        bc.op = g.op;
        in.push_back(bc);
    }
    const int rc = build_batch(in, 256, 128, b);
    if (rc != FM_OK) {
        fm_limb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FM_OK;
}

int64_t fm_limb_batch_tiles(const FmLimbBatch* b)
{
    return b ? b->n_tiles : 0;
}

int fm_limb_batch_launches(const FmLimbBatch* b)
{
    if (!b) return 0;
    int n = (int)b->zero_subs.size();
    if (b->n_tiles > 0) n += b->fused ? 1 : 3;
    return n;
}

const std::vector<fm_gemm_call>& fm_limb_batch_zero_calls(const FmLimbBatch* b)
{
    return b->zero_calls;
}

int fm_limb_batch_run(FmLimbBatch* b, int* status, cudaStream_t s)
{
    for (const fm_gf2_sub& z : b->zero_subs) FM_TRY(fm_gf2_zero_sub(z, s));
    if (b->n_tiles == 0) return FM_OK;
    if (b->fused) return fm_fused_batch_run(b->fused, status, s);
    if (b->gf2) {
        FM_TRY(fm_gf2_split_batch_run(FM_LIMB_A, b->d_adesc, b->d_ajobs, b->n_ajobs, s));
        FM_TRY(fm_gf2_split_batch_run(FM_LIMB_B, b->d_bdesc, b->d_bjobs, b->n_bjobs, s));
    } else {
        FM_TRY(fm_limb_split_batch_run(b->q, FM_LIMB_A, b->d_adesc, b->d_ajobs, b->n_ajobs, b->p, s));
        FM_TRY(fm_limb_split_batch_run(b->q, FM_LIMB_B, b->d_bdesc, b->d_bjobs, b->n_bjobs, b->p, s));
    }
    LimbGemmArgs a;
    fill_common(b->q, b->p, status, a);
    a.calls = b->d_calls;
    a.tiles = b->d_tiles;
    a.n_tiles = b->n_tiles;
    const int grid = std::min(b->n_tiles, fm_sm_count());
    if (b->gf2) return launch_gemm<256, true, kE4M3Gf2, true>(a, grid, s);
    if (b->q.fold) {
        if (b->q.block_n == 256) return launch_gemm<256, true, kF16Res, true>(a, grid, s);
        if ((int64_t)b->max_kb * kBK <= kTwoMaxK)
            return launch_gemm<128, true, kF16Res, true, true>(a, std::min(b->n_tiles, 2 * fm_sm_count()), s);
        return launch_gemm<128, true, kF16Res, true>(a, grid, s);
    }
    return launch_gemm<128, false, kF16Res, true>(a, grid, s);
}

// ---- C entry points of the step-by-step limb form --------------------------
extern "C" int64_t fm_limb_planes_size(int64_t rows, int64_t cols, int32_t role, uint32_t p,
                                       const fm_opts* opts)
{
    if (rows < 0 || cols < 0) return FM_EINVAL;
    if (role != FM_LIMB_A && role != FM_LIMB_B) return FM_EINVAL;
    FmLimbPlan q;
    // A is M x K; B is K x N
    const int rc = role == FM_LIMB_A ? fm_limb_plan(rows, 1, cols, p, opts, &q)
                                     : fm_limb_plan(1, cols, rows, p, opts, &q);
    if (rc != FM_OK) return rc;
    return (int64_t)q.n_planes * (int64_t)(role == FM_LIMB_A ? q.a_plane_bytes : q.b_plane_bytes);
}

extern "C" int fm_limb_gemm(fm_sub C, const void* a_planes, const void* b_planes, int64_t K,
                            uint32_t p, int32_t op, const fm_opts* opts, fm_stream stream)
{
    if (op < FM_OP_SET || op > FM_OP_SUB || K < 0) return FM_EINVAL;
    FM_TRY(fm_check_sub(C));
    if (((uintptr_t)a_planes & 15) || ((uintptr_t)b_planes & 15)) return FM_EINVAL;
    FmLimbPlan q;
    FM_TRY(fm_limb_plan(C.rows, C.cols, K, p, opts, &q));
    if (C.rows == 0 || C.cols == 0) return FM_OK;
    if (K == 0) return FM_EUNSUPPORTED;  // nothing to multiply: use fm_gemm_modp
    if (!a_planes || !b_planes) return FM_EINVAL;
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    return fm_limb_gemm_run(q, C, a_planes, b_planes, p, op, status, (cudaStream_t)stream);
}
