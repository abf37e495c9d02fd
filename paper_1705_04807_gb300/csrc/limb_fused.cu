// limb_fused.cu -- a whole batch of C <- C op A*B mod p in ONE persistent launch
// of the tensor-core limb form, with the limb split done on the fly.
//
// The batching form of Sec. 2.2 issues many small, uneven products. Splitting
// every operand into limb planes in HBM first (three launches, limb_split.cu +
// limb_gemm.cu) moves six bytes of planes per entry through HBM twice; here the
// residues themselves are read (4 bytes per entry, mostly from L2, since the
// tiles of one call run side by side) and split in registers into the f16
// planes the tensor cores read from shared memory.
//
// Two-limb Karatsuba form (odd p < 2^16): with r = x if x <= 127*257 else x - p,
// s = r + 128 + 128*256 is a 16-bit number whose low and high bytes are the
// balanced digits d0 + 128 and d1 + 128 of r (Sec. 2.1's base-256 split into
// signed 8-bit limbs, restated). The IEEE half with bits 0x64 << 8 | byte is
// 1024 + byte, so one byte permute and one packed half subtraction of 1152 give
// two digits d exactly; d0 + d1 (|.| <= 255) is one more packed addition. The
// three planes d0, d0 + d1 and d1 of A and of B feed the three products
//     A*B == (1 - 256) A0B0 + 256 (A0+A1)(B0+B1) + (2^16 - 256) A1B1   (mod p).
//
// Per CTA (one per SM, walking 128 x 128 output tiles): eight converter warps
// load a 64-wide K stage of A (128 x 64) and B (64 x 128) from the
// Morton-hybrid layout with 16-byte loads, split it and store the six planes in
// the 128-byte-swizzled K-major layout (two stages in shared memory, the next
// stage's loads in flight while the current one is converted); once all eight
// have stored a stage, lane 0 of converter warp 0 issues its tcgen05.mma
// kind::f16 for the three products into three FP32 accumulators in tensor
// memory; four epilogue warps fold the accumulators at exact-chunk boundaries,
// combine them at the tile end into residues (a fourth tensor-memory slice,
// so the accumulators are free for the next tile at once) and update C in the
// Morton-hybrid layout.
//
// Each operand entry is split once per output tile that uses it, which costs
// more than the planes' round trip through HBM on batches of products a few
// hundred wide: the plane form is the default and this one is requested with
// fm_opts.fused_batch (one launch and no plane workspace).
//
// 16-byte loads need 4-aligned columns: a call's K window is shifted by A's
// column offset mod 4 (ra zero entries in front, the same shift on B's rows),
// so every 16-byte load of A starts on a multiple of 4 inside one tile row
// (T' >= 8). B is read with 16-byte loads when its first column is a multiple
// of 4 and with 4-byte loads otherwise; C's columns are never shifted.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fm_internal.cuh"
#include "fm_kernels.h"
#include "limb_common.cuh"
#include "limb_drain.cuh"

namespace {

using namespace fm_limb;

// Warps 0-7 convert; lane 0 of warp 0 also issues the MMAs of each stage once
// all eight have stored it; warps 8-11 are the epilogue (one per TMEM lane
// quarter). Twelve warps, three per SM sub-partition, leave 168 registers per
// thread (a thirteenth warp would cut that to 128).
constexpr int kFzConvWarps = 8;
constexpr int kFzEpiWarps = 4;
constexpr int kFzThreads = 32 * (kFzConvWarps + kFzEpiWarps);
constexpr int kFzBN = 128;                                   // output columns per tile
constexpr uint32_t kFzPlane = kATileBytes;                   // one plane, one operand, one stage
constexpr uint32_t kFzStageBytes = 6 * kFzPlane;             // A: planes 0-2, B: planes 3-5
constexpr int kFzStages = 2;
constexpr size_t kFzSmem = (size_t)kFzStages * kFzStageBytes + 1024;  // + alignment slack
constexpr uint32_t kFzHi = 127u * 257u;                      // largest residue kept as r = x
constexpr uint32_t kFzSoff = 128u + 128u * 256u;             // s = r + kFzSoff

// What the converters read of a call at every stage, held by value (see CView).
struct ConvCall {
    const uint32_t* A;
    const uint32_t* B;
    int64_t a_col0, b_row0;
    uint32_t a_cmask, a_c64, b_rmask, b_r64;
    int a_lt, b_lt;
};

// One call of a fused batch. a_col0 is A's first column rounded down to a
// multiple of 4, ra the remainder.
struct FusedCall {
    const uint32_t* A;
    const uint32_t* B;
    uint32_t* C;
    int64_t a_row0, a_col0, b_row0, b_col0, c_row0, c_col0;
    int64_t M, N, K;
    int a_lt, b_lt, c_lt, op;
    int ra;
    int KB;                 // 64-wide K stages: ceil((K + ra) / 64)
    uint32_t a_cmask, a_c64;  // A: column bits of an offset, column part of 64
    uint32_t b_rmask, b_r64;  // B: row bits of an offset, row part of 64
};

struct FusedArgs {
    const FusedCall* calls;
    const int4* tiles;  // (call, mb, nb) per output tile; a call's tiles are adjacent
    int n_tiles;
    int cs[3];          // K stages per exact chunk of product k
    uint32_t p, mu32;
    float invp, pf;
    int* status;
};

// Morton-hybrid offset = row part | column part (disjoint bits): tile (I, J)
// at Z(I, J) T'^2 with Z = spread(I) << 1 | spread(J), entry (u, v) at
// u T' + v. Fused batches take operands of at most 2^32 entries, so offsets
// are 32-bit. Row (column) parts add like dilated integers:
// part(i + d) = ((part(i) | ~mask) + part(d)) & mask, mask = the row (column)
// bits, which moves a row or column index along without re-interleaving.
__host__ __device__ __forceinline__ uint32_t spread16(uint32_t x)
{
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__host__ __device__ __forceinline__ uint32_t row_part(uint32_t i, int lt)
{
    return (spread16(i >> lt) << (2 * lt + 1)) | ((i & ((1u << lt) - 1)) << lt);
}

__host__ __device__ __forceinline__ uint32_t col_part(uint32_t j, int lt)
{
    return (spread16(j >> lt) << (2 * lt)) | (j & ((1u << lt) - 1));
}

__host__ __device__ __forceinline__ uint32_t part_add(uint32_t x, uint32_t d, uint32_t mask)
{
    return ((x | ~mask) + d) & mask;
}

// Bits e (0..7) with 0 <= lo + e < K.
__device__ __forceinline__ uint32_t range_bits(int64_t lo, int64_t K)
{
    const int s = lo < 0 ? (int)(lo < -8 ? 8 : -lo) : 0;
    const int64_t left = K - lo;
    const int e = left <= 0 ? 0 : (left >= 8 ? 8 : (int)left);
    return e > s ? ((0xFFu >> (8 - e)) & (0xFFu << s)) : 0u;
}

// Loads that leave their destination unchanged when pred is false: no select
// after the load, so nothing waits for the data until it is used.
__device__ __forceinline__ void ldg16_if(uint4& v, const uint32_t* p, bool pred)
{
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t"
        "@q ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
        : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
        : "l"(p), "r"((int)pred));
}

__device__ __forceinline__ void ldg4_if(uint32_t& v, const uint32_t* p, bool pred)
{
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.global.nc.u32 %0, [%1];\n\t}"
        : "+r"(v)
        : "l"(p), "r"((int)pred));
}

__device__ __forceinline__ void sts16(uint32_t addr, uint4 v)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ uint32_t elem(const uint4& v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

// s of two residues packed as 16-bit halves (the first in the low half).
__device__ __forceinline__ uint32_t pack_s(uint32_t x0, uint32_t x1, uint32_t p)
{
    const uint32_t s0 = x0 + kFzSoff - (x0 > kFzHi ? p : 0u);
    const uint32_t s1 = x1 + kFzSoff - (x1 > kFzHi ? p : 0u);
    return prmt(s0, s1, 0x5410);
}

// Digit pair (low byte or high byte of each 16-bit s) as two exact halves.
__device__ __forceinline__ uint32_t digits(uint32_t w, uint32_t sel)
{
    const uint32_t h = prmt(w, 0x64646464u, sel);
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(h), "r"(0x64806480u));  // 1152, 1152
    return d;
}

__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Four packed words (8 consecutive k of one row or column) -> the 16-byte
// chunk of each plane at byte offset off of the three planes starting at base.
__device__ __forceinline__ void store_chunk(uint32_t base, uint32_t off, const uint32_t (&w)[4])
{
    uint4 p0, p1, p2;
    p0.x = digits(w[0], 0x4240);
    p0.y = digits(w[1], 0x4240);
    p0.z = digits(w[2], 0x4240);
    p0.w = digits(w[3], 0x4240);
    p1.x = digits(w[0], 0x4341);
    p1.y = digits(w[1], 0x4341);
    p1.z = digits(w[2], 0x4341);
    p1.w = digits(w[3], 0x4341);
    p2.x = hadd2(p0.x, p1.x);
    p2.y = hadd2(p0.y, p1.y);
    p2.z = hadd2(p0.z, p1.z);
    p2.w = hadd2(p0.w, p1.w);
    sts16(base + off, p0);                 // product 0: A0 B0
    sts16(base + kFzPlane + off, p2);      // product 1: (A0 + A1)(B0 + B1)
    sts16(base + 2 * kFzPlane + off, p1);  // product 2: A1 B1
}

// A wait for a whole warp: lane 0 polls, the warp synchronises and every lane
// gets the one outcome (the warp then runs .sync.aligned instructions or
// leaves its loop together).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* status, volatile int* abort)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = fm_mbar_wait(bar, parity, status, abort) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Final residues of 32 columns from the three Karatsuba accumulators, exactly
// in packed FP32: with f_k = acc_k folded (|f_k| <= 3p/4),
//     (1 - 256) f0 + 256 f1 + (2^16 - 256) f2 = f0 + 256 (f1 - f0 - f2) + 256 (256 f2),
// every product by 256 taken of a folded value (below 192 p < 2^24) and folded
// again. The result, in [0, p), replaces v0.
__device__ __forceinline__ void karatsuba_residue(uint32_t (&v0)[32], const uint32_t (&v1)[32],
                                                  const uint32_t (&v2)[32], uint32_t p, float invp, float pf)
{
    const uint64_t ip = f2_splat(invp), bs = f2_splat(kRoundBias), np = f2_splat(-pf);
    const uint64_t k256 = f2_splat(256.0f);
#pragma unroll
    for (int e = 0; e < 32; e += 2) {
        const uint64_t f0 = f2_fold(((uint64_t)v0[e + 1] << 32) | v0[e], ip, bs, np);
        const uint64_t f1 = f2_fold(((uint64_t)v1[e + 1] << 32) | v1[e], ip, bs, np);
        const uint64_t f2 = f2_fold(((uint64_t)v2[e + 1] << 32) | v2[e], ip, bs, np);
        const uint64_t m = f2_fold(f2_sub(f2_sub(f1, f0), f2), ip, bs, np);
        const uint64_t g = f2_fold(f2_mul(m, k256), ip, bs, np);
        const uint64_t t = f2_fold(f2_mul(f2, k256), ip, bs, np);
        const uint64_t h = f2_fold(f2_mul(t, k256), ip, bs, np);
        const uint64_t r = f2_fold(f2_add(f2_add(f0, g), h), ip, bs, np);
        const int32_t a = (int32_t)(__float_as_uint(__fadd_rn(__uint_as_float((uint32_t)r), kRoundBias)) -
                                    kRoundBiasBits);
        const int32_t b = (int32_t)(__float_as_uint(__fadd_rn(__uint_as_float((uint32_t)(r >> 32)), kRoundBias)) -
                                    kRoundBiasBits);
        v0[e] = (uint32_t)(a + (a < 0 ? (int32_t)p : 0));
        v0[e + 1] = (uint32_t)(b + (b < 0 ? (int32_t)p : 0));
    }
}

// 128-byte swizzle: 16-byte chunk kc of row r (rows of 128 bytes).
__device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t kc)
{
    return r * 128u + ((kc ^ (r & 7u)) << 4);
}

__global__ void __launch_bounds__(kFzThreads, 1) limb_fused_kernel(const __grid_constant__ FusedArgs args)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    __shared__ __align__(8) uint64_t full_bar[kFzStages];
    __shared__ __align__(8) uint64_t empty_bar[kFzStages];
    __shared__ __align__(8) uint64_t midf_bar[3];  // product k's chunk complete (MMA -> epilogue)
    __shared__ __align__(8) uint64_t mide_bar[3];  // product k's chunk folded (epilogue -> MMA)
    __shared__ __align__(8) uint64_t endf_bar;     // the tile's accumulators complete
    __shared__ __align__(8) uint64_t ende_bar;     // the tile's accumulators read
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t p = args.p;

    if (tid == 0) {
        for (int s = 0; s < kFzStages; ++s) {
            fm_mbar_init(&full_bar[s], kFzConvWarps);
            fm_mbar_init(&empty_bar[s], 1);
        }
        for (int k = 0; k < 3; ++k) {
            fm_mbar_init(&midf_bar[k], 1);
            fm_mbar_init(&mide_bar[k], kFzEpiWarps);
        }
        fm_mbar_init(&endf_bar, 1);
        fm_mbar_init(&ende_bar, kFzEpiWarps);
        fm_mbar_init(&done_bar, 1);
        fm_fence_mbar_init();
        s_abort = 0;
    }
    if (warp == 0) {
        fm_tmem_alloc(&tmem_slot, 512);
        fm_tmem_relinquish();
    }
    fm_tc_fence_before();
    __syncthreads();
    fm_tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t smem0 = fm_smem_u32(smem);

    if (warp < kFzConvWarps) {
        // ---- converters ----
        const int ct = tid;
        const int kca = ct & 7, arow0 = ct >> 3;                    // A: chunk kca of rows arow0 + 32 it
        const int kcb = lane & 7, n0 = (warp * 4 + (lane >> 3)) * 4;  // B: chunk kcb of columns n0 .. n0+3

        // state of the stage whose loads are in flight
        int tile = blockIdx.x, kb = 0;
        ConvCall cv{};
        int64_t K = 0;
        int ra = 0, KB = 0;
        uint32_t idesc = 0;
        uint32_t arow[4] = {0, 0, 0, 0}, bcol[4] = {0, 0, 0, 0};
        uint32_t arow_ok = 0, bcol_ok = 0, ak_ok = 0, brow_ok = 0;
        uint32_t ac0 = 0, ac1 = 0, bR = 0;  // A chunk column parts, B row-block row part
        bool bvec = true;
        uint4 xa[4][2], xb[8];

        auto setup_tile = [&]() {
            const int4 e = args.tiles[tile];
            const FusedCall& c = args.calls[e.x];
            cv = ConvCall{c.A, c.B, c.a_col0, c.b_row0, c.a_cmask, c.a_c64, c.b_rmask, c.b_r64, c.a_lt, c.b_lt};
            K = c.K;
            ra = c.ra;
            KB = c.KB;
            const int64_t left = c.N - (int64_t)e.z * kFzBN;
            idesc = fm_idesc_f16_f32(kBM, (int)(((left < kFzBN ? left : kFzBN) + 15) & ~15));
            arow_ok = 0;
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int64_t i = (int64_t)e.y * kBM + arow0 + 32 * it;
                const bool ok = i < c.M;
                arow[it] = ok ? row_part((uint32_t)(c.a_row0 + i), c.a_lt) : 0u;
                arow_ok |= (ok ? 1u : 0u) << it;
            }
            const int64_t js = (int64_t)e.z * kFzBN + n0;  // sub-matrix column of n0
            bcol_ok = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) bcol_ok |= (js + q < c.N ? 1u : 0u) << q;
            // column parts of B's four columns (one tile-row crossing at most)
            const uint32_t gb = (uint32_t)(c.b_col0 + js), bm = (1u << c.b_lt) - 1;
            bvec = (gb & 3u) == 0;
            const uint32_t cp0 = col_part(gb, c.b_lt), cp1 = col_part((gb | bm) + 1, c.b_lt);
#pragma unroll
            for (int q = 0; q < 4; ++q) bcol[q] = (gb & bm) + q <= bm ? cp0 + q : cp1 + ((gb & bm) + q - bm - 1);
        };
        auto load_stage = [&]() {
            const ConvCall& c = cv;
            const int64_t k0 = (int64_t)kb * kBK - ra;  // sub-matrix K index of slot 0
            const bool full = k0 >= 0 && k0 + kBK <= K;
            // A: columns k0 + 8 kca .. +7 (column parts advance by 64 per stage)
            if (kb == 0) {
                const uint32_t gj = (uint32_t)(c.a_col0 + kca * 8);
                ac0 = col_part(gj, c.a_lt);
                ac1 = col_part(gj + 4, c.a_lt);
            } else {
                ac0 = part_add(ac0, c.a_c64, c.a_cmask);
                ac1 = part_add(ac1, c.a_c64, c.a_cmask);
            }
            ak_ok = full ? 0xFFu : range_bits(k0 + kca * 8, K);
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const bool r = (arow_ok >> it) & 1u;
                xa[it][0] = xa[it][1] = make_uint4(0, 0, 0, 0);
                ldg16_if(xa[it][0], c.A + (arow[it] | ac0), r && (ak_ok & 0x0Fu));
                ldg16_if(xa[it][1], c.A + (arow[it] | ac1), r && (ak_ok & 0xF0u));
            }
            // B: rows k0 + 8 kcb .. +7 of the sub-matrix, columns n0 .. n0+3 of the tile
            const int64_t r0 = k0 + kcb * 8;
            brow_ok = bcol_ok ? (full ? 0xFFu : range_bits(r0, K)) : 0u;
            int ef = 0;
            if (kb == 0) {
                // rows before the first valid one are negative: start there
                if (brow_ok) {
                    ef = __ffs(brow_ok) - 1;
                    bR = row_part((uint32_t)(c.b_row0 + r0 + ef), c.b_lt);
                }
            } else if (kb == 1) {
                bR = row_part((uint32_t)(c.b_row0 + r0), c.b_lt);
            } else {
                bR = part_add(bR, c.b_r64, c.b_rmask);
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool row = (brow_ok >> e) & 1u;
                const uint32_t rp = part_add(bR, (uint32_t)(e - ef) << c.b_lt, c.b_rmask);
                xb[e] = make_uint4(0, 0, 0, 0);
                if (bvec) {
                    ldg16_if(xb[e], c.B + (rp | bcol[0]), row);
                } else {
                    ldg4_if(xb[e].x, c.B + (rp | bcol[0]), row && (bcol_ok & 1u));
                    ldg4_if(xb[e].y, c.B + (rp | bcol[1]), row && (bcol_ok & 2u));
                    ldg4_if(xb[e].z, c.B + (rp | bcol[2]), row && (bcol_ok & 4u));
                    ldg4_if(xb[e].w, c.B + (rp | bcol[3]), row && (bcol_ok & 8u));
                }
            }
            if (kb == 0) bR = 0;  // stage 1 recomputes it (stage 0 may start before row 0)
        };

        // MMA issue (lane 0 of warp 0) for stage g = (st of KB) of a tile
        uint32_t tcount = 0, mcnt[3] = {0, 0, 0};
        bool pend[3] = {false, false, false};
        auto issue = [&](uint32_t g, int st, int nst, uint32_t id) -> bool {
            const int s = g & 1;
            if (st == 0 && tcount > 0) {
                if (!fm_mbar_wait(&ende_bar, (tcount - 1) & 1u, args.status, &s_abort)) return false;
                fm_tc_fence_after();
            }
            if (!fm_mbar_wait(&full_bar[s], (g >> 1) & 1u, args.status, &s_abort)) return false;
            fm_tc_fence_after();
            const uint32_t base = smem0 + (uint32_t)s * kFzStageBytes;
            for (int k = 0; k < 3; ++k) {
                if (pend[k]) {
                    if (!fm_mbar_wait(&mide_bar[k], mcnt[k] & 1u, args.status, &s_abort)) return false;
                    fm_tc_fence_after();
                    ++mcnt[k];
                    pend[k] = false;
                }
                const uint32_t a = base + (uint32_t)k * kFzPlane;
                const uint32_t b = base + (uint32_t)(3 + k) * kFzPlane;
#pragma unroll
                for (int ks = 0; ks < kBK / 16; ++ks)
                    fm_mma_f16(tmem + (uint32_t)(k * kFzBN), fm_smem_desc_sw128(a + ks * 32),
                               fm_smem_desc_sw128(b + ks * 32), id, (st > 0 || ks > 0) ? 1u : 0u);
                if ((st + 1) % args.cs[k] == 0 && st + 1 < nst) {
                    fm_mma_commit(&midf_bar[k]);
                    pend[k] = true;
                }
            }
            fm_mma_commit(&empty_bar[s]);
            if (st + 1 == nst) {
                fm_mma_commit(&endf_bar);
                ++tcount;
            }
            return true;
        };
        const bool mma_thread = warp == 0 && lane == 0;

        // one call site each for the tile setup and the stage loads: the first
        // pass only loads stage 0, every later pass splits the loaded stage,
        // starts the next stage's loads and stores the split one
        uint32_t g = 0;
        bool first = true;
        while (true) {
            uint32_t w[32];
            const int cur_kb = kb, cur_KB = KB;  // the loaded stage, before advancing
            const uint32_t cur_idesc = idesc;
            if (!first) {
                // split the loaded stage into packed s pairs (zero outside the sub-matrix)
                const bool a_full = ak_ok == 0xFFu, b_full = bcol_ok == 0xFu;
#pragma unroll
                for (int it = 0; it < 4; ++it)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint32_t x0 = elem(xa[it][j >> 1], (2 * j) & 3);
                        uint32_t x1 = elem(xa[it][j >> 1], (2 * j + 1) & 3);
                        if (!a_full) {
                            x0 = ((ak_ok >> (2 * j)) & 1u) ? x0 : 0u;
                            x1 = ((ak_ok >> (2 * j + 1)) & 1u) ? x1 : 0u;
                        }
                        w[it * 4 + j] = pack_s(x0, x1, p);
                    }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint32_t x0 = elem(xb[2 * j], q), x1 = elem(xb[2 * j + 1], q);
                        if (!b_full && !((bcol_ok >> q) & 1u)) x0 = x1 = 0u;
                        w[16 + q * 4 + j] = pack_s(x0, x1, p);
                    }
            }
            // next stage: its loads fly while this one is stored
            bool fresh = first;
            if (!first && ++kb >= KB) {
                kb = 0;
                tile += gridDim.x;
                fresh = true;
            }
            const bool more = tile < args.n_tiles;
            if (more) {
                if (fresh) setup_tile();
                load_stage();
            }
            if (first) {
                first = false;
                if (!more) break;
                continue;
            }

            const int s = g & 1;
            if (!warp_wait(&empty_bar[s], ((g >> 1) & 1u) ^ 1u, args.status, &s_abort)) break;
            const uint32_t base = smem0 + (uint32_t)s * kFzStageBytes;
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const uint32_t wa[4] = {w[it * 4], w[it * 4 + 1], w[it * 4 + 2], w[it * 4 + 3]};
                store_chunk(base, sw128((uint32_t)(arow0 + 32 * it), (uint32_t)kca), wa);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t wb[4] = {w[16 + q * 4], w[16 + q * 4 + 1], w[16 + q * 4 + 2], w[16 + q * 4 + 3]};
                store_chunk(base + 3 * kFzPlane, sw128((uint32_t)(n0 + q), (uint32_t)kcb), wb);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) fm_mbar_arrive(&full_bar[s]);
            if (mma_thread && !issue(g, cur_kb, cur_KB, cur_idesc)) s_abort = 1;
            __syncwarp();
            ++g;
            if (!more || __any_sync(0xffffffffu, s_abort != 0)) break;
        }
        if (mma_thread) {
            // every MMA issued has completed before TMEM is freed
            fm_mma_commit(&done_bar);
            fm_mbar_wait(&done_bar, 0, args.status, nullptr);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, all 128 columns ----
        const int quarter = warp & 3;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const uint32_t slot3 = tmem + lane_base + 3u * kFzBN;
        uint32_t tcount = 0, ecnt[3] = {0, 0, 0};
        bool ok = true;
        for (int tile = blockIdx.x; tile < args.n_tiles && ok; tile += gridDim.x) {
            const int4 e = args.tiles[tile];
            const CView c = c_view(args.calls[e.x]);
            const int KB = args.calls[e.x].KB;
            const int64_t j0 = (int64_t)e.z * kFzBN;  // sub-matrix column of TMEM column 0
            const int64_t cols = c.N - j0 < kFzBN ? c.N - j0 : kFzBN;
            const int n32 = (int)((cols + 31) / 32);
            const int64_t gi = (int64_t)e.y * kBM + quarter * 32 + lane;
            const bool row_ok = gi < c.M;
            if (c.op != FM_OP_SET && row_ok) prefetch_c_row(c, gi, j0, cols);
            // exact-chunk boundaries inside the tile: fold product k in place
            for (int st = 0; st + 1 < KB && ok; ++st)
                for (int k = 0; k < 3; ++k) {
                    if ((st + 1) % args.cs[k] != 0) continue;
                    if (!warp_wait(&midf_bar[k], ecnt[k] & 1u, args.status, &s_abort)) {
                        ok = false;
                        break;
                    }
                    fm_tc_fence_after();
                    ++ecnt[k];
                    const uint32_t acc = tmem + lane_base + (uint32_t)(k * kFzBN);
#pragma unroll 1
                    for (int cc = 0; cc < n32; ++cc) {
                        uint32_t v[32];
                        fm_tmem_ld32(acc + cc * 32, v);
                        fm_tmem_wait_ld();
                        fold_fp(v, args.invp, args.pf);
                        fm_tmem_st32(acc + cc * 32, v);
                    }
                    fm_tmem_wait_st();
                    fm_tc_fence_before();
                    __syncwarp();
                    if (lane == 0) fm_mbar_arrive(&mide_bar[k]);
                }
            if (!ok) break;
            if (!warp_wait(&endf_bar, tcount & 1u, args.status, &s_abort)) break;
            fm_tc_fence_after();
            ++tcount;
            // residue of the three products, into slot 3; the accumulators are then free
#pragma unroll 1
            for (int cc = 0; cc < n32; ++cc) {
                uint32_t v0[32], v1[32], v2[32];
                fm_tmem_ld32(tmem + lane_base + (uint32_t)cc * 32, v0);
                fm_tmem_ld32(tmem + lane_base + (uint32_t)(kFzBN + cc * 32), v1);
                fm_tmem_ld32(tmem + lane_base + (uint32_t)(2 * kFzBN + cc * 32), v2);
                fm_tmem_wait_ld();
                karatsuba_residue(v0, v1, v2, p, args.invp, args.pf);
                fm_tmem_st32(slot3 + cc * 32, v0);
            }
            fm_tmem_wait_st();
            fm_tc_fence_before();
            __syncwarp();
            if (lane == 0) fm_mbar_arrive(&ende_bar);
            // C update from slot 3 (overlaps the next tile's MMAs)
            const uint64_t cmask = (1ull << c.c_lt) - 1;
#pragma unroll 1
            for (int cc = 0; cc < n32; ++cc) {
                uint32_t r[32];
                fm_tmem_ld32(slot3 + cc * 32, r);
                fm_tmem_wait_ld();
                if (row_ok) write_c_run<32>(c, p, args.mu32, gi, j0 + cc * 32, cmask, r);
            }
        }
    }

    fm_tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        fm_tc_fence_after();
        fm_tmem_dealloc(tmem, 512);
    }
}

}  // namespace

// ---- host -------------------------------------------------------------------
struct FmFusedBatch {
    FusedArgs args;
    FusedCall* d_calls = nullptr;
    int4* d_tiles = nullptr;
};

int fm_fused_batch_create(const fm_gemm_call* calls, int64_t n, uint32_t p, const FmLimbPlan& q,
                          FmFusedBatch** out)
{
    *out = nullptr;
    if (!q.fold || q.n_products != 3 || q.w != 2 || q.block_n != kFzBN) return FM_EUNSUPPORTED;
    std::vector<FusedCall> fc;
    for (int64_t i = 0; i < n; ++i) {
        const fm_gemm_call& g = calls[i];
        if (g.C.rows == 0 || g.C.cols == 0 || g.A.cols == 0) continue;  // K = 0: the caller's
        // T' >= 8 (a stage's 8-row runs of B cross at most one tile row) and
        // operands of at most 2^32 entries (32-bit offsets)
        if (g.A.m.log2_T < 3 || g.B.m.log2_T < 3 || g.A.m.log2_T > 14 || g.B.m.log2_T > 14)
            return FM_EUNSUPPORTED;
        if (g.A.m.log2_grid + g.A.m.log2_T > 16 || g.B.m.log2_grid + g.B.m.log2_T > 16) return FM_EUNSUPPORTED;
        if (((uintptr_t)g.A.m.base & 15) || ((uintptr_t)g.B.m.base & 15)) return FM_EUNSUPPORTED;
        FusedCall c;
        std::memset(&c, 0, sizeof(c));
        c.A = static_cast<const uint32_t*>(g.A.m.base);
        c.B = static_cast<const uint32_t*>(g.B.m.base);
        c.C = static_cast<uint32_t*>(g.C.m.base);
        c.ra = (int)(g.A.col0 & 3);
        c.a_row0 = g.A.row0;
        c.a_col0 = g.A.col0 - c.ra;
        c.b_row0 = g.B.row0;
        c.b_col0 = g.B.col0;
        c.c_row0 = g.C.row0;
        c.c_col0 = g.C.col0;
        c.M = g.C.rows;
        c.N = g.C.cols;
        c.K = g.A.cols;
        c.a_lt = g.A.m.log2_T;
        c.b_lt = g.B.m.log2_T;
        c.c_lt = g.C.m.log2_T;
        c.op = g.op;
        c.KB = (int)((c.K + c.ra + kBK - 1) / kBK);
        c.a_cmask = (0x55555555u << (2 * c.a_lt)) | ((1u << c.a_lt) - 1);
        c.a_c64 = col_part(64, c.a_lt);
        c.b_rmask = (0xAAAAAAAAu << (2 * c.b_lt)) | (((1u << c.b_lt) - 1) << c.b_lt);
        c.b_r64 = row_part(64, c.b_lt);
        fc.push_back(c);
    }
    // longest calls first; a call's tiles stay adjacent, so the CTAs that run
    // them at the same time share its operands in L2
    std::vector<size_t> order(fc.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return fc[x].KB > fc[y].KB; });
    std::vector<FusedCall> sorted;
    std::vector<int4> tiles;
    for (size_t i : order) {
        const FusedCall& c = fc[i];
        const int ci = (int)sorted.size();
        sorted.push_back(c);
        const int64_t MB = (c.M + kBM - 1) / kBM, NB = (c.N + kFzBN - 1) / kFzBN;
        for (int64_t mb = 0; mb < MB; ++mb)
            for (int64_t nb = 0; nb < NB; ++nb) tiles.push_back(make_int4(ci, (int)mb, (int)nb, 0));
    }
    if (tiles.size() > 0x7fffffff) return FM_EINVAL;
    FmFusedBatch* b = new FmFusedBatch();
    std::memset(&b->args, 0, sizeof(b->args));
    auto fail = [&](int rc) {
        fm_fused_batch_destroy(b);
        return rc;
    };
    if (!sorted.empty()) {
        if (cudaMalloc(&b->d_calls, sorted.size() * sizeof(FusedCall)) != cudaSuccess) return fail(FM_ENOMEM);
        if (cudaMemcpy(b->d_calls, sorted.data(), sorted.size() * sizeof(FusedCall), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(FM_ECUDA);
        if (cudaMalloc(&b->d_tiles, tiles.size() * sizeof(int4)) != cudaSuccess) return fail(FM_ENOMEM);
        if (cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(FM_ECUDA);
    }
    FusedArgs& a = b->args;
    a.calls = b->d_calls;
    a.tiles = b->d_tiles;
    a.n_tiles = (int)tiles.size();
    for (int k = 0; k < 3; ++k) a.cs[k] = q.prod_cs[k];
    a.p = p;
    a.mu32 = (uint32_t)(((uint64_t)1 << 32) / p);
    a.invp = 1.0f / (float)p;
    a.pf = (float)p;
    *out = b;
    return FM_OK;
}

int fm_fused_batch_run(FmFusedBatch* b, int* status, cudaStream_t s)
{
    if (b->args.n_tiles == 0) return FM_OK;
    FusedArgs a = b->args;
    a.status = status;
    FM_CUDA_TRY(cudaFuncSetAttribute(limb_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFzSmem));
    const int grid = std::min(a.n_tiles, fm_sm_count());
    limb_fused_kernel<<<grid, kFzThreads, kFzSmem, s>>>(a);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

int64_t fm_fused_batch_tiles(const FmFusedBatch* b)
{
    return b ? b->args.n_tiles : 0;
}

void fm_fused_batch_destroy(FmFusedBatch* b)
{
    if (!b) return;
    cudaFree(b->d_calls);
    cudaFree(b->d_tiles);
    delete b;
}
