// limb_drain.cuh -- exact FP32 drains of tensor-memory accumulators and the
// write of final residues into a Morton-hybrid C, shared by the limb GEMM
// kernels. A call type passed to write_c_run / prefetch_c_row has the fields
// C, c_lt, c_row0, c_col0, N and op of its C sub-matrix.
#pragma once

#include <stdint.h>

#include "fm_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t barrett32(uint32_t x, uint32_t p, uint32_t mu)
{
    const uint32_t q = __umulhi(x, mu);
    uint32_t r = x - q * p;
    return r >= p ? r - p : r;
}

__device__ __forceinline__ uint32_t op_combine(uint32_t c, uint32_t s, uint32_t p, uint32_t mu32, int op)
{
    if (op == FM_OP_SET) return s;
    const uint32_t cc = barrett32(c, p, mu32);  // C holds residues; any 32-bit value is reduced
    if (op == FM_OP_ADD) {
        const uint32_t r = cc + s;
        return r >= p ? r - p : r;
    }
    return cc >= s ? cc - s : cc + (p - s);
}

// Fold-form drains. Every accumulator value v is an integer with |v| <= 2^24
// and |v / p| < 2^22: for p > 4 because |v| <= 2^24, for p <= 4 because the
// limbs are then below p in magnitude, so |v| <= 960 p^2 + 2p. In that range
// round-to-nearest of v / p is one FMA with the constant 1.5 * 2^23 (the sum
// lands where the float spacing is 1) and one subtraction, both on the FMA
// pipe; conversions between small integers and floats use the same bias.
// fold_fp: v - q p with q = the rounded quotient (within 3/4 of v / p, as 1/p
// is rounded), exact, a carried value of magnitude <= 3p/4 < p.
// fold_int: that value times mul mod p, as a float to carry on (to_float) or
// as the final residue in [0, p).
constexpr float kRoundBias = 12582912.0f;  // 1.5 * 2^23
constexpr uint32_t kRoundBiasBits = 0x4B400000u;

// Packed FP32 helpers (fma/sub/mul .f32x2): two lanes per instruction, each
// rounded as the scalar FP32 operation. f2_fold: x - round(x / p) p per lane.
__device__ __forceinline__ uint64_t f2_fold(uint64_t x, uint64_t ip, uint64_t bs, uint64_t np)
{
    uint64_t r;
    asm("{\n\t.reg .b64 t, q;\n\t"
        "fma.rn.f32x2 t, %1, %2, %3;\n\t"
        "sub.rn.f32x2 q, t, %3;\n\t"
        "fma.rn.f32x2 %0, q, %4, %1;\n\t}"
        : "=l"(r)
        : "l"(x), "l"(ip), "l"(bs), "l"(np));
    return r;
}

__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ uint64_t f2_splat(float f)
{
    return (uint64_t)__float_as_uint(f) * 0x100000001ull;
}

// The same-product drain is the drain that runs most often (the Karatsuba
// middle product's 256-deep chunks): like every drain it uses Blackwell's
// packed FP32 arithmetic, two accumulator values per instruction, which halves
// its instruction issue.
__device__ __forceinline__ void fold_fp(uint32_t (&v)[32], float invp, float pf)
{
    const uint64_t ip = f2_splat(invp), bs = f2_splat(kRoundBias), np = f2_splat(-pf);
#pragma unroll
    for (int e = 0; e < 32; e += 2) {
        const uint64_t x = f2_fold(((uint64_t)v[e + 1] << 32) | v[e], ip, bs, np);
        v[e] = (uint32_t)x;
        v[e + 1] = (uint32_t)(x >> 32);
    }
}

// Product-boundary and final drains: x = v folded (|x| <= 3p/4, since the
// rounded quotient is off by at most 3/4), then x * mul mod p in exact FP32
// steps with mul = 256 c1 + c0 (c0, c1 < 256): x c0 and x c1 are below 2^24 in
// magnitude and are folded, and r0 + 256 r1 (at most 257 * 3p/4 < 2^24) is
// folded once more. The result, a value in (-p, p), is carried on as a float
// (to_float) or converted to the residue in [0, p) through the same bias.
__device__ __forceinline__ void fold_int(uint32_t (&v)[32], uint32_t mul, bool to_float, uint32_t p,
                                         float invp, float pf)
{
    const uint64_t ip = f2_splat(invp), bs = f2_splat(kRoundBias), np = f2_splat(-pf);
    const uint64_t c0 = f2_splat((float)(mul & 255u)), c1 = f2_splat((float)(mul >> 8));
    const uint64_t k256 = f2_splat(256.0f);
#pragma unroll
    for (int e = 0; e < 32; e += 2) {
        uint64_t x = ((uint64_t)v[e + 1] << 32) | v[e];
        x = f2_fold(x, ip, bs, np);
        const uint64_t r0 = f2_fold(f2_mul(x, c0), ip, bs, np);
        const uint64_t r1 = f2_fold(f2_mul(x, c1), ip, bs, np);
        const uint64_t y = f2_fold(f2_fma(r1, k256, r0), ip, bs, np);
        uint32_t y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
        if (!to_float) {
            int32_t a = (int32_t)(__float_as_uint(__fadd_rn(__uint_as_float(y0), kRoundBias)) - kRoundBiasBits);
            int32_t b = (int32_t)(__float_as_uint(__fadd_rn(__uint_as_float(y1), kRoundBias)) - kRoundBiasBits);
            y0 = (uint32_t)(a + (a < 0 ? (int32_t)p : 0));
            y1 = (uint32_t)(b + (b < 0 ? (int32_t)p : 0));
        }
        v[e] = y0;
        v[e + 1] = y1;
    }
}

// The C sub-matrix of a call, held by value. Call tables of batches live in
// global memory; an epilogue that read their fields through a reference
// between its stores to C would have each field fetched again after every
// store (the compiler cannot rule out that a store to C changed it).
struct CView {
    uint32_t* C;
    int64_t c_row0, c_col0, M, N;
    int c_lt, op;
};

template <class Call>
__device__ __forceinline__ CView c_view(const Call& c)
{
    return CView{c.C, c.c_row0, c.c_col0, c.M, c.N, c.c_lt, c.op};
}

// C(gi, j0 .. j0+W-1) <- C op sres (mod p), in the Morton-hybrid layout, for the
// columns j in [0, N) of the sub-matrix (j0 may be negative). Loads are issued
// before stores; a run inside one tile row moves as 16-byte vectors.
template <int W, class Call>
__device__ __forceinline__ void write_c_run(const Call& c, uint32_t p, uint32_t mu32, int64_t gi, int64_t j0,
                                            uint64_t cmask, const uint32_t (&sres)[W])
{
    const uint64_t ci = (uint64_t)(c.c_row0 + gi);
    const uint64_t cj0 = (uint64_t)(c.c_col0 + j0);
    const uint64_t base = fm_encode(ci, cj0, c.c_lt);
    const bool run = j0 >= 0 && j0 + W <= c.N && (cj0 & cmask) + W <= cmask + 1 && (base & 3) == 0;
    if (run) {
        uint4* dst = reinterpret_cast<uint4*>(c.C + base);
        uint4 old[W / 4];
        if (c.op != FM_OP_SET) {
#pragma unroll
            for (int q = 0; q < W / 4; ++q) old[q] = dst[q];
        }
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            uint4 o = c.op != FM_OP_SET ? old[q] : make_uint4(0, 0, 0, 0);
            o.x = op_combine(o.x, sres[4 * q + 0], p, mu32, c.op);
            o.y = op_combine(o.y, sres[4 * q + 1], p, mu32, c.op);
            o.z = op_combine(o.z, sres[4 * q + 2], p, mu32, c.op);
            o.w = op_combine(o.w, sres[4 * q + 3], p, mu32, c.op);
            dst[q] = o;
        }
        return;
    }
    // ragged edge or a tile boundary inside the run: groups of 8, loads then
    // stores (a group's stores keep the next group's loads from being hoisted,
    // which bounds the live registers)
#pragma unroll
    for (int g = 0; g < W; g += 8) {
        uint32_t old[8];
        uint64_t a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            a[e] = fm_encode(ci, cj0 + g + e, c.c_lt);
            const int64_t j = j0 + g + e;
            old[e] = (c.op != FM_OP_SET && j >= 0 && j < c.N) ? c.C[a[e]] : 0u;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (j0 + g + e >= 0 && j0 + g + e < c.N)
                c.C[a[e]] = op_combine(old[e], sres[g + e], p, mu32, c.op);
    }
}

// Prefetch into L2 the C entries of row gi, columns j0 .. j0+n-1 (n > 0): one
// request per 128-byte line of each run that is contiguous in the
// Morton-hybrid layout (a tile row).
template <class Call>
__device__ __forceinline__ void prefetch_c_row(const Call& c, int64_t gi, int64_t j0, int64_t n)
{
    const int lt = c.c_lt;
    const int64_t T = (int64_t)1 << lt;
    const uint64_t ci = (uint64_t)(c.c_row0 + gi);
    int64_t j = c.c_col0 + j0;
    const int64_t end = j + n;
    while (j < end) {
        const int64_t run = min(end, (j | (T - 1)) + 1) - j;
        const uint32_t* a = c.C + fm_encode(ci, (uint64_t)j, lt);
        const uintptr_t lo = (uintptr_t)a & ~(uintptr_t)127, hi = (uintptr_t)(a + run);
        for (uintptr_t q = lo; q < hi; q += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
        j += run;
    }
}

}  // namespace
