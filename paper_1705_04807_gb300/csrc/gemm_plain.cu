// gemm_plain.cu -- base-case modular GEMM on the CUDA cores (Sec. 2.1-2.2).
//
// One CTA computes one output part (a contained piece of C inside one T' x T'
// tile) of C <- C op A*B mod p. For every inner-index piece it stages the
// whole tiles of A and B that the piece touches -- each one a contiguous
// T'^2 block of the Morton-hybrid array, thanks to the aligned/contained
// decomposition (Prop. of Sec. 2.1) -- with one 1-D bulk copy (TMA) per tile
// into shared memory, in a ring of kPlainStages<T'> stages on mbarriers (four
// of 16 KB at T' = 32, two of 64 KB at T' = 64). Inside a staged tile the
// element (u, v) is at u*T' + v (Sec. 2.1, P2), so the inner loop is a plain
// row-major product.
//
// Arithmetic (delayed reduction, reduce once per output):
//   narrow: residues < 2^32, accumulate a*b in 64 bits when K*(p-1)^2 < 2^64;
//   wide:   96-bit carry-chain accumulation for any p < 2^31;
//   dfma:   FP64 fused multiply-add, exact while K*(p-1)^2 < 2^53.
#include "fm_internal.cuh"
#include "fm_sched.h"
#include "fm_kernels.h"

namespace {

struct AccNarrow {
    uint64_t v;
    __device__ __forceinline__ void zero() { v = 0; }
    __device__ __forceinline__ void mac(uint32_t a, uint32_t b) { v += (uint64_t)a * b; }
    __device__ __forceinline__ uint32_t mod(uint32_t p) const { return (uint32_t)(v % p); }
};

struct AccWide {
    uint32_t l0, l1, h;
    __device__ __forceinline__ void zero() { l0 = l1 = h = 0; }
    __device__ __forceinline__ void mac(uint32_t a, uint32_t b)
    {
        asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
            "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(l0), "+r"(l1), "+r"(h)
            : "r"(a), "r"(b));
    }
    __device__ __forceinline__ uint32_t mod(uint32_t p) const
    {
        // value = h * 2^64 + (l1 * 2^32 + l0)
        const uint64_t lo = ((uint64_t)l1 << 32) | l0;
        const uint64_t two64 = (uint64_t)((~0ull) % p + 1) % p;  // 2^64 mod p
        const uint64_t hv = ((uint64_t)(h % p) * two64) % p;
        return (uint32_t)((hv + lo % p) % p);
    }
};

struct AccDfma {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void mac(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ uint32_t mod(uint32_t p) const
    {
        return (uint32_t)((unsigned long long)v % p);
    }
};

template <int ARITH>
struct Traits;
template <>
struct Traits<kArithNarrow> {
    using Acc = AccNarrow;
    using Val = uint32_t;
    __device__ __forceinline__ static Val cvt(uint32_t x) { return x; }
};
template <>
struct Traits<kArithWide> {
    using Acc = AccWide;
    using Val = uint32_t;
    __device__ __forceinline__ static Val cvt(uint32_t x) { return x; }
};
template <>
struct Traits<kArithDfma> {
    using Acc = AccDfma;
    using Val = double;
    __device__ __forceinline__ static Val cvt(uint32_t x) { return (double)x; }
};

__device__ __forceinline__ uint32_t combine(uint32_t c, uint32_t s, uint32_t p, int op)
{
    if (op == FM_OP_SET) return s;
    const uint32_t cc = c % p;
    if (op == FM_OP_ADD) {
        const uint32_t r = cc + s;  // < 2^32 since both < 2^31
        return r >= p ? r - p : r;
    }
    return cc >= s ? cc - s : cc + (p - s);
}

// Stages of the copy ring: at T' = 32 a stage (up to four tiles) is 16 KB, so
// four fit in 64 KB and keep three pieces' copies in flight behind the one
// being multiplied; at T' = 64 two stages already take 128 KB.
template <int LT>
__host__ __device__ constexpr int plain_stages()
{
    return LT == 5 ? 4 : 2;
}

// Output rows per warp: a CTA has T' / rows_per_warp warps. Each integer
// multiply-add's 64-bit accumulation waits on the previous one into the same
// accumulator; four rows a warp (instead of eight) doubles the warps per SM
// sub-partition that hide that latency, for more shared-memory loads per
// multiply-add. The FP64 form is bound by its pipe and keeps eight (four
// measured 9 % slower there).
template <int ARITH>
__host__ __device__ constexpr int rows_per_warp()
{
    return ARITH == kArithDfma ? 8 : 4;
}

template <int LT, int ARITH>
__host__ __device__ constexpr int plain_threads()
{
    return (1 << LT) / rows_per_warp<ARITH>() * 32;
}

template <int LT, int ARITH>
__global__ void __launch_bounds__(plain_threads<LT, ARITH>())
    plain_kernel(const FmCallDesc* __restrict__ calls, const FmWorkItem* __restrict__ items,
                 const FmLPiece* __restrict__ lps, int64_t n_items, uint32_t p, int* queue,
                 int* status)
{
    using Acc = typename Traits<ARITH>::Acc;
    using Val = typename Traits<ARITH>::Val;
    constexpr int T = 1 << LT;
    constexpr int TE = T * T;             // elements per tile
    constexpr int RPW = rows_per_warp<ARITH>();  // output rows per warp
    constexpr int CPL = T / 32;           // output columns per lane
    constexpr uint32_t kTileBytes = TE * 4;
    constexpr int S = plain_stages<LT>();

    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint32_t* tiles = reinterpret_cast<uint32_t*>(smem_raw);  // [S stages][4 tiles][TE]
    __shared__ __align__(8) uint64_t full[S];
    __shared__ int s_item;
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) fm_mbar_init(&full[s], 1);
        fm_fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    uint32_t g = 0;  // stages consumed so far by this CTA (same in every thread)
    int64_t next = blockIdx.x;
    while (true) {
        if (queue) {
            if (tid == 0) s_item = atomicAdd(queue, 1);
            __syncthreads();
            next = s_item;
        }
        if (next >= n_items || s_abort) break;
        const FmWorkItem w = items[next];
        const FmCallDesc cd = calls[w.call];
        const int n = cd.lp_count;
        const bool a2 = w.a_split < w.rows, b2 = w.b_split < w.cols;

        auto issue = [&](int q, uint32_t buf) {
            const FmLPiece lp = lps[cd.lp_begin + q];
            uint32_t* st = tiles + (size_t)buf * 4 * TE;
            const uint32_t bytes = kTileBytes * (2 + (a2 ? 1 : 0) + (b2 ? 1 : 0));
            fm_mbar_arrive_expect_tx(&full[buf], bytes);
            fm_bulk_g2s(st, cd.A + fm_tile_base(w.a_ti, lp.a_tj, LT), kTileBytes, &full[buf]);
            if (a2)
                fm_bulk_g2s(st + TE, cd.A + fm_tile_base(w.a_ti + 1, lp.a_tj, LT), kTileBytes,
                            &full[buf]);
            fm_bulk_g2s(st + 2 * TE, cd.B + fm_tile_base(lp.b_ti, w.b_tj, LT), kTileBytes,
                        &full[buf]);
            if (b2)
                fm_bulk_g2s(st + 3 * TE, cd.B + fm_tile_base(lp.b_ti, w.b_tj + 1, LT), kTileBytes,
                            &full[buf]);
        };

        if (tid == 0)
            for (int q = 0; q < n && q < S; ++q) issue(q, (g + q) % S);

        // my rows and columns inside the output part
        int my_r[RPW], my_c[CPL];
#pragma unroll
        for (int r = 0; r < RPW; ++r) my_r[r] = warp * RPW + r;
#pragma unroll
        for (int c = 0; c < CPL; ++c) my_c[c] = lane + 32 * c;

        Acc acc[RPW][CPL];
#pragma unroll
        for (int r = 0; r < RPW; ++r)
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[r][c].zero();

        for (int q = 0; q < n; ++q) {
            const uint32_t gq = g + q;
            const uint32_t buf = gq % S;
            if (!fm_mbar_wait(&full[buf], (gq / S) & 1, status, &s_abort)) break;
            const FmLPiece lp = lps[cd.lp_begin + q];
            const uint32_t* st = tiles + (size_t)buf * 4 * TE;
            // row pointers into A, column pointers into B (clamped for idle lanes)
            const uint32_t* arow[RPW];
            const uint32_t* bcol[CPL];
#pragma unroll
            for (int r = 0; r < RPW; ++r) {
                const int x = my_r[r] < w.rows ? my_r[r] : 0;
                const int tr = w.a_r + x;  // in-tile row, continues into the next tile
                arow[r] = (x < w.a_split ? st + (size_t)tr * T : st + TE + (size_t)(tr - T) * T) +
                          lp.a_c;
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int y = my_c[c] < w.cols ? my_c[c] : 0;
                const int tc = w.b_c + y;
                bcol[c] = (y < w.b_split ? st + 2 * TE + tc : st + 3 * TE + (tc - T)) +
                          (size_t)lp.b_r * T;
            }
            const int len = lp.len;
            if ((lp.a_c & 3) == 0) {
                int l = 0;
                for (; l + 4 <= len; l += 4) {
                    uint4 a4[RPW];
#pragma unroll
                    for (int r = 0; r < RPW; ++r) a4[r] = *reinterpret_cast<const uint4*>(arow[r] + l);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        Val b[CPL];
#pragma unroll
                        for (int c = 0; c < CPL; ++c) b[c] = Traits<ARITH>::cvt(bcol[c][(l + k) * T]);
#pragma unroll
                        for (int r = 0; r < RPW; ++r) {
                            const uint32_t av =
                                k == 0 ? a4[r].x : (k == 1 ? a4[r].y : (k == 2 ? a4[r].z : a4[r].w));
                            const Val a = Traits<ARITH>::cvt(av);
#pragma unroll
                            for (int c = 0; c < CPL; ++c) acc[r][c].mac(a, b[c]);
                        }
                    }
                }
                for (; l < len; ++l) {
                    Val b[CPL];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) b[c] = Traits<ARITH>::cvt(bcol[c][l * T]);
#pragma unroll
                    for (int r = 0; r < RPW; ++r) {
                        const Val a = Traits<ARITH>::cvt(arow[r][l]);
#pragma unroll
                        for (int c = 0; c < CPL; ++c) acc[r][c].mac(a, b[c]);
                    }
                }
            } else {
                for (int l = 0; l < len; ++l) {
                    Val b[CPL];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) b[c] = Traits<ARITH>::cvt(bcol[c][l * T]);
#pragma unroll
                    for (int r = 0; r < RPW; ++r) {
                        const Val a = Traits<ARITH>::cvt(arow[r][l]);
#pragma unroll
                        for (int c = 0; c < CPL; ++c) acc[r][c].mac(a, b[c]);
                    }
                }
            }
            __syncthreads();  // every thread is done with this buffer
            if (tid == 0 && q + S < n) issue(q + S, buf);
        }
        if (s_abort) {
            // let copies still in flight land before the CTA exits
            if (tid == 0)
                for (int q = 0; q < n && q < S; ++q)
                    fm_mbar_wait(&full[(g + q) % S], ((g + q) / S) & 1, status, nullptr);
            break;
        }
        g += n;

        // epilogue: reduce once, combine with C, write the contained part
        uint32_t* cbase = cd.C + fm_tile_base(w.c_ti, w.c_tj, LT);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            if (my_r[r] >= w.rows) continue;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                if (my_c[c] >= w.cols) continue;
                uint32_t* dst = cbase + (size_t)(w.c_r + my_r[r]) * T + (w.c_c + my_c[c]);
                const uint32_t s = acc[r][c].mod(p);
                const uint32_t old = cd.op == FM_OP_SET ? 0u : *dst;
                *dst = combine(old, s, p, cd.op);
            }
        }
        if (!queue) break;
        __syncthreads();
    }
}

template <int LT, int ARITH>
int launch_t(const FmCallDesc* calls, const FmWorkItem* items, const FmLPiece* lps,
             int64_t n_items, uint32_t p, int* queue, int grid, int* status, cudaStream_t s)
{
    constexpr int T = 1 << LT;
    const size_t smem = (size_t)plain_stages<LT>() * 4 * T * T * 4;
    auto k = plain_kernel<LT, ARITH>;
    FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, plain_threads<LT, ARITH>(), smem, s>>>(calls, items, lps, n_items, p, queue, status);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

}  // namespace

int fm_plain_launch(int lt, int arith, const FmCallDesc* calls, const FmWorkItem* items,
                    const FmLPiece* lps, int64_t n_items, uint32_t p, int* queue, int grid,
                    int* status, cudaStream_t s)
{
    if (n_items <= 0) return FM_OK;
#define FM_CASE(L, A) \
    if (lt == L && arith == A) return launch_t<L, A>(calls, items, lps, n_items, p, queue, grid, status, s);
    FM_CASE(5, kArithNarrow)
    FM_CASE(5, kArithWide)
    FM_CASE(5, kArithDfma)
    FM_CASE(6, kArithNarrow)
    FM_CASE(6, kArithWide)
    FM_CASE(6, kArithDfma)
#undef FM_CASE
    return FM_EUNSUPPORTED;
}

int fm_plain_occupancy(int lt, int arith)
{
    int blocks = 1;
    const int T = 1 << lt;
    const size_t smem = (size_t)(lt == 5 ? plain_stages<5>() : plain_stages<6>()) * 4 * T * T * 4;
#define FM_OCC(L, A)                                                                             \
    if (lt == L && arith == A) {                                                                 \
        cudaFuncSetAttribute(plain_kernel<L, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                             (int)smem);                                                         \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, plain_kernel<L, A>, plain_threads<L, A>(), smem); \
    }
    FM_OCC(5, kArithNarrow)
    FM_OCC(5, kArithWide)
    FM_OCC(5, kArithDfma)
    FM_OCC(6, kArithNarrow)
    FM_OCC(6, kArithWide)
    FM_OCC(6, kArithDfma)
#undef FM_OCC
    return blocks > 0 ? blocks : 1;
}
