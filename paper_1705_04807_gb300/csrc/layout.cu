// layout.cu -- row-major <-> Morton-hybrid conversion and permutations.
//
// Sec. 1: matrices live in the Morton-hybrid layout (Z-order over T' x T'
// row-major tiles); TURBO needs row and column permutations, which require
// index conversion between the curve and Cartesian order. These kernels are
// HBM-bound gathers: each CTA walks whole tiles of the Morton matrix, so the
// Morton side is read or written as contiguous 16-byte vectors and the
// row-major side in row segments of T' elements. The row-major side holds
// 32-bit entries, or 16-bit ones (residues mod p < 2^16: half the bytes to
// move, e.g. across the host link); the Morton-hybrid side is always 32-bit.
// The same kernels also lay the tiles along the Hilbert curve instead of the
// Z curve (the Hilbert-hybrid variant, for comparing the curves' index
// conversion cost).
#include <algorithm>

#include "fm_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Four consecutive row-major entries starting at p (4-entry aligned).
__device__ __forceinline__ uint4 ld4(const uint32_t* p)
{
    return __ldg(reinterpret_cast<const uint4*>(p));
}

__device__ __forceinline__ uint4 ld4(const uint16_t* p)
{
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    return make_uint4(v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16);
}

__device__ __forceinline__ void st4(uint32_t* p, uint4 v)
{
    *reinterpret_cast<uint4*>(p) = v;
}

// 16-bit destination: the low 16 bits of every entry
__device__ __forceinline__ void st4(uint16_t* p, uint4 v)
{
    *reinterpret_cast<uint2*>(p) = make_uint2((v.x & 0xFFFFu) | (v.y << 16), (v.z & 0xFFFFu) | (v.w << 16));
}

// byte alignment of a 4-entry vector of T
template <typename T>
constexpr uintptr_t kVec4Align = 4 * sizeof(T) - 1;

// The curve the tiles follow: the Z curve (Morton-hybrid) or the Hilbert
// curve (Hilbert-hybrid); tiles are T' x T' row-major in both.
enum { kMorton = 0, kHilbert = 1 };

template <int CURVE>
__device__ __forceinline__ uint64_t curve_tile_base(uint64_t I, uint64_t J, int lg, int lt)
{
    return CURVE == kHilbert ? fm_hilbert_tile(I, J, lg) << (2 * lt) : fm_tile_base(I, J, lt);
}

template <int CURVE>
__device__ __forceinline__ uint64_t curve_encode(uint64_t i, uint64_t j, int lg, int lt)
{
    return CURVE == kHilbert ? fm_hilbert_encode(i, j, lg, lt) : fm_encode(i, j, lt);
}

// Offsets of the entries (i, j0), (i, j0 + kStride), (i, j0 + 2 kStride), ...
// of one row of a curve-layout matrix (T' = 2^lt <= 1024 divides kStride, so
// the offset inside a tile row is the same for all of them). On the Z curve the
// tile index advances by dilated-integer addition: the column part of Z(I, J)
// is spread(J) on the even bits, and spread(J + d) = ((spread(J) | odd) +
// spread(d)) & even -- three operations per step instead of a full bit
// interleave. The Hilbert curve recomputes the tile's position.
constexpr uint32_t kStride = 4 * kThreads;
constexpr uint64_t kEvenBits = 0x5555555555555555ull;

template <int CURVE>
struct RowWalk {
    uint64_t rowz, sj, step, off;
    uint64_t I, J, dJ;
    int lg, lt;
    __device__ __forceinline__ RowWalk(uint64_t i, uint64_t j0, int lg_, int lt_) : lg(lg_), lt(lt_)
    {
        const uint64_t t1 = (1ull << lt) - 1;
        off = ((i & t1) << lt) | (j0 & t1);
        I = i >> lt;
        J = j0 >> lt;
        dJ = (uint64_t)kStride >> lt;
        rowz = fm_spread_bits(I) << 1;
        sj = fm_spread_bits(J);
        step = fm_spread_bits(dJ);
    }
    __device__ __forceinline__ uint64_t at() const
    {
        return CURVE == kHilbert ? (fm_hilbert_tile(I, J, lg) << (2 * lt)) | off : ((rowz | sj) << (2 * lt)) | off;
    }
    __device__ __forceinline__ void next()
    {
        if (CURVE == kHilbert)
            J += dJ;
        else
            sj = ((sj | ~kEvenBits) + step) & kEvenBits;
    }
};

// dst(i, j) = src[rp(i) * ld + cp(j)] (0 outside rows x cols), dst Morton.
// A permutation entry outside [0, rows) / [0, cols) is not dereferenced: the
// entries it would fill become 0 and FM_EINVAL is raised in *status.
template <bool kPerm, typename T, int CURVE = kMorton>
__global__ void __launch_bounds__(kThreads) to_morton_kernel(const T* __restrict__ src,
                                                             int64_t rows, int64_t cols, int64_t ld,
                                                             const int32_t* __restrict__ rp,
                                                             const int32_t* __restrict__ cp,
                                                             uint32_t* __restrict__ dst, int lg,
                                                             int lt, int* status)
{
    const int64_t tiles = (int64_t)1 << (2 * lg);
    const int64_t tile_elems = (int64_t)1 << (2 * lt);
    // 16-byte row segments whenever no column permutation scatters them
    const bool vec_ok = (!kPerm || cp == nullptr) && lt >= 2 && ((ld & 3) == 0) &&
                        (((uintptr_t)src & kVec4Align<T>) == 0);
    bool bad = false;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // Walking the tiles in the curve's own order (Z or Hilbert) keeps the
        // destination writes sequential; with a permutation the reads are a
        // random gather inside each source row, so tiles are walked row band
        // by row band to keep one band of source rows in L2.
        uint64_t I, J;
        uint32_t* tile;
        if (kPerm) {
            I = (uint64_t)t >> lg;
            J = (uint64_t)t & ((1ull << lg) - 1);
            tile = dst + curve_tile_base<CURVE>(I, J, lg, lt);
        } else {
            if (CURVE == kHilbert) {
                fm_hilbert_cell((uint64_t)t, lg, &I, &J);
            } else {
                I = fm_compact_bits((uint64_t)t >> 1);
                J = fm_compact_bits((uint64_t)t);
            }
            tile = dst + ((uint64_t)t << (2 * lt));
        }
        const int64_t i_base = (int64_t)I << lt, j_base = (int64_t)J << lt;
        if (lt >= 2) {
            for (int64_t e = 4 * (int64_t)threadIdx.x; e < tile_elems; e += 4 * kThreads) {
                const int64_t i = i_base + (e >> lt);
                const int64_t j = j_base + (e & ((1 << lt) - 1));
                uint4 v = make_uint4(0, 0, 0, 0);
                int64_t si = i < rows ? i : -1;
                if (kPerm && rp && si >= 0) {
                    si = (int64_t)__ldg(rp + i);
                    if (si < 0 || si >= rows) {
                        bad = true;
                        si = -1;
                    }
                }
                if (si >= 0) {
                    if (vec_ok && j + 3 < cols) {
                        v = ld4(src + si * ld + j);
                    } else {
                        uint32_t w[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int64_t jj = j + q;
                            int64_t sj = jj < cols ? jj : -1;
                            if (kPerm && cp && sj >= 0) {
                                sj = (int64_t)__ldg(cp + jj);
                                if (sj < 0 || sj >= cols) {
                                    bad = true;
                                    sj = -1;
                                }
                            }
                            w[q] = sj >= 0 ? (uint32_t)__ldg(src + si * ld + sj) : 0u;
                        }
                        v = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                *reinterpret_cast<uint4*>(tile + e) = v;
            }
        } else {
            for (int64_t e = threadIdx.x; e < tile_elems; e += kThreads) {
                const int64_t i = i_base + (e >> lt);
                const int64_t j = j_base + (e & ((1 << lt) - 1));
                uint32_t v = 0;
                if (i < rows && j < cols) {
                    const int64_t si = kPerm && rp ? (int64_t)__ldg(rp + i) : i;
                    const int64_t sj = kPerm && cp ? (int64_t)__ldg(cp + j) : j;
                    if (si >= 0 && si < rows && sj >= 0 && sj < cols)
                        v = (uint32_t)__ldg(src + si * ld + sj);
                    else
                        bad = true;
                }
                tile[e] = v;
            }
        }
    }
    if (kPerm && __syncthreads_or(bad) && threadIdx.x == 0) fm_raise(status, FM_EINVAL);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Permuted conversion: dst(i, j) = src[rp(i) * ld + cp(j)] (either permutation
// may be the identity, NULL). Each CTA
// walks destination rows i = blockIdx.x, + gridDim.x, ...: it stages the
// source row rp(i) in shared memory (16-byte asynchronous copies of whole
// vectors, entries past the last whole vector one by one) in its own entry
// type, gathers the permuted columns from shared memory and writes the
// destination row as contiguous runs of T' entries (one per Morton tile it
// crosses), so HBM sees one read and one write per element. With NBUF = 2
// (rows of 16-byte aligned vectors only) the copies of the CTA's next row are
// in flight while it gathers the current one. Out-of-range permutation
// entries are not dereferenced (0 and FM_EINVAL, as above).
template <typename T, int NBUF>
__global__ void __launch_bounds__(kThreads)
    to_morton_rowgather_kernel(const T* __restrict__ src, int64_t rows, int64_t cols,
                               int64_t ld, const int32_t* __restrict__ rp,
                               const int32_t* __restrict__ cp, uint32_t* __restrict__ dst, int lg,
                               int lt, int* status)
{
    extern __shared__ __align__(16) uint8_t sraw[];
    constexpr int kVec = 16 / sizeof(T);  // entries per 16-byte vector
    const int64_t n = (int64_t)1 << (lg + lt);
    const bool vec = ((ld % kVec) == 0) && (((uintptr_t)src & 15) == 0);
    const int64_t cv = vec ? cols / kVec : 0;             // whole vectors of a row
    const int64_t stride = (cols + kVec - 1) / kVec * kVec;  // entries per row buffer
    T* sbuf = reinterpret_cast<T*>(sraw);
    bool bad = false;

    auto source_row = [&](int64_t i) -> int64_t {
        if (i >= rows) return -1;
        const int64_t si = rp ? (int64_t)__ldg(rp + i) : i;
        if (si < 0 || si >= rows) {
            bad = true;
            return -1;
        }
        return si;
    };
    auto fetch = [&](int64_t si, T* row) {
        if (si < 0) return;
        const T* sr = src + si * ld;
        for (int64_t q = threadIdx.x; q < cv; q += kThreads) cp_async16(row + kVec * q, sr + kVec * q);
        for (int64_t j = kVec * cv + threadIdx.x; j < cols; j += kThreads) row[j] = __ldg(sr + j);
    };
    const bool cp_vec = cp != nullptr && (((uintptr_t)cp & 15) == 0);
    const int ncols = (int)cols;
    auto gather = [&](int64_t i, int64_t si, const T* row) {
        RowWalk<kMorton> w_(i, 4 * threadIdx.x, lg, lt);
        for (int j = 4 * (int)threadIdx.x; j < (int)n; j += (int)kStride, w_.next()) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (si >= 0 && j < ncols) {
                int32_t sj[4];
                if (cp_vec && j + 3 < ncols) {
                    const int4 v = __ldg(reinterpret_cast<const int4*>(cp + j));
                    sj[0] = v.x;
                    sj[1] = v.y;
                    sj[2] = v.z;
                    sj[3] = v.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) sj[q] = j + q < ncols ? (cp ? __ldg(cp + j + q) : j + q) : -1;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (j + q < ncols) {
                        if ((unsigned)sj[q] < (unsigned)ncols)
                            w[q] = (uint32_t)row[sj[q]];
                        else
                            bad = true;
                    }
                }
            }
            *reinterpret_cast<uint4*>(dst + w_.at()) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    };

    int64_t i = blockIdx.x;
    int64_t si = i < n ? source_row(i) : -1;
    if (NBUF == 2) {
        fetch(si, sbuf);
        cp_async_commit();
    }
    for (int k = 0; i < n; ++k, i += gridDim.x) {
        T* cur = sbuf + (NBUF == 2 ? (int64_t)(k & 1) * stride : 0);
        int64_t si_next = -1;
        if (NBUF == 2) {
            const int64_t inext = i + gridDim.x;
            si_next = inext < n ? source_row(inext) : -1;
            fetch(si_next, sbuf + (int64_t)((k + 1) & 1) * stride);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            fetch(si, cur);
            cp_async_commit();
            cp_async_wait<0>();
        }
        __syncthreads();
        gather(i, si, cur);
        __syncthreads();
        if (NBUF == 2) si = si_next;
        else if (i + gridDim.x < n) si = source_row(i + gridDim.x);
    }
    cp_async_wait<0>();
    if (__syncthreads_or(bad) && threadIdx.x == 0) fm_raise(status, FM_EINVAL);
}

// dst[i * ld + j] = src(i, j) for i < rows, j < cols, src Morton.
template <typename E, int CURVE = kMorton>
__global__ void __launch_bounds__(kThreads) from_morton_kernel(const uint32_t* __restrict__ src,
                                                               int lg, int lt, int64_t rows,
                                                               int64_t cols, E* __restrict__ dst,
                                                               int64_t ld)
{
    const int64_t tiles_side = (int64_t)1 << lg;
    const int64_t T = (int64_t)1 << lt;
    // only tiles that intersect the rows x cols corner
    const int64_t tr = (rows + T - 1) >> lt, tc = (cols + T - 1) >> lt;
    const int64_t ntiles = tr * tc;
    const int64_t tile_elems = T * T;
    const bool vec_ok = lt >= 2 && ((ld & 3) == 0) && (((uintptr_t)dst & kVec4Align<E>) == 0);
    (void)tiles_side;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t I = t / tc, J = t % tc;
        const uint32_t* tile = src + curve_tile_base<CURVE>((uint64_t)I, (uint64_t)J, lg, lt);
        const int64_t i_base = I << lt, j_base = J << lt;
        if (lt >= 2) {
            for (int64_t e = 4 * (int64_t)threadIdx.x; e < tile_elems; e += 4 * kThreads) {
                const int64_t i = i_base + (e >> lt);
                const int64_t j = j_base + (e & (T - 1));
                if (i >= rows || j >= cols) continue;
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(tile + e));
                if (vec_ok && j + 3 < cols) {
                    st4(dst + i * ld + j, v);
                } else {
                    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j + q < cols) dst[i * ld + j + q] = (E)w[q];
                }
            }
        } else {
            for (int64_t e = threadIdx.x; e < tile_elems; e += kThreads) {
                const int64_t i = i_base + (e >> lt);
                const int64_t j = j_base + (e & (T - 1));
                if (i < rows && j < cols) dst[i * ld + j] = (E)__ldg(tile + e);
            }
        }
    }
}

// dst(i, j) = src(rp[i], cp[j]) for i < rows, j < cols, else 0; both on the
// same curve. Every entry's source index is converted from Cartesian order.
// The general form (any T'); permutations between layouts with T' >= 4 take
// permute_staged_kernel below. Out-of-range permutation entries are not
// dereferenced (0 and FM_EINVAL).
template <int CURVE = kMorton>
__global__ void __launch_bounds__(kThreads) permute_kernel(const uint32_t* __restrict__ src, int lgs,
                                                           int lts, uint32_t* __restrict__ dst,
                                                           int lgd, int ltd, int64_t rows,
                                                           int64_t cols,
                                                           const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ cp, int* status)
{
    const int64_t tiles = (int64_t)1 << (2 * lgd);
    const int64_t tile_elems = (int64_t)1 << (2 * ltd);
    const int64_t Td = (int64_t)1 << ltd;
    bool bad = false;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t I = CURVE == kHilbert ? (uint64_t)t >> lgd : fm_compact_bits((uint64_t)t >> 1);
        const uint64_t J = CURVE == kHilbert ? (uint64_t)t & ((1ull << lgd) - 1) : fm_compact_bits((uint64_t)t);
        uint32_t* tile = dst + curve_tile_base<CURVE>(I, J, lgd, ltd);
        const int64_t i_base = (int64_t)I << ltd, j_base = (int64_t)J << ltd;
        for (int64_t e = threadIdx.x; e < tile_elems; e += kThreads) {
            const int64_t i = i_base + (e >> ltd);
            const int64_t j = j_base + (e & (Td - 1));
            uint32_t v = 0;
            if (i < rows && j < cols) {
                const int64_t si = rp ? (int64_t)__ldg(rp + i) : i;
                const int64_t sj = cp ? (int64_t)__ldg(cp + j) : j;
                if (si >= 0 && si < rows && sj >= 0 && sj < cols)
                    v = __ldg(src + curve_encode<CURVE>((uint64_t)si, (uint64_t)sj, lgs, lts));
                else
                    bad = true;
            }
            tile[e] = v;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) fm_raise(status, FM_EINVAL);
}

// The same permutation, row-staged, for layouts with T' >= 4 on both sides:
// each CTA walks destination rows i = blockIdx.x, + gridDim.x, ... The source
// row rp[i] is copied from the tiles it crosses, runs of T'_src contiguous
// entries, into shared memory by 16-byte asynchronous copies (one curve index
// conversion per vector); the destination row is written as runs of T'_dst
// contiguous entries (16-byte vectors), each entry gathered from shared memory
// through cp. With NBUF = 2 the copies of the CTA's next row are in flight
// while it gathers the current one. HBM sees each entry read once and written
// once in whole 16-byte vectors, against one scattered 4-byte read per entry
// in permute_kernel. The last vector of a source row may read past cols, but
// not past the tile (T'_src is a multiple of 4), and those entries are never
// gathered. Out-of-range permutation entries are not dereferenced (0 and
// FM_EINVAL).
template <int CURVE, int NBUF>
__global__ void __launch_bounds__(kThreads)
    permute_staged_kernel(const uint32_t* __restrict__ src, int lgs, int lts, uint32_t* __restrict__ dst,
                          int lgd, int ltd, int64_t rows, int64_t cols, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ cp, int* status)
{
    extern __shared__ __align__(16) uint32_t sbuf[];
    const int64_t nd = (int64_t)1 << (lgd + ltd);
    const int64_t c4 = (cols + 3) >> 2;
    const bool cp_vec = cp != nullptr && (((uintptr_t)cp & 15) == 0);
    bool bad = false;

    // source row of destination row i, or -1 (a row past rows, or a bad entry)
    auto source_row = [&](int64_t i) -> int64_t {
        if (i >= rows) return -1;
        const int64_t si = rp ? (int64_t)__ldg(rp + i) : i;
        if (si < 0 || si >= rows) {
            bad = true;
            return -1;
        }
        return si;
    };
    const int ncols = (int)cols, c4i = (int)c4;
    auto fetch = [&](int64_t si, uint32_t* row) {
        if (si < 0) return;
        RowWalk<CURVE> w_(si, 4 * threadIdx.x, lgs, lts);
        for (int q = threadIdx.x; q < c4i; q += kThreads, w_.next()) cp_async16(row + 4 * q, src + w_.at());
    };
    auto gather = [&](int64_t i, int64_t si, const uint32_t* row) {
        RowWalk<CURVE> w_(i, 4 * threadIdx.x, lgd, ltd);
        for (int j = 4 * (int)threadIdx.x; j < (int)nd; j += (int)kStride, w_.next()) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (si >= 0 && j < ncols) {
                int32_t sj[4];
                if (cp_vec && j + 3 < ncols) {
                    const int4 v = __ldg(reinterpret_cast<const int4*>(cp + j));
                    sj[0] = v.x;
                    sj[1] = v.y;
                    sj[2] = v.z;
                    sj[3] = v.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        sj[q] = j + q < ncols ? (cp ? __ldg(cp + j + q) : j + q) : -1;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (j + q < ncols) {
                        if ((unsigned)sj[q] < (unsigned)ncols)
                            w[q] = row[sj[q]];
                        else
                            bad = true;
                    }
                }
            }
            *reinterpret_cast<uint4*>(dst + w_.at()) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    };

    int64_t i = blockIdx.x;
    int64_t si = i < nd ? source_row(i) : -1;
    if (NBUF == 2) {
        fetch(si, sbuf);
        cp_async_commit();
    }
    for (int k = 0; i < nd; ++k, i += gridDim.x) {
        uint32_t* cur = sbuf + (NBUF == 2 ? (int64_t)(k & 1) * 4 * c4 : 0);
        int64_t si_next = -1;
        if (NBUF == 2) {
            const int64_t inext = i + gridDim.x;
            si_next = inext < nd ? source_row(inext) : -1;
            fetch(si_next, sbuf + (int64_t)((k + 1) & 1) * 4 * c4);
            cp_async_commit();
            cp_async_wait<1>();  // this thread's copies of the current row have landed
        } else {
            fetch(si, cur);
            cp_async_commit();
            cp_async_wait<0>();
        }
        __syncthreads();
        gather(i, si, cur);
        __syncthreads();  // the buffer is free before the next copies into it
        if (NBUF == 2) si = si_next;
        else if (i + gridDim.x < nd) si = source_row(i + gridDim.x);
    }
    cp_async_wait<0>();
    if (__syncthreads_or(bad) && threadIdx.x == 0) fm_raise(status, FM_EINVAL);
}

// Raises FM_ERANGE in *status when an entry of the rows x cols sub-matrix at
// (row0, col0) of a Morton-hybrid matrix is >= p. One warp per sub-matrix row:
// the row's entries inside one tile row are contiguous, so the lanes read
// consecutive entries.
__global__ void __launch_bounds__(kThreads) validate_kernel(const uint32_t* __restrict__ base, int lt,
                                                            int64_t row0, int64_t col0, int64_t rows,
                                                            int64_t cols, uint32_t p, int* status)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    const int64_t T = (int64_t)1 << lt;
    bool bad = false;
    for (int64_t r = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); r < rows; r += warps) {
        const uint64_t gi = (uint64_t)(row0 + r);
        for (int64_t j = 0; j < cols;) {
            const uint64_t gj = (uint64_t)(col0 + j);
            const int64_t left = T - (int64_t)(gj & (uint64_t)(T - 1));
            const int64_t run = cols - j < left ? cols - j : left;
            const uint32_t* seg = base + fm_encode(gi, gj, lt);
            for (int64_t e = lane; e < run; e += 32) bad |= __ldg(seg + e) >= p;
            j += run;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) fm_raise(status, FM_ERANGE);
}

// Shared memory the row-staged kernels may use: one or two source rows.
constexpr size_t kStagedRowMax = 200 * 1024;

int grid_for(int64_t tiles)
{
    const int64_t cap = (int64_t)fm_sm_count() * 8;
    return (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
}

template <typename T, int CURVE = kMorton>
int to_morton_impl(const T* src, int64_t rows, int64_t cols, int64_t ld, const int32_t* rp,
                   const int32_t* cp, fm_matrix dst, fm_stream stream)
{
    FM_TRY(fm_check_matrix(dst));
    const int64_t n = fm_side(dst);
    if (rows < 0 || cols < 0 || rows > n || cols > n || ld < cols) return FM_EINVAL;
    if ((rows > 0 && cols > 0) && src == nullptr) return FM_EINVAL;
    int* status = nullptr;
    if (rp || cp) {
        status = fm_device_status();
        if (!status) return FM_ECUDA;
    }
    const int64_t tiles = (int64_t)1 << (2 * dst.log2_grid);
    constexpr int kVec = 16 / sizeof(T);
    const size_t row_bytes = (size_t)((cols + kVec - 1) / kVec * kVec) * sizeof(T);
    if (CURVE == kMorton && (rp || cp) && dst.log2_T >= 2 && row_bytes <= kStagedRowMax) {
        // two row buffers (the next row's copies overlap the gather) when the
        // rows are whole 16-byte vectors and two fit, else one
        const bool two = ((ld % kVec) == 0) && (((uintptr_t)src & 15) == 0) && 2 * row_bytes <= kStagedRowMax;
        auto k = two ? to_morton_rowgather_kernel<T, 2> : to_morton_rowgather_kernel<T, 1>;
        const size_t smem = two ? 2 * row_bytes : row_bytes;
        FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedRowMax));
        int per_sm = 0;
        FM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)fm_sm_count() * std::max(1, per_sm)));
        k<<<grid, kThreads, smem, (cudaStream_t)stream>>>(src, rows, cols, ld, rp, cp, dst.base, dst.log2_grid,
                                                         dst.log2_T, status);
    } else if (rp || cp)
        to_morton_kernel<true, T, CURVE><<<grid_for(tiles), kThreads, 0, (cudaStream_t)stream>>>(
            src, rows, cols, ld, rp, cp, dst.base, dst.log2_grid, dst.log2_T, status);
    else
        to_morton_kernel<false, T, CURVE><<<grid_for(tiles), kThreads, 0, (cudaStream_t)stream>>>(
            src, rows, cols, ld, nullptr, nullptr, dst.base, dst.log2_grid, dst.log2_T, nullptr);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

template <typename E, int CURVE = kMorton>
int from_morton_impl(fm_matrix src, int64_t rows, int64_t cols, E* dst, int64_t ld, fm_stream stream)
{
    FM_TRY(fm_check_matrix(src));
    const int64_t n = fm_side(src);
    if (rows < 0 || cols < 0 || rows > n || cols > n || ld < cols) return FM_EINVAL;
    if (rows == 0 || cols == 0) return FM_OK;
    if (dst == nullptr) return FM_EINVAL;
    const int64_t T = (int64_t)1 << src.log2_T;
    const int64_t tiles = ((rows + T - 1) / T) * ((cols + T - 1) / T);
    from_morton_kernel<E, CURVE><<<grid_for(tiles), kThreads, 0, (cudaStream_t)stream>>>(
        src.base, src.log2_grid, src.log2_T, rows, cols, dst, ld);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

}  // namespace

extern "C" int fm_layout_to_morton(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                                   fm_matrix dst, fm_stream stream)
{
    FmRange range("fm_layout_to_morton");
    return to_morton_impl(src, rows, cols, ld, nullptr, nullptr, dst, stream);
}

extern "C" int fm_layout_to_morton_permuted(const uint32_t* src, int64_t rows, int64_t cols,
                                            int64_t ld, const int32_t* row_perm,
                                            const int32_t* col_perm, fm_matrix dst,
                                            fm_stream stream)
{
    FmRange range("fm_layout_to_morton_permuted");
    return to_morton_impl(src, rows, cols, ld, row_perm, col_perm, dst, stream);
}

extern "C" int fm_layout_from_morton(fm_matrix src, int64_t rows, int64_t cols, uint32_t* dst,
                                     int64_t ld, fm_stream stream)
{
    FmRange range("fm_layout_from_morton");
    return from_morton_impl(src, rows, cols, dst, ld, stream);
}

extern "C" int fm_layout_to_morton_u16(const uint16_t* src, int64_t rows, int64_t cols, int64_t ld,
                                       fm_matrix dst, fm_stream stream)
{
    FmRange range("fm_layout_to_morton_u16");
    return to_morton_impl(src, rows, cols, ld, nullptr, nullptr, dst, stream);
}

extern "C" int fm_layout_to_morton_permuted_u16(const uint16_t* src, int64_t rows, int64_t cols,
                                                int64_t ld, const int32_t* row_perm,
                                                const int32_t* col_perm, fm_matrix dst,
                                                fm_stream stream)
{
    FmRange range("fm_layout_to_morton_permuted_u16");
    return to_morton_impl(src, rows, cols, ld, row_perm, col_perm, dst, stream);
}

extern "C" int fm_layout_from_morton_u16(fm_matrix src, int64_t rows, int64_t cols, uint16_t* dst,
                                         int64_t ld, fm_stream stream)
{
    FmRange range("fm_layout_from_morton_u16");
    return from_morton_impl(src, rows, cols, dst, ld, stream);
}

extern "C" int fm_validate_residues(fm_sub X, uint32_t p, fm_stream stream)
{
    FmRange range("fm_validate_residues");
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    FM_TRY(fm_check_sub(X));
    if (X.rows == 0 || X.cols == 0) return FM_OK;
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    const int64_t blocks = (X.rows + kThreads / 32 - 1) / (kThreads / 32);
    validate_kernel<<<grid_for(blocks), kThreads, 0, (cudaStream_t)stream>>>(
        X.m.base, X.m.log2_T, X.row0, X.col0, X.rows, X.cols, p, status);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

namespace {

template <int CURVE>
int permute_impl(fm_matrix src, fm_matrix dst, int64_t rows, int64_t cols, const int32_t* row_perm,
                 const int32_t* col_perm, fm_stream stream)
{
    FM_TRY(fm_check_matrix(src));
    FM_TRY(fm_check_matrix(dst));
    const int64_t ns = fm_side(src), nd = fm_side(dst);
    if (rows < 0 || cols < 0 || rows > ns || cols > ns || rows > nd || cols > nd) return FM_EINVAL;
    const uint64_t sbytes = (uint64_t)ns * ns * 4, dbytes = (uint64_t)nd * nd * 4;
    const uintptr_t s0 = (uintptr_t)src.base, d0 = (uintptr_t)dst.base;
    if (s0 < d0 + dbytes && d0 < s0 + sbytes) return FM_EINVAL;  // src and dst overlap
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t row_bytes = (size_t)((cols + 3) & ~(int64_t)3) * 4;
    if (src.log2_T >= 2 && dst.log2_T >= 2 && row_bytes <= kStagedRowMax) {
        // two row buffers (copies of the next row overlap the gather) when
        // they fit, else one
        const bool two = 2 * row_bytes <= kStagedRowMax;
        auto k = two ? permute_staged_kernel<CURVE, 2> : permute_staged_kernel<CURVE, 1>;
        const size_t smem = two ? 2 * row_bytes : row_bytes;
        FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedRowMax));
        int per_sm = 0;
        FM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem));
        const int64_t cap = (int64_t)fm_sm_count() * std::max(1, per_sm);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nd, cap));
        k<<<grid, kThreads, smem, s>>>(src.base, src.log2_grid, src.log2_T, dst.base, dst.log2_grid,
                                       dst.log2_T, rows, cols, row_perm, col_perm, status);
    } else {
        const int64_t tiles = (int64_t)1 << (2 * dst.log2_grid);
        permute_kernel<CURVE><<<grid_for(tiles), kThreads, 0, s>>>(
            src.base, src.log2_grid, src.log2_T, dst.base, dst.log2_grid, dst.log2_T, rows, cols, row_perm,
            col_perm, status);
    }
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

}  // namespace

extern "C" int fm_permute_rows_cols(fm_matrix src, fm_matrix dst, int64_t rows, int64_t cols,
                                    const int32_t* row_perm, const int32_t* col_perm,
                                    fm_stream stream)
{
    FmRange range("fm_permute_rows_cols");
    return permute_impl<kMorton>(src, dst, rows, cols, row_perm, col_perm, stream);
}

extern "C" int fm_layout_to_hilbert(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                                    fm_matrix dst, fm_stream stream)
{
    FmRange range("fm_layout_to_hilbert");
    return to_morton_impl<uint32_t, kHilbert>(src, rows, cols, ld, nullptr, nullptr, dst, stream);
}

extern "C" int fm_layout_from_hilbert(fm_matrix src, int64_t rows, int64_t cols, uint32_t* dst,
                                      int64_t ld, fm_stream stream)
{
    FmRange range("fm_layout_from_hilbert");
    return from_morton_impl<uint32_t, kHilbert>(src, rows, cols, dst, ld, stream);
}

extern "C" int fm_permute_rows_cols_hilbert(fm_matrix src, fm_matrix dst, int64_t rows, int64_t cols,
                                            const int32_t* row_perm, const int32_t* col_perm,
                                            fm_stream stream)
{
    FmRange range("fm_permute_rows_cols_hilbert");
    return permute_impl<kHilbert>(src, dst, rows, cols, row_perm, col_perm, stream);
}
