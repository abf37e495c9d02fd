// limb_split.cu -- residues -> balanced signed 8-bit limb planes (f16 carrier).
//
// Each residue x in [0, p) becomes w balanced digits in [-128, 127] (base 256)
// of its representative r = x if x <= Hi else x - p, Hi = 127 * sum_{t<w} 256^t;
// with Karatsuba further planes hold the digit sums d_i + d_j, i < j < w (one
// for w = 2, three for w = 3, six for w = 4). The kernels read the
// (sub-)matrices from the Morton-hybrid layout (Sec. 1), re-base them to an
// aligned grid and write the planes as tiles in the 128-byte-swizzled K-major
// layout the tensor-core descriptors expect, so that every pipeline stage of
// the limb GEMM is ONE contiguous 1-D bulk copy per operand (the paper's
// contiguous base case, Sec. 2.1). HBM-bound.
#include <cuda_fp16.h>

#include <algorithm>

#include "fm_internal.cuh"
#include "fm_kernels.h"
#include "limb_common.cuh"

namespace {

using namespace fm_limb;
constexpr int kSplitThreads = 256;

// ---- limb digits ----------------------------------------------------------
template <int W>
__device__ __forceinline__ void limb_digits(uint32_t x, uint32_t p, int32_t hi, int (&d)[4])
{
    int32_t r = (x <= (uint32_t)hi) ? (int32_t)x : (int32_t)((int64_t)x - (int64_t)p);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (t < W) {
            const int32_t dt = ((r + 128) & 255) - 128;
            d[t] = dt;
            r = (r - dt) >> 8;
        } else {
            d[t] = 0;
        }
    }
}

// Two integers in [-512, 511] as a packed pair of IEEE halves, exactly: the
// half with bits 0x6400 + m (0 <= m < 1024) is 1024 + m, so 0x6400 + (d + 512)
// encodes 1536 + d and one packed subtraction of 1536 leaves d (exact, since d
// is representable). Avoids the slower integer-to-half conversions.
__device__ __forceinline__ uint32_t pack_half2(int lo, int hi)
{
    const uint32_t bits = (0x6400u + (uint32_t)(lo + 512)) | ((0x6400u + (uint32_t)(hi + 512)) << 16);
    const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&bits), __float2half2_rn(1536.0f));
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Planes per operand: W digits, plus the digit sums of every pair of them
// with Karatsuba.
template <int W, bool KARA>
constexpr int kPlanes = W + (KARA ? W * (W - 1) / 2 : 0);

// Value of plane T for one residue's digits d: digit T for T < W, else the
// Karatsuba digit sum d_i + d_j of pair T - W (|.| <= 256; the pair order of
// karatsuba_pair). T and W are compile-time, so d stays in registers.
template <int T, int W>
__device__ __forceinline__ int plane_value(const int (&d)[4])
{
    if constexpr (T < W) {
        return d[T];
    } else {
        constexpr int u = T - W;
        constexpr int j = u < 1 ? 1 : (u < 3 ? 2 : 3);
        constexpr int i = u - j * (j - 1) / 2;
        return d[i] + d[j];
    }
}

// Writes planes T.. of 8 consecutive entries (digits d) as f16 at out + off of
// each plane.
template <int W, bool KARA, int T = 0>
__device__ __forceinline__ void store_planes(const int (&d)[8][4], uint8_t* out, size_t plane_bytes,
                                             uint32_t off)
{
    if constexpr (T < kPlanes<W, KARA>) {
        int q[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) q[e] = plane_value<T, W>(d[e]);
        uint4 v;
        v.x = pack_half2(q[0], q[1]);
        v.y = pack_half2(q[2], q[3]);
        v.z = pack_half2(q[4], q[5]);
        v.w = pack_half2(q[6], q[7]);
        *reinterpret_cast<uint4*>(out + (size_t)T * plane_bytes + off) = v;
        store_planes<W, KARA, T + 1>(d, out, plane_bytes, off);
    }
}

// Byte offset of the 16-byte chunk kc (8 f16 values) of row r inside a tile
// whose rows are 128 bytes, in the 128-byte swizzle pattern (chunk index XOR
// row index mod 8), identical to what a TMA SWIZZLE_128B load produces.
__device__ __forceinline__ uint32_t sw128_offset(uint32_t r, uint32_t kc)
{
    return r * 128u + ((kc ^ (r & 7u)) << 4);
}

// Loads 8 consecutive entries (row gi, columns gj..gj+7) of a Morton-hybrid
// matrix, zero outside [0, rows) x [0, cols) of the sub-matrix. When the 8
// entries are one aligned run inside a tile row they come as two 16-byte loads.
__device__ __forceinline__ void load8_morton(const uint32_t* __restrict__ base, int lt, int64_t row0,
                                             int64_t col0, int64_t i, int64_t j, int64_t rows,
                                             int64_t cols, uint32_t (&x)[8])
{
    if (i >= rows) {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0;
        return;
    }
    const uint64_t gi = (uint64_t)(row0 + i);
    const uint64_t mask = (1ull << lt) - 1;
    const uint64_t gj0 = (uint64_t)(col0 + j);
    const uint64_t a0 = fm_encode(gi, gj0, lt);
    if (j + 8 <= cols && (gj0 & mask) + 8 <= mask + 1 && (a0 & 3) == 0) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(base + a0));
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(base + a0) + 1);
        x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
        x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
        return;
    }
    uint64_t addr = a0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int64_t jj = j + e;
        const uint64_t gj = gj0 + e;
        if (e > 0) addr = ((gj & mask) == 0) ? fm_encode(gi, gj, lt) : addr + 1;
        x[e] = jj < cols ? __ldg(base + addr) : 0u;
    }
}

// A (M x K) -> w planes of [MB][KB] tiles, each 128 rows x 64 k f16, swizzled.
// One CTA writes tile (mb, kb) of every plane. Rows at or past M are not
// written: a row of the product depends on its own row of A only, and the
// GEMM writes no output row past M (whatever such a plane row holds only
// reaches accumulator rows that are never stored). Columns past K inside the
// last K tile are written as zeros: they enter every row's sums.
template <int W, bool KARA>
__device__ __forceinline__ void split_a_tile(const uint32_t* __restrict__ A, int lt, int64_t row0,
                                             int64_t col0, int64_t M, int64_t K, int KB, int tile, uint32_t p,
                                             int32_t hi, uint8_t* __restrict__ planes, size_t plane_bytes)
{
    const int mb = tile / KB, kb = tile % KB;
    uint8_t* out = planes + (size_t)tile * kATileBytes;
    constexpr int kIters = kBM * 8 / kSplitThreads;  // 16-byte chunks per thread
    uint32_t x[kIters][8];
#pragma unroll
    for (int it = 0; it < kIters; ++it) {  // every load in flight before any digit work
        const int c = threadIdx.x + it * kSplitThreads;
        const int r = c >> 3, kc = c & 7;
        load8_morton(A, lt, row0, col0, (int64_t)mb * kBM + r, (int64_t)kb * kBK + kc * 8, M, K,
                     x[it]);
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
        const int c = threadIdx.x + it * kSplitThreads;
        const int r = c >> 3, kc = c & 7;
        if ((int64_t)mb * kBM + r >= M) continue;
        int d[8][4];
#pragma unroll
        for (int e = 0; e < 8; ++e) limb_digits<W>(x[it][e], p, hi, d[e]);
        store_planes<W, KARA>(d, out, plane_bytes, sw128_offset(r, kc));
    }
}

// B (K x N) -> w planes of [NB][KB] tiles, each BN rows (n) x 64 k f16 (B
// transposed to K-major), swizzled. Staged through shared memory so that both
// the Morton reads (along n, 16-byte vectors) and the tile writes (along k)
// are coalesced. One CTA writes tile (nb, kb) of every plane; rows n at or
// past N are not written (they reach only output columns that are never
// stored), k past K is written as zeros.
template <int BN, int W, bool KARA>
__device__ __forceinline__ void split_b_tile(const uint32_t* __restrict__ B, int lt, int64_t row0,
                                             int64_t col0, int64_t K, int64_t N, int KB, int tile, uint32_t p,
                                             int32_t hi,
                                             uint8_t* __restrict__ planes, size_t plane_bytes,
                                             uint32_t* sb)
{
    // sb: [kBK][BN] staging; column n of row kk lives at n ^ ((kk / 8) * 4),
    // which keeps 4-aligned runs contiguous and makes the column reads below
    // hit 32 distinct banks
    const int nb = tile / KB, kb = tile % KB;
    const uint64_t mask = (1ull << lt) - 1;
    constexpr int kIters = kBK * BN / 4 / kSplitThreads;  // 16-byte loads per thread
    uint4 v[kIters];
#pragma unroll
    for (int it = 0; it < kIters; ++it) {  // every load in flight before the staging stores
        const int idx = threadIdx.x + it * kSplitThreads;
        const int kk = idx / (BN / 4), nn = (idx % (BN / 4)) * 4;
        const int64_t gk = (int64_t)kb * kBK + kk, gn = (int64_t)nb * BN + nn;
        v[it] = make_uint4(0, 0, 0, 0);
        if (gk < K) {
            const uint64_t gi = (uint64_t)(row0 + gk), gj = (uint64_t)(col0 + gn);
            const uint64_t a = fm_encode(gi, gj, lt);
            if (gn + 4 <= N && (gj & mask) + 4 <= mask + 1 && (a & 3) == 0) {
                v[it] = __ldg(reinterpret_cast<const uint4*>(B + a));
            } else {
                // misaligned or ragged: entries along the tile row follow one
                // another, a new encode only where the run crosses into the next tile
                uint32_t t[4];
                uint64_t aq = a;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q > 0) aq = ((gj + q) & mask) == 0 ? fm_encode(gi, gj + q, lt) : aq + 1;
                    t[q] = gn + q < N ? __ldg(B + aq) : 0u;
                }
                v[it] = make_uint4(t[0], t[1], t[2], t[3]);
            }
        }
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
        const int idx = threadIdx.x + it * kSplitThreads;
        const int kk = idx / (BN / 4), nn = (idx % (BN / 4)) * 4;
        *reinterpret_cast<uint4*>(sb + kk * BN + (nn ^ ((kk >> 3) << 2))) = v[it];
    }
    __syncthreads();
    uint8_t* out = planes + (size_t)tile * BN * 128;
    // 8 lanes per output row (its 8 chunks of 8 k), 4 rows per warp: every warp
    // store covers 512 contiguous bytes of the tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kc = lane & 7;
    const int n_end = (int)min((int64_t)BN, N - (int64_t)nb * BN);
    for (int n = warp * 4 + (lane >> 3); n < n_end; n += kSplitThreads / 8) {
        int d[8][4];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int kk = kc * 8 + e;
            limb_digits<W>(sb[kk * BN + (n ^ ((kk >> 3) << 2))], p, hi, d[e]);
        }
        store_planes<W, KARA>(d, out, plane_bytes, sw128_offset(n, kc));
    }
}

template <int W, bool KARA>
__global__ void __launch_bounds__(kSplitThreads)
    split_a_kernel(const uint32_t* __restrict__ A, int lt, int64_t row0, int64_t col0, int64_t M,
                   int64_t K, int KB, uint32_t p, int32_t hi, uint8_t* __restrict__ planes, size_t plane_bytes)
{
    split_a_tile<W, KARA>(A, lt, row0, col0, M, K, KB, blockIdx.x, p, hi, planes, plane_bytes);
}

template <int BN, int W, bool KARA>
__global__ void __launch_bounds__(kSplitThreads)
    split_b_kernel(const uint32_t* __restrict__ B, int lt, int64_t row0, int64_t col0, int64_t K,
                   int64_t N, int KB, uint32_t p, int32_t hi, uint8_t* __restrict__ planes, size_t plane_bytes)
{
    extern __shared__ __align__(16) uint32_t sb[];
    split_b_tile<BN, W, KARA>(B, lt, row0, col0, K, N, KB, blockIdx.x, p, hi, planes, plane_bytes, sb);
}

// Batched: CTA b splits tile jobs[b].y of operand jobs[b].x (one launch for the
// A (or B) operands of every call of a plan).
template <int W, bool KARA>
__global__ void __launch_bounds__(kSplitThreads)
    split_a_batch_kernel(const FmSplitDesc* __restrict__ descs, const int2* __restrict__ jobs, uint32_t p,
                         int32_t hi)
{
    const int2 j = jobs[blockIdx.x];
    const FmSplitDesc d = descs[j.x];
    split_a_tile<W, KARA>(d.src, d.lt, d.row0, d.col0, d.rows, d.cols, d.KB, j.y, p, hi, d.out, d.plane_bytes);
}

template <int BN, int W, bool KARA>
__global__ void __launch_bounds__(kSplitThreads)
    split_b_batch_kernel(const FmSplitDesc* __restrict__ descs, const int2* __restrict__ jobs, uint32_t p,
                         int32_t hi)
{
    extern __shared__ __align__(16) uint32_t sb[];
    const int2 j = jobs[blockIdx.x];
    const FmSplitDesc d = descs[j.x];
    split_b_tile<BN, W, KARA>(d.src, d.lt, d.row0, d.col0, d.rows, d.cols, d.KB, j.y, p, hi, d.out,
                              d.plane_bytes, sb);
}

// The split kernels for a plan's limb count and Karatsuba choice.
template <int W, bool KARA>
struct SplitKernels {
    static constexpr auto a = split_a_kernel<W, KARA>;
    static constexpr auto b128 = split_b_kernel<128, W, KARA>;
    static constexpr auto b256 = split_b_kernel<256, W, KARA>;
    static constexpr auto ab = split_a_batch_kernel<W, KARA>;
    static constexpr auto bb128 = split_b_batch_kernel<128, W, KARA>;
    static constexpr auto bb256 = split_b_batch_kernel<256, W, KARA>;
};

struct SplitSet {
    decltype(&split_a_kernel<1, false>) a;
    decltype(&split_b_kernel<128, 1, false>) b128, b256;
    decltype(&split_a_batch_kernel<1, false>) ab;
    decltype(&split_b_batch_kernel<128, 1, false>) bb128, bb256;
};

template <int W, bool KARA>
SplitSet split_set()
{
    return SplitSet{SplitKernels<W, KARA>::a,  SplitKernels<W, KARA>::b128, SplitKernels<W, KARA>::b256,
                    SplitKernels<W, KARA>::ab, SplitKernels<W, KARA>::bb128, SplitKernels<W, KARA>::bb256};
}

// Kernels for plan q: w digits, Karatsuba when the plan carries pair planes.
int split_kernels(const FmLimbPlan& q, SplitSet* out)
{
    const bool kara = q.n_planes > q.w;
    if (kara && q.n_planes != q.w + q.w * (q.w - 1) / 2) return FM_EINVAL;
    switch (q.w * 2 + (kara ? 1 : 0)) {
    case 2: *out = split_set<1, false>(); return FM_OK;
    case 4: *out = split_set<2, false>(); return FM_OK;
    case 5: *out = split_set<2, true>(); return FM_OK;
    case 6: *out = split_set<3, false>(); return FM_OK;
    case 7: *out = split_set<3, true>(); return FM_OK;
    case 8: *out = split_set<4, false>(); return FM_OK;
    case 9: *out = split_set<4, true>(); return FM_OK;
    default: return FM_EINVAL;
    }
}

}  // namespace

namespace {
int32_t limb_hi(int w)
{
    int32_t hi = 0;
    for (int t = 0; t < w; ++t) hi += 127 * (1 << (8 * t));  // 127 * sum 256^t
    return hi;
}
}  // namespace

int fm_limb_split_run(const FmLimbPlan& q, fm_sub X, int role, uint32_t p, void* planes,
                      cudaStream_t s)
{
    uint8_t* out = static_cast<uint8_t*>(planes);
    const int32_t hi = limb_hi(q.w);
    SplitSet ks;
    FM_TRY(split_kernels(q, &ks));
    if (role == FM_LIMB_A) {
        if (q.MB * q.KB == 0) return FM_OK;
        ks.a<<<q.MB * q.KB, kSplitThreads, 0, s>>>(X.m.base, X.m.log2_T, X.row0, X.col0, q.M, q.K, q.KB, p, hi,
                                                   out, q.a_plane_bytes);
    } else {
        if (q.NB * q.KB == 0) return FM_OK;
        const size_t sb_smem = (size_t)kBK * q.block_n * 4;
        auto k = q.block_n == 256 ? ks.b256 : ks.b128;
        FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb_smem));
        k<<<q.NB * q.KB, kSplitThreads, sb_smem, s>>>(X.m.base, X.m.log2_T, X.row0, X.col0, q.K, q.N, q.KB, p,
                                                      hi, out, q.b_plane_bytes);
    }
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

int fm_limb_split_batch_run(const FmLimbPlan& q, int role, const FmSplitDesc* d_descs,
                            const int2* d_jobs, int64_t n_jobs, uint32_t p, cudaStream_t s)
{
    if (n_jobs == 0) return FM_OK;
    if (n_jobs > 0x7fffffff) return FM_EINVAL;
    const int32_t hi = limb_hi(q.w);
    SplitSet ks;
    FM_TRY(split_kernels(q, &ks));
    if (role == FM_LIMB_A) {
        ks.ab<<<(unsigned)n_jobs, kSplitThreads, 0, s>>>(d_descs, d_jobs, p, hi);
    } else {
        const size_t sb_smem = (size_t)kBK * q.block_n * 4;
        auto k = q.block_n == 256 ? ks.bb256 : ks.bb128;
        FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb_smem));
        k<<<(unsigned)n_jobs, kSplitThreads, sb_smem, s>>>(d_descs, d_jobs, p, hi);
    }
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

// ---- C entry point ----
extern "C" int fm_limb_split(fm_sub X, int32_t role, uint32_t p, const fm_opts* opts, void* planes,
                             fm_stream stream)
{
    if (role != FM_LIMB_A && role != FM_LIMB_B) return FM_EINVAL;
    FM_TRY(fm_check_sub(X));
    if (!planes || ((uintptr_t)planes & 15)) return FM_EINVAL;
    FmLimbPlan q;
    FM_TRY(role == FM_LIMB_A ? fm_limb_plan(X.rows, 1, X.cols, p, opts, &q)
                             : fm_limb_plan(1, X.cols, X.rows, p, opts, &q));
    return fm_limb_split_run(q, X, role, p, planes, (cudaStream_t)stream);
}

