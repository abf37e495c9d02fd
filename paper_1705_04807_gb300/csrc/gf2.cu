// gf2.cu -- the product over GF(2) on bit-packed Morton-hybrid matrices.
//
// GF(2) is the field of the paper's experiments (Sec. 2.2, "Performance
// Analysis": random sub-matrix products in Morton-hybrid matrices of N = 2048
// with T' = 32). With T' = 32 a tile row is exactly one 32-bit word, so the
// bit-packed Morton-hybrid matrix stores tile (I, J) as 32 consecutive words at
// Z(I, J) * 32, word u = tile row u, bit v = entry (u, v): the element order of
// the Morton-hybrid layout with 32 entries per word.
//
// The product runs on the tensor cores: each operand is expanded to one plane of
// E4M3 bytes (0x00 = 0, 0x38 = 1.0) in the same tiled, 128-byte-swizzled layout
// as the limb planes, but with 128 elements per 128-byte row (one K stage), and
// the persistent limb GEMM multiplies them with kind::f8f6f4 (twice the f16
// rate). Sums of 0/1 products are exact in FP32 up to 2^24 terms, so a product
// with K < 2^24 is one accumulation per output tile; its parity is packed back
// into words of C.
#include "fm_internal.cuh"
#include "fm_kernels.h"
#include "limb_common.cuh"

namespace {

using namespace fm_limb;

constexpr int kGf2Threads = 256;
constexpr uint32_t kOneE4M3 = 0x38u;  // 1.0 in E4M3

// Word of row i holding columns [32 jw, 32 jw + 32) of a bit-packed matrix.
__device__ __forceinline__ const uint32_t* gf2_word(const uint32_t* base, uint64_t i, uint64_t jw)
{
    return base + (fm_encode(i, jw << 5, 5) >> 5);
}

// 32 bits of row i starting at column c (bit 0 = column c); columns at or
// beyond the matrix side read as 0. words = words per row (2^log2_grid).
__device__ __forceinline__ uint32_t gf2_bits32(const uint32_t* base, uint64_t i, uint64_t c,
                                               uint64_t words)
{
    const uint64_t jw = c >> 5;
    const uint32_t sh = (uint32_t)(c & 31);
    const uint32_t w0 = jw < words ? *gf2_word(base, i, jw) : 0u;
    if (sh == 0) return w0;
    const uint32_t w1 = jw + 1 < words ? *gf2_word(base, i, jw + 1) : 0u;
    return __funnelshift_r(w0, w1, sh);
}

__device__ __forceinline__ uint32_t low_mask(int64_t n)
{
    return n >= 32 ? ~0u : (n <= 0 ? 0u : ((1u << n) - 1u));
}

// 4 bits -> 4 bytes of E4M3 (bit t -> byte t). Multiplying by 1 + 2^7 + 2^14 +
// 2^21 puts bit t at position 8t among 16 distinct positions (no carries).
__device__ __forceinline__ uint32_t expand4(uint32_t nib)
{
    return ((nib * 0x00204081u) & 0x01010101u) * kOneE4M3;
}

__device__ __forceinline__ uint4 expand16(uint32_t bits16)
{
    return make_uint4(expand4(bits16 & 15u), expand4((bits16 >> 4) & 15u), expand4((bits16 >> 8) & 15u),
                      expand4((bits16 >> 12) & 15u));
}

// Chunk c (16 bytes) of row r of a 128-byte-row swizzled tile.
__device__ __forceinline__ uint4* tile_chunk(uint8_t* tile, int r, int c)
{
    return reinterpret_cast<uint4*>(tile + r * 128 + ((c ^ (r & 7)) << 4));
}

// Row-major entries (bit 0 of each) -> bit-packed Morton-hybrid, zero outside
// [0, rows) x [0, cols). One warp per tile; lane u builds tile row u.
__global__ void gf2_pack_kernel(const uint32_t* __restrict__ src, int64_t rows, int64_t cols,
                                int64_t ld, uint32_t* __restrict__ dst, int lg, bool vec)
{
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (int64_t)1 << (2 * lg);
    for (int64_t z = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; z < ntiles;
         z += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t I = (int64_t)fm_compact_bits((uint64_t)z >> 1);
        const int64_t J = (int64_t)fm_compact_bits((uint64_t)z);
        const int64_t i = I * 32 + lane, j0 = J * 32;
        uint32_t w = 0;
        if (i < rows && j0 < cols) {
            const uint32_t* row = src + i * ld + j0;
            if (vec && j0 + 32 <= cols) {
                const uint4* r4 = reinterpret_cast<const uint4*>(row);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint4 v = r4[q];
                    w |= ((v.x & 1u) << (4 * q)) | ((v.y & 1u) << (4 * q + 1)) |
                         ((v.z & 1u) << (4 * q + 2)) | ((v.w & 1u) << (4 * q + 3));
                }
            } else {
                const int64_t n = cols - j0 < 32 ? cols - j0 : 32;
                for (int e = 0; e < n; ++e) w |= (row[e] & 1u) << e;
            }
        }
        dst[z * 32 + lane] = w;
    }
}

// Bit-packed Morton-hybrid -> row-major entries 0 / 1 of [0, rows) x [0, cols).
__global__ void gf2_unpack_kernel(const uint32_t* __restrict__ src, int lg, int64_t rows,
                                  int64_t cols, uint32_t* __restrict__ dst, int64_t ld, bool vec)
{
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (int64_t)1 << (2 * lg);
    for (int64_t z = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; z < ntiles;
         z += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t I = (int64_t)fm_compact_bits((uint64_t)z >> 1);
        const int64_t J = (int64_t)fm_compact_bits((uint64_t)z);
        const int64_t i = I * 32 + lane, j0 = J * 32;
        if (i >= rows || j0 >= cols) continue;
        const uint32_t w = src[z * 32 + lane];
        uint32_t* row = dst + i * ld + j0;
        if (vec && j0 + 32 <= cols) {
            uint4* r4 = reinterpret_cast<uint4*>(row);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                r4[q] = make_uint4((w >> (4 * q)) & 1u, (w >> (4 * q + 1)) & 1u, (w >> (4 * q + 2)) & 1u,
                                   (w >> (4 * q + 3)) & 1u);
        } else {
            const int64_t n = cols - j0 < 32 ? cols - j0 : 32;
            for (int e = 0; e < n; ++e) row[e] = (w >> e) & 1u;
        }
    }
}

// A (M x K sub-matrix) -> plane of [MB][KB] tiles, 128 rows x 128 k bytes.
// Thread item (r, q): row r of the tile, k bits [32 q, 32 q + 32) -> chunks 2q, 2q+1.
__device__ __forceinline__ void gf2_split_a_tile(const uint32_t* __restrict__ base, int lg, int64_t row0,
                                                 int64_t col0, int64_t M, int64_t K, int KB, int t,
                                                 uint8_t* __restrict__ out)
{
    const int mb = t / KB, kb = t % KB;
    uint8_t* tile = out + (size_t)t * kATileBytes;
    const uint64_t words = (uint64_t)1 << lg;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int idx = threadIdx.x + h * kGf2Threads;
        const int r = idx & 127, q = idx >> 7;
        const int64_t i = (int64_t)mb * kBM + r;
        const int64_t k0 = (int64_t)kb * 128 + 32 * q;
        uint32_t bits = 0;
        if (i < M && k0 < K)
            bits = gf2_bits32(base, (uint64_t)(row0 + i), (uint64_t)(col0 + k0), words) & low_mask(K - k0);
        *tile_chunk(tile, r, 2 * q) = expand16(bits & 0xFFFFu);
        *tile_chunk(tile, r, 2 * q + 1) = expand16(bits >> 16);
    }
}

// B (K x N sub-matrix) -> plane of [NB][KB] tiles, 256 rows (n) x 128 k bytes
// (B transposed). A warp takes 32 x 32 blocks: lane i reads 32 column bits of
// B row l0 + i, and 32 ballots turn them into lane j's 32 row bits of column
// n0 + j.
__device__ __forceinline__ void gf2_split_b_tile(const uint32_t* __restrict__ base, int lg, int64_t row0,
                                                 int64_t col0, int64_t K, int64_t N, int KB, int t,
                                                 uint8_t* __restrict__ out)
{
    const int nb = t / KB, kb = t % KB;
    uint8_t* tile = out + (size_t)t * (256 * 128);
    const uint64_t words = (uint64_t)1 << lg;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
    for (int blk = warp; blk < 32; blk += kGf2Threads / 32) {
        const int lb = blk & 3, nq = blk >> 2;  // 4 blocks along k, 8 along n
        const int64_t l = (int64_t)kb * 128 + 32 * lb + lane;
        const int64_t n0 = (int64_t)nb * 256 + 32 * nq;
        uint32_t w = 0;
        if (l < K && n0 < N)
            w = gf2_bits32(base, (uint64_t)(row0 + l), (uint64_t)(col0 + n0), words) & low_mask(N - n0);
        uint32_t col = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint32_t t = __ballot_sync(0xFFFFFFFFu, (w >> j) & 1u);
            if (lane == j) col = t;
        }
        const int r = 32 * nq + lane;
        *tile_chunk(tile, r, 2 * lb) = expand16(col & 0xFFFFu);
        *tile_chunk(tile, r, 2 * lb + 1) = expand16(col >> 16);
    }
}

__global__ void __launch_bounds__(kGf2Threads) gf2_split_a_kernel(
    const uint32_t* __restrict__ base, int lg, int64_t row0, int64_t col0, int64_t M, int64_t K,
    int KB, uint8_t* __restrict__ out)
{
    gf2_split_a_tile(base, lg, row0, col0, M, K, KB, blockIdx.x, out);
}

__global__ void __launch_bounds__(kGf2Threads) gf2_split_b_kernel(
    const uint32_t* __restrict__ base, int lg, int64_t row0, int64_t col0, int64_t K, int64_t N,
    int KB, uint8_t* __restrict__ out)
{
    gf2_split_b_tile(base, lg, row0, col0, K, N, KB, blockIdx.x, out);
}

// Batched: CTA b splits tile jobs[b].y of operand jobs[b].x (lt carries the
// operand's log2_grid).
__global__ void __launch_bounds__(kGf2Threads) gf2_split_a_batch_kernel(const FmSplitDesc* __restrict__ d,
                                                                        const int2* __restrict__ jobs)
{
    const int2 j = jobs[blockIdx.x];
    const FmSplitDesc x = d[j.x];
    gf2_split_a_tile(x.src, x.lt, x.row0, x.col0, x.rows, x.cols, x.KB, j.y, x.out);
}

__global__ void __launch_bounds__(kGf2Threads) gf2_split_b_batch_kernel(const FmSplitDesc* __restrict__ d,
                                                                        const int2* __restrict__ jobs)
{
    const int2 j = jobs[blockIdx.x];
    const FmSplitDesc x = d[j.x];
    gf2_split_b_tile(x.src, x.lt, x.row0, x.col0, x.rows, x.cols, x.KB, j.y, x.out);
}

// C <- 0 on a sub-matrix (the product with K = 0 under FM_OP_SET).
__global__ void gf2_zero_kernel(uint32_t* base, int64_t row0, int64_t col0, int64_t rows, int64_t cols)
{
    const int64_t w0 = col0 >> 5, w1 = (col0 + cols + 31) >> 5;
    const int64_t per_row = w1 - w0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * per_row;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = row0 + t / per_row, jw = w0 + t % per_row;
        const int64_t lo = col0 > jw * 32 ? col0 - jw * 32 : 0;
        const int64_t hi = col0 + cols < jw * 32 + 32 ? col0 + cols - jw * 32 : 32;
        const uint32_t m = low_mask(hi) & ~low_mask(lo);
        uint32_t* w = base + (fm_encode((uint64_t)i, (uint64_t)jw << 5, 5) >> 5);
        if (m == ~0u)
            *w = 0u;
        else
            atomicAnd(w, ~m);
    }
}

int grid_for_tiles(int64_t ntiles)
{
    const int64_t blocks = (ntiles * 32 + 255) / 256;
    return (int)std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)fm_sm_count() * 16);
}

int check_gf2_matrix(const fm_gf2_matrix& m)
{
    if (m.base == nullptr || ((uintptr_t)m.base & 15) != 0) return FM_EINVAL;
    if (m.log2_grid < 0 || m.log2_grid > 15) return FM_EINVAL;
    return FM_OK;
}

fm_sub as_sub(const fm_gf2_sub& s)
{
    fm_sub r;
    r.m.base = s.m.base;
    r.m.log2_grid = s.m.log2_grid;
    r.m.log2_T = 5;
    r.row0 = s.row0;
    r.col0 = s.col0;
    r.rows = s.rows;
    r.cols = s.cols;
    return r;
}

}  // namespace

int fm_gf2_split_batch_run(int role, const FmSplitDesc* d_descs, const int2* d_jobs, int64_t n_jobs,
                           cudaStream_t s)
{
    if (n_jobs == 0) return FM_OK;
    if (n_jobs > 0x7fffffff) return FM_EINVAL;
    if (role == FM_LIMB_A)
        gf2_split_a_batch_kernel<<<(unsigned)n_jobs, kGf2Threads, 0, s>>>(d_descs, d_jobs);
    else
        gf2_split_b_batch_kernel<<<(unsigned)n_jobs, kGf2Threads, 0, s>>>(d_descs, d_jobs);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

int fm_gf2_zero_sub(const fm_gf2_sub& C, cudaStream_t s)
{
    if (C.rows == 0 || C.cols == 0) return FM_OK;
    gf2_zero_kernel<<<fm_sm_count() * 4, 256, 0, s>>>(C.m.base, C.row0, C.col0, C.rows, C.cols);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

extern "C" int fm_gf2_pack(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                           fm_gf2_matrix dst, fm_stream stream)
{
    FM_TRY(check_gf2_matrix(dst));
    const int64_t n = (int64_t)32 << dst.log2_grid;
    if (rows < 0 || cols < 0 || rows > n || cols > n || ld < cols) return FM_EINVAL;
    if ((rows > 0 && cols > 0) && src == nullptr) return FM_EINVAL;
    const bool vec = ((uintptr_t)src & 15) == 0 && (ld & 3) == 0;
    const int64_t ntiles = (int64_t)1 << (2 * dst.log2_grid);
    gf2_pack_kernel<<<grid_for_tiles(ntiles), 256, 0, (cudaStream_t)stream>>>(src, rows, cols, ld, dst.base,
                                                                                dst.log2_grid, vec);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

extern "C" int fm_gf2_unpack(fm_gf2_matrix src, int64_t rows, int64_t cols, uint32_t* dst, int64_t ld,
                             fm_stream stream)
{
    FM_TRY(check_gf2_matrix(src));
    const int64_t n = (int64_t)32 << src.log2_grid;
    if (rows < 0 || cols < 0 || rows > n || cols > n || ld < cols) return FM_EINVAL;
    if (rows == 0 || cols == 0) return FM_OK;
    if (dst == nullptr) return FM_EINVAL;
    const bool vec = ((uintptr_t)dst & 15) == 0 && (ld & 3) == 0;
    const int64_t ntiles = (int64_t)1 << (2 * src.log2_grid);
    gf2_unpack_kernel<<<grid_for_tiles(ntiles), 256, 0, (cudaStream_t)stream>>>(src.base, src.log2_grid,
                                                                                  rows, cols, dst, ld, vec);
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}

extern "C" int64_t fm_gf2_workspace_size(int64_t M, int64_t N, int64_t K)
{
    if (M < 0 || N < 0 || K < 0) return FM_EINVAL;
    FmLimbPlan q;
    FM_TRY(fm_gf2_plan(M, N, K, false, &q));
    return (int64_t)(q.a_plane_bytes + q.b_plane_bytes);
}

int fm_gf2_check_call(const fm_gf2_call& g)
{
    if (g.op < FM_OP_SET || g.op > FM_OP_SUB) return FM_EINVAL;
    FM_TRY(check_gf2_matrix(g.C.m));
    FM_TRY(check_gf2_matrix(g.A.m));
    FM_TRY(check_gf2_matrix(g.B.m));
    return fm_check_product(as_sub(g.C), as_sub(g.A), as_sub(g.B), false);
}

extern "C" int fm_gf2_gemm(fm_gf2_sub C, fm_gf2_sub A, fm_gf2_sub B, int32_t op, const fm_opts* opts,
                           fm_stream stream)
{
    FmRange range("fm_gf2_gemm");
    fm_gf2_call g;
    g.C = C;
    g.A = A;
    g.B = B;
    g.op = op;
    g.reserved = 0;
    FM_TRY(fm_gf2_check_call(g));
    const fm_sub Cs = as_sub(C);
    const int64_t M = C.rows, N = C.cols, K = A.cols;
    if (M == 0 || N == 0) return FM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) {
        if (op != FM_OP_SET) return FM_OK;
        gf2_zero_kernel<<<fm_sm_count() * 4, 256, 0, s>>>(C.m.base, C.row0, C.col0, M, N);
        FM_CUDA_TRY(cudaGetLastError());
        return FM_OK;
    }
    FmLimbPlan q;
    FM_TRY(fm_gf2_plan(M, N, K, opts && opts->cta_pair == 1, &q));
    uint8_t* Ap = static_cast<uint8_t*>(fm_workspace(0, q.a_plane_bytes + q.b_plane_bytes));
    if (!Ap) return FM_ENOMEM;
    uint8_t* Bp = Ap + q.a_plane_bytes;
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    gf2_split_a_kernel<<<q.MB * q.KB, kGf2Threads, 0, s>>>(A.m.base, A.m.log2_grid, A.row0, A.col0, M, K,
                                                           q.KB, Ap);
    FM_CUDA_TRY(cudaGetLastError());
    gf2_split_b_kernel<<<q.NB * q.KB, kGf2Threads, 0, s>>>(B.m.base, B.m.log2_grid, B.row0, B.col0, K, N,
                                                           q.KB, Bp);
    FM_CUDA_TRY(cudaGetLastError());
    fm_trace("gf2_gemm M=%lld N=%lld K=%lld op=%d tiles=%d planes=%llu B", (long long)M, (long long)N,
             (long long)K, op, q.MB * q.NB, (unsigned long long)(q.a_plane_bytes + q.b_plane_bytes));
    return fm_limb_gemm_run(q, Cs, Ap, Bp, 2u, op, status, s);
}
