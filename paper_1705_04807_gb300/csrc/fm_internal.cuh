// fm_internal.cuh -- shared internals of libfm (host + device).
//
// Morton-hybrid index math (Sec. 1; Sec. 2.2 Step 1; Sec. 2.1 P2), status
// handling, the workspace cache, and thin inline-PTX wrappers for mbarriers,
// 1-D bulk (TMA) copies and tcgen05 (5th-generation tensor core) instructions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fm.h"

#define FM_VERSION_NUM 100  // 0.1.0

// ---------------------------------------------------------------------------
// Morton-hybrid index. Tile (I, J) starts at Z(I, J) * T'^2 where Z interleaves
// the bits of I (odd positions, more significant) and J (even positions): the
// Z-curve with quadrants NW=0, NE=1, SW=2, SE=3 (Sec. 2.2 Step 1). Entry (u, v)
// inside a tile is at u*T' + v (Sec. 2.1 P2).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t fm_spread_bits(uint64_t x)
{
    x &= 0xFFFFFFFFull;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

__host__ __device__ __forceinline__ uint64_t fm_compact_bits(uint64_t x)
{
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return x;
}

// Z index of tile (I, J).
__host__ __device__ __forceinline__ uint64_t fm_tile_z(uint64_t I, uint64_t J)
{
    return (fm_spread_bits(I) << 1) | fm_spread_bits(J);
}

// Element offset of tile (I, J)'s first entry (its sigma), T' = 2^lt.
__host__ __device__ __forceinline__ uint64_t fm_tile_base(uint64_t I, uint64_t J, int lt)
{
    return fm_tile_z(I, J) << (2 * lt);
}

// Morton-hybrid index of Cartesian (i, j), T' = 2^lt.
__host__ __device__ __forceinline__ uint64_t fm_encode(uint64_t i, uint64_t j, int lt)
{
    const uint64_t mask = (1ull << lt) - 1;
    return fm_tile_base(i >> lt, j >> lt, lt) | ((i & mask) << lt) | (j & mask);
}

__host__ __device__ __forceinline__ void fm_extract(uint64_t z, int lt, uint64_t* i, uint64_t* j)
{
    const uint64_t mask = (1ull << lt) - 1;
    const uint64_t off = z & ((1ull << (2 * lt)) - 1);
    const uint64_t tz = z >> (2 * lt);
    *i = (fm_compact_bits(tz >> 1) << lt) | (off >> lt);
    *j = (fm_compact_bits(tz) << lt) | (off & mask);
}

// Hilbert-hybrid variant (the curve Sec. 1 weighs against Morton's for index
// conversion cost): tile (I, J) of a 2^lg x 2^lg grid sits at position
// H(I, J) of the Hilbert curve, whose order-1 pattern visits (I, J) = (0, 0),
// (0, 1), (1, 1), (1, 0). Going down one level per bit: the quadrant's rank
// along the curve is appended to the index, and the coordinates inside the
// quadrant are mapped onto the order-(level-1) curve -- the first quadrant is
// traversed transposed, the last anti-transposed (reflected across the other
// diagonal), the middle two as they are.
__host__ __device__ __forceinline__ uint64_t fm_hilbert_tile(uint64_t I, uint64_t J, int lg)
{
    uint64_t d = 0;
    for (int b = lg - 1; b >= 0; --b) {
        const uint64_t qi = (I >> b) & 1, qj = (J >> b) & 1;
        d = (d << 2) | (qi << 1) | (qi ^ qj);
        const uint64_t low = (1ull << b) - 1;
        const uint64_t i = I & low, j = J & low;
        if (!qi && !qj) {
            I = j;
            J = i;
        } else if (qi && !qj) {
            I = low - j;
            J = low - i;
        } else {
            I = i;
            J = j;
        }
    }
    return d;
}

// The tile at position d of the Hilbert curve (the inverse of fm_hilbert_tile):
// built up from the lowest level, each level's quadrant rank placing the cell
// found so far inside that quadrant of the next larger curve (transposed in the
// first quadrant, reflected across the anti-diagonal in the last).
__host__ __device__ __forceinline__ void fm_hilbert_cell(uint64_t d, int lg, uint64_t* I, uint64_t* J)
{
    uint64_t i = 0, j = 0;
    for (int b = 0; b < lg; ++b) {
        const uint64_t q = (d >> (2 * b)) & 3, s = 1ull << b;
        if (q == 0) {
            const uint64_t t = i;
            i = j;
            j = t;
        } else if (q == 1) {
            j += s;
        } else if (q == 2) {
            i += s;
            j += s;
        } else {
            const uint64_t ni = 2 * s - 1 - j, nj = s - 1 - i;
            i = ni;
            j = nj;
        }
    }
    *I = i;
    *J = j;
}

// Hilbert-hybrid index of Cartesian (i, j): tile base H(I, J) T'^2 plus the
// row-major offset inside the tile, T' = 2^lt, 2^lg tiles per side.
__host__ __device__ __forceinline__ uint64_t fm_hilbert_encode(uint64_t i, uint64_t j, int lg, int lt)
{
    const uint64_t mask = (1ull << lt) - 1;
    return (fm_hilbert_tile(i >> lt, j >> lt, lg) << (2 * lt)) | ((i & mask) << lt) | (j & mask);
}

__host__ __device__ __forceinline__ int64_t fm_side(const fm_matrix& m)
{
    return (int64_t)1 << (m.log2_grid + m.log2_T);
}

// ---------------------------------------------------------------------------
// Host helpers (defined in api.cu).
// ---------------------------------------------------------------------------
#define FM_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t fm_err__ = (expr);                      \
        if (fm_err__ != cudaSuccess) return FM_ECUDA;       \
    } while (0)

#define FM_TRY(expr)                                        \
    do {                                                    \
        int fm_rc__ = (expr);                               \
        if (fm_rc__ != FM_OK) return fm_rc__;               \
    } while (0)

int fm_check_matrix(const fm_matrix& m);
int fm_check_sub(const fm_sub& s);
// Device status word of the current device (allocated once, zero = OK).
int* fm_device_status();
// Growable cached device workspace of the current device, at least `bytes`;
// slot 0..3 are independent buffers. Returns nullptr on failure.
void* fm_workspace(int slot, size_t bytes);
// Pinned host staging buffer (slot 0..3) of at least `bytes`.
void* fm_host_staging(int slot, size_t bytes);
int fm_sm_count();

// FM_TRACE: when the environment variable is set, every public call appends one
// line (call, shapes, work) to stderr, or to the file it names if it is not "1".
bool fm_trace_on();
void fm_trace(const char* fmt, ...);

// NVTX range around a public entry point (visible in Nsight timelines).
struct FmRange {
    explicit FmRange(const char* name);
    ~FmRange();
};

// ---------------------------------------------------------------------------
// Device-side: bounded waits and status.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Every device-side wait gives up after this long, raises FM_ETIMEOUT in the
// status word and lets the kernel wind down instead of hanging the GPU.
#define FM_WAIT_LIMIT_NS 2000000000ull

__device__ __forceinline__ uint64_t fm_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void fm_raise(int* status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// Grid-wide barrier of a cooperative launch (bar[0] = arrivals, bar[1] =
// generation, zeroed before the launch). A wait that expires raises FM_ETIMEOUT
// and sets *s_abort (shared), after which every later barrier of the CTA
// returns false at once.
__device__ __forceinline__ bool fm_grid_barrier(unsigned* bar, int* status, volatile int* s_abort)
{
    __syncthreads();
    if (threadIdx.x == 0 && !*s_abort) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = fm_globaltimer();
            while (*gen == g) {
                if (fm_globaltimer() - t0 > FM_WAIT_LIMIT_NS) {
                    fm_raise(status, FM_ETIMEOUT);
                    *s_abort = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return !*s_abort;
}

__device__ __forceinline__ uint32_t fm_smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier ----
__device__ __forceinline__ void fm_mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(fm_smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fm_fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fm_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fm_smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void fm_mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fm_smem_u32(bar)) : "memory");
}

// A thread whose phase is not complete sleeps in the instruction until it
// completes, for at most the suspend-time hint (1 ms): a waiting warp then
// takes no issue slots from the warps doing the work on its SM sub-partition.
__device__ __forceinline__ bool fm_mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(fm_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; false if the wait limit expired
// (then FM_ETIMEOUT is raised) or *abort became non-zero.
__device__ __forceinline__ bool fm_mbar_wait(uint64_t* bar, uint32_t parity, int* status,
                                             volatile int* abort)
{
    if (fm_mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = fm_globaltimer();
    while (true) {
        if (fm_mbar_try_wait(bar, parity)) return true;
        if (abort && *abort) return false;
        if (fm_globaltimer() - t0 > FM_WAIT_LIMIT_NS) {
            fm_raise(status, FM_ETIMEOUT);
            if (abort) *abort = 1;
            return false;
        }
    }
}

// ---- 1-D bulk copy global -> shared (TMA engine), completes on an mbarrier ----
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void fm_bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            fm_smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(fm_smem_u32(bar))
        : "memory");
}

// ---- tcgen05 (5th-gen tensor core, tensor memory) ----
__device__ __forceinline__ void fm_tmem_alloc(uint32_t* smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     fm_smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void fm_tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fm_tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void fm_tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fm_tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16, one CTA.
__device__ __forceinline__ void fm_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D (+)= A * B with 8-bit E4M3 operands (kind::f8f6f4, FP32 accumulation). In
// the 128-byte swizzled K-major layout a row holds 128 elements; one MMA takes
// K = 32 of them (32 bytes), so descriptors advance as for the f16 kind. The
// instruction descriptor is the f16 one: format code 0 is E4M3 for this kind.
__device__ __forceinline__ void fm_mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on an mbarrier once all previously issued tcgen05 ops of this thread
// have completed.
__device__ __forceinline__ void fm_mma_commit(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            fm_smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fm_tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fm_tmem_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 32 lanes x 32 columns of 32-bit: thread t gets columns [col, col+32) of lane
// (warp's lane quarter)*32 + t.
__device__ __forceinline__ void fm_tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// 16 columns of the warp's 32 lanes (32x32b.x16): half the registers of the
// 32-column forms, for kernels with a tight register budget.
__device__ __forceinline__ void fm_tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void fm_tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void fm_tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
        "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
        "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// ---- clusters and the CTA-pair (cta_group::2) forms ----
__device__ __forceinline__ uint32_t fm_cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t fm_mapa(uint32_t saddr, uint32_t rank)
{
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(saddr), "r"(rank));
    return d;
}

// Arrive on an mbarrier of any CTA of the cluster with the default (CTA-scope
// release) semantics: orders this thread's tcgen05 work fenced before it, not
// its global stores, so it costs no cluster-wide fence.
__device__ __forceinline__ void fm_mbar_arrive_remote(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void fm_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                     "memory");
}

// Tensor memory of a CTA pair: one warp of each CTA of the pair executes these together.
__device__ __forceinline__ void fm_tmem_alloc_pair(uint32_t* smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     fm_smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void fm_tmem_relinquish_pair()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fm_tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// D (+)= A * B on a CTA pair (issued by the even CTA): A and D split by rows
// (each CTA holds M/2 rows of A at the same shared-memory offset and M/2 lanes
// of D), B split by columns (each CTA holds N/2 rows of the K-major B tile).
__device__ __forceinline__ void fm_mma_f16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void fm_mma_e4m3_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                 uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier at this shared-memory offset in every CTA of cta_mask
// once all previously issued tcgen05 ops of this thread have completed.
__device__ __forceinline__ void fm_mma_commit_pair(uint64_t* bar, uint16_t cta_mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(fm_smem_u32(bar)),
        "h"(cta_mask)
        : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzled layout: rows of 64 f16 (128 B), 8-row groups 1024 B apart. The tile
// base must be 1024-byte aligned; advancing along K by 16 elements adds 32 B
// to the start address.
__device__ __forceinline__ uint64_t fm_smem_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address       [0, 14)
    d |= (uint64_t)1 << 16;                    // leading byte offset [16, 30) (unused)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset  [32, 46)
    d |= (uint64_t)1 << 46;                    // descriptor version  [46, 48)
    d |= (uint64_t)2 << 61;                    // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: F16 x F16 -> F32, both K-major, M x N.
__host__ __device__ __forceinline__ uint32_t fm_idesc_f16_f32(int M, int N)
{
    return (1u << 4)                        // D format F32
           | (0u << 7) | (0u << 10)          // A, B format F16
           | ((uint32_t)(N >> 3) << 17)      // N / 8
           | ((uint32_t)(M >> 4) << 24);     // M / 16
}

#endif  // __CUDACC__
