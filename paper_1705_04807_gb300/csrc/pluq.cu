// pluq.cu -- rank-revealing TU / PLUQ decomposition over GF(p) on the device.
//
// Sec. 1: the matrix product serves TU decomposition of rectangular, possibly
// singular matrices over finite fields (TURBO), which also yields the rank; the
// paper defers the algorithm itself to its reference. This is a blocked
// right-looking elimination with the same kind of result, P A Q = L U with L
// unit lower trapezoidal (m x r), U upper trapezoidal (r x n), r = rank:
//
//   for each panel of 128 columns:
//     1. factor the panel (rows r..m-1): pivot = first row with a nonzero in
//        the column, row swap, exact modular rank-1 update; a column with no
//        nonzero below row r is skipped (it belongs to the non-pivot columns);
//     2. move the panel's pivot columns in front of its skipped ones;
//     3. apply the panel's row swaps to the rest of the matrix;
//     4. U12 <- L11^-1 A12: the inverse of the unit lower triangle L11 (one
//        CTA), then one limb product X * A12 written over A12;
//     5. A22 <- A22 - L21 U12 mod p: one fm_gemm_modp call on three disjoint
//        sub-matrices of the Morton-hybrid matrix -- the MM call the paper's
//        decomposition issues (Sec. 2: S_A = S_B * S_C on sub-matrices).
//   finally the skipped columns of every panel are moved behind all pivot
//   columns.
//
// Step 1 runs as one cooperative launch: each CTA keeps its share of the panel
// rows in shared memory and one grid barrier per column selects the pivot (a
// global-memory variant serves panels too tall for shared memory). The barrier
// is bounded: a wait that expires raises FM_ETIMEOUT and every CTA leaves the
// kernel.
#include <algorithm>
#include <atomic>
#include <climits>
#include <unordered_map>
#include <vector>

#include "fm_internal.cuh"
#include "fm_kernels.h"

namespace {

constexpr int kNb = 128;          // panel width
constexpr int kPanelThreads = 256;

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p, uint64_t mu)
{
    const uint64_t t = (uint64_t)a * b;
    const uint64_t q = __umul64hi(t, mu);
    uint64_t r = t - q * p;
    while (r >= p) r -= p;
    return (uint32_t)r;
}

__device__ __forceinline__ uint32_t submod(uint32_t a, uint32_t b, uint32_t p)
{
    return a >= b ? a - b : a + (p - b);
}

// a^(p-2) mod p: the inverse of a unit of the prime field GF(p).
__device__ uint32_t invmod_prime(uint32_t a, uint32_t p, uint64_t mu)
{
    uint32_t r = 1, b = a;
    uint32_t e = p - 2;
    while (e) {
        if (e & 1) r = mulmod(r, b, p, mu);
        b = mulmod(b, b, p, mu);
        e >>= 1;
    }
    return r;
}

struct PanelArgs {
    uint32_t* A;
    int lt;
    int64_t m;       // rows of the matrix
    int64_t r0;      // first row of the panel region (rank found so far)
    int64_t c0;      // first column of the panel
    int w;           // panel width (<= kNb)
    uint32_t p;
    uint64_t mu;
    int* piv_slot;   // [w] first nonzero row per column (INT_MAX before the search)
    int* piv_row;    // out [w]: pivot row of panel column t, or -1 if skipped
    int* n_piv;      // out: pivots found
    unsigned* bar;   // [2]: arrival count, generation
    int* status;
};

__device__ __forceinline__ uint32_t* elem(const PanelArgs& a, int64_t i, int64_t j)
{
    return a.A + fm_encode((uint64_t)i, (uint64_t)j, a.lt);
}

// Factors rows [r0, m) x columns [c0, c0 + w) in place (see the file comment).
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(const PanelArgs a)
{
    __shared__ uint32_t prow[kNb];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)blockIdx.x * (kPanelThreads / 32) + warp;
    const int64_t nwarps = (int64_t)gridDim.x * (kPanelThreads / 32);
    int64_t r = a.r0;
    int found = 0;
    for (int t = 0; t < a.w; ++t) {
        const int64_t j = a.c0 + t;
        if (!fm_grid_barrier(a.bar, a.status, &s_abort)) return;  // updates of column t-1 done
        if (r >= a.m) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.piv_row[t] = -1;
            continue;
        }
        // pivot: row r itself when nonzero, else the first nonzero row below
        int piv;
        if (*elem(a, r, j) != 0) {
            piv = (int)r;
        } else {
            for (int64_t base = r + 1 + gwarp * 32; base < a.m; base += nwarps * 32) {
                const int64_t i = base + lane;
                const bool nz = i < a.m && *elem(a, i, j) != 0;
                const unsigned bal = __ballot_sync(0xffffffffu, nz);
                if (bal) {
                    if (lane == 0) atomicMin(&a.piv_slot[t], (int)(base + __ffs(bal) - 1));
                    break;
                }
            }
            if (!fm_grid_barrier(a.bar, a.status, &s_abort)) return;
            piv = *(volatile int*)&a.piv_slot[t];
            if (piv == INT_MAX) {  // no nonzero below row r: a non-pivot column
                if (blockIdx.x == 0 && threadIdx.x == 0) a.piv_row[t] = -1;
                continue;
            }
            if (blockIdx.x == 0) {  // swap rows r and piv across the panel
                for (int c = threadIdx.x; c < a.w; c += kPanelThreads) {
                    uint32_t* x = elem(a, r, a.c0 + c);
                    uint32_t* y = elem(a, piv, a.c0 + c);
                    const uint32_t tmp = *x;
                    *x = *y;
                    *y = tmp;
                }
            }
            if (!fm_grid_barrier(a.bar, a.status, &s_abort)) return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.piv_row[t] = piv;
        // pivot row to shared memory
        for (int c = threadIdx.x; c < a.w; c += kPanelThreads) prow[c] = *elem(a, r, a.c0 + c);
        __syncthreads();
        const uint32_t inv = invmod_prime(prow[t], a.p, a.mu);
        // rank-1 update of rows below r: a_i <- a_i - l_i * pivot row, l_i stored in column t
        for (int64_t i = r + 1 + gwarp; i < a.m; i += nwarps) {
            const uint32_t l = mulmod(*elem(a, i, j), inv, a.p, a.mu);
            for (int c = t + 1 + lane; c < a.w; c += 32) {
                uint32_t* x = elem(a, i, a.c0 + c);
                *x = submod(*x, mulmod(l, prow[c], a.p, a.mu), a.p);
            }
            __syncwarp();
            if (lane == 0) *elem(a, i, j) = l;
        }
        ++r;
        ++found;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.n_piv = found;
}

// *nz = 1 if rows [r0, m) x columns [c0, c0 + w) hold a nonzero (left at 0
// otherwise): a panel with no nonzero has no pivot, and all its columns are
// skipped without a search. One warp per row, contiguous runs inside tile rows.
__global__ void panel_nonzero_kernel(const uint32_t* __restrict__ A, int lt, int64_t r0, int64_t m, int64_t c0,
                                     int w, int* nz)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t T = (int64_t)1 << lt;
    bool any = false;
    for (int64_t i = r0 + (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < m && !any; i += warps) {
        for (int64_t j = 0; j < w;) {
            const uint64_t gj = (uint64_t)(c0 + j);
            const int64_t run = min((int64_t)w - j, T - (int64_t)(gj & (uint64_t)(T - 1)));
            const uint32_t* seg = A + fm_encode((uint64_t)i, gj, lt);
            for (int64_t e = lane; e < run; e += 32) any |= __ldg(seg + e) != 0u;
            j += run;
        }
        any = __any_sync(0xffffffffu, any);
    }
    if (any && lane == 0) atomicOr(nz, 1);
}

// Columns [c0, c0 + w) of rows [0, m) reordered: new column t = old order[t].
__global__ void permute_panel_cols_kernel(uint32_t* A, int lt, int64_t m, int64_t c0, int w,
                                          const int* __restrict__ order)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x / 32) + warp; i < m;
         i += (int64_t)gridDim.x * (blockDim.x / 32)) {
        uint32_t v[kNb / 32];
#pragma unroll
        for (int q = 0; q < kNb / 32; ++q) {
            const int t = lane + 32 * q;
            v[q] = t < w ? A[fm_encode((uint64_t)i, (uint64_t)(c0 + order[t]), lt)] : 0u;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kNb / 32; ++q) {
            const int t = lane + 32 * q;
            if (t < w) A[fm_encode((uint64_t)i, (uint64_t)(c0 + t), lt)] = v[q];
        }
    }
}

// The panel's row swaps (in order) applied to columns outside [c0, c0 + w).
__global__ void row_swaps_kernel(uint32_t* A, int lt, int64_t n, int64_t c0, int w, int64_t r0,
                                 const int* __restrict__ piv_row, int w_piv)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (j >= c0 && j < c0 + w) continue;
        int64_t r = r0;
        for (int t = 0; t < w_piv; ++t) {
            const int pv = piv_row[t];
            if (pv < 0) continue;
            if (pv != r) {
                uint32_t* x = A + fm_encode((uint64_t)r, (uint64_t)j, lt);
                uint32_t* y = A + fm_encode((uint64_t)pv, (uint64_t)j, lt);
                const uint32_t tmp = *x;
                *x = *y;
                *y = tmp;
            }
            ++r;
        }
    }
}

// The same swaps on the row permutation (gather convention).
__global__ void perm_swaps_kernel(int32_t* rp, int64_t r0, const int* __restrict__ piv_row, int w)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t r = r0;
        for (int t = 0; t < w; ++t) {
            const int pv = piv_row[t];
            if (pv < 0) continue;
            if (pv != r) {
                const int32_t tmp = rp[r];
                rp[r] = rp[pv];
                rp[pv] = tmp;
            }
            ++r;
        }
    }
}

// Columns of rows [0, m) reordered in place: new column t = old column ord[t],
// t < n. One CTA per row at a time, the row staged in shared memory.
__global__ void permute_cols_rows_kernel(uint32_t* A, int lt, int64_t m, int64_t n,
                                         const int32_t* __restrict__ ord)
{
    extern __shared__ uint32_t row[];
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
            row[j] = A[fm_encode((uint64_t)i, (uint64_t)j, lt)];
        __syncthreads();
        for (int64_t t = threadIdx.x; t < n; t += blockDim.x)
            A[fm_encode((uint64_t)i, (uint64_t)t, lt)] = row[ord[t]];
        __syncthreads();
    }
}

// Extended Euclid: inverse of a unit a modulo p < 2^31, in 32-bit arithmetic
// (every remainder and coefficient stays below p in magnitude).
__host__ __device__ __forceinline__ uint32_t inv_euclid(uint32_t a, uint32_t p)
{
    int32_t t = 0, nt = 1;
    uint32_t r = p, nr = a;
    while (nr != 0) {
        const uint32_t q = r / nr;
        const int32_t tmp = t - (int32_t)q * nt;
        t = nt;
        nt = tmp;
        const uint32_t rr = r - q * nr;
        r = nr;
        nr = rr;
    }
    return (uint32_t)(t < 0 ? t + (int32_t)p : t);
}

struct SmemPanelArgs {
    uint32_t* A;
    int lt;
    int64_t m, r0, c0;
    int w;
    int rows_per_cta;  // R: CTA b owns rows [r0 + b R, r0 + (b+1) R) of the panel
    uint32_t p;
    uint64_t mu;
    uint2* stat;       // [w][gridDim.x] (code, tag): code 1 = no candidate,
                       // 2 + i = candidate is this CTA's row i
    uint2* cand;       // [w][gridDim.x][w + 2] (value, tag): candidate row values,
                       // inverse, global row index
    uint32_t tag0;     // tags of this launch: tag0 + t for column t (never reused)
    int* piv_row;      // out [w]: pivot row of column t (original index) or -1
    int* n_piv;        // out
    unsigned* bar;
    int* status;
};

// a * b mod p for a, b < p: one 32-bit Barrett step when p < 2^16 (the product
// fits 32 bits), the 64-bit one otherwise (mu32 = 2^32 / p, mu = 2^64 / p).
__device__ __forceinline__ uint32_t mul_p(uint32_t a, uint32_t b, uint32_t p, uint32_t mu32, uint64_t mu)
{
    if (p < 65536u) {
        const uint32_t x = a * b;
        uint32_t r = x - __umulhi(x, mu32) * p;
        return r >= p ? r - p : r;
    }
    return mulmod(a, b, p, mu);
}

// Published words are (value, tag) pairs written by one aligned 64-bit store and
// read by one 64-bit load (single-copy atomic), so a reader that sees the tag it
// expects also sees the value: no fences, no clearing between launches.
__device__ __forceinline__ void put_tagged(uint2* p, uint32_t v, uint32_t tag)
{
    asm volatile("st.relaxed.gpu.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(v), "r"(tag) : "memory");
}

__device__ __forceinline__ uint2 get_tagged(const uint2* p)
{
    uint2 r;
    asm volatile("ld.relaxed.gpu.global.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p) : "memory");
    return r;
}

// Waits (bounded) until *p carries the tag; false if the wait expired or
// *abort became non-zero.
__device__ __forceinline__ bool wait_tagged(const uint2* p, uint32_t tag, uint32_t* v, int* status,
                                            volatile int* abort)
{
    uint2 r = get_tagged(p);
    if (r.y == tag) {
        *v = r.x;
        return true;
    }
    const uint64_t t0 = fm_globaltimer();
    while (true) {
        r = get_tagged(p);
        if (r.y == tag) {
            *v = r.x;
            return true;
        }
        if (*abort) return false;
        if (fm_globaltimer() - t0 > FM_WAIT_LIMIT_NS) {
            fm_raise(status, FM_ETIMEOUT);
            *abort = 1;
            return false;
        }
    }
}

// Panel factorisation with the panel rows resident in shared memory. CTA b owns
// rows [r0 + b R, r0 + (b+1) R). The pivot of column t is the first row (in row
// order) that is not yet a pivot and has a nonzero in column t, so it belongs to
// the lowest-numbered CTA that has such a row. Per column every CTA publishes
// its candidate (row values, inverse, index) in a slot of its own and then a
// status word (release); it reads the status words of CTAs 0, 1, ... (acquire)
// only up to the first one that has a candidate, takes that row and updates its
// own non-pivot rows. The CTA that owns the pivot reads only lower-numbered
// CTAs' status words (already published: they have no candidate) and uses its
// own row, so it runs at its own pace; there is no grid-wide barrier per
// column. Every published word is tagged with the launch and column, so no
// fence orders it. A CTA publishes column t before it reads anything of column
// t, so the waits form no cycle. Rows are not moved; the pivot order is
// returned. Every wait is bounded.
__global__ void __launch_bounds__(kPanelThreads, 1) smem_panel_kernel(const SmemPanelArgs a)
{
    extern __shared__ uint32_t sm[];
    const int R = a.rows_per_cta, w = a.w, P = gridDim.x;
    uint32_t* rows = sm;                                   // [R][w]
    uint32_t* prow = rows + (size_t)R * w;                 // [w]
    int* piv_flag = reinterpret_cast<int*>(prow + kNb);    // [R]
    uint32_t* lbuf = reinterpret_cast<uint32_t*>(piv_flag + R);  // [R] multipliers
    const uint32_t mu32 = (uint32_t)(0x100000000ull / a.p);
    __shared__ int s_abort, s_first, s_owner;
    __shared__ uint32_t s_myinv;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = a.r0 + (int64_t)blockIdx.x * R;
    const int64_t left = a.m - row0;
    const int nrows = left <= 0 ? 0 : (left < R ? (int)left : R);
    if (tid == 0) s_abort = 0;
    for (int e = tid; e < R * w; e += kPanelThreads) {
        const int i = e / w, c = e % w;
        rows[e] = i < nrows ? a.A[fm_encode((uint64_t)(row0 + i), (uint64_t)(a.c0 + c), a.lt)] : 0u;
    }
    for (int i = tid; i < R; i += kPanelThreads) piv_flag[i] = 0;
    __syncthreads();
    if (tid == 0) s_first = INT_MAX;
    __syncthreads();
    int found = 0;
    for (int t = 0; t < w; ++t) {
        // 1. this CTA's candidate: first non-pivot row with a nonzero in column t
        // (s_first was reset after the previous column's publication)
        for (int i = tid; i < nrows; i += kPanelThreads)
            if (!piv_flag[i] && rows[(size_t)i * w + t] != 0) atomicMin(&s_first, i);
        __syncthreads();
        const int li = s_first;
        const int mycode = li != INT_MAX ? 2 + li : 1;
        const uint32_t tag = a.tag0 + (uint32_t)t;
        // warp 0 publishes the candidate row, its inverse and row index, then the
        // status word, all tagged
        if (warp == 0) {
            if (li != INT_MAX) {
                uint2* cbuf = a.cand + ((size_t)t * P + blockIdx.x) * (w + 2);
                for (int c = lane; c < w; c += 32) put_tagged(cbuf + c, rows[(size_t)li * w + c], tag);
                if (lane == 0) {
                    s_myinv = inv_euclid(rows[(size_t)li * w + t], a.p);
                    put_tagged(cbuf + w, s_myinv, tag);
                    put_tagged(cbuf + w + 1, (uint32_t)(row0 + li), tag);
                }
            }
            if (lane == 0) {
                put_tagged(&a.stat[(size_t)t * P + blockIdx.x], (uint32_t)mycode, tag);
                s_owner = INT_MAX;
            }
        }
        __syncthreads();
        if (tid == 0) s_first = INT_MAX;  // every thread holds li by now
        // 2. find the first CTA with a candidate: thread b reads CTA b's status
        // word, all at once (only lower CTAs when this one has a candidate); a
        // thread stops as soon as a lower CTA is known to have one, so only CTAs
        // up to the owner are waited for
        const int limit = mycode >= 2 ? (int)blockIdx.x + 1 : P;
        for (int b = tid; b < limit; b += kPanelThreads) {
            uint32_t code = b == (int)blockIdx.x ? (uint32_t)mycode : 0u;
            if (code == 0) {
                const uint2* sp = &a.stat[(size_t)t * P + b];
                const uint64_t t0 = fm_globaltimer();
                while (true) {
                    const uint2 r = get_tagged(sp);
                    if (r.y == tag) {
                        code = r.x;
                        break;
                    }
                    if (*(volatile int*)&s_owner < b || s_abort) break;
                    if (fm_globaltimer() - t0 > FM_WAIT_LIMIT_NS) {
                        fm_raise(a.status, FM_ETIMEOUT);
                        s_abort = 1;
                        break;
                    }
                }
            }
            if (code >= 2) atomicMin(&s_owner, b);
        }
        __syncthreads();
        if (s_abort) return;
        const int owner = s_owner == INT_MAX ? -1 : s_owner;
        if (owner < 0) {  // no nonzero left in this column: a non-pivot column
            if (blockIdx.x == 0 && tid == 0) a.piv_row[t] = -1;
            continue;
        }
        // 3. the pivot row (this CTA's own row, or the owner's published copy) and
        // its inverse; every thread takes the inverse itself
        uint32_t inv;
        if (owner == (int)blockIdx.x) {
            for (int c = tid; c < w; c += kPanelThreads) prow[c] = rows[(size_t)li * w + c];
            inv = s_myinv;
            if (tid == 0) {
                piv_flag[li] = 1;
                if (blockIdx.x == 0) a.piv_row[t] = (int)(row0 + li);
            }
        } else {
            const uint2* ob = a.cand + ((size_t)t * P + owner) * (w + 2);
            for (int c = tid; c < w; c += kPanelThreads) {
                uint32_t v = 0;
                wait_tagged(ob + c, tag, &v, a.status, &s_abort);
                prow[c] = v;
            }
            wait_tagged(ob + w, tag, &inv, a.status, &s_abort);
            if (blockIdx.x == 0 && tid == 0) {
                uint32_t g = 0;
                wait_tagged(ob + w + 1, tag, &g, a.status, &s_abort);
                a.piv_row[t] = (int)g;
            }
        }
        // 4. the multipliers l_i (column t) of all non-pivot rows at once, then
        // a_i <- a_i - l_i * pivot row on columns > t (warps over rows, lanes
        // over columns); l_i is kept in column t
        for (int i = tid; i < nrows; i += kPanelThreads)
            if (i != li || owner != (int)blockIdx.x)
                lbuf[i] = piv_flag[i] ? 0u : mul_p(rows[(size_t)i * w + t], inv, a.p, mu32, a.mu);
            else
                lbuf[i] = 0u;
        __syncthreads();
        if (s_abort) return;
        for (int i = warp; i < nrows; i += kPanelThreads / 32) {
            const uint32_t l = lbuf[i];
            if (l == 0) continue;
            uint32_t* ri = rows + (size_t)i * w;
            for (int c = t + 1 + lane; c < w; c += 32) ri[c] = submod(ri[c], mul_p(l, prow[c], a.p, mu32, a.mu), a.p);
        }
        for (int i = tid; i < nrows; i += kPanelThreads)
            if (!piv_flag[i]) rows[(size_t)i * w + t] = lbuf[i];
        __syncthreads();
        ++found;
    }
    for (int e = tid; e < nrows * w; e += kPanelThreads) {
        const int i = e / w, c = e % w;
        a.A[fm_encode((uint64_t)(row0 + i), (uint64_t)(a.c0 + c), a.lt)] = rows[e];
    }
    if (blockIdx.x == 0 && tid == 0) *a.n_piv = found;
}

// Tags of a panel launch: 256 fresh values (one per column), never zero (the
// slots are cleared at every fm_pluq call; the counter wraps after 2^24 launches).
uint32_t next_tags()
{
    static std::atomic<uint32_t> counter{1};
    return counter.fetch_add(256u);
}

// Row swaps (pairs (x, y) in order) on columns [0, n) and on the permutation.
__global__ void swap_pairs_kernel(uint32_t* A, int lt, int64_t n, const int* __restrict__ pairs,
                                  int npairs, int32_t* rp)
{
    if (rp && blockIdx.x == 0 && threadIdx.x == 0) {
        for (int q = 0; q < npairs; ++q) {
            const int x = pairs[2 * q], y = pairs[2 * q + 1];
            const int32_t tmp = rp[x];
            rp[x] = rp[y];
            rp[y] = tmp;
        }
    }
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        for (int q = 0; q < npairs; ++q) {
            uint32_t* x = A + fm_encode((uint64_t)pairs[2 * q], (uint64_t)j, lt);
            uint32_t* y = A + fm_encode((uint64_t)pairs[2 * q + 1], (uint64_t)j, lt);
            const uint32_t tmp = *x;
            *x = *y;
            *y = tmp;
        }
    }
}

// a * b mod p for p < 2^16 (a, b < p): the product fits 32 bits; one Barrett
// step with mu32 = floor(2^32 / p) leaves it below 2p
__device__ __forceinline__ uint32_t mulmod16(uint32_t a, uint32_t b, uint32_t p, uint32_t mu32)
{
    const uint32_t x = a * b;
    uint32_t r = x - __umulhi(x, mu32) * p;
    return r >= p ? r - p : r;
}

// a * b mod p, products of residues below 2^16 in 32 bits, else 64-bit Barrett
template <bool SMALL>
__device__ __forceinline__ uint32_t mulm(uint32_t a, uint32_t b, uint32_t p, uint32_t mu32, uint64_t mu)
{
    return SMALL ? mulmod16(a, b, p, mu32) : mulmod(a, b, p, mu);
}

// a^e mod p by square-and-multiply
template <bool SMALL>
__device__ __forceinline__ uint32_t powm(uint32_t a, uint32_t e, uint32_t p, uint32_t mu32, uint64_t mu)
{
    uint32_t r = 1 % p, b = a;
    while (e) {
        if (e & 1) r = mulm<SMALL>(r, b, p, mu32, mu);
        b = mulm<SMALL>(b, b, p, mu32, mu);
        e >>= 1;
    }
    return r;
}

// sum of a * b over 32 terms, reduced once: raw products below 2^32 when
// p < 2^16, reduced products otherwise (the sum stays below 2^37 either way)
template <bool SMALL>
__device__ __forceinline__ uint64_t mac(uint64_t acc, uint32_t a, uint32_t b, uint32_t p, uint64_t mu)
{
    return acc + (SMALL ? (uint64_t)a * b : (uint64_t)mulmod(a, b, p, mu));
}

// X <- L11^-1 (k x k, k <= 128), L11 the unit lower triangle of rows
// [r0, r0+k) x columns [c0, c0+k); X is written to the Morton-hybrid matrix Xm
// (zero above the diagonal, ones on it). Blocked in 32 x 32 blocks (the
// identity pads k to a multiple of 32): the diagonal blocks by forward
// substitution, one column of each per warp (unit_lower_inv_cols); then block
// row bi follows from the rows above it, X(bi, bj) = -X(bi, bi) sum_{bj <= m < bi}
// L(bi, m) X(m, bj), for all bj at once. Sums accumulate in 64 bits: raw
// products below p^2 < 2^32 when p < 2^16, products reduced mod p otherwise.
// L and X live in shared memory with a row stride of K + 1 words, so that a
// warp reading one column touches 32 different banks.
constexpr int kInvThreads = 1024;
constexpr int kInvStride = kNb + 1;

// x mod p for x < 2^40 (sums of at most 256 products below 2^32): Barrett with
// mu = floor((2^64 - 1) / p) leaves the remainder below 2p
__device__ __forceinline__ uint32_t red64(uint64_t x, uint32_t p, uint64_t mu)
{
    const uint64_t r = x - __umul64hi(x, mu) * p;
    return (uint32_t)(r >= p ? r - p : r);
}

__device__ __forceinline__ uint32_t neg_mod(uint64_t acc, uint32_t p, uint64_t mu)
{
    const uint32_t r = red64(acc, p, mu);
    return r == 0 ? 0u : p - r;
}

// NC columns of inverses of unit lower 32 x 32 triangles, one warp, by forward
// substitution: column c has index j[c] and its triangle's strictly lower part
// W (W(i, t) = 0 for t >= i); lrow[c] points at row `lane` of W. Lane i ends
// with X(i, j) in x[c]: X(i, j) = 0 for i < j, X(j, j) = 1 and
// X(i, j) = -sum_{j <= t < i} W(i, t) X(t, j) for i > j. Step t broadcasts the
// final X(t, j) from lane t, after which lane t + 1's sum is complete; the NC
// columns interleave, so their dependency chains overlap. Every lane runs every
// step, so the per-step work is what counts: for p < 2^16 each product is
// reduced at once (32-bit Barrett) and the sum of at most 31 residues stays
// below 2^21 in 32 bits; otherwise the sum of reduced products is kept in 64
// bits.
template <int NC, bool SMALL>
__device__ __forceinline__ void unit_lower_inv_cols(const uint32_t* const (&lrow)[NC], const int (&j)[NC],
                                                    uint32_t (&x)[NC], uint32_t p, uint32_t mu32, uint64_t mu,
                                                    int lane)
{
    uint64_t acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        acc[c] = 0;
        x[c] = lane == j[c] ? 1u : 0u;
    }
#pragma unroll
    for (int t = 0; t < 31; ++t) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const uint32_t xt = __shfl_sync(0xffffffffu, x[c], t);
            if (SMALL) {
                const uint32_t a = (uint32_t)acc[c] + mulmod16(lrow[c][t], xt, p, mu32);
                acc[c] = a;
                if (lane == t + 1 && t + 1 > j[c]) {
                    const uint32_t r = mulmod16(a, 1u, p, mu32);  // a < 2^21
                    x[c] = r == 0 ? 0u : p - r;
                }
            } else {
                acc[c] += mulmod(lrow[c][t], xt, p, mu);
                if (lane == t + 1 && t + 1 > j[c]) x[c] = neg_mod(acc[c], p, mu);
            }
        }
    }
}

// UPPER = false: X = L^-1 for the unit lower triangle L of A (as above).
// UPPER = true: X = U^-1 for the upper triangle U of A rows [r0, r0+k) x
// columns [c0, c0+k) with dinv[t] = 1 / U(t, t): U = diag(U) V with V unit
// upper, so the same inversion runs on the unit lower V^T, and
// U^-1 (i, j) = (V^T)^-1 (j, i) / U(j, j). The diagonal blocks of the inverse
// of a lower triangle are the inverses of its diagonal blocks: when dg is not
// null (k = 128) they are taken from there (block b's inverse column-major at
// dg + b * 2048 + (UPPER ? 1024 : 0), as diag_lu_kernel leaves them).
// A column block of the lower inverse depends on no other column block, so
// with cb >= 0 (k = 128) only block column cb is computed and stored: the
// columns [32 cb, 32 cb + 32) of X, or for UPPER the rows [32 cb, 32 cb + 32)
// of U^-1, which come from those columns of the inverse of V^T.
template <bool UPPER, bool SMALL>
__device__ __forceinline__ void tri_inv_body(const uint32_t* A, int lt, int64_t r0, int64_t c0, int k, uint32_t* X,
                                             int xlt, uint32_t p, uint64_t mu, const uint32_t* dinv,
                                             const uint32_t* dg, int cb = -1)
{
    const uint32_t mu32 = (uint32_t)(0xFFFFFFFFu / p);
    extern __shared__ uint32_t smx[];
    constexpr int K = kNb, S = kInvStride;  // padded size, 4 blocks of 32
    uint32_t* L = smx;                      // [K][S], strictly lower part
    uint32_t* Xs = smx + (size_t)K * S;     // [K][S]
    uint32_t* T = Xs + (size_t)K * S;       // [3][32][32]
    const int nb = (k + 31) / 32;
    // element e = (a, b) with b the fastest: a row of A is read along its
    // columns in both cases (UPPER: W(b, a) = U(a, b) / U(a, a))
#pragma unroll
    for (int q = 0; q < K * K / kInvThreads; ++q) {
        const int e = (int)threadIdx.x + q * kInvThreads;
        const int a = e / K, b = e % K;
        uint32_t v = 0;
        if (UPPER) {
            if (a < b && b < k) v = mulmod(A[fm_encode((uint64_t)(r0 + a), (uint64_t)(c0 + b), lt)], dinv[a], p, mu);
            L[b * S + a] = v;
        } else {
            if (b < a && a < k) v = A[fm_encode((uint64_t)(r0 + a), (uint64_t)(c0 + b), lt)];
            L[a * S + b] = v;
        }
        Xs[a * S + b] = a == b ? 1u : 0u;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 1. the diagonal blocks: column `warp` of each, one warp (or loaded)
    if (dg) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            Xs[(32 * b + lane) * S + 32 * b + warp] = dg[b * 2048 + (UPPER ? 1024 : 0) + warp * 32 + lane];
    } else {
        const uint32_t* lrow[4];
        int jj[4];
        uint32_t x[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            lrow[b] = L + (size_t)(32 * b + lane) * S + 32 * b;
            jj[b] = warp;
        }
        unit_lower_inv_cols<4, SMALL>(lrow, jj, x, p, mu32, mu, lane);
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (b < nb) Xs[(32 * b + lane) * S + 32 * b + warp] = x[b];
    }
    __syncthreads();
    // 2. block rows below the first: thread (r, c) = (warp, lane) of each 32 x 32 block
    for (int bi = 1; bi < nb; ++bi) {
        const int i = 32 * bi + warp;
        const int bj0 = cb < 0 ? 0 : cb, bj1 = cb < 0 ? bi : min(bi, cb + 1);
        if (bj0 >= bj1) continue;  // the same for every thread
        for (int bj = bj0; bj < bj1; ++bj) {
            uint64_t acc = 0;
#pragma unroll 8
            for (int t = 32 * bj; t < 32 * bi; ++t) acc = mac<SMALL>(acc, L[i * S + t], Xs[t * S + 32 * bj + lane], p, mu);
            T[(bj * 32 + warp) * 32 + lane] = red64(acc, p, mu);
        }
        __syncthreads();
        for (int bj = bj0; bj < bj1; ++bj) {
            uint64_t acc = 0;
#pragma unroll 8
            for (int s2 = 0; s2 < 32; ++s2)
                acc = mac<SMALL>(acc, Xs[i * S + 32 * bi + s2], T[(bj * 32 + s2) * 32 + lane], p, mu);
            Xs[i * S + 32 * bj + lane] = neg_mod(acc, p, mu);
        }
        __syncthreads();
    }
    if (cb >= 0) {
        for (int e = threadIdx.x; e < 32 * k; e += blockDim.x) {
            const int i = UPPER ? 32 * cb + e / k : e / 32, j = UPPER ? e % k : 32 * cb + e % 32;
            X[fm_encode((uint64_t)i, (uint64_t)j, xlt)] =
                UPPER ? mulmod(Xs[j * S + i], dinv[j], p, mu) : Xs[i * S + j];
        }
        return;
    }
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        X[fm_encode((uint64_t)i, (uint64_t)j, xlt)] =
            UPPER ? mulmod(Xs[j * S + i], dinv[j], p, mu) : Xs[i * S + j];
    }
}

template <bool SMALL>
__global__ void __launch_bounds__(kInvThreads) tri_inv_kernel(const uint32_t* A, int lt, int64_t r0, int64_t c0,
                                                              int k, uint32_t* X, int xlt, uint32_t p,
                                                              uint64_t mu)
{
    tri_inv_body<false, SMALL>(A, lt, r0, c0, k, X, xlt, p, mu, nullptr, nullptr);
}

// Both inverses of a diagonal block factored by diag_lu_kernel, one 32-wide
// block column each of eight CTAs: CTAs 0-3 write the block columns of
// X = L11^-1, CTAs 4-7 the block rows of Y = U11^-1. Launched right behind
// diag_lu_kernel, before the host has read its flag: when the fast path failed
// (*flag != 0) it returns at once.
template <bool SMALL>
__global__ void __launch_bounds__(kInvThreads) tri_inv2_kernel(const uint32_t* A, int lt, int64_t r0, int64_t c0,
                                                               uint32_t* X, uint32_t* Y, int xlt, uint32_t p,
                                                               uint64_t mu, const uint32_t* dinv, const int* flag,
                                                               const uint32_t* dg)
{
    if (*flag != 0) return;
    const int cb = (int)(blockIdx.x & 3);
    if (blockIdx.x < 4)
        tri_inv_body<false, SMALL>(A, lt, r0, c0, kNb, X, xlt, p, mu, nullptr, dg, cb);
    else
        tri_inv_body<true, SMALL>(A, lt, r0, c0, kNb, Y, xlt, p, mu, dinv, dg, cb);
}

// ---- diagonal-block fast path -------------------------------------------------
// In a panel whose 128 diagonal entries are all nonzero when elimination
// reaches them, the first-nonzero rule picks row r + t for column t: no row
// exchanges, and the panel factors as [L11; L21] U11 with L21 = A21 U11^-1.
// diag_lu_kernel factors the 128 x 128 diagonal block in one CTA, in shared
// memory, without divisions: step t replaces row i > t by c_t S_i - S_i[t] S_t
// (c_t = S_t[t]), which keeps every row a multiple sigma_t = c_0 ... c_{t-1} of
// the row the division form computes; afterwards l_it = S_i[t] / c_t and
// U row t = S_t / sigma_t, with all 2 x 128 inverses taken at once. A zero c_t
// means the rule would search below the block: *flag = 1 and the block is left
// unchanged (the column-by-column kernel then factors the panel). On success
// L11 (strictly lower) and U11 (upper) are written into A and dinv[t] =
// 1 / U11(t, t).
constexpr int kDiagThreads = 1024;

// Blocked in 32-wide block columns o = 0, 32, 64, 96 (the same L and U as the
// unblocked elimination without row exchanges, which are unique):
//   1. the 32 x 32 diagonal block by the division-free steps above, one entry
//      per thread per step (rows on warps, columns on lanes), then its 32
//      inverses at once; L_kk and U_kk written back;
//   2. L_kk^-1 and U_kk^-1 (as (V^T)^-1 transposed, U_kk = diag(U_kk) V) by
//      forward substitution, one column of each per warp; both inverses are
//      also left in dg for tri_inv2_kernel;
//   3. the panel below, L_ik = A_ik U_kk^-1, and the row to the right,
//      U_kj = L_kk^-1 A_kj, as 32-term dot products reduced once;
//   4. the trailing update A_ij -= L_ik U_kj, likewise.
template <bool SMALL>
__global__ void __launch_bounds__(kDiagThreads) diag_lu_kernel(uint32_t* A, int lt, int64_t r0, int64_t c0,
                                                               uint32_t p, uint64_t mu, uint32_t* dinv, int* flag,
                                                               uint32_t* dg)
{
    constexpr int K = kNb, B = 32;
    extern __shared__ uint32_t sm[];
    constexpr int S = B + 1;          // padded row stride: a column read hits 32 banks
    uint32_t* D = sm;                 // [K][K]
    uint32_t* Li = D + K * K;         // [B][S]  L_kk^-1
    uint32_t* Ui = Li + B * S;        // [B][B]  U_kk^-1
    uint32_t* Z = Ui + B * B;         // [B][S]  (V^T)^-1
    uint32_t* TL = Z + B * S;         // [K - B][B]  new panel below
    uint32_t* TU = TL + (K - B) * B;  // [B][K - B]  new row to the right
    __shared__ uint32_t cpiv[B], cinv[B], sinv[B], sig[B], dv[K];
    __shared__ int s_zero;
    const uint32_t mu32 = (uint32_t)(0xFFFFFFFFu / p);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < K * K / kDiagThreads; ++q) {
        const int e = tid + q * kDiagThreads;
        D[e] = A[fm_encode((uint64_t)(r0 + e / K), (uint64_t)(c0 + e % K), lt)];
    }
    if (tid == 0) s_zero = 0;
    for (int o = 0; o < K; o += B) {
        // 1. division-free LU of the diagonal block
        for (int t = 0; t < B; ++t) {
            __syncthreads();
            const uint32_t c = D[(o + t) * K + o + t];
            if (c == 0) {
                if (tid == 0) s_zero = 1;
                break;
            }
            if (tid == 0) cpiv[t] = c;
            if (warp < B - 1 - t && lane < B - 1 - t) {
                const int i = o + t + 1 + warp, j = o + t + 1 + lane;
                D[i * K + j] = submod(mulm<SMALL>(c, D[i * K + j], p, mu32, mu),
                                      mulm<SMALL>(D[i * K + o + t], D[(o + t) * K + j], p, mu32, mu), p);
            }
        }
        __syncthreads();
        if (s_zero) {
            if (tid == 0) *flag = 1;
            return;
        }
        if (warp == 0) {
            // sigma_t = c_0 ... c_{t-1}: an exclusive prefix product (warp scan),
            // then 1 / sigma_t
            uint32_t v = cpiv[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v = mulm<SMALL>(v, u, p, mu32, mu);
            }
            const uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
            const uint32_t g = lane == 0 ? 1 % p : ex;
            sig[lane] = g;
            sinv[lane] = powm<SMALL>(g, p - 2, p, mu32, mu);
        } else if (warp == 1) {
            cinv[lane] = powm<SMALL>(cpiv[lane], p - 2, p, mu32, mu);
        }
        __syncthreads();
        {  // normalise: l_it = S_i[t] / c_t below the diagonal, U row t = S_t / sigma_t
            const int i = warp, j = lane;
            uint32_t& v = D[(o + i) * K + o + j];
            v = mulm<SMALL>(v, i > j ? cinv[j] : sinv[i], p, mu32, mu);
            if (i == 0) dv[o + j] = mulm<SMALL>(sig[j], cinv[j], p, mu32, mu);  // 1 / u_jj
        }
        __syncthreads();
        // 2. L_kk^-1 and (V^T)^-1 with V^T(i, t) = U(t, i) / u_tt, both unit
        //    lower: their strictly lower parts W1, W2 are copied to padded
        //    [B][S] arrays in TL (free until step 3), then warp w solves for
        //    column w of both inverses by forward substitution
        {
            uint32_t* W1 = TL;
            uint32_t* W2 = TL + B * S;
            const int i = warp, t = lane;
            W1[i * S + t] = t < i ? D[(o + i) * K + o + t] : 0u;
            // thread (warp, lane) = (t', i'): reads row t' of U along its columns
            W2[lane * S + warp] = warp < lane ? mulm<SMALL>(D[(o + warp) * K + o + lane], dv[o + warp], p, mu32, mu) : 0u;
        }
        __syncthreads();
        {
            const uint32_t* lrow[2] = {TL + lane * S, TL + B * S + lane * S};
            const int jj[2] = {warp, warp};
            uint32_t x[2];
            unit_lower_inv_cols<2, SMALL>(lrow, jj, x, p, mu32, mu, lane);
            Li[lane * S + warp] = x[0];
            Z[lane * S + warp] = x[1];
            // both, column-major, for tri_inv2_kernel (the diagonal blocks of
            // L11^-1 and of (V^T)^-1)
            dg[(o / B) * 2048 + warp * 32 + lane] = x[0];
            dg[(o / B) * 2048 + 1024 + warp * 32 + lane] = x[1];
        }
        __syncthreads();
        Ui[warp * B + lane] = warp <= lane ? mulm<SMALL>(Z[lane * S + warp], dv[o + lane], p, mu32, mu) : 0u;
        __syncthreads();
        if (o + B >= K) break;
        // 3. the panel below and the row to the right
        //    (all 32 terms: U_kk^-1 is zero below its diagonal, L_kk^-1 above)
        for (int i = o + B + warp; i < K; i += 32) {
            uint64_t acc = 0;
#pragma unroll 8
            for (int t = 0; t < B; ++t) acc = mac<SMALL>(acc, D[i * K + o + t], Ui[t * B + lane], p, mu);
            TL[(i - o - B) * B + lane] = red64(acc, p, mu);
        }
        for (int j = o + B + lane; j < K; j += 32) {
            uint64_t acc = 0;
#pragma unroll 8
            for (int t = 0; t < B; ++t) acc = mac<SMALL>(acc, Li[warp * S + t], D[(o + t) * K + j], p, mu);
            TU[warp * (K - B) + (j - o - B)] = red64(acc, p, mu);
        }
        __syncthreads();
        for (int i = o + B + warp; i < K; i += 32) D[i * K + o + lane] = TL[(i - o - B) * B + lane];
        for (int j = o + B + lane; j < K; j += 32) D[(o + warp) * K + j] = TU[warp * (K - B) + (j - o - B)];
        __syncthreads();
        // 4. trailing update
        for (int i = o + B + warp; i < K; i += 32) {
            for (int j = o + B + lane; j < K; j += 32) {
                uint64_t acc = 0;
#pragma unroll 8
                for (int t = 0; t < B; ++t) acc = mac<SMALL>(acc, D[i * K + o + t], D[(o + t) * K + j], p, mu);
                D[i * K + j] = submod(D[i * K + j], red64(acc, p, mu), p);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K * K / kDiagThreads; ++q) {
        const int e = tid + q * kDiagThreads;
        A[fm_encode((uint64_t)(r0 + e / K), (uint64_t)(c0 + e % K), lt)] = D[e];
    }
    if (tid < K) dinv[tid] = dv[tid];
    if (tid == 0) *flag = 0;
}

}  // namespace

extern "C" int fm_pluq(fm_matrix Am, int64_t m, int64_t n, uint32_t p, int32_t* row_perm,
                       int32_t* col_perm, int64_t* rank, fm_stream stream)
{
    FmRange range("fm_pluq");
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    FM_TRY(fm_check_matrix(Am));
    if (m < 0 || n < 0 || m > fm_side(Am) || n > fm_side(Am) || !rank) return FM_EINVAL;
    if (m >= INT_MAX || n >= INT_MAX) return FM_EINVAL;
    if ((m > 0 && !row_perm) || (n > 0 && !col_perm)) return FM_EINVAL;
    if (Am.log2_T < 2) return FM_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    *rank = 0;
    // identity row permutation
    {
        std::vector<int32_t> id((size_t)m);
        for (int64_t i = 0; i < m; ++i) id[(size_t)i] = (int32_t)i;
        if (m) FM_CUDA_TRY(cudaMemcpyAsync(row_perm, id.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
        FM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // device workspace: piv_slot[kNb], piv_row[kNb], order[kNb], n_piv, barrier[2],
    // swap pairs[2 kNb], candidate rows [kNb][grid][kNb + 2], status words [kNb][grid]
    int dev = 0, coop = 0, per_sm = 0, max_smem = 0;
    FM_CUDA_TRY(cudaGetDevice(&dev));
    FM_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    FM_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (!coop) return FM_EUNSUPPORTED;
    const int sms = fm_sm_count();
    const size_t ws_ints = 3 * kNb + 4 + 2 * kNb + 2 * ((size_t)kNb * sms * (kNb + 2) + (size_t)kNb * sms);
    int* ws = static_cast<int*>(fm_workspace(1, sizeof(int) * ws_ints));
    if (!ws) return FM_ENOMEM;
    int* d_slot = ws;
    int* d_piv = ws + kNb;
    int* d_order = ws + 2 * kNb;
    int* d_npiv = ws + 3 * kNb;
    unsigned* d_bar = reinterpret_cast<unsigned*>(ws + 3 * kNb + 2);
    int* d_pairs = ws + 3 * kNb + 4;
    // tagged candidate slots and status words (8-byte aligned: 5 kNb + 4 ints in)
    uint2* d_cand = reinterpret_cast<uint2*>(ws + 5 * kNb + 4);
    uint2* d_stat = d_cand + (size_t)kNb * sms * (kNb + 2);
    FM_CUDA_TRY(cudaMemsetAsync(d_cand, 0, sizeof(uint2) * ((size_t)kNb * sms * (kNb + 2) + (size_t)kNb * sms), s));
    FM_CUDA_TRY(cudaMemsetAsync(d_bar, 0, 2 * sizeof(unsigned), s));

    FM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel, kPanelThreads, 0));
    if (per_sm < 1) return FM_EUNSUPPORTED;
    const int grid_g = sms * std::min(per_sm, 2);  // global-memory panel kernel
    const uint64_t mu = ~0ull / p;

    // After a panel with k pivots in rows [r, r + k) and columns [c0, c0 + k):
    // U12 <- L11^-1 A12 as a product (Sec. 2: S_A = S_B * S_C) with X = L11^-1
    // (written into A12 itself: the limb product splits A12 into planes before
    // A12 is written), then A22 <- A22 - L21 U12 by fm_gemm_modp on three
    // disjoint sub-matrices of A.
    // Two-level blocking: up to kOuter consecutive panels form an outer block.
    // Inside it each panel's update reaches only the block's own columns; the
    // columns behind the block receive the whole block's update at once, as
    // U12 <- L11^-1 A12 by block forward substitution over its panels and one
    // product A22 <- A22 - L21 U12 with K = the block's pivots (up to 512),
    // which has a quarter of the epilogue work of four K = 128 updates. A block
    // ends after a panel with fewer than 128 pivots (its pivot columns stay
    // contiguous: a panel moves its pivot columns in front of its skipped ones).
    // Look-ahead: at the end of a block, stream s (the caller's) updates only
    // the next block's columns and goes on with its panels; the columns behind
    // those take the block's update on a second stream u, which waits (an event)
    // for the block's panels on s. s waits for u before it touches those columns
    // itself (at the next block's end), before row swaps of a searched panel
    // (they reach every column) and before the final column permutation. u's
    // products run in their own plane workspace on a capped number of CTAs, so
    // that the panels' one-CTA kernels and thin products find SMs free;
    // the panels' inverses X alternate between two sets by block parity (u reads
    // a block's set while the next block writes the other).
    constexpr int kOuter = 4;
    int64_t c0 = 0, c_out = 0, r_out = 0;
    int nbk = 0;           // panels in the open outer block
    int bk[kOuter] = {0};  // pivots of each
    int blk = 0;           // outer blocks opened so far
    int cur_set = 0;       // the open block's set of inverses
    int fast_panels = 0, searched_panels = 0, zero_panels = 0;
    struct LookAhead {
        cudaStream_t u = nullptr;
        cudaStream_t v = nullptr;  // side stream: a panel row's product beside its L21 product
        cudaEvent_t ev_v0 = nullptr, ev_v1 = nullptr;
        cudaEvent_t ev_s = nullptr, ev_u = nullptr, ev_flag = nullptr;
        int* h_flag = nullptr;  // pinned: the fast path's flag arrives without blocking the host
        bool pending = false;  // work enqueued on u since s last waited for it
        int64_t lo = 0;        // while pending: u may still write columns [lo, n)
        int set = 0;           // while pending: the set of inverses u reads
        ~LookAhead()
        {
            if (u) {
                cudaStreamSynchronize(u);
                cudaStreamDestroy(u);
            }
            if (v) {
                cudaStreamSynchronize(v);
                cudaStreamDestroy(v);
            }
            if (ev_v0) cudaEventDestroy(ev_v0);
            if (ev_v1) cudaEventDestroy(ev_v1);
            if (ev_s) cudaEventDestroy(ev_s);
            if (ev_u) cudaEventDestroy(ev_u);
            if (ev_flag) cudaEventDestroy(ev_flag);
            if (h_flag) cudaFreeHost(h_flag);
        }
    } la;
    FM_CUDA_TRY(cudaStreamCreateWithFlags(&la.u, cudaStreamNonBlocking));
    FM_CUDA_TRY(cudaStreamCreateWithFlags(&la.v, cudaStreamNonBlocking));
    FM_CUDA_TRY(cudaEventCreateWithFlags(&la.ev_v0, cudaEventDisableTiming));
    FM_CUDA_TRY(cudaEventCreateWithFlags(&la.ev_v1, cudaEventDisableTiming));
    FM_CUDA_TRY(cudaEventCreateWithFlags(&la.ev_s, cudaEventDisableTiming));
    FM_CUDA_TRY(cudaEventCreateWithFlags(&la.ev_u, cudaEventDisableTiming));
    FM_CUDA_TRY(cudaEventCreateWithFlags(&la.ev_flag, cudaEventDisableTiming));
    FM_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&la.h_flag), sizeof(int), cudaHostAllocDefault));
    auto wait_u = [&]() -> int {  // s waits for everything enqueued on u so far
        if (!la.pending) return FM_OK;
        FM_CUDA_TRY(cudaEventRecord(la.ev_u, la.u));
        FM_CUDA_TRY(cudaStreamWaitEvent(s, la.ev_u, 0));
        la.pending = false;
        return FM_OK;
    };
    // u waits for everything enqueued on s so far, then takes columns [lo, n)
    // (s has waited for u's earlier work before every call)
    auto start_u = [&](int64_t lo) -> int {
        FM_CUDA_TRY(cudaEventRecord(la.ev_s, s));
        FM_CUDA_TRY(cudaStreamWaitEvent(la.u, la.ev_s, 0));
        la.pending = true;
        la.lo = lo;
        la.set = cur_set;
        return FM_OK;
    };
    // u's GEMM CTAs: all but one SM in twelve (140 of 152). With the side stream
    // v also running, a 16384 x 12288 rank-10000 factorization took 29.7 / 27.8 /
    // 27.5 / 31.5 / 30.1 ms at 100 / 121 / 140 / 152 / 170 CTAs: at 152 or more u
    // reaches every SM and the one-CTA panel kernels, which take a whole SM's
    // registers, wait for it; at 121 or fewer u is starved
    const int u_ctas = std::max(2, sms - sms / 12);
    // plane workspaces sized once for the largest product (K = a block's pivots),
    // so that neither stream's workspace is reallocated while the other runs
    {
        size_t most = 0;
        for (int bn : {128, 256}) {
            fm_opts o{};
            o.block_n = bn;
            FmLimbPlan lq;
            if (fm_limb_plan(m, n, (int64_t)kOuter * kNb, p, &o, &lq) == FM_OK)
                most = std::max(most, fm_limb_workspace_bytes(lq));
        }
        if (most && (!fm_workspace(0, most) || !fm_workspace(5, most) || !fm_workspace(6, most)))
            return FM_ENOMEM;
    }
    // C op A * B with every operand a sub-matrix of A (the limb product writes
    // C over the B operand when they are the same part: it splits B first):
    // product on s (fm_gemm_modp's own choice of form), product_v on the side
    // stream v in a workspace of its own, product_u on the look-ahead stream u
    // in another, on capped CTAs
    auto product_v = [&](const fm_sub& C, const fm_sub& Aop, const fm_sub& Bop, int op) -> int {
        if (C.rows == 0 || C.cols == 0 || Aop.cols == 0) return FM_OK;
        FmLimbPlan lq;
        FM_TRY(fm_limb_plan_shaped(C.rows, C.cols, Aop.cols, p, nullptr, &lq));
        void* lws = fm_workspace(6, fm_limb_workspace_bytes(lq));
        if (!lws) return FM_ENOMEM;
        return fm_limb_run(lq, C, Aop, Bop, p, op, lws, status, la.v);
    };
    auto product_u = [&](const fm_sub& C, const fm_sub& Aop, const fm_sub& Bop, int op) -> int {
        if (C.rows == 0 || C.cols == 0 || Aop.cols == 0) return FM_OK;
        FmLimbPlan lq;
        FM_TRY(fm_limb_plan_shaped(C.rows, C.cols, Aop.cols, p, nullptr, &lq));
        lq.max_ctas = u_ctas;
        void* lws = fm_workspace(5, fm_limb_workspace_bytes(lq));
        if (!lws) return FM_ENOMEM;
        return fm_limb_run(lq, C, Aop, Bop, p, op, lws, status, la.u);
    };
    auto product = [&](const fm_sub& C, const fm_sub& Aop, const fm_sub& Bop, int op) -> int {
        if (C.rows == 0 || C.cols == 0 || Aop.cols == 0) return FM_OK;
        if (op == FM_OP_SET) {
            FmLimbPlan lq;
            FM_TRY(fm_limb_plan_shaped(C.rows, C.cols, Aop.cols, p, nullptr, &lq));
            void* lws = fm_workspace(0, fm_limb_workspace_bytes(lq));
            if (!lws) return FM_ENOMEM;
            return fm_limb_run(lq, C, Aop, Bop, p, FM_OP_SET, lws, status, s);
        }
        return fm_gemm_modp(C, Aop, Bop, p, op, FM_ALGO_AUTO, nullptr, stream);
    };
    // After a panel with k pivots in rows [r_, r_ + k) and columns [c0, c0 + k):
    // U12 <- L11^-1 A12 (X = L11^-1) and A22 <- A22 - L21 U12 on columns
    // [c_from, c_to).
    auto update_cols = [&](int64_t r_, int k_, fm_matrix Xm, int64_t c_from, int64_t c_to, bool on_u = false) -> int {
        if (c_from >= c_to || k_ == 0) return FM_OK;
        const int64_t cols = c_to - c_from;
        const fm_sub A12{Am, r_, c_from, k_, cols};
        auto prod = [&](const fm_sub& C, const fm_sub& Aop, const fm_sub& Bop, int op) {
            return on_u ? product_u(C, Aop, Bop, op) : product(C, Aop, Bop, op);
        };
        FM_TRY(prod(A12, fm_sub{Xm, 0, 0, k_, k_}, A12, FM_OP_SET));
        return prod(fm_sub{Am, r_ + k_, c_from, m - r_ - k_, cols}, fm_sub{Am, r_ + k_, c0, m - r_ - k_, k_}, A12,
                    FM_OP_SUB);
    };
    uint32_t* xs_base = nullptr;  // X of each panel, two sets of kOuter (set per panel below)
    // Closes the open block after its last panel (ending at column c_end, rows
    // up to r_now). Columns [c_end, c_lim) -- the block's own columns behind
    // that panel, when the block ended early -- already hold the updates of
    // the block's earlier panels and take only the last panel's; columns
    // [c_lim, n) take the whole block's: on s up to la_end, the end of the next
    // block's columns, and on u beyond.
    auto finish_outer = [&](int64_t c_end, int64_t c_lim, int64_t r_now) -> int {
        const int n_bk = nbk;
        nbk = 0;
        const int64_t k_out = r_now - r_out;
        if (k_out == 0) return FM_OK;
        uint32_t* xset = xs_base + (size_t)cur_set * kOuter * kNb * kNb;
        const int64_t la_end = std::min<int64_t>(n, c_end + (int64_t)kOuter * kNb);
        FM_TRY(wait_u());  // u's columns of the previous block are about to be touched
        const int k_last = bk[n_bk - 1];
        if (n_bk == 1) {  // a block of one panel: no column has any of its update yet
            const fm_matrix X0{xset, 0, 7};
            FM_TRY(update_cols(r_out, k_last, X0, c_end, la_end));
            if (la_end >= n) return FM_OK;
            FM_TRY(start_u(la_end));
            return update_cols(r_out, k_last, X0, la_end, n, true);
        }
        if (c_end < c_lim && k_last > 0) {
            const fm_matrix Xl{xset + (size_t)(n_bk - 1) * kNb * kNb, 0, 7};
            FM_TRY(update_cols(r_now - k_last, k_last, Xl, c_end, c_lim));
        }
        c_end = std::max(c_end, c_lim);
        // columns [lo, hi): U12 <- L11^-1 A12 by block forward substitution over
        // the block's panels, then A22 <- A22 - L21 U12 with K = the block's pivots
        auto block_cols = [&](int64_t lo, int64_t hi, bool on_u) -> int {
            if (lo >= hi) return FM_OK;
            auto prod = [&](const fm_sub& C, const fm_sub& Aop, const fm_sub& Bop, int op) {
                return on_u ? product_u(C, Aop, Bop, op) : product(C, Aop, Bop, op);
            };
            const int64_t cols = hi - lo;
            for (int i = 0; i < n_bk; ++i) {
                if (bk[i] == 0) continue;
                const int64_t ri = r_out + (int64_t)kNb * i;
                const fm_sub Ai{Am, ri, lo, bk[i], cols};
                if (i > 0)
                    FM_TRY(prod(Ai, fm_sub{Am, ri, c_out, bk[i], (int64_t)kNb * i},
                                fm_sub{Am, r_out, lo, (int64_t)kNb * i, cols}, FM_OP_SUB));
                const fm_matrix Xi{xset + (size_t)i * kNb * kNb, 0, 7};
                FM_TRY(prod(Ai, fm_sub{Xi, 0, 0, bk[i], bk[i]}, Ai, FM_OP_SET));
            }
            return prod(fm_sub{Am, r_now, lo, m - r_now, cols}, fm_sub{Am, r_now, c_out, m - r_now, k_out},
                        fm_sub{Am, r_out, lo, k_out, cols}, FM_OP_SUB);
        };
        const int64_t mid = std::max(c_end, la_end);
        FM_TRY(block_cols(c_end, mid, false));
        if (mid >= n) return FM_OK;
        FM_TRY(start_u(mid));
        return block_cols(mid, n, true);
    };
    std::vector<int> colid((size_t)n);  // original column at each storage position
    for (int64_t j = 0; j < n; ++j) colid[(size_t)j] = (int)j;
    std::vector<int> pivot_pos, skipped_pos;
    int64_t r = 0;
    for (c0 = 0; c0 < n; c0 += kNb) {
        const int w = (int)std::min<int64_t>(kNb, n - c0);
        if (r >= m) {
            for (int t = 0; t < w; ++t) skipped_pos.push_back((int)(c0 + t));
            continue;
        }
        // X = L11^-1 of each panel of the open block, Y = U11^-1 (the fast
        // path), 1 / U11(t, t), and the flags
        xs_base = static_cast<uint32_t*>(
            fm_workspace(4, (size_t)((2 * kOuter + 1) * kNb * kNb + kNb + 4 + 8 * 1024) * 4));
        if (!xs_base) return FM_ENOMEM;
        if (nbk == 0) {
            c_out = c0;
            r_out = r;
            cur_set = (blk++) & 1;
            if (la.pending && la.set == cur_set) FM_TRY(wait_u());  // u still reads this set
        }
        uint32_t* xs = xs_base + ((size_t)cur_set * kOuter + nbk) * kNb * kNb;
        uint32_t* ys = xs_base + (size_t)2 * kOuter * kNb * kNb;
        uint32_t* dinv = ys + kNb * kNb;
        int* d_flag = reinterpret_cast<int*>(dinv + kNb);
        uint32_t* dgs = reinterpret_cast<uint32_t*>(d_flag + 4);  // diagonal 32 x 32 inverses
        const int64_t c_lim = std::min<int64_t>(c_out + (int64_t)kOuter * kNb, n);
        // this panel and its block's updates touch columns [c0, c_lim): u must
        // be done with them (a block that follows an all-zero one starts past
        // the columns the previous block end left to s)
        if (la.pending && c_lim > la.lo) FM_TRY(wait_u());
        // after a panel with k pivots: the rest of the block's columns now, or,
        // when the panel ends the block, everything behind it
        auto after_panel = [&](int k, fm_matrix Xm) -> int {
            bk[nbk++] = k;
            const bool ends = k < kNb || nbk == kOuter || c0 + w >= n || r + k >= m;
            if (!ends) return update_cols(r, k, Xm, c0 + w, c_lim);
            return finish_outer(c0 + w, c_lim, r + k);
        };
        const size_t ismem = ((size_t)2 * kNb * kInvStride + 3 * 32 * 32) * 4;
        // diagonal-block fast path, tried first: a full panel whose 128 diagonal
        // pivots are nonzero (the rows the first-nonzero rule picks) factors
        // without the column-by-column search
        if (w == kNb && r + kNb <= m) {
            const size_t dsmem = ((size_t)kNb * kNb + 2 * 32 * 33 + 32 * 32 + 2 * (kNb - 32) * 32) * 4;
            auto dk = p < (1u << 16) ? diag_lu_kernel<true> : diag_lu_kernel<false>;
            FM_CUDA_TRY(cudaFuncSetAttribute(dk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
            dk<<<1, kDiagThreads, dsmem, s>>>(Am.base, Am.log2_T, r, c0, p, mu, dinv, d_flag, dgs);
            FM_CUDA_TRY(cudaGetLastError());
            // the flag goes to the host right behind the block; both inverses
            // run meanwhile (they return at once if the fast path failed), and
            // the host, which waits for the flag only, queues what follows
            // while they run
            FM_CUDA_TRY(cudaMemcpyAsync(la.h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            FM_CUDA_TRY(cudaEventRecord(la.ev_flag, s));
            auto ik = p < (1u << 16) ? tri_inv2_kernel<true> : tri_inv2_kernel<false>;
            FM_CUDA_TRY(cudaFuncSetAttribute(ik, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
            ik<<<8, kInvThreads, ismem, s>>>(Am.base, Am.log2_T, r, c0, xs, ys, 7, p, mu, dinv, d_flag, dgs);
            FM_CUDA_TRY(cudaGetLastError());
            FM_CUDA_TRY(cudaEventSynchronize(la.ev_flag));
            const int flag = *la.h_flag;
            if (flag == 0) {
                ++fast_panels;
                for (int t = 0; t < kNb; ++t) pivot_pos.push_back((int)(c0 + t));
                const fm_matrix Xm{xs, 0, 7}, Ym{ys, 0, 7};
                // A panel that does not end its block updates the block's columns
                // behind it: U12 <- L11^-1 A12, then A22 <- A22 - L21 U12. U12
                // does not depend on L21, so it runs on the side stream v (once
                // the inverses are done) beside the L21 product, and s waits for
                // it before the update.
                const bool inner = nbk + 1 < kOuter && c0 + w < n && r + kNb < m && c0 + w < c_lim;
                const fm_sub A12{Am, r, c0 + w, kNb, c_lim - (c0 + w)};
                if (inner) {
                    FM_CUDA_TRY(cudaEventRecord(la.ev_v0, s));
                    FM_CUDA_TRY(cudaStreamWaitEvent(la.v, la.ev_v0, 0));
                    FM_TRY(product_v(A12, fm_sub{Xm, 0, 0, kNb, kNb}, A12, FM_OP_SET));
                    FM_CUDA_TRY(cudaEventRecord(la.ev_v1, la.v));
                }
                if (r + kNb < m) {
                    // L21 <- A21 U11^-1, over A21 itself (its planes are split before it is written)
                    const fm_sub A21{Am, r + kNb, c0, m - r - kNb, kNb};
                    FmLimbPlan lq;
                    FM_TRY(fm_limb_plan_shaped(m - r - kNb, kNb, kNb, p, nullptr, &lq));
                    void* lws = fm_workspace(0, fm_limb_workspace_bytes(lq));
                    if (!lws) return FM_ENOMEM;
                    FM_TRY(fm_limb_run(lq, A21, A21, fm_sub{Ym, 0, 0, kNb, kNb}, p, FM_OP_SET, lws, status, s));
                }
                if (inner) {
                    FM_CUDA_TRY(cudaStreamWaitEvent(s, la.ev_v1, 0));
                    bk[nbk++] = kNb;
                    FM_TRY(product(fm_sub{Am, r + kNb, c0 + w, m - r - kNb, A12.cols},
                                   fm_sub{Am, r + kNb, c0, m - r - kNb, kNb}, A12, FM_OP_SUB));
                } else {
                    FM_TRY(after_panel(kNb, Xm));
                }
                r += kNb;
                continue;
            }
        }
        // otherwise: a panel without a nonzero in rows [r, m) has no pivot: skip it
        {
            FM_CUDA_TRY(cudaMemsetAsync(d_flag + 1, 0, sizeof(int), s));
            const int64_t ctas = (m - r + 7) / 8;  // one warp per row, 8 warps a CTA
            panel_nonzero_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)sms * 8)), 256, 0, s>>>(
                Am.base, Am.log2_T, r, m, c0, w, d_flag + 1);
            FM_CUDA_TRY(cudaGetLastError());
            int nz = 1;
            FM_CUDA_TRY(cudaMemcpyAsync(&nz, d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
            FM_CUDA_TRY(cudaStreamSynchronize(s));
            if (!nz) {
                ++zero_panels;
                for (int t = 0; t < w; ++t) skipped_pos.push_back((int)(c0 + t));
                FM_TRY(after_panel(0, fm_matrix{xs, 0, 7}));
                continue;
            }
        }
        ++searched_panels;
        FM_TRY(wait_u());  // its row swaps reach every column
        std::vector<int> slots(kNb, INT_MAX);
        FM_CUDA_TRY(cudaMemcpyAsync(d_slot, slots.data(), sizeof(int) * kNb, cudaMemcpyHostToDevice, s));
        // panel rows resident in shared memory when a CTA's share fits
        const int R = (int)((m - r + sms - 1) / sms);
        const size_t psmem = ((size_t)R * w + kNb + 2 * (size_t)R) * 4;
        const bool smem_path = psmem <= (size_t)max_smem;
        if (smem_path) {
            SmemPanelArgs pa;
            pa.A = Am.base;
            pa.lt = Am.log2_T;
            pa.m = m;
            pa.r0 = r;
            pa.c0 = c0;
            pa.w = w;
            pa.rows_per_cta = R;
            pa.p = p;
            pa.mu = mu;
            pa.stat = d_stat;
            pa.cand = d_cand;
            pa.tag0 = next_tags();
            pa.piv_row = d_piv;
            pa.n_piv = d_npiv;
            pa.bar = d_bar;
            pa.status = status;
            FM_CUDA_TRY(cudaFuncSetAttribute(smem_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)psmem));
            void* kargs[] = {&pa};
            FM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)smem_panel_kernel, sms, kPanelThreads,
                                                    kargs, psmem, s));
        } else {
            PanelArgs pa;
            pa.A = Am.base;
            pa.lt = Am.log2_T;
            pa.m = m;
            pa.r0 = r;
            pa.c0 = c0;
            pa.w = w;
            pa.p = p;
            pa.mu = mu;
            pa.piv_slot = d_slot;
            pa.piv_row = d_piv;
            pa.n_piv = d_npiv;
            pa.bar = d_bar;
            pa.status = status;
            void* kargs[] = {&pa};
            FM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_kernel, grid_g, kPanelThreads,
                                                    kargs, 0, s));
        }
        std::vector<int> piv(kNb);
        int npiv = 0;
        FM_CUDA_TRY(cudaMemcpyAsync(piv.data(), d_piv, sizeof(int) * w, cudaMemcpyDeviceToHost, s));
        FM_CUDA_TRY(cudaMemcpyAsync(&npiv, d_npiv, sizeof(int), cudaMemcpyDeviceToHost, s));
        FM_CUDA_TRY(cudaStreamSynchronize(s));
        int st = 0;
        FM_CUDA_TRY(cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st != 0) return st;
        // pivot columns of the panel first, then its skipped columns
        std::vector<int> order;
        for (int t = 0; t < w; ++t)
            if (piv[t] >= 0) order.push_back(t);
        const int k = (int)order.size();
        for (int t = 0; t < w; ++t)
            if (piv[t] < 0) order.push_back(t);
        bool moved = false;
        for (int t = 0; t < w; ++t) moved |= order[t] != t;
        if (moved) {
            FM_CUDA_TRY(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * w, cudaMemcpyHostToDevice, s));
            permute_panel_cols_kernel<<<std::max<int64_t>(1, std::min<int64_t>((m + 7) / 8, 4096)), 256, 0, s>>>(
                Am.base, Am.log2_T, m, c0, w, d_order);
            FM_CUDA_TRY(cudaGetLastError());
            std::vector<int> ids(colid.begin() + c0, colid.begin() + c0 + w);
            for (int t = 0; t < w; ++t) colid[(size_t)(c0 + t)] = ids[(size_t)order[t]];
        }
        for (int t = 0; t < k; ++t) pivot_pos.push_back((int)(c0 + t));
        for (int t = k; t < w; ++t) skipped_pos.push_back((int)(c0 + t));
        if (k > 0) {
            const int sgrid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048));
            if (smem_path) {
                // the panel left rows in place: bring the k pivot rows to r .. r+k-1
                std::unordered_map<int, int> pos_of, row_at;  // rows moved so far
                auto where = [&](int row) {
                    auto it = pos_of.find(row);
                    return it == pos_of.end() ? row : it->second;
                };
                auto who = [&](int pos) {
                    auto it = row_at.find(pos);
                    return it == row_at.end() ? pos : it->second;
                };
                std::vector<int> pairs;
                int q = 0;
                for (int t = 0; t < w; ++t) {
                    if (piv[t] < 0) continue;
                    const int target = (int)(r + q);
                    const int cur = where(piv[t]);
                    if (cur != target) {
                        const int displaced = who(target);
                        pairs.push_back(target);
                        pairs.push_back(cur);
                        pos_of[piv[t]] = target;
                        row_at[target] = piv[t];
                        pos_of[displaced] = cur;
                        row_at[cur] = displaced;
                    }
                    ++q;
                }
                const int npairs = (int)pairs.size() / 2;
                if (npairs > 0) {
                    FM_CUDA_TRY(cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(int) * pairs.size(),
                                                cudaMemcpyHostToDevice, s));
                    swap_pairs_kernel<<<sgrid, 256, 0, s>>>(Am.base, Am.log2_T, n, d_pairs, npairs, row_perm);
                    FM_CUDA_TRY(cudaGetLastError());
                }
            } else {
                row_swaps_kernel<<<sgrid, 256, 0, s>>>(Am.base, Am.log2_T, n, c0, w, r, d_piv, w);
                FM_CUDA_TRY(cudaGetLastError());
                perm_swaps_kernel<<<1, 32, 0, s>>>(row_perm, r, d_piv, w);
                FM_CUDA_TRY(cudaGetLastError());
            }
            auto ik = p < (1u << 16) ? tri_inv_kernel<true> : tri_inv_kernel<false>;
            FM_CUDA_TRY(cudaFuncSetAttribute(ik, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
            ik<<<1, kInvThreads, ismem, s>>>(Am.base, Am.log2_T, r, c0, k, xs, 7, p, mu);
            FM_CUDA_TRY(cudaGetLastError());
        }
        FM_TRY(after_panel(k, fm_matrix{xs, 0, 7}));
        r += k;
    }
    FM_TRY(wait_u());
    // move every skipped column behind all pivot columns
    std::vector<int> final_order(pivot_pos);
    final_order.insert(final_order.end(), skipped_pos.begin(), skipped_pos.end());
    bool moved = false;
    for (int64_t t = 0; t < n; ++t) moved |= final_order[(size_t)t] != t;
    std::vector<int32_t> cp((size_t)n);
    for (int64_t t = 0; t < n; ++t) cp[(size_t)t] = colid[(size_t)final_order[(size_t)t]];
    if (n) FM_CUDA_TRY(cudaMemcpyAsync(col_perm, cp.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    if (moved) {
        if ((size_t)n * 4 > 200 * 1024) return FM_EUNSUPPORTED;  // a row must fit in shared memory
        int32_t* d_ord = static_cast<int32_t*>(fm_workspace(3, (size_t)n * 4));
        if (!d_ord) return FM_ENOMEM;
        std::vector<int32_t> ord32(final_order.begin(), final_order.end());
        FM_CUDA_TRY(cudaMemcpyAsync(d_ord, ord32.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        const size_t rsmem = (size_t)n * 4;
        FM_CUDA_TRY(cudaFuncSetAttribute(permute_cols_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem));
        permute_cols_rows_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>(m, (int64_t)fm_sm_count() * 4)),
                                   256, rsmem, s>>>(Am.base, Am.log2_T, m, n, d_ord);
        FM_CUDA_TRY(cudaGetLastError());
    }
    FM_CUDA_TRY(cudaStreamSynchronize(s));
    *rank = r;
    fm_trace("pluq m=%lld n=%lld p=%u rank=%lld panels of %d columns: %d diagonal-block, %d searched, %d zero",
             (long long)m, (long long)n, p, (long long)r, kNb, fast_panels, searched_panels, zero_panels);
    return FM_OK;
}
