/*
 * fm.h -- C ABI of libfm: exact modular matrix multiply on Morton-hybrid
 * matrices for NVIDIA GB300 (sm_103a).
 *
 * Abu Salem and Al Arab, "Cache-oblivious Matrix Multiplication for Exact
 * Factorisation" (arXiv 1705.04807):
 *   Sec. 1   the Morton-hybrid layout: Z-order over T' x T' tiles, each tile
 *            row-major; TU decomposition with row and column permutations.
 *   Sec. 2   the problem: multiply sub-matrices S_A = S_B * S_C (accumulated
 *            as S_A += S_B * S_C) of Morton-hybrid matrices over a finite field.
 *   Sec. 2.1 aligned and contained sub-matrices; base cases on contained parts.
 *   Sec. 2.2 Steps 1-4: recursion on the aligned parents, so every base case
 *            multiplies parts that each lie inside one row-major tile.
 *
 * Naming. The library writes the update as C <- C op A*B (mod p); the paper's
 * S_A, S_B, S_C are this C, A, B.
 *
 * Conventions for every entry point:
 *   - All matrix and index pointers are DEVICE pointers owned by the caller,
 *     unless a parameter says "host". The library never frees caller memory.
 *   - Calls are asynchronous on the given stream (NULL = legacy default
 *     stream); the return code reports argument and launch errors only.
 *     Errors raised inside a kernel (a bounded wait that expired) are read
 *     with fm_get_last_device_status.
 *   - Return value: FM_OK (0) or a negative fm_status.
 *   - Residues are uint32 in [0, p); 2 <= p < 2^31. Outputs are canonical
 *     residues in [0, p). Results are bit-exact: every algorithm returns the
 *     same integers as the definition.
 */
#ifndef FM_H
#define FM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (identical to cudaStream_t / CUstream). */
typedef struct CUstream_st* fm_stream;

typedef enum fm_status {
    FM_OK = 0,
    FM_EINVAL = -1,       /* bad shape, descriptor, pointer or overlap           */
    FM_EMODULUS = -2,     /* p < 2 or p >= 2^31                                  */
    FM_ERANGE = -3,       /* a residue >= p (only reported by validating calls)   */
    FM_ECUDA = -4,        /* a CUDA runtime call failed                           */
    FM_ETIMEOUT = -5,     /* a bounded device-side wait expired                   */
    FM_ENOMEM = -6,       /* workspace allocation failed                          */
    FM_EUNSUPPORTED = -7, /* valid request this build does not implement          */
    FM_ETOOBIG = -8       /* larger than the fixed scratch of fm_gemm_modp_noalloc */
} fm_status;

/* A Morton-hybrid matrix (Sec. 1): n x n with n = 2^log2_grid * T',
 * T' = 2^log2_T, stored as n*n uint32 entries. Tile (I, J) (T' x T',
 * row-major inside) starts at element Z(I, J) * T'^2, where Z interleaves the
 * bits of I and J with the row bit more significant (quadrants NW=0, NE=1,
 * SW=2, SE=3, Sec. 2.2 Step 1). Entry (i, j) of a tile starting at sigma is at
 * sigma + i*T' + j (Sec. 2.1, problem P2). base must be 16-byte aligned.
 * Limits: 0 <= log2_T <= 10, 0 <= log2_grid, n <= 2^20. */
typedef struct fm_matrix {
    uint32_t* base;
    int32_t log2_grid;
    int32_t log2_T;
} fm_matrix;

/* A sub-matrix (M, sigma, r, c) of Sec. 2.2: rows x cols starting at Cartesian
 * (row0, col0) of m, so sigma = encode(row0, col0). Any offset is allowed
 * (aligned or not); the part must lie inside the matrix. */
typedef struct fm_sub {
    fm_matrix m;
    int64_t row0, col0, rows, cols;
} fm_sub;

typedef enum fm_op { FM_OP_SET = 0, FM_OP_ADD = 1, FM_OP_SUB = 2 } fm_op;

typedef enum fm_algo {
    FM_ALGO_AUTO = 0,      /* library choice (limb tensor-core form when it pays) */
    FM_ALGO_PLAIN = 1,     /* CUDA-core integer GEMM with delayed reduction       */
    FM_ALGO_LIMB_TC = 2,   /* balanced 8-bit limbs on tcgen05 tensor cores         */
    FM_ALGO_LIMB_MMA_S8 = 3, /* reserved: legacy int8 mma.sync form (unsupported)  */
    FM_ALGO_DFMA = 4       /* FP64 FMA with delayed reduction (exact while the
                              accumulated sum stays below 2^53)                    */
} fm_algo;

/* Optional tuning; pass NULL for defaults. Zero fields mean "default". */
typedef struct fm_opts {
    int32_t k_chunk;        /* limb form: K elements per exact accumulation chunk  */
    int32_t block_n;        /* limb form: output tile width, 128 or 256            */
    int32_t no_karatsuba;   /* limb form: 1 = four limb products instead of three  */
    int32_t cta_pair;       /* limb form: 1 = a CTA pair (cta_group::2) per
                               256 x 256 output tile (fold form, block_n 256) or
                               per 256 x 128 tile (residue form, block_n 128;
                               FM_EINVAL with any other block_n), -1 = one CTA per
                               128 x block_n tile, 0 = automatic (pairs for the
                               fold form when M, N > 256 and K >= 1024; one CTA
                               in the residue form and for GF(2))               */
    int32_t fused_batch;    /* limb batches: 1 = ONE launch that splits the
                               operands into limbs on the fly, instead of limb
                               planes of every call in a workspace and three
                               launches (Karatsuba form, block_n 128, T' >= 8) */
    int32_t reserved[3];
} fm_opts;

/* ---- layout and permutation (Sec. 1; HBM-bound gathers) ---------------- */

/* Row-major src (rows x cols, leading dimension ld >= cols, device) into the
 * Morton-hybrid matrix dst: dst(i, j) = src[i*ld + j] for i < rows, j < cols
 * and 0 elsewhere (the zero padding fills the whole n x n grid).
 * Errors: FM_EINVAL if rows or cols exceed n, ld < cols, or a pointer is
 * null or misaligned. */
int fm_layout_to_morton(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                        fm_matrix dst, fm_stream stream);

/* Same, with TURBO's permutations applied first (Sec. 1):
 * dst(i, j) = src[row_perm[i]*ld + col_perm[j]]; a NULL permutation is the
 * identity. Permutation entries must lie in [0, rows) / [0, cols). The kernel
 * checks every entry it uses: one outside that range is never used as an
 * index; the destination entries it would fill are set to 0 and FM_EINVAL is
 * raised in the device status word (read with fm_get_last_device_status). */
int fm_layout_to_morton_permuted(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                                 const int32_t* row_perm, const int32_t* col_perm,
                                 fm_matrix dst, fm_stream stream);

/* The leading rows x cols of the Morton-hybrid src into row-major dst
 * (leading dimension ld >= cols). */
int fm_layout_from_morton(fm_matrix src, int64_t rows, int64_t cols, uint32_t* dst, int64_t ld,
                          fm_stream stream);

/* The same three conversions with 16-bit row-major entries, for residues
 * mod p <= 65536: half the bytes on the row-major side (for example across
 * the host link). The Morton-hybrid matrix stays 32-bit; the _u16 reads
 * widen every entry, fm_layout_from_morton_u16 stores the low 16 bits of
 * every entry. Arguments and errors as for the 32-bit calls. */
int fm_layout_to_morton_u16(const uint16_t* src, int64_t rows, int64_t cols, int64_t ld,
                            fm_matrix dst, fm_stream stream);
int fm_layout_to_morton_permuted_u16(const uint16_t* src, int64_t rows, int64_t cols, int64_t ld,
                                     const int32_t* row_perm, const int32_t* col_perm,
                                     fm_matrix dst, fm_stream stream);
int fm_layout_from_morton_u16(fm_matrix src, int64_t rows, int64_t cols, uint16_t* dst,
                              int64_t ld, fm_stream stream);

/* Morton-hybrid to Morton-hybrid permutation (Sec. 1, TURBO's virtual row and
 * column permutations made explicit): dst(i, j) = src(row_perm[i], col_perm[j])
 * for i < rows, j < cols; the rest of dst is set to 0. src and dst must not
 * overlap and may have different T'. NULL permutation = identity. Permutation
 * entries must lie in [0, rows) / [0, cols); an entry outside is never used as
 * an index: the entries it would fill are set to 0 and FM_EINVAL is raised in
 * the device status word (read with fm_get_last_device_status). With T' >= 4
 * on both sides and cols <= 51200 each source row is staged whole in shared
 * memory (16-byte vectors in and out); otherwise entries are gathered one by
 * one. */
int fm_permute_rows_cols(fm_matrix src, fm_matrix dst, int64_t rows, int64_t cols,
                         const int32_t* row_perm, const int32_t* col_perm, fm_stream stream);

/* ---- curve variant: Hilbert-hybrid ----------------------------------------
 * Sec. 1 picks the Morton-hybrid order because its index conversion costs the
 * least among the Hilbert, Peano and Morton orders. A Hilbert-hybrid matrix is
 * an fm_matrix whose T' x T' row-major tiles follow the Hilbert curve over the
 * 2^log2_grid x 2^log2_grid tile grid instead of the Z curve: tile (I, J)
 * starts at H(I, J) * T'^2, where the order-1 curve visits (I, J) = (0, 0),
 * (0, 1), (1, 1), (1, 0) and each quadrant holds the order-(k-1) curve, the
 * first transposed and the last reflected across the anti-diagonal. Only the
 * three calls below take Hilbert-hybrid matrices (the products take
 * Morton-hybrid ones); arguments and errors as for their Morton-hybrid
 * counterparts. */
int fm_layout_to_hilbert(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                         fm_matrix dst, fm_stream stream);
int fm_layout_from_hilbert(fm_matrix src, int64_t rows, int64_t cols, uint32_t* dst, int64_t ld,
                           fm_stream stream);
int fm_permute_rows_cols_hilbert(fm_matrix src, fm_matrix dst, int64_t rows, int64_t cols,
                                 const int32_t* row_perm, const int32_t* col_perm,
                                 fm_stream stream);

/* ---- the modular product (Sec. 2, 2.2) ---------------------------------- */

/* C <- C op A*B mod p on sub-matrices: C is rows x cols, A is C.rows x K,
 * B is K x C.cols with K = A.cols = B.rows. A and B may share a matrix; C must
 * not overlap A or B (FM_EINVAL). All three matrices must have the same T'
 * for FM_ALGO_PLAIN and FM_ALGO_DFMA (which run the aligned/contained tile
 * decomposition of Sec. 2.2); the limb form accepts any T'.
 * FM_ALGO_DFMA requires (p-1)^2 * K < 2^53 (FM_EUNSUPPORTED otherwise).
 * Workspace (decomposition lists, limb planes) is owned by the library, cached
 * per device and reused; the first call at a new size allocates. */
int fm_gemm_modp(fm_sub C, fm_sub A, fm_sub B, uint32_t p, int32_t op, int32_t algo,
                 const fm_opts* opts, fm_stream stream);

/* Bytes of device workspace fm_gemm_modp needs for these operands and algo. */
int64_t fm_gemm_modp_workspace_size(fm_sub C, fm_sub A, fm_sub B, uint32_t p, int32_t algo,
                                    const fm_opts* opts);

/* ---- tensor-core limb form, step by step ------------------------------
 * fm_gemm_modp with FM_ALGO_LIMB_TC runs these two steps on cached workspace.
 * They are exposed so that a caller can split an operand once and reuse its
 * limb planes for several products (as a TU decomposition does with a panel).
 * The paper has no limbs (its base case is a plain triple loop over GF(2)).
 *
 * Limb planes. Every residue x in [0, p) is written as w balanced digits in
 * [-128, 127] (w = least w with 256^w >= p), low digit first, of the
 * representative r = x if x <= Hi else x - p, Hi = 127 * sum_{t<w} 256^t,
 * so that r == x (mod p) and r = sum_t d_t 256^t. Digit t of every entry forms
 * plane t, stored as IEEE half (exact for these integers). When w = 2, p < 2^16
 * is odd and fm_opts.no_karatsuba is 0, a third plane holds d_0 + d_1 and the
 * product runs three limb GEMMs (Karatsuba: A*B = (1-256) A0*B0
 * + 256 (A0+A1)*(B0+B1) + (2^16-256) A1*B1) instead of four.
 *   role FM_LIMB_A (an M x K operand): plane t holds MB x ceil(K/64) tiles in
 *     row-block-major order, each 128 rows x 64 k (16 KB); MB = ceil(M/128),
 *     rounded up to even when BN = 256 or in the residue form (p >= 2^16 or
 *     p even), where a CTA pair may take two row blocks.
 *   role FM_LIMB_B (a K x N operand, stored transposed): plane t holds
 *     ceil(N/BN) x ceil(K/64) tiles, each BN rows (n) x 64 k (BN * 128 bytes),
 *     BN = the product's output tile width (fm_opts.block_n; default 256 when
 *     p < 2^16 and p is odd or p < 256, else 128).
 *   Inside a tile, row r is 128 bytes; its 16-byte chunk c (8 consecutive k)
 *   is stored at r*128 + ((c ^ (r % 8)) * 16) (the 128-byte swizzle of the
 *   tensor core's shared-memory operand layout). Entries past the operand's
 *   K extent are zero; rows past its M (A) or N (B) extent, a padding row
 *   block included, are not written, since they reach only output rows or
 *   columns that are never stored. Planes follow each other without gaps. */
enum { FM_LIMB_A = 0, FM_LIMB_B = 1 };

/* Bytes of the limb planes of an operand (rows x cols as the operand is
 * used: M x K for FM_LIMB_A, K x N for FM_LIMB_B), or a negative fm_status. */
int64_t fm_limb_planes_size(int64_t rows, int64_t cols, int32_t role, uint32_t p,
                            const fm_opts* opts);

/* Splits the sub-matrix X (Morton-hybrid, any T' and offset) into limb planes
 * at the device pointer planes (fm_limb_planes_size bytes, 16-byte aligned). */
int fm_limb_split(fm_sub X, int32_t role, uint32_t p, const fm_opts* opts, void* planes,
                  fm_stream stream);

/* C <- C op A*B mod p from limb planes of A (C.rows x K) and B (K x C.cols),
 * both produced by fm_limb_split with the same p and opts. Exact: the limb
 * products run on tcgen05 tensor cores (FP16 carrier, FP32 accumulation) in K
 * chunks of at most 1024 (960 when the running residue is folded into the
 * accumulator), each drained to exact integers and reduced mod p. */
int fm_limb_gemm(fm_sub C, const void* a_planes, const void* b_planes, int64_t K, uint32_t p,
                 int32_t op, const fm_opts* opts, fm_stream stream);

/* ---- the limb product without allocation ----------------------------------
 * The paper has no counterpart: this is a library service. fm_gemm_modp
 * allocates its limb-plane workspace with cudaMalloc on first use. Some callers
 * cannot let a library do that: programs whose device memory comes only from
 * their own allocator or a fixed budget (a serving process that reserves the
 * GPU's memory for its pool at start-up, where a hidden cudaMalloc can fail at
 * any point or take memory a co-tenant counted on), and code that must not
 * stall on the device synchronisation cudaMalloc and cudaFree imply. They use
 * this entry point instead. It computes exactly what fm_gemm_modp with
 * FM_ALGO_LIMB_TC computes (C <- C op A*B mod p on Morton-hybrid sub-matrices,
 * any T', default fm_opts) and allocates nothing: its scratch is a fixed
 * device array of 64 MiB of limb planes plus a status word, compiled into the
 * library (every GPU that loads it holds that array until the process exits).
 * A product whose limb planes need more than 64 MiB returns FM_ETOOBIG (e.g.
 * M = N = K = 2048 fits for p < 2^16; the planes take 6 * K * (M + N) bytes for
 * odd p < 2^16 with three planes, 20 * K * (M + N) for p = 2^31 - 1 with ten
 * (four limbs and their six pair sums), rounded up to whole tiles). Calls with M, N or K equal to 0 touch no scratch (K = 0
 * with FM_OP_SET zeroes the C sub-matrix; with ADD or SUB it leaves C as is).
 * The first call on a device that multiplies (K > 0) does that device's
 * one-time set-up: it looks up the array's device address and queries how
 * many CTA pairs of the limb kernel fit at once; make that first call before
 * any stream capture. All calls share the one array, so calls that can overlap
 * on the GPU (different streams without ordering) race and must be serialised
 * by the caller; the array keeps the last call's contents, and every call
 * rewrites all of it that its stored results depend on (what it leaves, the
 * planes' rows past M or N, reaches only outputs that are never stored). A
 * device-side wait that expires raises
 * FM_ETIMEOUT in the array's own status word; fm_get_last_device_status reads
 * (and clears) that word together with the library's, without allocating. */
int fm_gemm_modp_noalloc(fm_sub C, fm_sub A, fm_sub B, uint32_t p, int32_t op, fm_stream stream);

/* ---- TU decomposition (Sec. 1: the consumer of the product) ------------
 * Rank-revealing PLUQ over the prime field GF(p) of the leading m x n corner
 * of the Morton-hybrid matrix A (T' >= 4), in place: P A Q = L U with L unit
 * lower trapezoidal (m x r), U upper trapezoidal (r x n, nonzero diagonal),
 * r = rank(A). On return A holds L strictly below the diagonal of its first r
 * columns and U on and above the diagonal of its first r rows (entries of rows
 * >= r outside L are zero); row_perm (device, m) and col_perm (device, n) are
 * gathers: (P A Q)(i, j) = A_in(row_perm[i], col_perm[j]). *rank (host) gets r.
 * Blocked right-looking elimination with 128-column panels (first-nonzero
 * pivoting, zero columns moved behind the pivot columns) grouped four to an
 * outer block; the trailing updates are limb products on sub-matrices of A
 * (C <- C - L21 * U12). The bulk of each outer block's update runs on a second
 * stream the call creates (ordered against `stream` by events) while the next
 * block's panels factor on `stream`, and a panel's U12 product on a third one
 * beside its L21 product; the call also holds a 4-byte pinned host buffer for
 * the panels' flags. p must be prime; n <= 51200. Synchronous:
 * returns after the factorisation, with both streams idle.
 * The paper defers the TU algorithm itself (TURBO) to its reference; this is
 * the textbook elimination that produces the same kind of result. */
int fm_pluq(fm_matrix A, int64_t m, int64_t n, uint32_t p, int32_t* row_perm, int32_t* col_perm,
            int64_t* rank, fm_stream stream);

/* ---- batching form (Sec. 2.2, Prop. on work and span: the base-case
 * products are independent and may run in parallel) ---------------------- */

/* One call of a batch: C <- C op A*B mod p on sub-matrices (all fields as in
 * fm_gemm_modp). */
typedef struct fm_gemm_call {
    fm_sub C, A, B;
    int32_t op;
    int32_t reserved;
} fm_gemm_call;

typedef struct fm_plan fm_plan;

/* Plans a batch of n calls (host array calls[0..n-1]) for one modulus p.
 * Calls of one batch must write disjoint C regions. The plan owns its device
 * workspace until fm_plan_destroy.
 *   FM_ALGO_AUTO / FM_ALGO_PLAIN / FM_ALGO_DFMA: decomposes every call into
 *     contained tile products (Sec. 2.2; all matrices with T' = 32 or 64), packs
 *     them into one work list and uploads it.
 *   FM_ALGO_LIMB_TC: the tensor-core limb form for the whole batch (any T'):
 *     limb planes for every call's operands in one workspace (cached in the
 *     plan). With opts->fused_batch == 1, the two-limb Karatsuba form (odd
 *     p < 2^16, block_n 128, the default for batches) and every A and B with
 *     8 <= T', at most 2^32 entries and a 16-byte aligned base, the batch is
 *     FUSED instead: one launch that splits the operands into limbs on the
 *     fly (FM_EUNSUPPORTED when the batch does not qualify). opts as for
 *     fm_gemm_modp except cta_pair (FM_EUNSUPPORTED). */
int fm_plan_create(fm_plan** plan, const fm_gemm_call* calls, int64_t n, uint32_t p,
                   int32_t algo, const fm_opts* opts);

/* Runs every call of the plan on stream. Decomposed forms: ONE persistent
 * kernel launch whose CTAs pull work items from a device queue. Fused limb
 * form: ONE persistent launch over the 128 x 128 output tiles of every call
 * (longest calls first, a call's tiles adjacent). Limb form with planes: three
 * launches (limb split of every A, of every B, and one persistent GEMM over
 * the output tiles of every call, longest first). Limb forms add one small
 * launch per call with K = 0 under FM_OP_SET. May be captured in a CUDA
 * graph; the plan must outlive the graph. */
int fm_gemm_modp_batched(fm_plan* plan, fm_stream stream);

/* Work items (decomposed forms: base-case tile products; limb form: output
 * tiles) of the plan (host). */
int64_t fm_plan_work_items(const fm_plan* plan);

/* Kernel launches of this library in one fm_gemm_modp_batched run of the plan
 * (host): 1 for the decomposed forms and for a fused limb batch, 3 for a limb
 * batch with limb planes in a workspace, plus one per K = 0 call under
 * FM_OP_SET. */
int64_t fm_plan_launches(const fm_plan* plan);

int fm_plan_destroy(fm_plan* plan);

/* ---- autotuning ---------------------------------------------------------
 * Sec. 1 takes the Morton-hybrid threshold T' from prior measurements; here the
 * threshold of the decomposed forms and the limb form's options (output tile
 * width, K chunk, Karatsuba) are measured on the device instead. */
typedef struct fm_tune_result {
    int32_t algo;        /* FM_ALGO_PLAIN or FM_ALGO_LIMB_TC                       */
    int32_t log2_T;      /* T' the winner ran with (for the plain form: the layout) */
    fm_opts opts;        /* options of the winning limb form (zero for plain)        */
    double ms;           /* one call of the winner, milliseconds                     */
    double gops;         /* 2 M N K / time, Gop/s                                    */
    int32_t candidates;  /* candidates that ran                                      */
    int32_t reserved;
} fm_tune_result;

enum { FM_TUNE_NO_LIMB = 1, FM_TUNE_NO_PLAIN = 2 };

/* Times every candidate form for C (M x N) -= A (M x K) * B (K x N) mod p on
 * scratch Morton matrices it allocates (and frees) on the current device:
 * the plain form at T' = 32 and 64, the limb form with output tile width 256 and
 * 128, the full and half exact K chunk, with and without Karatsuba. Writes the
 * fastest to *out and remembers it for the problem class (M, N, K rounded up to
 * powers of two; p < 2^8, odd p < 2^16, other p); fm_gemm_modp with
 * FM_ALGO_AUTO and opts == NULL then uses the remembered choice when the
 * caller's operands allow it. Synchronises stream. */
int fm_autotune(int64_t M, int64_t N, int64_t K, uint32_t p, int32_t flags, fm_stream stream,
                fm_tune_result* out);

/* 1 and *out filled if the problem class has a remembered choice, else 0. */
int fm_autotune_lookup(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out);

/* Saves / loads the remembered choices as text (host only). load returns the
 * number of classes read or a negative fm_status. */
int fm_autotune_save(const char* path);
int fm_autotune_load(const char* path);
int fm_autotune_clear(void);

/* Times the candidate forms of the batch calls[0..n-1] (host array, as for
 * fm_plan_create) on the current device and remembers the fastest for its
 * batch class (number of calls, mean M, N and K rounded up to powers of two,
 * modulus class, T'); fm_plan_create with FM_ALGO_AUTO and opts == NULL then
 * builds that form for batches of the class. Candidates: the decomposed plain
 * plan (all matrices with T' = 32 or 64), the limb plan with planes at output
 * tile width 128 and 256 (256 for odd p < 2^16 only), full and half K chunk,
 * with and without Karatsuba, and the fused limb plan. Each runs once untimed
 * and three times timed (CUDA events) on the batch itself, with every C matrix
 * replaced by a scratch copy (allocated and freed here), so the caller's
 * matrices do not change. The batch's layout T' is the caller's: to tune T',
 * lay the batch out at each T' and tune each. Synchronises stream. */
int fm_autotune_batch(const fm_gemm_call* calls, int64_t n, uint32_t p, int32_t flags, fm_stream stream,
                      fm_tune_result* out);

/* ---- decomposition (host only; Sec. 2.2 Steps 1-4) ---------------------- */

/* Writes the base-case products of C <- C op A*B as local index ranges
 * (i_lo, i_hi, j_lo, j_hi, l_lo, l_hi), 6 int64 per product, into the host
 * array out (capacity cap products). Each product multiplies parts of A, B and
 * C that each lie inside one T' x T' tile (contained, Sec. 2.1). Returns the
 * number of products (which may exceed cap; only cap are written) or a
 * negative fm_status. Needs no GPU. */
int64_t fm_decompose(fm_sub C, fm_sub A, fm_sub B, int64_t* out, int64_t cap);

/* ---- GF(2) on bit-packed matrices ---------------------------------------
 * The field of the paper's experiments (Sec. 2.2, "Performance Analysis":
 * random sub-matrix products in Morton-hybrid matrices with T' = 32 over the
 * binary field). A bit-packed Morton-hybrid matrix has T' = 32 fixed, so a
 * tile row is one 32-bit word: n x n entries, n = 32 * 2^log2_grid, stored as
 * 4^log2_grid tiles of 32 words (128 bytes); tile (I, J) starts at word
 * Z(I, J) * 32 (Z as for fm_matrix), word u of a tile is tile row u and its
 * bit v is entry (32 I + u, 32 J + v). The matrix takes n * n / 8 bytes; base
 * must be 16-byte aligned. Sub-matrices use any row, column, size. */
typedef struct fm_gf2_matrix {
    uint32_t* base;     /* device pointer, 16-byte aligned                     */
    int32_t log2_grid;  /* 2^log2_grid tiles per side, 0..15                   */
    int32_t reserved;
} fm_gf2_matrix;

typedef struct fm_gf2_sub {
    fm_gf2_matrix m;
    int64_t row0, col0, rows, cols;
} fm_gf2_sub;

/* Row-major entries (device, leading dimension ld >= cols; bit 0 of each entry
 * is taken) -> the bit-packed matrix dst; entries outside rows x cols become 0. */
int fm_gf2_pack(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld, fm_gf2_matrix dst,
                fm_stream stream);

/* The leading rows x cols entries of src -> row-major 0 / 1 words at dst. */
int fm_gf2_unpack(fm_gf2_matrix src, int64_t rows, int64_t cols, uint32_t* dst, int64_t ld,
                  fm_stream stream);

/* C <- A*B (FM_OP_SET) or C <- C + A*B (FM_OP_ADD; FM_OP_SUB is the same in
 * GF(2)) on bit-packed sub-matrices: C is rows x cols, A is C.rows x K, B is
 * K x C.cols. A and B may share a matrix; C must not overlap A or B
 * (FM_EINVAL). Bits of C outside the sub-matrix are unchanged, also where they
 * share a word with it. Runs on the tensor cores with E4M3 0 / 1 operands and
 * FP32 accumulation (exact: at most 2^24 - 2 terms per accumulation, folded
 * to parity between chunks). opts may be NULL; only opts->cta_pair is read
 * (1 = CTA pairs on 256 x 256 output tiles). Workspace: fm_gf2_workspace_size
 * bytes, cached per device as for fm_gemm_modp. */
int fm_gf2_gemm(fm_gf2_sub C, fm_gf2_sub A, fm_gf2_sub B, int32_t op, const fm_opts* opts,
                fm_stream stream);

/* Device workspace bytes of fm_gf2_gemm for an M x N x K product. */
int64_t fm_gf2_workspace_size(int64_t M, int64_t N, int64_t K);

/* One call of a GF(2) batch: C <- A*B (FM_OP_SET) or C + A*B (FM_OP_ADD /
 * FM_OP_SUB) on bit-packed sub-matrices (fields as in fm_gf2_gemm). */
typedef struct fm_gf2_call {
    fm_gf2_sub C, A, B;
    int32_t op;
    int32_t reserved;
} fm_gf2_call;

/* Plans a batch of n GF(2) calls (the experiments' workload of Sec. 2.2 is such
 * a batch of independent sub-matrix products). Calls of one batch must write
 * disjoint C regions (they may share words). Run it with fm_gemm_modp_batched (three
 * launches: the E4M3 split of every A, of every B, one persistent GEMM over
 * the output tiles of every call; plus one launch per call with K = 0 under
 * FM_OP_SET) and free it with fm_plan_destroy. opts may be NULL (cta_pair is
 * not supported: FM_EUNSUPPORTED). */
int fm_gf2_plan_create(fm_plan** plan, const fm_gf2_call* calls, int64_t n, const fm_opts* opts);

/* ---- failure detection (the paper has no counterpart) ---------------------
 * Every device-side wait of the library is bounded: after 2 s it raises
 * FM_ETIMEOUT in the device status word and the kernel winds down, leaving the
 * context usable. This hook launches a kernel whose wait cannot complete so
 * that tests can watch that happen: which = 0, an mbarrier phase that nothing
 * completes; which = 1, a grid barrier that one CTA of the grid never reaches;
 * which = 2, the mbarrier of which = 0 raising into the status word of
 * fm_gemm_modp_noalloc's fixed scratch. Returns launch errors only (FM_EINVAL
 * for another which); the outcome is read with fm_get_last_device_status.
 * Nothing faults or hangs.
 *
 * Tracing: with the environment variable FM_TRACE set (to "1" for stderr, or
 * to a file path), every fm_gemm_modp, fm_gemm_modp_batched, fm_gf2_gemm and
 * fm_pluq call appends one line with its shapes and work (products, tiles,
 * plane bytes). The public entry points are also NVTX ranges. */
int fm_debug_expire_wait(int32_t which, fm_stream stream);

/* ---- measured pipe rates (the paper has no counterpart) -------------------
 * The roofline of the non-tensor forms: the plain form spends one 32 x 32 ->
 * 64-bit integer multiply-add (mad.wide.u32) per (i, j, l), the DFMA form one
 * FP64 fused multiply-add; the legacy warp-level int8 MMA (mma.sync m16n8k32,
 * s8 x s8 -> s32) is the true-INT8 alternative to the f16 carrier on tcgen05.
 * fm_measure_peak runs a probe kernel of that one instruction (4 CTAs of 256
 * threads per SM, independent chains, no memory traffic in the loop; iters
 * loop iterations, 8 multiply-adds per thread each, or four m16n8k32 MMAs per
 * warp) after one shorter warm-up launch, times it with CUDA events on stream
 * and writes multiply-adds per second to *ops_per_s (host; for the MMA, its
 * m * n * k products per second). Synchronous. FM_EINVAL for an unknown kind
 * or iters <= 0. */
enum { FM_PEAK_IMAD_WIDE = 0, FM_PEAK_IMAD32 = 1, FM_PEAK_DFMA = 2, FM_PEAK_FFMA = 3, FM_PEAK_MMA_S8 = 4 };
int fm_measure_peak(int32_t kind, int64_t iters, fm_stream stream, double* ops_per_s);

/* ---- status ------------------------------------------------------------- */

/* Synchronises stream, returns and clears the device status words that
 * kernels raise into (FM_ETIMEOUT on an expired bounded wait, FM_ERANGE from
 * fm_validate_residues, FM_EINVAL for an out-of-range permutation entry): the
 * library's own word and that of fm_gemm_modp_noalloc's fixed scratch. Each
 * word keeps the first code raised since it was last read; FM_OK if none.
 * Allocates nothing. */
int fm_get_last_device_status(fm_stream stream);

/* Validation: every entry of the sub-matrix X must be a residue in [0, p)
 * (the inputs the paper's arithmetic assumes; the library's kernels do not
 * check them). Scans X on stream and, if an entry is >= p, records FM_ERANGE
 * in the device status word, read with fm_get_last_device_status.
 * Errors (returned): FM_EMODULUS if p < 2 or p >= 2^31, FM_EINVAL for a bad
 * descriptor. */
int fm_validate_residues(fm_sub X, uint32_t p, fm_stream stream);

/* Static string for a status code. */
const char* fm_strerror(int status);

/* Frees the library's cached per-device workspace (current device). */
int fm_release_workspace(void);

/* Library version as major*10000 + minor*100 + patch. */
int fm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FM_H */
