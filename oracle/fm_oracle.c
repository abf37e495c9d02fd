/*
 * fm_oracle.c -- plain, slow, obviously correct CPU reference for the exact
 * modular matrix multiply on Morton-hybrid matrices.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the bench's CPU-baseline
 * leg use it, through oracle/__init__.py. It shares no code with the CUDA path.
 *
 * Contents (each function cites the passage of the paper it follows):
 *   - Morton-hybrid index encode / extract   (Sec. 1 and Sec. 2.2, Step 1)
 *   - layout conversion row-major <-> Morton-hybrid (Sec. 1, Sec. 2.1)
 *   - row / column permutation                (Sec. 1, TURBO's permutations)
 *   - C <- C op A*B mod p, triple loop        (Sec. 2, S_A = S_B * S_C; the
 *                                               paper's field arithmetic is GF(p))
 *   - sampled entries of the same product, mat-vec mod p (Freivalds' check)
 *   - rank-revealing PLUQ by Gaussian elimination mod p (Sec. 1, TU / rank)
 *
 * All matrices here are plain row-major uint32 arrays with a leading dimension.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------- */
/* Morton-hybrid index.                                                       */
/*                                                                            */
/* Sec. 1: the Morton order is the recursive Z-shaped curve; the hybrid stops */
/* decomposing at T' x T' blocks, which are stored row-major. Sec. 2.2, Step  */
/* 1: the four quadrants of a block with lambda elements starting at alpha     */
/* are laid out NW, NE, SW, SE at alpha, alpha + lambda/4, alpha + 2 lambda/4, */
/* alpha + 3 lambda/4. Sec. 2.1 (P2): inside a row-major T' x T' block that    */
/* starts at sigma, entry (i, j) sits at sigma + i*T' + j.                     */
/*                                                                            */
/* The matrix is (2^m T') x (2^m T'). encode descends the quadrant recursion   */
/* one level at a time, exactly as Step 1 states it.                          */
/* ------------------------------------------------------------------------- */
uint64_t or_encode(int64_t i, int64_t j, int32_t m, int64_t T)
{
    uint64_t alpha = 0;                         /* start of the current block */
    int64_t n = ((int64_t)1 << m) * T;          /* side of the current block  */
    int64_t r = i, c = j;                       /* position inside the block  */
    while (n > T) {
        int64_t h = n / 2;
        uint64_t lambda_q = (uint64_t)h * (uint64_t)h;  /* lambda' = lambda/4 */
        int q;
        if (r < h && c < h)       q = 0;   /* NW */
        else if (r < h)           q = 1;   /* NE */
        else if (c < h)           q = 2;   /* SW */
        else                      q = 3;   /* SE */
        alpha += (uint64_t)q * lambda_q;
        if (r >= h) r -= h;
        if (c >= h) c -= h;
        n = h;
    }
    return alpha + (uint64_t)r * (uint64_t)T + (uint64_t)c;   /* sigma + i*T' + j */
}

/* Inverse of or_encode: walk the same quadrant recursion from the index. */
static void or_extract(uint64_t z, int32_t m, int64_t T, int64_t* pi, int64_t* pj)
{
    int64_t n = ((int64_t)1 << m) * T;
    int64_t i0 = 0, j0 = 0;
    uint64_t alpha = 0;
    while (n > T) {
        int64_t h = n / 2;
        uint64_t lambda_q = (uint64_t)h * (uint64_t)h;
        int q = (int)((z - alpha) / lambda_q);
        alpha += (uint64_t)q * lambda_q;
        if (q == 1 || q == 3) j0 += h;
        if (q == 2 || q == 3) i0 += h;
        n = h;
    }
    uint64_t off = z - alpha;
    *pi = i0 + (int64_t)(off / (uint64_t)T);
    *pj = j0 + (int64_t)(off % (uint64_t)T);
}

int64_t or_extract_i(uint64_t z, int32_t m, int64_t T)
{
    int64_t i, j;
    or_extract(z, m, T, &i, &j);
    return i;
}

int64_t or_extract_j(uint64_t z, int32_t m, int64_t T)
{
    int64_t i, j;
    or_extract(z, m, T, &i, &j);
    return j;
}

void or_encode_many(const int64_t* i, const int64_t* j, int64_t n, int32_t m, int64_t T,
                    uint64_t* z)
{
    for (int64_t t = 0; t < n; ++t) z[t] = or_encode(i[t], j[t], m, T);
}

void or_extract_many(const uint64_t* z, int64_t n, int32_t m, int64_t T, int64_t* i, int64_t* j)
{
    for (int64_t t = 0; t < n; ++t) or_extract(z[t], m, T, &i[t], &j[t]);
}

/* Row-major rows x cols (leading dimension ld) -> Morton-hybrid (2^m T')^2;  */
/* entries outside rows x cols are zero.                                      */
void or_to_morton(const uint32_t* src, int64_t rows, int64_t cols, int64_t ld,
                  uint32_t* dst, int32_t m, int64_t T)
{
    int64_t n = ((int64_t)1 << m) * T;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            dst[or_encode(i, j, m, T)] = (i < rows && j < cols) ? src[i * ld + j] : 0u;
}

/* Morton-hybrid -> row-major, the leading rows x cols corner. */
void or_from_morton(const uint32_t* src, int32_t m, int64_t T, int64_t rows, int64_t cols,
                    uint32_t* dst, int64_t ld)
{
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j)
            dst[i * ld + j] = src[or_encode(i, j, m, T)];
}

/* out(i, j) = in(rp[i], cp[j]); a null permutation means the identity. */
void or_permute(const uint32_t* src, int64_t lds, int64_t rows, int64_t cols,
                const int32_t* rp, const int32_t* cp, uint32_t* dst, int64_t ldd)
{
    for (int64_t i = 0; i < rows; ++i) {
        int64_t si = rp ? rp[i] : i;
        for (int64_t j = 0; j < cols; ++j) {
            int64_t sj = cp ? cp[j] : j;
            dst[i * ldd + j] = src[si * lds + sj];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* C <- C op A*B mod p  (op: 0 set, 1 add, 2 subtract).                        */
/*                                                                            */
/* Sec. 2 states the problem as S_A = S_B * S_C on sub-matrices, accumulated   */
/* as S_A += S_B * S_C in the recursion; the paper works over a finite field.  */
/* This is the definition written out: for every (i, j) the exact integer      */
/* sum_l A[i][l]*B[l][j] (held in 128 bits, which cannot overflow for any      */
/* K < 2^64 and p < 2^32), reduced mod p, then combined with C mod p.          */
/* Loop order i, l, j; rows are shared out over threads when OpenMP is on.     */
/* ------------------------------------------------------------------------- */
static uint32_t combine(uint32_t c, uint64_t s, uint32_t p, int op)
{
    uint64_t cc = (uint64_t)c % p;
    if (op == 0) return (uint32_t)s;
    if (op == 1) return (uint32_t)((cc + s) % p);
    return (uint32_t)((cc + (uint64_t)p - s) % p);
}

int or_gemm_modp(const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                 uint32_t* C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                 uint32_t p, int32_t op)
{
    if (p < 2 || op < 0 || op > 2 || M < 0 || N < 0 || K < 0) return -1;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < M; ++i) {
        u128* acc = (u128*)calloc((size_t)(N > 0 ? N : 1), sizeof(u128));
        for (int64_t l = 0; l < K; ++l) {
            uint64_t a = A[i * lda + l];
            const uint32_t* brow = B + l * ldb;
            for (int64_t j = 0; j < N; ++j) acc[j] += (u128)(a * (uint64_t)brow[j]);
        }
        for (int64_t j = 0; j < N; ++j) {
            uint64_t s = (uint64_t)(acc[j] % p);
            C[i * ldc + j] = combine(C[i * ldc + j], s, p, op);
        }
        free(acc);
    }
    return 0;
}

/* Entries (ij[2t], ij[2t+1]) of C op A*B mod p, one at a time (for sampled   */
/* checks at sizes where the full product is too slow on a CPU).              */
int or_gemm_modp_entries(const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                         const uint32_t* C, int64_t ldc, int64_t K, uint32_t p, int32_t op,
                         const int64_t* ij, int64_t n, uint32_t* out)
{
    if (p < 2 || op < 0 || op > 2) return -1;
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < n; ++t) {
        int64_t i = ij[2 * t], j = ij[2 * t + 1];
        u128 acc = 0;
        for (int64_t l = 0; l < K; ++l)
            acc += (u128)((uint64_t)A[i * lda + l] * (uint64_t)B[l * ldb + j]);
        uint32_t c = (op == 0) ? 0u : C[i * ldc + j];
        out[t] = combine(c, (uint64_t)(acc % p), p, op);
    }
    return 0;
}

/* y = A x mod p for a row-major rows x cols A. */
int or_matvec_modp(const uint32_t* A, int64_t lda, int64_t rows, int64_t cols,
                   const uint32_t* x, uint32_t p, uint32_t* y)
{
    if (p < 2) return -1;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < rows; ++i) {
        u128 acc = 0;
        for (int64_t j = 0; j < cols; ++j) acc += (u128)((uint64_t)A[i * lda + j] * x[j]);
        y[i] = (uint32_t)(acc % p);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Rank-revealing PLUQ by Gaussian elimination over GF(p).                    */
/*                                                                            */
/* Sec. 1: TU decomposition triangulates a rectangular, possibly singular     */
/* matrix and recovers its rank exactly. The paper defers the algorithm to    */
/* TURBO; this is the textbook elimination that produces the same kind of      */
/* result: P A Q = L U with L unit lower trapezoidal (m x r), U upper          */
/* trapezoidal (r x n) with r nonzero pivots, r = rank(A).                    */
/*                                                                            */
/* Step k searches the trailing block A[k:, k:] in row-major order for the    */
/* first nonzero entry, swaps it to (k, k), stores the multipliers in column  */
/* k below the pivot and updates the trailing block. It stops when the        */
/* trailing block is zero. On return a (m x n, row-major, in place) holds L   */
/* strictly below the diagonal of its first r columns and U on and above the  */
/* diagonal of its first r rows; rp, cp are gathers: (P A Q)[i][j] =           */
/* A[rp[i]][cp[j]].                                                           */
/* ------------------------------------------------------------------------- */
static uint64_t inv_modp(uint64_t a, uint64_t p)
{
    /* extended Euclid on (a, p); a != 0 mod p and p prime */
    int64_t t = 0, newt = 1;
    int64_t r = (int64_t)p, newr = (int64_t)(a % p);
    while (newr != 0) {
        int64_t q = r / newr, tmp;
        tmp = t - q * newt; t = newt; newt = tmp;
        tmp = r - q * newr; r = newr; newr = tmp;
    }
    if (t < 0) t += (int64_t)p;
    return (uint64_t)t;
}

int64_t or_pluq(uint32_t* a, int64_t m, int64_t n, uint32_t p, int32_t* rp, int32_t* cp)
{
    if (p < 2) return -1;
    for (int64_t i = 0; i < m; ++i) rp[i] = (int32_t)i;
    for (int64_t j = 0; j < n; ++j) cp[j] = (int32_t)j;
    int64_t kmax = m < n ? m : n;
    int64_t k;
    for (k = 0; k < kmax; ++k) {
        int64_t pi = -1, pj = -1;
        for (int64_t i = k; i < m && pi < 0; ++i)
            for (int64_t j = k; j < n; ++j)
                if (a[i * n + j] % p != 0) { pi = i; pj = j; break; }
        if (pi < 0) break;
        if (pi != k) {
            for (int64_t j = 0; j < n; ++j) {
                uint32_t t = a[k * n + j]; a[k * n + j] = a[pi * n + j]; a[pi * n + j] = t;
            }
            int32_t t = rp[k]; rp[k] = rp[pi]; rp[pi] = t;
        }
        if (pj != k) {
            for (int64_t i = 0; i < m; ++i) {
                uint32_t t = a[i * n + k]; a[i * n + k] = a[i * n + pj]; a[i * n + pj] = t;
            }
            int32_t t = cp[k]; cp[k] = cp[pj]; cp[pj] = t;
        }
        uint64_t inv = inv_modp(a[k * n + k], p);
        for (int64_t i = k + 1; i < m; ++i) {
            uint64_t l = ((uint64_t)a[i * n + k] % p) * inv % p;
            a[i * n + k] = (uint32_t)l;
            if (l == 0) continue;
            for (int64_t j = k + 1; j < n; ++j) {
                uint64_t u = (uint64_t)a[k * n + j] % p;
                uint64_t v = (uint64_t)a[i * n + j] % p;
                a[i * n + j] = (uint32_t)((v + (uint64_t)p - (l * u) % p) % p);
            }
        }
    }
    return k;
}

/* ------------------------------------------------------------------------- */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
