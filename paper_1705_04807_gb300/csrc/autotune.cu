// autotune.cu -- measured choice of the GEMM form and its options per problem class.
//
// The threshold T' of the decomposed forms (Sec. 1: the Morton-hybrid order
// stops at T' x T' tiles; the paper takes T' = 32 from prior work), and the
// limb form's output tile width, K chunk and Karatsuba use, are picked by
// timing every candidate on scratch matrices of the requested shape on the
// current device. The fastest is remembered per problem class (M, N, K rounded
// up to powers of two, and the modulus class) and used by FM_ALGO_AUTO when the
// caller passes no options. The table can be saved to and loaded from a text
// file so that tuning runs once per machine.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "fm_internal.cuh"
#include "fm_kernels.h"

namespace {

struct TuneKey {
    int mc, nc, kc, pc;
    bool operator<(const TuneKey& o) const
    {
        if (mc != o.mc) return mc < o.mc;
        if (nc != o.nc) return nc < o.nc;
        if (kc != o.kc) return kc < o.kc;
        return pc < o.pc;
    }
};

std::mutex g_tune_mu;
std::map<TuneKey, fm_tune_result> g_tune;

int ceil_log2(int64_t x)
{
    int l = 0;
    while (((int64_t)1 << l) < x) ++l;
    return l;
}

int p_class(uint32_t p)
{
    if (p < 256) return 0;
    if (p < (1u << 16) && (p & 1)) return 1;
    return 2;
}

TuneKey key_of(int64_t M, int64_t N, int64_t K, uint32_t p)
{
    return TuneKey{ceil_log2(M), ceil_log2(N), ceil_log2(K), p_class(p)};
}

// Deterministic residues in [0, p) for scratch operands (a hash of the index;
// the timing does not depend on the values, only on their range).
__global__ void fill_kernel(uint32_t* x, int64_t n, uint32_t p, uint32_t salt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + salt;
        z ^= z >> 31;
        z *= 0xBF58476D1CE4E5B9ull;
        z ^= z >> 29;
        x[i] = (uint32_t)(z % p);
    }
}

struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch()
    {
        for (void* q : ptrs) cudaFree(q);
    }
    uint32_t* alloc_matrix(int64_t rows, int64_t cols, int lt, uint32_t p, uint32_t salt,
                           fm_matrix* m, cudaStream_t s)
    {
        int lg = 0;
        while ((((int64_t)1 << lg) << lt) < std::max(rows, cols)) ++lg;
        const int64_t n = ((int64_t)1 << lg) << lt;
        void* q = nullptr;
        if (cudaMalloc(&q, (size_t)n * n * 4) != cudaSuccess) return nullptr;
        ptrs.push_back(q);
        fill_kernel<<<1024, 256, 0, s>>>(static_cast<uint32_t*>(q), n * n, p, salt);
        m->base = static_cast<uint32_t*>(q);
        m->log2_grid = lg;
        m->log2_T = lt;
        return m->base;
    }
};

struct Candidate {
    int algo;
    int lt;
    fm_opts opts;
};

}  // namespace

extern "C" int fm_autotune(int64_t M, int64_t N, int64_t K, uint32_t p, int32_t flags,
                           fm_stream stream, fm_tune_result* out)
{
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    if (M <= 0 || N <= 0 || K <= 0 || !out) return FM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // candidates
    std::vector<Candidate> cands;
    auto limb = [&](int bn, int kchunk, int no_kara, int pair) {
        Candidate c;
        std::memset(&c, 0, sizeof(c));
        c.algo = FM_ALGO_LIMB_TC;
        c.lt = 7;
        c.opts.block_n = bn;
        c.opts.k_chunk = kchunk;
        c.opts.no_karatsuba = no_kara;
        c.opts.cta_pair = pair;
        cands.push_back(c);
    };
    if (!(flags & FM_TUNE_NO_LIMB)) {
        FmLimbPlan q;
        if (fm_limb_plan(M, N, K, p, nullptr, &q) == FM_OK) {
            const int full = q.prod_cs[0] * 64;
            for (int bn : {256, 128}) {
                if (!q.fold && bn == 256) continue;
                for (int kc : {full, full / 2}) {
                    if (kc < 64 || kc % 64) continue;
                    for (int pair : {-1, 1}) {
                        if (pair == 1 && bn != 256) continue;
                        limb(bn, kc, 0, pair);
                        if (q.n_planes == 3) limb(bn, kc, 1, pair);
                    }
                }
            }
        }
    }
    if (!(flags & FM_TUNE_NO_PLAIN)) {
        for (int lt : {5, 6}) {
            Candidate c;
            std::memset(&c, 0, sizeof(c));
            c.algo = FM_ALGO_PLAIN;
            c.lt = lt;
            cands.push_back(c);
        }
    }
    if (cands.empty()) return FM_EINVAL;

    Scratch scratch;
    std::map<int, std::vector<fm_matrix>> by_lt;  // C, A, B per T'
    cudaEvent_t e0, e1;
    FM_CUDA_TRY(cudaEventCreate(&e0));
    FM_CUDA_TRY(cudaEventCreate(&e1));
    fm_tune_result best;
    std::memset(&best, 0, sizeof(best));
    best.ms = -1.0;
    int tried = 0;
    for (const Candidate& c : cands) {
        if (!by_lt.count(c.lt)) {
            std::vector<fm_matrix> ms(3);
            if (!scratch.alloc_matrix(M, N, c.lt, p, 1, &ms[0], s) ||
                !scratch.alloc_matrix(M, K, c.lt, p, 2, &ms[1], s) ||
                !scratch.alloc_matrix(K, N, c.lt, p, 3, &ms[2], s)) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return FM_ENOMEM;
            }
            by_lt[c.lt] = ms;
        }
        const std::vector<fm_matrix>& ms = by_lt[c.lt];
        const fm_sub C{ms[0], 0, 0, M, N}, A{ms[1], 0, 0, M, K}, B{ms[2], 0, 0, K, N};
        const fm_opts* o = c.algo == FM_ALGO_LIMB_TC ? &c.opts : nullptr;
        if (fm_gemm_modp(C, A, B, p, FM_OP_SUB, c.algo, o, stream) != FM_OK) continue;  // warm-up
        const int reps = 3;
        cudaEventRecord(e0, s);
        int rc = FM_OK;
        for (int r = 0; r < reps && rc == FM_OK; ++r)
            rc = fm_gemm_modp(C, A, B, p, FM_OP_SUB, c.algo, o, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || rc != FM_OK) continue;
        float ms_total = 0.f;
        cudaEventElapsedTime(&ms_total, e0, e1);
        const double ms_one = ms_total / reps;
        ++tried;
        if (best.ms < 0 || ms_one < best.ms) {
            best.algo = c.algo;
            best.log2_T = c.lt;
            best.opts = c.opts;
            best.ms = ms_one;
            best.gops = 2.0 * (double)M * N * K / (ms_one * 1e-3) / 1e9;
            best.candidates = (int32_t)cands.size();
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (tried == 0) return FM_EUNSUPPORTED;
    best.candidates = tried;
    *out = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key_of(M, N, K, p)] = best;
    return FM_OK;
}

// Tuned choice for a problem class, if any (used by FM_ALGO_AUTO).
bool fm_tuned_choice(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key_of(M, N, K, p));
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

// Text format, one class per line:
//   mc nc kc pc algo log2_T block_n k_chunk no_karatsuba ms gops [cta_pair]
// (a missing last field reads as 0).
extern "C" int fm_autotune_save(const char* path)
{
    if (!path) return FM_EINVAL;
    FILE* f = std::fopen(path, "w");
    if (!f) return FM_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::fprintf(f, "# libfm autotune table v1: mc nc kc pc algo log2_T block_n k_chunk "
                    "no_karatsuba ms gops cta_pair\n");
    for (const auto& kv : g_tune) {
        const TuneKey& k = kv.first;
        const fm_tune_result& r = kv.second;
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d %.6f %.3f %d\n", k.mc, k.nc, k.kc, k.pc, r.algo,
                     r.log2_T, r.opts.block_n, r.opts.k_chunk, r.opts.no_karatsuba, r.ms, r.gops,
                     r.opts.cta_pair);
    }
    std::fclose(f);
    return FM_OK;
}

extern "C" int fm_autotune_load(const char* path)
{
    if (!path) return FM_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return FM_EINVAL;
    char line[512];
    int loaded = 0;
    std::map<TuneKey, fm_tune_result> table;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        TuneKey k;
        fm_tune_result r;
        std::memset(&r, 0, sizeof(r));
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d %lf %lf %d", &k.mc, &k.nc,
                                    &k.kc, &k.pc, &r.algo, &r.log2_T, &r.opts.block_n,
                                    &r.opts.k_chunk, &r.opts.no_karatsuba, &r.ms, &r.gops,
                                    &r.opts.cta_pair);
        if (got != 11 && got != 12) {
            std::fclose(f);
            return FM_EINVAL;
        }
        if (r.algo != FM_ALGO_PLAIN && r.algo != FM_ALGO_LIMB_TC) {
            std::fclose(f);
            return FM_EINVAL;
        }
        table[k] = r;
        ++loaded;
    }
    std::fclose(f);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : table) g_tune[kv.first] = kv.second;
    return loaded;
}

extern "C" int fm_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return FM_OK;
}

extern "C" int fm_autotune_lookup(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out)
{
    if (!out) return FM_EINVAL;
    return fm_tuned_choice(M, N, K, p, out) ? 1 : 0;
}
