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
                        if (pair == 1 && bn != (q.fold ? 256 : 128)) continue;  // pair tile widths
                        limb(bn, kc, 0, pair);
                        if (q.n_planes > q.w) limb(bn, kc, 1, pair);
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

// ---- batches ---------------------------------------------------------------
// A batch's layout (T') is the caller's; what the tuner picks for it is the
// form (decomposed plain plan, limb plan with planes, fused limb plan) and the
// limb options (output tile width, K chunk, Karatsuba). Candidates run on the
// caller's batch itself, with every C matrix replaced by a scratch copy, so the
// caller's data is not changed. The winner is remembered per batch class:
// number of calls, mean M, N and K (each rounded up to a power of two), the
// modulus class and T'.
namespace {

struct BatchKey {
    int nc, mc, ncol, kc, pc, lt;
    bool operator<(const BatchKey& o) const
    {
        const int a[6] = {nc, mc, ncol, kc, pc, lt}, b[6] = {o.nc, o.mc, o.ncol, o.kc, o.pc, o.lt};
        return std::lexicographical_compare(a, a + 6, b, b + 6);
    }
};

std::map<BatchKey, fm_tune_result> g_tune_batch;

bool batch_key(const fm_gemm_call* calls, int64_t n, uint32_t p, BatchKey* k)
{
    if (n <= 0) return false;
    double sm = 0, sn = 0, sk = 0;
    const int lt = calls[0].C.m.log2_T;
    for (int64_t c = 0; c < n; ++c) {
        sm += (double)calls[c].C.rows;
        sn += (double)calls[c].C.cols;
        sk += (double)calls[c].A.cols;
    }
    *k = BatchKey{ceil_log2(n), ceil_log2((int64_t)(sm / n + 0.5)), ceil_log2((int64_t)(sn / n + 0.5)),
                  ceil_log2((int64_t)(sk / n + 0.5)), p_class(p), lt};
    return true;
}

}  // namespace

// Tuned choice for a problem class, if any (used by FM_ALGO_AUTO).
bool fm_tuned_choice(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key_of(M, N, K, p));
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

bool fm_tuned_batch_choice(const fm_gemm_call* calls, int64_t n, uint32_t p, fm_tune_result* out)
{
    BatchKey k;
    if (!batch_key(calls, n, p, &k)) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_batch.find(k);
    if (it == g_tune_batch.end()) return false;
    *out = it->second;
    return true;
}

extern "C" int fm_autotune_batch(const fm_gemm_call* calls, int64_t n, uint32_t p, int32_t flags,
                                 fm_stream stream, fm_tune_result* out)
{
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    if (!calls || n <= 0 || !out) return FM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    bool same_lt = true, plain_lt = true;
    double ops = 0;
    for (int64_t c = 0; c < n; ++c) {
        const fm_gemm_call& g = calls[c];
        FM_TRY(fm_check_product(g.C, g.A, g.B, false));
        same_lt = same_lt && g.C.m.log2_T == calls[0].C.m.log2_T && g.A.m.log2_T == calls[0].C.m.log2_T &&
                  g.B.m.log2_T == calls[0].C.m.log2_T;
        ops += 2.0 * (double)g.C.rows * g.C.cols * g.A.cols;
    }
    plain_lt = same_lt && (calls[0].C.m.log2_T == 5 || calls[0].C.m.log2_T == 6);
    // candidates: (algo, opts)
    std::vector<Candidate> cands;
    auto add = [&](int algo, int bn, int kchunk, int no_kara, int fused) {
        Candidate c;
        std::memset(&c, 0, sizeof(c));
        c.algo = algo;
        c.lt = calls[0].C.m.log2_T;
        c.opts.block_n = bn;
        c.opts.k_chunk = kchunk;
        c.opts.no_karatsuba = no_kara;
        c.opts.fused_batch = fused;
        cands.push_back(c);
    };
    if (!(flags & FM_TUNE_NO_LIMB)) {
        FmLimbPlan q;
        if (fm_limb_plan(512, 512, 1024, p, nullptr, &q) == FM_OK) {
            const int full = q.prod_cs[0] * 64;
            for (int bn : {128, 256}) {
                if (!q.fold && bn == 256) continue;
                for (int kc : {full, full / 2}) {
                    if (kc < 64 || kc % 64) continue;
                    add(FM_ALGO_LIMB_TC, bn, kc, 0, 0);
                    if (q.n_planes > q.w) add(FM_ALGO_LIMB_TC, bn, kc, 1, 0);
                }
            }
            if (q.fold && q.n_planes == 3) add(FM_ALGO_LIMB_TC, 128, 0, 0, 1);  // fused: Karatsuba, 128 wide
        }
    }
    if (!(flags & FM_TUNE_NO_PLAIN) && plain_lt) add(FM_ALGO_PLAIN, 0, 0, 0, 0);
    if (cands.empty()) return FM_EINVAL;

    // scratch copies of every C matrix the batch writes
    Scratch scratch;
    std::vector<fm_gemm_call> work(calls, calls + n);
    std::map<uint32_t*, uint32_t*> copy_of;
    for (fm_gemm_call& g : work) {
        uint32_t* base = g.C.m.base;
        auto it = copy_of.find(base);
        if (it == copy_of.end()) {
            const size_t bytes = (size_t)fm_side(g.C.m) * fm_side(g.C.m) * 4;
            void* q = nullptr;
            if (cudaMalloc(&q, bytes) != cudaSuccess) return FM_ENOMEM;
            scratch.ptrs.push_back(q);
            FM_CUDA_TRY(cudaMemcpyAsync(q, base, bytes, cudaMemcpyDeviceToDevice, s));
            it = copy_of.emplace(base, static_cast<uint32_t*>(q)).first;
        }
        g.C.m.base = it->second;
    }
    cudaEvent_t e0, e1;
    FM_CUDA_TRY(cudaEventCreate(&e0));
    FM_CUDA_TRY(cudaEventCreate(&e1));
    fm_tune_result best;
    std::memset(&best, 0, sizeof(best));
    best.ms = -1.0;
    int tried = 0;
    for (const Candidate& c : cands) {
        fm_plan* plan = nullptr;
        const fm_opts* o = c.algo == FM_ALGO_LIMB_TC ? &c.opts : nullptr;
        if (fm_plan_create(&plan, work.data(), n, p, c.algo, o) != FM_OK) continue;
        int rc = fm_gemm_modp_batched(plan, stream);  // warm-up (and the plane workspace)
        const int reps = 3;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && rc == FM_OK; ++r) rc = fm_gemm_modp_batched(plan, stream);
        cudaEventRecord(e1, s);
        const bool ok = cudaEventSynchronize(e1) == cudaSuccess && rc == FM_OK;
        fm_plan_destroy(plan);
        if (!ok) continue;
        float ms_total = 0.f;
        cudaEventElapsedTime(&ms_total, e0, e1);
        const double ms_one = ms_total / reps;
        ++tried;
        if (best.ms < 0 || ms_one < best.ms) {
            best.algo = c.algo;
            best.log2_T = c.lt;
            best.opts = c.opts;
            best.ms = ms_one;
            best.gops = ops / (ms_one * 1e-3) / 1e9;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (tried == 0) return FM_EUNSUPPORTED;
    best.candidates = tried;
    *out = best;
    BatchKey k;
    batch_key(calls, n, p, &k);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_batch[k] = best;
    return FM_OK;
}

// Text format, one class per line:
//   mc nc kc pc algo log2_T block_n k_chunk no_karatsuba ms gops [cta_pair]
// (a missing last field reads as 0); batch classes on lines of their own:
//   batch calls mc nc kc pc log2_T algo block_n k_chunk no_karatsuba fused_batch ms gops
extern "C" int fm_autotune_save(const char* path)
{
    if (!path) return FM_EINVAL;
    FILE* f = std::fopen(path, "w");
    if (!f) return FM_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::fprintf(f, "# libfm autotune table v2: mc nc kc pc algo log2_T block_n k_chunk "
                    "no_karatsuba ms gops cta_pair\n");
    for (const auto& kv : g_tune) {
        const TuneKey& k = kv.first;
        const fm_tune_result& r = kv.second;
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d %.6f %.3f %d\n", k.mc, k.nc, k.kc, k.pc, r.algo,
                     r.log2_T, r.opts.block_n, r.opts.k_chunk, r.opts.no_karatsuba, r.ms, r.gops,
                     r.opts.cta_pair);
    }
    for (const auto& kv : g_tune_batch) {
        const BatchKey& k = kv.first;
        const fm_tune_result& r = kv.second;
        std::fprintf(f, "batch %d %d %d %d %d %d %d %d %d %d %d %.6f %.3f\n", k.nc, k.mc, k.ncol, k.kc, k.pc,
                     k.lt, r.algo, r.opts.block_n, r.opts.k_chunk, r.opts.no_karatsuba, r.opts.fused_batch,
                     r.ms, r.gops);
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
    std::map<BatchKey, fm_tune_result> btable;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        fm_tune_result r;
        std::memset(&r, 0, sizeof(r));
        if (std::strncmp(line, "batch ", 6) == 0) {
            BatchKey k;
            const int got = std::sscanf(line + 6, "%d %d %d %d %d %d %d %d %d %d %d %lf %lf", &k.nc, &k.mc,
                                        &k.ncol, &k.kc, &k.pc, &k.lt, &r.algo, &r.opts.block_n,
                                        &r.opts.k_chunk, &r.opts.no_karatsuba, &r.opts.fused_batch, &r.ms,
                                        &r.gops);
            if (got != 13 || (r.algo != FM_ALGO_PLAIN && r.algo != FM_ALGO_LIMB_TC)) {
                std::fclose(f);
                return FM_EINVAL;
            }
            r.log2_T = k.lt;
            btable[k] = r;
            ++loaded;
            continue;
        }
        TuneKey k;
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
    for (const auto& kv : btable) g_tune_batch[kv.first] = kv.second;
    return loaded;
}

extern "C" int fm_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    g_tune_batch.clear();
    return FM_OK;
}

extern "C" int fm_autotune_lookup(int64_t M, int64_t N, int64_t K, uint32_t p, fm_tune_result* out)
{
    if (!out) return FM_EINVAL;
    return fm_tuned_choice(M, N, K, p, out) ? 1 : 0;
}
