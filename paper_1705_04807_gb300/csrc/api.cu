// api.cu -- C entry points of libfm: validation, algorithm dispatch, cached
// workspace, device status word, and the batched plan.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

#include "fm_internal.cuh"
#include "fm_kernels.h"
#include "fm_sched.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kSlots = 7;

struct DeviceState {
    int* status = nullptr;
    void* ws[kSlots] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t ws_bytes[kSlots] = {0, 0, 0, 0, 0, 0, 0};
    int sm_count = 0;
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return (d >= 0 && d < kMaxDevices) ? d : -1;
}

// ---- cached decomposition lists for single calls ----
struct ListKey {
    fm_sub C, A, B;
    int32_t op;
    static bool same(const fm_sub& x, const fm_sub& y)
    {
        return x.m.base == y.m.base && x.m.log2_grid == y.m.log2_grid &&
               x.m.log2_T == y.m.log2_T && x.row0 == y.row0 && x.col0 == y.col0 &&
               x.rows == y.rows && x.cols == y.cols;
    }
    bool operator==(const ListKey& o) const
    {
        return same(C, o.C) && same(A, o.A) && same(B, o.B) && op == o.op;
    }
};

struct ListEntry {
    ListKey key;
    int device;
    FmCallDesc* d_calls = nullptr;
    FmWorkItem* d_items = nullptr;
    FmLPiece* d_lps = nullptr;
    int64_t n_items = 0;
};

std::list<ListEntry> g_lists;  // most recently used first
constexpr size_t kMaxLists = 64;

void free_entry(ListEntry& e)
{
    cudaFree(e.d_calls);
    cudaFree(e.d_items);
    cudaFree(e.d_lps);
}

template <class T>
int upload(const std::vector<T>& v, T** out)
{
    *out = nullptr;
    if (v.empty()) return FM_OK;
    if (cudaMalloc(reinterpret_cast<void**>(out), v.size() * sizeof(T)) != cudaSuccess) return FM_ENOMEM;
    if (cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return FM_ECUDA;
    return FM_OK;
}

int get_lists(const fm_sub& C, const fm_sub& A, const fm_sub& B, int op, ListEntry** out)
{
    ListKey key;
    std::memset(&key, 0, sizeof(key));
    key.C = C;
    key.A = A;
    key.B = B;
    key.op = op;
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_lists.begin(); it != g_lists.end(); ++it) {
        if (it->device == dev && it->key == key) {
            g_lists.splice(g_lists.begin(), g_lists, it);
            *out = &g_lists.front();
            return FM_OK;
        }
    }
    std::vector<FmWorkItem> items;
    std::vector<FmLPiece> lps;
    FmCallDesc cd;
    cd.C = C.m.base;
    cd.A = A.m.base;
    cd.B = B.m.base;
    cd.lt = C.m.log2_T;
    cd.op = op;
    fm_decompose_call(C, A, B, 0, items, lps, &cd.lp_begin, &cd.lp_count);
    std::vector<FmCallDesc> calls(1, cd);
    ListEntry e;
    e.key = key;
    e.device = dev;
    e.n_items = (int64_t)items.size();
    int rc = upload(calls, &e.d_calls);
    if (rc == FM_OK) rc = upload(items, &e.d_items);
    if (rc == FM_OK) rc = upload(lps, &e.d_lps);
    if (rc != FM_OK) {
        free_entry(e);
        return rc;
    }
    if (g_lists.size() >= kMaxLists) {
        free_entry(g_lists.back());
        g_lists.pop_back();
    }
    g_lists.push_front(e);
    *out = &g_lists.front();
    return FM_OK;
}

bool narrow_ok(uint32_t p, int64_t K)
{
    const unsigned __int128 bound = (unsigned __int128)(p - 1) * (p - 1) * (unsigned __int128)K;
    return bound < ((unsigned __int128)1 << 64);
}

bool dfma_ok(uint32_t p, int64_t K)
{
    const unsigned __int128 bound = (unsigned __int128)(p - 1) * (p - 1) * (unsigned __int128)K;
    return bound < ((unsigned __int128)1 << 53);
}

__global__ void zero_sub_kernel(uint32_t* base, int lt, int64_t row0, int64_t col0, int64_t rows,
                                int64_t cols)
{
    const int64_t n = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        base[fm_encode((uint64_t)(row0 + i), (uint64_t)(col0 + j), lt)] = 0;
    }
}

int resolve_algo(const fm_sub& C, const fm_sub& A, const fm_sub& B, int algo)
{
    if (algo != FM_ALGO_AUTO) return algo;
    const bool same = A.m.log2_T == C.m.log2_T && B.m.log2_T == C.m.log2_T;
    const bool plain_tiles = same && (C.m.log2_T == 5 || C.m.log2_T == 6);
    const int64_t M = C.rows, N = C.cols, K = A.cols;
    const bool big = M >= 256 && N >= 256 && K >= 256;
    if (big || !plain_tiles) return FM_ALGO_LIMB_TC;
    return FM_ALGO_PLAIN;
}

}  // namespace

// ---------------------------------------------------------------------------
int* fm_device_status()
{
    const int d = current_device();
    if (d < 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState& s = g_dev[d];
    if (!s.status) {
        if (cudaMalloc(&s.status, sizeof(int)) != cudaSuccess) {
            s.status = nullptr;
            return nullptr;
        }
        if (cudaMemset(s.status, 0, sizeof(int)) != cudaSuccess) return nullptr;
    }
    return s.status;
}

void* fm_workspace(int slot, size_t bytes)
{
    const int d = current_device();
    if (d < 0 || slot < 0 || slot >= kSlots) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState& s = g_dev[d];
    if (s.ws_bytes[slot] >= bytes && s.ws[slot]) return s.ws[slot];
    if (s.ws[slot]) {
        cudaFree(s.ws[slot]);  // synchronises the device: no kernel still uses it
        s.ws[slot] = nullptr;
        s.ws_bytes[slot] = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 256) != cudaSuccess) return nullptr;
    s.ws[slot] = p;
    s.ws_bytes[slot] = bytes;
    return p;
}

int fm_sm_count()
{
    const int d = current_device();
    if (d < 0) return 148;
    DeviceState& s = g_dev[d];
    if (!s.sm_count) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0)
            n = 148;
        s.sm_count = n;
    }
    return s.sm_count;
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Tracing (FM_TRACE) and NVTX ranges.
bool fm_trace_on()
{
    const char* v = std::getenv("FM_TRACE");
    return v && *v && std::strcmp(v, "0") != 0;
}

void fm_trace(const char* fmt, ...)
{
    if (!fm_trace_on()) return;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    const char* v = std::getenv("FM_TRACE");
    FILE* f = std::strcmp(v, "1") == 0 ? stderr : std::fopen(v, "a");
    if (!f) return;
    va_list ap;
    va_start(ap, fmt);
    std::fprintf(f, "fm: ");
    std::vfprintf(f, fmt, ap);
    std::fprintf(f, "\n");
    va_end(ap);
    if (f != stderr) std::fclose(f);
}

FmRange::FmRange(const char* name) { nvtxRangePushA(name); }
FmRange::~FmRange() { nvtxRangePop(); }

extern "C" int fm_gemm_modp(fm_sub C, fm_sub A, fm_sub B, uint32_t p, int32_t op, int32_t algo,
                            const fm_opts* opts, fm_stream stream)
{
    FmRange range("fm_gemm_modp");
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    if (op < FM_OP_SET || op > FM_OP_SUB) return FM_EINVAL;
    if (algo < FM_ALGO_AUTO || algo > FM_ALGO_DFMA) return FM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    FM_TRY(fm_check_product(C, A, B, false));
    const int64_t M = C.rows, N = C.cols, K = A.cols;
    if (M == 0 || N == 0) return FM_OK;
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    if (K == 0) {
        if (op == FM_OP_SET) {
            zero_sub_kernel<<<256, 256, 0, s>>>(C.m.base, C.m.log2_T, C.row0, C.col0, M, N);
            FM_CUDA_TRY(cudaGetLastError());
        }
        return FM_OK;
    }
    fm_opts tuned_opts;
    if (algo == FM_ALGO_AUTO && opts == nullptr) {
        fm_tune_result r;
        if (fm_tuned_choice(M, N, K, p, &r)) {
            const bool same = A.m.log2_T == C.m.log2_T && B.m.log2_T == C.m.log2_T;
            const bool plain_ok = same && (C.m.log2_T == 5 || C.m.log2_T == 6);
            if (r.algo == FM_ALGO_LIMB_TC || !plain_ok) {
                algo = FM_ALGO_LIMB_TC;
                if (r.algo == FM_ALGO_LIMB_TC) {
                    tuned_opts = r.opts;
                    opts = &tuned_opts;
                }
            } else {
                algo = FM_ALGO_PLAIN;
            }
        }
    }
    algo = resolve_algo(C, A, B, algo);
    if (algo == FM_ALGO_LIMB_MMA_S8) return FM_EUNSUPPORTED;
    if (algo == FM_ALGO_LIMB_TC) {
        FmLimbPlan plan;
        FM_TRY(fm_limb_plan_shaped(M, N, K, p, opts, &plan));
        void* ws = fm_workspace(0, fm_limb_workspace_bytes(plan));
        if (!ws) return FM_ENOMEM;
        fm_trace("gemm_modp limb M=%lld N=%lld K=%lld p=%u op=%d products=%d tiles=%d jobs/tile=%d planes=%zu B",
                 (long long)M, (long long)N, (long long)K, p, op, plan.n_products, plan.MB * plan.NB,
                 plan.n_products ? (plan.KB + plan.prod_cs[0] - 1) / plan.prod_cs[0] : 0,
                 fm_limb_workspace_bytes(plan));
        return fm_limb_run(plan, C, A, B, p, op, ws, status, s);
    }
    // decomposed paths (Sec. 2.2): equal T', T' in {32, 64}
    FM_TRY(fm_check_product(C, A, B, true));
    const int lt = C.m.log2_T;
    if (lt != 5 && lt != 6) return FM_EUNSUPPORTED;
    int arith;
    if (algo == FM_ALGO_DFMA) {
        if (!dfma_ok(p, K)) return FM_EUNSUPPORTED;
        arith = kArithDfma;
    } else {
        arith = narrow_ok(p, K) ? kArithNarrow : kArithWide;
    }
    ListEntry* e = nullptr;
    FM_TRY(get_lists(C, A, B, op, &e));
    fm_trace("gemm_modp %s T'=%d M=%lld N=%lld K=%lld p=%u op=%d base-case products=%lld",
             algo == FM_ALGO_DFMA ? "dfma" : "plain", 1 << lt, (long long)M, (long long)N, (long long)K, p,
             op, (long long)e->n_items);
    return fm_plain_launch(lt, arith, e->d_calls, e->d_items, e->d_lps, e->n_items, p, nullptr,
                           (int)e->n_items, status, s);
}

extern "C" int64_t fm_gemm_modp_workspace_size(fm_sub C, fm_sub A, fm_sub B, uint32_t p,
                                               int32_t algo, const fm_opts* opts)
{
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    int rc = fm_check_product(C, A, B, false);
    if (rc != FM_OK) return rc;
    algo = resolve_algo(C, A, B, algo);
    if (algo != FM_ALGO_LIMB_TC) return 0;
    FmLimbPlan plan;
    rc = fm_limb_plan_shaped(C.rows, C.cols, A.cols, p, opts, &plan);
    if (rc != FM_OK) return rc;
    return (int64_t)fm_limb_workspace_bytes(plan);
}

// ---------------------------------------------------------------------------
// Batched plan: every call decomposed into work items of one shared list,
// executed by one persistent launch that pulls items from a device queue.
struct fm_plan {
    int device = 0;
    uint32_t p = 0;
    int lt = 0;
    int arith = kArithNarrow;
    int64_t n_items = 0;
    FmCallDesc* d_calls = nullptr;
    FmWorkItem* d_items = nullptr;
    FmLPiece* d_lps = nullptr;
    int* d_queue = nullptr;
    int grid = 0;
    FmLimbBatch* limb = nullptr;  // FM_ALGO_LIMB_TC: the batched tensor-core form
};

extern "C" int fm_plan_create(fm_plan** out, const fm_gemm_call* calls, int64_t n, uint32_t p,
                              int32_t algo, const fm_opts* opts)
{
    if (!out || (n > 0 && !calls) || n < 0) return FM_EINVAL;
    *out = nullptr;
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    if (algo == FM_ALGO_AUTO && opts == nullptr && n > 0) {
        // the form fm_autotune_batch measured fastest for batches of this class
        fm_tune_result r;
        if (fm_tuned_batch_choice(calls, n, p, &r) &&
            fm_plan_create(out, calls, n, p, r.algo, r.algo == FM_ALGO_LIMB_TC ? &r.opts : nullptr) == FM_OK)
            return FM_OK;
    }
    if (algo == FM_ALGO_LIMB_TC) {
        for (int64_t c = 0; c < n; ++c) {
            const fm_gemm_call& g = calls[c];
            if (g.op < FM_OP_SET || g.op > FM_OP_SUB) return FM_EINVAL;
            FM_TRY(fm_check_product(g.C, g.A, g.B, false));
        }
        fm_plan* pl = new fm_plan();
        pl->device = current_device();
        pl->p = p;
        const int rc = fm_limb_batch_create(calls, n, p, opts, &pl->limb);
        if (rc != FM_OK) {
            delete pl;
            return rc;
        }
        pl->n_items = fm_limb_batch_tiles(pl->limb);
        *out = pl;
        return FM_OK;
    }
    if (algo != FM_ALGO_AUTO && algo != FM_ALGO_PLAIN && algo != FM_ALGO_DFMA) return FM_EUNSUPPORTED;
    int lt = -1;
    int64_t kmax = 0;
    for (int64_t c = 0; c < n; ++c) {
        const fm_gemm_call& g = calls[c];
        if (g.op < FM_OP_SET || g.op > FM_OP_SUB) return FM_EINVAL;
        FM_TRY(fm_check_product(g.C, g.A, g.B, true));
        if (lt < 0) lt = g.C.m.log2_T;
        if (g.C.m.log2_T != lt) return FM_EINVAL;
        kmax = std::max<int64_t>(kmax, g.A.cols);
    }
    if (n > 0 && lt != 5 && lt != 6) return FM_EUNSUPPORTED;
    std::vector<FmCallDesc> cds((size_t)n);
    std::vector<FmWorkItem> items;
    std::vector<FmLPiece> lps;
    for (int64_t c = 0; c < n; ++c) {
        const fm_gemm_call& g = calls[c];
        FmCallDesc& cd = cds[(size_t)c];
        cd.C = g.C.m.base;
        cd.A = g.A.m.base;
        cd.B = g.B.m.base;
        cd.lt = lt;
        cd.op = g.op;
        fm_decompose_call(g.C, g.A, g.B, (int32_t)c, items, lps, &cd.lp_begin, &cd.lp_count);
    }
    // longest work first: better balance for the persistent queue
    std::stable_sort(items.begin(), items.end(), [&](const FmWorkItem& x, const FmWorkItem& y) {
        return cds[x.call].lp_count > cds[y.call].lp_count;
    });
    fm_plan* pl = new fm_plan();
    pl->device = current_device();
    pl->p = p;
    pl->lt = lt < 0 ? 6 : lt;
    if (algo == FM_ALGO_DFMA) {
        if (!dfma_ok(p, kmax)) {
            delete pl;
            return FM_EUNSUPPORTED;
        }
        pl->arith = kArithDfma;
    } else {
        pl->arith = narrow_ok(p, kmax) ? kArithNarrow : kArithWide;
    }
    pl->n_items = (int64_t)items.size();
    int rc = upload(cds, &pl->d_calls);
    if (rc == FM_OK) rc = upload(items, &pl->d_items);
    if (rc == FM_OK) rc = upload(lps, &pl->d_lps);
    if (rc == FM_OK && cudaMalloc(&pl->d_queue, sizeof(int)) != cudaSuccess) rc = FM_ENOMEM;
    if (rc != FM_OK) {
        fm_plan_destroy(pl);
        return rc;
    }
    pl->grid = fm_sm_count() * fm_plain_occupancy(pl->lt, pl->arith);
    *out = pl;
    return FM_OK;
}

extern "C" int fm_gf2_plan_create(fm_plan** out, const fm_gf2_call* calls, int64_t n, const fm_opts* opts)
{
    if (!out || (n > 0 && !calls) || n < 0) return FM_EINVAL;
    *out = nullptr;
    for (int64_t c = 0; c < n; ++c) FM_TRY(fm_gf2_check_call(calls[c]));
    fm_plan* pl = new fm_plan();
    pl->device = current_device();
    pl->p = 2;
    const int rc = fm_gf2_batch_create(calls, n, opts, &pl->limb);
    if (rc != FM_OK) {
        delete pl;
        return rc;
    }
    pl->n_items = fm_limb_batch_tiles(pl->limb);
    *out = pl;
    return FM_OK;
}

extern "C" int fm_gemm_modp_batched(fm_plan* plan, fm_stream stream)
{
    FmRange range("fm_gemm_modp_batched");
    if (!plan) return FM_EINVAL;
    fm_trace("gemm_modp_batched %s work items=%lld launches=%lld",
             plan->limb ? "tensor-core" : "decomposed", (long long)plan->n_items,
             (long long)fm_plan_launches(plan));
    if (plan->limb) {
        for (const fm_gemm_call& g : fm_limb_batch_zero_calls(plan->limb))
            if (g.op == FM_OP_SET) FM_TRY(fm_gemm_modp(g.C, g.A, g.B, plan->p, g.op, FM_ALGO_LIMB_TC, nullptr, stream));
        int* status = fm_device_status();
        if (!status) return FM_ECUDA;
        return fm_limb_batch_run(plan->limb, status, (cudaStream_t)stream);
    }
    if (plan->n_items == 0) return FM_OK;
    int* status = fm_device_status();
    if (!status) return FM_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    FM_CUDA_TRY(cudaMemsetAsync(plan->d_queue, 0, sizeof(int), s));
    const int grid = (int)std::min<int64_t>(plan->grid, plan->n_items);
    return fm_plain_launch(plan->lt, plan->arith, plan->d_calls, plan->d_items, plan->d_lps,
                           plan->n_items, plan->p, plan->d_queue, grid, status, s);
}

extern "C" int64_t fm_plan_work_items(const fm_plan* plan)
{
    return plan ? plan->n_items : (int64_t)FM_EINVAL;
}

extern "C" int64_t fm_plan_launches(const fm_plan* plan)
{
    if (!plan) return FM_EINVAL;
    if (plan->limb) {
        int64_t n = fm_limb_batch_launches(plan->limb);
        for (const fm_gemm_call& g : fm_limb_batch_zero_calls(plan->limb)) n += g.op == FM_OP_SET ? 1 : 0;
        return n;
    }
    return plan->n_items > 0 ? 1 : 0;
}

extern "C" int fm_plan_destroy(fm_plan* plan)
{
    if (!plan) return FM_OK;
    cudaFree(plan->d_calls);
    cudaFree(plan->d_items);
    cudaFree(plan->d_lps);
    cudaFree(plan->d_queue);
    fm_limb_batch_destroy(plan->limb);
    delete plan;
    return FM_OK;
}

// ---------------------------------------------------------------------------
extern "C" int fm_get_last_device_status(fm_stream stream)
{
    const int d = current_device();
    if (d < 0) return FM_ECUDA;
    FM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    // No allocation here: a status word that does not exist yet has had no
    // kernel raise into it.
    int* st = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        st = g_dev[d].status;
    }
    int h = FM_OK;
    if (st) {
        FM_CUDA_TRY(cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost));
        FM_CUDA_TRY(cudaMemset(st, 0, sizeof(int)));
    }
    // the word fm_gemm_modp_noalloc's kernels raise into
    int h2 = FM_OK;
    FM_TRY(fm_noalloc_take_status((cudaStream_t)stream, &h2));
    return h != FM_OK ? h : h2;
}

extern "C" const char* fm_strerror(int status)
{
    switch (status) {
    case FM_OK: return "ok";
    case FM_EINVAL: return "invalid argument (shape, descriptor, pointer or overlap)";
    case FM_EMODULUS: return "modulus out of range (need 2 <= p < 2^31)";
    case FM_ERANGE: return "residue out of range";
    case FM_ECUDA: return "CUDA runtime error";
    case FM_ETIMEOUT: return "bounded device wait expired";
    case FM_ENOMEM: return "out of device memory";
    case FM_EUNSUPPORTED: return "unsupported configuration";
    case FM_ETOOBIG: return "product too large for the fixed scratch of fm_gemm_modp_noalloc";
    default: return "unknown status";
    }
}

extern "C" int fm_release_workspace(void)
{
    const int d = current_device();
    if (d < 0) return FM_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState& s = g_dev[d];
    for (int k = 0; k < kSlots; ++k) {
        if (s.ws[k]) cudaFree(s.ws[k]);
        s.ws[k] = nullptr;
        s.ws_bytes[k] = 0;
    }
    for (auto it = g_lists.begin(); it != g_lists.end();) {
        if (it->device == d) {
            free_entry(*it);
            it = g_lists.erase(it);
        } else {
            ++it;
        }
    }
    return FM_OK;
}

extern "C" int fm_version(void) { return FM_VERSION_NUM; }
