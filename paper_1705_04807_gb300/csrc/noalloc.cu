// noalloc.cu -- the tensor-core limb product for callers that cannot allocate.
//
// fm_gemm_modp keeps its limb planes in workspace it allocates with
// cudaMalloc on first use. Some callers cannot let a library allocate device
// memory: programs whose device memory is handed out by their own allocator
// (a serving process that reserves the GPU's memory for its pool at start-up)
// or capped by a fixed budget, where an allocation behind the allocator's back
// can fail at an arbitrary point or push a co-tenant out of memory, and code
// that must not stall on cudaMalloc's implicit device synchronisation. This
// file gives them fm_gemm_modp_noalloc: the same limb form, with its scratch
// in a fixed, file-scope device array instead of allocated memory. The caller
// still owns and passes A, B and C.
#include <mutex>

#include "fm_internal.cuh"
#include "fm_kernels.h"

namespace {

// Limb planes of A and B for one product, at most 64 MiB, followed by a status
// word. Lives in device memory of every GPU that loads this module, until the
// process exits.
constexpr size_t kNoallocPlaneBytes = (size_t)64 << 20;
constexpr size_t kNoallocBytes = kNoallocPlaneBytes + 256;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Host code cannot use g_noalloc_scratch's name as a device address (on the
// host it names a shadow variable), so the device address is looked up once
// per device, with that device current, and cached. The same first call also
// does the limb kernels' other one-time query (how many CTA pairs fit on the
// device at once), so that no later call of any shape makes one.
void* scratch_on_current_device()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return nullptr;
        if (fm_limb_prepare_device() != FM_OK) return nullptr;
        g_noalloc_addr[dev] = p;
    }
    return g_noalloc_addr[dev];
}

// The address of the array on the current device if a call has set it up,
// else nullptr (no lookup: a device no call has used has nothing to report).
void* scratch_if_set_up()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    return g_noalloc_addr[dev];
}

__global__ void noalloc_zero_kernel(uint32_t* base, int lt, int64_t row0, int64_t col0,
                                    int64_t rows, int64_t cols)
{
    const int64_t n = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        base[fm_encode((uint64_t)(row0 + i), (uint64_t)(col0 + j), lt)] = 0;
    }
}

}  // namespace

extern "C" int fm_gemm_modp_noalloc(fm_sub C, fm_sub A, fm_sub B, uint32_t p, int32_t op,
                                    fm_stream stream)
{
    if (p < 2 || p >= (1u << 31)) return FM_EMODULUS;
    if (op < FM_OP_SET || op > FM_OP_SUB) return FM_EINVAL;
    FM_TRY(fm_check_product(C, A, B, false));
    const int64_t M = C.rows, N = C.cols, K = A.cols;
    if (M == 0 || N == 0) return FM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    FmLimbPlan plan;
    if (K > 0) {
        FM_TRY(fm_limb_plan(M, N, K, p, nullptr, &plan));
        if (fm_limb_workspace_bytes(plan) > kNoallocPlaneBytes) return FM_ETOOBIG;
    }
    if (K == 0) {
        if (op == FM_OP_SET) {
            noalloc_zero_kernel<<<256, 256, 0, s>>>(C.m.base, C.m.log2_T, C.row0, C.col0, M, N);
            FM_CUDA_TRY(cudaGetLastError());
        }
        return FM_OK;
    }
    uint8_t* scratch = static_cast<uint8_t*>(scratch_on_current_device());
    if (!scratch) return FM_ECUDA;
    // The status word is not cleared here: like the library's own status word
    // it keeps the first error raised since fm_get_last_device_status last read
    // it. Nothing left in the planes by an earlier call needs clearing either:
    // the split writes every plane byte a stored output depends on, the zero
    // K padding included; plane rows past M (A) or N (B) keep older contents,
    // which reach only output rows and columns that are never stored.
    int* status = reinterpret_cast<int*>(scratch + kNoallocPlaneBytes);
    return fm_limb_run(plan, C, A, B, p, op, scratch, status, s);
}

int* fm_noalloc_status_word()
{
    uint8_t* scratch = static_cast<uint8_t*>(scratch_on_current_device());
    return scratch ? reinterpret_cast<int*>(scratch + kNoallocPlaneBytes) : nullptr;
}

int fm_noalloc_take_status(cudaStream_t s, int* out)
{
    *out = FM_OK;
    uint8_t* scratch = static_cast<uint8_t*>(scratch_if_set_up());
    if (!scratch) return FM_OK;
    int* status = reinterpret_cast<int*>(scratch + kNoallocPlaneBytes);
    // pageable host destination: the copies complete before they return
    FM_CUDA_TRY(cudaMemcpyAsync(out, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    FM_CUDA_TRY(cudaStreamSynchronize(s));
    FM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    FM_CUDA_TRY(cudaStreamSynchronize(s));
    return FM_OK;
}
