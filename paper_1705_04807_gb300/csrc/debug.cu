// debug.cu -- a test hook for failure detection (the paper has no counterpart).
//
// Every device-side wait of the library is bounded: after FM_WAIT_LIMIT_NS it
// raises FM_ETIMEOUT in the device status word and the kernel winds down. The
// hook launches a kernel whose wait cannot complete, through the same wait code
// the GEMM and PLUQ kernels use, so that a test can watch the limit expire and
// the status arrive while the context stays usable. Nothing faults or hangs.
// One kind raises into the status word of fm_gemm_modp_noalloc's fixed
// scratch instead of the library's own, which shows that a wait that runs out
// on that path reaches fm_get_last_device_status as well.
#include "fm_internal.cuh"
#include "fm_kernels.h"

namespace {

// An mbarrier that expects one arrival that never comes.
__global__ void expire_mbar_kernel(int* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        fm_mbar_init(&bar, 1);
        fm_fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) fm_mbar_wait(&bar, 0, status, nullptr);
}

// A grid barrier that CTA 1 of the two never reaches.
__global__ void expire_grid_kernel(unsigned* bar, int* status)
{
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    if (blockIdx.x == 1) return;
    fm_grid_barrier(bar, status, &s_abort);
}

}  // namespace

extern "C" int fm_debug_expire_wait(int32_t which, fm_stream stream)
{
    FmRange range("fm_debug_expire_wait");
    if (which < 0 || which > 2) return FM_EINVAL;
    int* status = which == 2 ? fm_noalloc_status_word() : fm_device_status();
    if (!status) return FM_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (which == 0 || which == 2) {
        expire_mbar_kernel<<<1, 32, 0, s>>>(status);
    } else if (which == 1) {
        unsigned* bar = static_cast<unsigned*>(fm_workspace(2, 2 * sizeof(unsigned)));
        if (!bar) return FM_ENOMEM;
        FM_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
        expire_grid_kernel<<<2, 32, 0, s>>>(bar, status);
    } else {
        return FM_EINVAL;
    }
    FM_CUDA_TRY(cudaGetLastError());
    return FM_OK;
}
