// Self-test of the failure path of the bounded device waits (idg_selftest_wait_timeout).
//
// The tensor-core kernels wait on shared-memory mbarriers for their matrix
// operations and bulk copies, every wait with an iteration limit; on a timeout
// a kernel records an error word, releases its tensor memory and returns.  This
// kernel exercises that path on purpose without any matrix operation: one CTA
// allocates tensor memory as the tensor-core kernels do, initialises an mbarrier
// that nothing ever arrives on, waits on it with a caller-given poll limit
// (which therefore runs out), records the timeout in its device error word
// (read and cleared by idg_device_errors with the others) and releases the
// tensor memory on the same, unconditional path as the success case.
#include <cuda_runtime.h>

#include "idg_internal.h"
#include "tc_common.cuh"

namespace idg {

// device error word of the self-test kernel (0 = ok)
__device__ int g_selftest_error = 0;

namespace {

constexpr int kThreads = 128;
constexpr int kColumns = 32;                 // smallest tensor-memory allocation

__global__ void __launch_bounds__(kThreads) wait_timeout_kernel(long max_polls) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc::smem_u32(&tmem_base)), "n"(kColumns));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // phase 0 of the barrier never completes: nothing arrives on it
    bool done = false;
    if (threadIdx.x == 0) {
        for (long it = 0; it < max_polls && !done; ++it) {
            uint32_t ok;
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(tc::smem_u32(&bar)), "r"(0u) : "memory");
            done = ok != 0;
        }
    }
    // the decision is uniform over the CTA, as in the tensor-core kernels
    const bool failed = __syncthreads_or(threadIdx.x == 0 && !done) != 0;
    if (failed && threadIdx.x == 0) atomicExch(&g_selftest_error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_base), "n"(kColumns));
    }
}

}  // namespace

idg_status read_selftest_error(int *code) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(code, g_selftest_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_selftest_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the self-test error word");
    return IDG_OK;
}

}  // namespace idg

using namespace idg;

extern "C" idg_status idg_selftest_wait_timeout(int64_t max_polls, idg_stream stream) {
    if (max_polls < 1 || max_polls > tc::kSpin)
        return fail(IDG_ERR_INVALID_ARG, "max_polls must be in 1 .. 2^20");
    wait_timeout_kernel<<<1, kThreads, 0, (cudaStream_t)stream>>>((long)max_polls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return IDG_OK;
}
