// fr_selftest.cu -- device check of the bounded waits (failure detection).
//
// Every wait in the fused and tensor-core kernels is an mbarrier wait
// bounded by the global timer: when an expected arrival never comes, the
// wait gives up after its limit, sets an abort flag and an error bit, and the
// kernel runs to its end, so the context stays usable and the host reads the
// error.  fr_wait_selftest runs both wait forms those kernels use on
// barriers that nothing completes, with a caller-given short limit, plus one
// wait on a barrier that does complete (a control that must not report).
#include "fr_common.cuh"
#include "fr_ptx.cuh"

namespace fr {
namespace {

// One block of 64 threads.  out[0]: error bits (1: single-thread wait gave
// up, 2: warp-wide wait gave up, 4: the control wait failed); out[1], out[2]:
// global-timer ns spent in the two waits that are meant to give up.
__global__ void __launch_bounds__(64) k_wait_selftest(unsigned long long *out, uint64_t limit_ns)
{
    using namespace ptx;
    __shared__ uint64_t bar[2];
    __shared__ int abort_flag[3];
    __shared__ unsigned err;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag[0] = abort_flag[1] = abort_flag[2] = 0;
        err = 0u;
        fence_mbar_init();
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (lane == 0) {                          // nothing arrives on bar[0]
            const uint64_t t0 = globaltimer();
            mbar_wait(&bar[0], 0u, &abort_flag[0], &err, 1u, limit_ns);
            out[1] = globaltimer() - t0;
        }
    } else {                                      // nothing arrives on bar[1]
        const uint64_t t0 = globaltimer();
        warp_wait_all(&bar[1], 0u, false, &abort_flag[1], &err, 2u, limit_ns);
        if (lane == 0) out[2] = globaltimer() - t0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // control: the arrival completes phase 0 of bar[0], so the wait
        // returns at once and sets no bit
        mbar_arrive(&bar[0]);
        mbar_wait(&bar[0], 0u, &abort_flag[2], &err, 4u, limit_ns);
        out[0] = err;
    }
}

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" int fr_wait_selftest(fr_ctx *ctx, int32_t limit_us, uint32_t *flags, uint64_t *waited_ns)
{
    FR_NVTX("fr_wait_selftest");
    FR_CHECK(ctx && flags, FR_EINVAL, "fr_wait_selftest: NULL argument");
    FR_CHECK(limit_us >= 1 && limit_us <= 2000000, FR_EINVAL, "fr_wait_selftest: limit_us %d not in 1..2e6",
             limit_us);
    FR_CUDA(cudaSetDevice(ctx->device));
    unsigned long long *d = nullptr;
    FR_CUDA(cudaMalloc(&d, 3 * sizeof(unsigned long long)));
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaMemset(d, 0, sizeof(h));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 64>>>(d, (uint64_t)limit_us * 1000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "fr_wait_selftest");
    *flags = (uint32_t)h[0];
    if (waited_ns) {
        waited_ns[0] = h[1];
        waited_ns[1] = h[2];
    }
    if (h[0] == 0) return FR_OK;
    set_error("fr_wait_selftest: bounded waits gave up (error bits 0x%x)", (unsigned)h[0]);
    return FR_ETIMEDOUT;
}
