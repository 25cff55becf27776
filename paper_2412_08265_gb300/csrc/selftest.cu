// selftest.cu -- self-test of the library's failure detection on the device:
// every wait in the kernels (the TMA slab loads of the deposit and adjoint)
// is bounded, records an error bit and lets the kernel return instead of
// hanging. This kernel waits on a shared-memory barrier that nothing will
// complete, with the same bounded wait and a short limit, so a test can check
// that the wait gives up, the status reaches the host and the context stays
// usable.
#include "../../include/rubix.h"
#include "common.cuh"
#include "engine.h"

namespace rubix {

__global__ void k_wait_selftest(long long max_cycles, unsigned* flag) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival completes phase 0; none is made
        fence_mbar_init();
    }
    __syncthreads();
    const bool done = mbar_wait_bounded(&bar, 0, max_cycles);
    if (!done && threadIdx.x == 0) atomicOr(flag, 1u);
}

}  // namespace rubix

using namespace rubix;

extern "C" rubix_status rubix_selftest_bounded_wait(double limit_s, int32_t* timed_out) {
    if (!timed_out) return fail(RUBIX_ERR_INVALID_ARG, "timed_out is NULL");
    if (!(limit_s > 0.0 && limit_s <= 10.0)) return fail(RUBIX_ERR_INVALID_ARG, "limit_s must be in (0, 10]");
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
        return fail(RUBIX_ERR_CUDA, "no CUDA device");
    unsigned* d_flag = nullptr;
    if (cudaMalloc(&d_flag, sizeof(unsigned)) != cudaSuccess) return fail(RUBIX_ERR_OOM, "selftest alloc");
    cudaMemset(d_flag, 0, sizeof(unsigned));
    const long long cycles = (long long)(limit_s * (double)khz * 1e3);
    k_wait_selftest<<<1, 32>>>(cycles, d_flag);
    unsigned h = 0;
    const cudaError_t e = cudaMemcpy(&h, d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d_flag);
    if (e != cudaSuccess) return fail(RUBIX_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
    *timed_out = h ? 1 : 0;
    return RUBIX_OK;
}
