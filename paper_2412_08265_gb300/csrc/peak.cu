// peak.cu -- measured FP32 FMA throughput of the current device: the
// denominator of the deposit's FP32 roofline, taken on the machine and at
// the clocks the deposit runs at. Independent dependent chains of FFMA (or
// packed FFMA2) in every thread of every SM, long enough that launch costs
// vanish; the SM clock during the run comes from clock64 against the global
// nanosecond timer.
#include <cstdio>

#include "../../include/rubix.h"
#include "common.cuh"
#include "kernels.h"

namespace rubix {
void set_last_error(const char* msg);
}

using namespace rubix;

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 512;

struct PeakClock {
    unsigned long long c0, c1, t0, t1;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float* out, int iters, float b, float c, PeakClock* clk) {
    const unsigned long long c0 = clock64(), t0 = global_ns();
    float s = 0.f;
    if constexpr (PACKED) {
        float2 a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
        const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
    } else {
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk->c0 = c0;
        clk->t0 = t0;
        clk->c1 = clock64();
        clk->t1 = global_ns();
    }
}

}  // namespace

extern "C" rubix_status rubix_measure_fp32_peak(int32_t packed, double* flops_per_s, double* fma_per_clk_per_sm,
                                                double* sm_mhz) {
    if (!flops_per_s) {
        set_last_error("flops_per_s is NULL");
        return RUBIX_ERR_INVALID_ARG;
    }
    const int n_sm = sm_count();
    const int blocks = 4 * n_sm;
    const int iters = 20000;
    float* out = nullptr;
    PeakClock* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rubix_status st = RUBIX_OK;
    float ms = 0.f;
    PeakClock h{};
    auto cuda_fail = [&](cudaError_t e) {
        char m[160];
        snprintf(m, sizeof(m), "FP32 peak measurement: %s", cudaGetErrorString(e));
        set_last_error(m);
        return (rubix_status)RUBIX_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * kPeakThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&clk, sizeof(PeakClock));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        auto launch = [&](int it) {
            if (packed) k_fma_peak<true><<<blocks, kPeakThreads>>>(out, it, 1.0001f, 1e-4f, clk);
            else k_fma_peak<false><<<blocks, kPeakThreads>>>(out, it, 1.0001f, 1e-4f, clk);
        };
        launch(200);  // warm-up
        cudaEventRecord(e0);
        launch(iters);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaMemcpy(&h, clk, sizeof(h), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) st = cuda_fail(e);
    if (st == RUBIX_OK) {
        const double fmas = (double)blocks * kPeakThreads * kChains * (packed ? 2.0 : 1.0) * iters;
        const double secs = ms * 1e-3;
        const double mhz = (h.t1 > h.t0) ? (double)(h.c1 - h.c0) / ((double)(h.t1 - h.t0) * 1e-3) : 0.0;
        *flops_per_s = 2.0 * fmas / secs;
        if (sm_mhz) *sm_mhz = mhz;
        if (fma_per_clk_per_sm) *fma_per_clk_per_sm = mhz > 0.0 ? fmas / secs / (mhz * 1e6) / n_sm : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (clk) cudaFree(clk);
    return st;
}
