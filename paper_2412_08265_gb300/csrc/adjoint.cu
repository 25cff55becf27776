// adjoint.cu -- pieces of the hand-written adjoint (gradients through the
// pipeline, Abstract and Sec. 1) that do not depend on the deposit's
// decomposition: zeroing the gradient outputs, and the FP64 sums of the
// per-particle contributions to the parameters every particle shares (a
// systemic velocity, a global mass scale, the inclination and the azimuth),
// added in a fixed order so that they are reproducible bit for bit.
#include "common.cuh"
#include "kernels.h"

namespace rubix {

__global__ void k_zero4(float* a, float* b, float* c, float* d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (a) a[i] = 0.f;
        if (b) b[i] = 0.f;
        if (c) c[i] = 0.f;
        if (d) d[i] = 0.f;
    }
}

int launch_zero_grads(float* a, float* b, float* c, float* d, long long n, cudaStream_t st) {
    if (n <= 0) return 0;
    long long nb = (n + 255) / 256;
    const long long cap = 8ll * sm_count();
    if (nb > cap) nb = cap;
    k_zero4<<<(int)nb, 256, 0, st>>>(a, b, c, d, n);
    return 1;
}

// K8: fixed-order FP64 reduction of contrib[n][kGlobal] -> out[kGlobal]: each
// of kRedBlocks blocks sums a contiguous range (strided per thread, then a
// tree), and one block adds the block sums by a tree.
constexpr int kRedBlocks = 256;
__global__ void __launch_bounds__(256) k_reduce_partial(const double* __restrict__ contrib, const int* __restrict__ n_dev,
                                                        double* __restrict__ part) {
    __shared__ double sh[kGlobal][256];
    const long long n = *n_dev;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long b = per * blockIdx.x, e = min(b + per, n);
    double a[kGlobal];
#pragma unroll
    for (int c = 0; c < kGlobal; ++c) a[c] = 0.0;
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x)
#pragma unroll
        for (int c = 0; c < kGlobal; ++c) a[c] += contrib[kGlobal * i + c];
#pragma unroll
    for (int c = 0; c < kGlobal; ++c) sh[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < kGlobal; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < kGlobal; ++c) part[kGlobal * blockIdx.x + c] = sh[c][0];
}

// Sum of the kRedBlocks partial sums: a fixed pairwise tree in shared memory
// (one thread per partial), so the order of the additions never changes.
__global__ void __launch_bounds__(kRedBlocks) k_reduce_final(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sh[kGlobal][kRedBlocks];
#pragma unroll
    for (int c = 0; c < kGlobal; ++c) sh[c][threadIdx.x] = part[kGlobal * threadIdx.x + c];
    __syncthreads();
    for (int o = kRedBlocks / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < kGlobal; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < kGlobal) out[threadIdx.x] = sh[threadIdx.x][0];
}

int launch_reduce_global(const double* contrib, const int* n_in_dev, double* out, double* scratch, cudaStream_t st) {
    k_reduce_partial<<<kRedBlocks, 256, 0, st>>>(contrib, n_in_dev, scratch);
    k_reduce_final<<<1, kRedBlocks, 0, st>>>(scratch, out);
    return 2;
}

}  // namespace rubix
