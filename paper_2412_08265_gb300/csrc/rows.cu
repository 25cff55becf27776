// rows.cu -- the cube rows the deposit does not write itself (the per-spaxel
// sum of Sec. 3): rows of spaxels without particles, and rows of split
// spaxels, summed from their work items' partial rows.
#include "common.cuh"
#include "kernels.h"
#include "twosum.cuh"

namespace rubix {

// ----------------------------------------------------------------------------
// Rows of spaxels without particles: zeros (one warp per row, 16-byte stores
// when the rows are 16-byte aligned). The deposit has no work item for them,
// so a small galaxy in a large field costs the deposit only its own spaxels.
// ----------------------------------------------------------------------------
__global__ void k_zero_empty(const int* __restrict__ seg_off, int n_s, int nb, float* __restrict__ cube, int pitch,
                             int n_lambda) {
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const bool vec = (pitch % 4) == 0 && (reinterpret_cast<uintptr_t>(cube) & 15) == 0;
    for (long long s = w0; s < n_s; s += nw) {
        if (seg_off[(s + 1) * nb] != seg_off[s * nb]) continue;
        float* row = cube + s * pitch;
        int j0 = 0;
        if (vec) {
            float4* r4 = reinterpret_cast<float4*>(row);
            const int n4 = n_lambda >> 2;
            for (int j = lane; j < n4; j += 32) r4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            j0 = n4 << 2;
        }
        for (int j = j0 + lane; j < n_lambda; j += 32) row[j] = 0.f;
    }
}

int launch_zero_empty(const int* seg_off, int n_s, int nb, float* cube, int pitch, int n_lambda, cudaStream_t st) {
    if (n_s <= 0) return 0;
    long long nb_blocks = ((long long)n_s * 32 + 255) / 256;
    const long long cap = 16ll * sm_count();
    if (nb_blocks > cap) nb_blocks = cap;
    k_zero_empty<<<(int)nb_blocks, 256, 0, st>>>(seg_off, n_s, nb, cube, pitch, n_lambda);
    return 1;
}

// ----------------------------------------------------------------------------
// K5: rows of split spaxels = the sum of their partial rows in item order: a
// plain FP32 sum for spaxels of at most kCombineF32Rows items, a compensated
// FP32 sum above (very high-count spaxels). The compensated sum carries the
// rounding error of every addition (Knuth's two-sum: s + e is exactly the
// sum of s and x) in a second FP32 accumulator: the error before the final
// rounding stays within about n^2 2^-48 of the rows' magnitudes, far below
// one FP32 rounding, as with an FP64 accumulator, without the FP64 pipe,
// which on this GPU runs at 1/64 of the FP32 rate.
// ----------------------------------------------------------------------------

// The split spaxels, compacted (in any order: each row's sum is in item order,
// so the result does not depend on it); list[n_s] counts them.
__global__ void k_split_list(const int* __restrict__ part_off, int n_s, int* __restrict__ list) {
    const int lane = threadIdx.x & 31;
    for (int s0 = blockIdx.x * blockDim.x; s0 < n_s; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool split = s < n_s && part_off[s + 1] > part_off[s];
        const unsigned m = __ballot_sync(0xffffffffu, split);
        int at = 0;
        if (lane == 0 && m) at = atomicAdd(list + n_s, __popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (split) list[at + __popc(m & ((1u << lane) - 1u))] = s;
    }
}

constexpr int kCombineBins = 128;  // bins of one row per combine unit: 4 per lane of one warp

// One unit = kCombineBins bins of one split spaxel's row, taken by one warp
// (lane l sums bins l, l + 32, l + 64, l + 96 of the unit: four independent
// loads per partial row in flight), so that the rows of a very high-count
// spaxel are summed by many warps at once and each warp has several loads
// in flight while it waits on the next unit's row offsets.
__global__ void __launch_bounds__(256) k_combine(const int* __restrict__ part_off, int n_s, int n_lambda,
                                                 const int* __restrict__ list, const float* __restrict__ partials,
                                                 float* __restrict__ cube, int pitch) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n_split = list[n_s];
    const int n_chunks = (n_lambda + kCombineBins - 1) / kCombineBins;
    const long long n_units = (long long)n_split * n_chunks;
    for (long long u = warp; u < n_units; u += n_warps) {
        const int s = list[u / n_chunks];
        const int j0 = (int)(u % n_chunks) * kCombineBins + lane;
        const int p0 = part_off[s], nr = part_off[s + 1] - p0;
        const float* __restrict__ col = partials + (long long)p0 * n_lambda;
        float acc[4] = {0.f, 0.f, 0.f, 0.f}, err[4] = {0.f, 0.f, 0.f, 0.f};
        bool in[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) in[k] = j0 + 32 * k < n_lambda;
        if (nr <= kCombineF32Rows) {
            // a few partial rows: FP32 adds lose nothing that the FP32 partial
            // sums have not already lost
            for (int r = 0; r < nr; ++r)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (in[k]) acc[k] += col[(long long)r * n_lambda + j0 + 32 * k];
        } else {
#pragma unroll 2
            for (int r = 0; r < nr; ++r)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (in[k]) two_sum_add(acc[k], err[k], col[(long long)r * n_lambda + j0 + 32 * k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += err[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (in[k]) cube[(long long)s * pitch + j0 + 32 * k] = acc[k];
    }
}

int launch_combine(const int* part_off, int n_s, int n_lambda, const float* partials, float* cube, int pitch,
                   int* list, cudaStream_t st) {
    if (n_s < 1) return 0;
    cudaMemsetAsync(list + n_s, 0, sizeof(int), st);  // an error here is the caller's next cudaGetLastError
    long long nb = ((long long)n_s + 255) / 256;
    if (nb > 4ll * sm_count()) nb = 4ll * sm_count();
    k_split_list<<<(int)nb, 256, 0, st>>>(part_off, n_s, list);
    k_combine<<<8 * sm_count(), 256, 0, st>>>(part_off, n_s, n_lambda, list, partials, cube, pitch);
    return 2;
}

}  // namespace rubix
