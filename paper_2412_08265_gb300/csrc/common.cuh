// common.cuh -- internal helpers shared by the library's kernels (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rubix {

constexpr double kC_kms = 299792.458;

// Error word written by kernels (bit flags), read by the host after a forward.
enum DeviceError : unsigned {
    kErrTmaTimeout = 1u,      // a bounded mbarrier wait on a TMA slab load expired
    kErrBadItem = 2u,         // a work item pointed outside its buffers
    kErrBounds = 4u,          // debug builds: a computed index fell outside its buffer
};

// Debug builds (RUBIX_DEBUG=1, a separate library built by the tests) check
// the shared-memory and record indices the deposit and the adjoint compute
// against their buffers and set kErrBounds instead of faulting; release
// builds compile none of it.
#ifndef RUBIX_DEBUG
#define RUBIX_DEBUG 0
#endif
__device__ __forceinline__ void dbg_check(bool ok, unsigned* err) {
#if RUBIX_DEBUG
    if (!ok && err) atomicOr(err, kErrBounds);
#else
    (void)ok;
    (void)err;
#endif
}

// ----------------------------------------------------------------------------
// Shared-memory barrier and TMA (inline PTX, sm_90+ forms valid on sm_103a)
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait on phase `parity` of an mbarrier. Returns false if it did not
// complete within ~max_cycles SM clocks (the caller records an error and
// stops using the buffer instead of spinning forever).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long max_cycles) {
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > max_cycles) return false;
    }
}

// 2-D tiled TMA load of box (c0 = innermost coordinate, c1 = row) into smem.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_addr(smem_dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// 3-D tiled TMA load (c0 innermost).
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// 4-byte asynchronous global -> shared copy; with `valid` false the shared word
// is zero-filled and nothing is read.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc, bool valid) {
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(smem_dst)), "l"(gsrc), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
// published round function: two 32x32->64 multiplies per round with the
// multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 /
// 0xBB67AE85.
// ----------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 ctr, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * ctr.x;
        uint64_t p1 = (uint64_t)M1 * ctr.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        U4 n;
        n.x = hi1 ^ ctr.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ ctr.w ^ k1;
        n.w = lo0;
        ctr = n;
        k0 += W0;
        k1 += W1;
    }
    return ctr;
}

// ----------------------------------------------------------------------------
// SSP cell search: half-open cell [node_i, node_i+1) holding q, clamped outside
// the grid (t = 0 below the first node, t = 1 at or above the last); dt = dt/dq
// inside the grid, 0 when clamped. Shared by the key, setup and adjoint kernels
// so that they always agree on the cell of a particle.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void ssp_cell(float q, const float* __restrict__ nodes, int n, int& i, float& t,
                                         float& dt) {
    if (n < 2 || !(q > nodes[0])) { i = 0; t = 0.f; dt = 0.f; return; }
    if (q >= nodes[n - 1]) { i = n - 2; t = 1.f; dt = 0.f; return; }
    int lo = 0, hi = n - 1;  // nodes[lo] <= q < nodes[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (nodes[mid] <= q) lo = mid; else hi = mid;
    }
    i = lo;
    const float h = nodes[lo + 1] - nodes[lo];
    t = (q - nodes[lo]) / h;
    dt = 1.f / h;
}

// Age band of an age cell: the template grid is split into n_bands groups of
// `apb` age cells so that one band's templates fit a wide shared-memory slab.
__device__ __forceinline__ int age_band(int ia, int apb, int n_bands) {
    const int b = (apb > 0) ? ia / apb : 0;
    return b < n_bands - 1 ? b : n_bands - 1;
}

// ----------------------------------------------------------------------------
// Work descriptors
// ----------------------------------------------------------------------------
// Per in-field particle, in sorted order: everything the deposit needs (32 B).
// Spectrum value at output bin j:  sum_c w[c] * lerp(T_c, t(j)), with the
// fractional SSP node position t(j) = bi + bf + j*(a_hi + a_lo). a_hi keeps 11
// significant bits, so j*a_hi is exact in FP32 for j < 2^13 and only the small
// term j*a_lo is rounded.
struct __align__(16) DepRec {
    float w[4];        // mass * flux_scale * bilinear weights: (ia,iz) (ia+1,iz) (ia,iz+1) (ia+1,iz+1)
    int c0_bi;         // (SSP cell ia * max(n_Z - 1, 1) + iz) << 16 | (floor(t(0)) & 0xffff)
    float bf;          // t(0) - floor(t(0)), in [0, 1)
    float a_hi;        // dt/dj, high part
    float a_lo;        // dt/dj, low part
};
static_assert(sizeof(DepRec) == 32, "DepRec layout");

__device__ __forceinline__ int rec_c0(int c0_bi) { return (int)((unsigned)c0_bi >> 16); }
__device__ __forceinline__ int rec_bi(int c0_bi) { return (c0_bi << 16) >> 16; }

// Per in-field particle, sorted order: the inputs of its spectrum, kept for backward.
struct __align__(16) PartRec {
    float mass, age, Z, v;
};

// One unit of deposit work: particles [begin, end) of spaxel `spaxel`,
// written to the cube row (part_row < 0) or to partial row `part_row`.
struct __align__(16) Item {
    int spaxel;
    int begin;
    int end;
    int part_row;
};

}  // namespace rubix
