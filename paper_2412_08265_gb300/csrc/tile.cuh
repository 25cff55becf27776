// tile.cuh -- device helpers shared by the deposit (K4) and the adjoint over
// the same (wavelength tile, work item, age band) decomposition: work-item
// search over the cost space, the bin -> SSP node map, and cell quads.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace rubix {

// First item index i in [0, n] with items[i].begin + c0 * i >= x (item n is
// the virtual end).
__device__ __forceinline__ long long item_lower_bound(const Item* __restrict__ items, long long n, long long c0,
                                                      long long x) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const long long pre = (long long)items[mid].begin + c0 * mid;
        if (pre < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Node position of output bin j: t(j) = K + phi, phi in [0, 1). j*a_hi is
// exact in FP32; only the small j*a_lo term is rounded.
__device__ __forceinline__ int node_pos(int j, int bi, float bf, float a_hi, float a_lo, float& phi) {
    const float jf = (float)j;
    const float pp = jf * a_hi;
    const float pi = floorf(pp);
    const float s = (pp - pi) + fmaf(jf, a_lo, bf);
    const float fl = floorf(s);
    phi = s - fl;
    return bi + (int)pi + (int)fl;
}

struct TileCtx {
    int j0, klo, slab_w, ncb, cell0, n_lambda, n_ls, n_cells;
};

// Quad of `cell` at node k from the global quad array (zero outside the
// template range: the template's zero extension).
__device__ __forceinline__ float4 quad_global(const float4* __restrict__ quad, int n_cells, int n_ls, int cell, int k) {
    return (k >= 0 && k < n_ls) ? __ldg(quad + (long long)k * n_cells + cell) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Mass-weighted bilinear template value at one node: sum_c w_c q_c.
__device__ __forceinline__ float quad_dot(const float4 w, const float4 q) {
    float2 p = __fmul2_rn(make_float2(w.x, w.y), make_float2(q.x, q.y));
    p = __ffma2_rn(make_float2(w.z, w.w), make_float2(q.z, q.w), p);
    return p.x + p.y;
}

// first index i in [0, n] with v[i] > x  (v non-decreasing)
__device__ __forceinline__ int upper_bound_ll(const long long* __restrict__ v, int n, long long x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace rubix
