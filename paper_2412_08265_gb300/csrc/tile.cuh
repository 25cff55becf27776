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
    const uint2* q16;  // 16-bit cell quads (qdt 1: BF16, 2: FP16); null: FP32 quads
    int qdt;
#if RUBIX_DEBUG
    unsigned* err;     // error word for the debug build's index checks
#endif
};

#if RUBIX_DEBUG
// Debug builds: the slab nodes the fast-path rounds of one particle will
// read, replayed with the rounds' own carry arithmetic (rounds of `step`
// bins; node K0 + o_r + lane for r < n_rounds, the last round read by lanes
// up to last_lanes only, plus the neighbours lo .. hi of each node) lie
// inside the slab.
__device__ __forceinline__ bool dbg_rounds_in_slab(int base, float f, float delta, const TileCtx& C, int lane,
                                                   int n_rounds, int step, int last_lanes, int lo, int hi) {
    const float d = (float)step * delta;
    const int n = C.slab_w * C.ncb;
    bool ok = true;
    int o = 0;
    for (int r = 0; r < n_rounds; ++r) {
        if (r < n_rounds - 1 || lane <= last_lanes) {
            ok = ok && base + (o + lane + lo) * C.ncb >= 0 && base + (o + lane + hi) * C.ncb < n;
        }
        f -= d;
        const bool carry = f < 0.f;
        f = carry ? f + 1.f : f;
        o += carry ? step - 1 : step;
    }
    return ok;
}
#endif

// The four corner templates of a 16-bit cell quad (x = corners 0 | 1 << 16,
// y = corners 2 | 3 << 16) as FP32 values (exact).
__device__ __forceinline__ float4 unpack_quad(const uint2 v, int qdt) {
    if (qdt == 1)
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u), __uint_as_float(v.y << 16),
                           __uint_as_float(v.y & 0xffff0000u));
    return make_float4(__half2float(__ushort_as_half((unsigned short)(v.x & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(v.x >> 16))),
                       __half2float(__ushort_as_half((unsigned short)(v.y & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(v.y >> 16))));
}

// Quad of `cell` at node k from the global quad array, FP32 or 16-bit (zero
// outside the template range: the template's zero extension).
__device__ __forceinline__ float4 quad_global(const float4* __restrict__ quad, const TileCtx& C, int cell, int k) {
    if (k < 0 || k >= C.n_ls) return make_float4(0.f, 0.f, 0.f, 0.f);
    const long long i = (long long)k * C.n_cells + cell;
    return C.qdt ? unpack_quad(__ldg(C.q16 + i), C.qdt) : __ldg(quad + i);
}

// Slab of a (tile, band) from 16-bit quads, by all threads of the CTA: node
// rows klo .. klo + slab_w of cells cell0 .. cell0 + ncb, converted to FP32
// (zero outside the template range and past the last cell, as TMA's fill
// does for FP32 quads). Thread i fills slab entries i, i + T, ... (T threads,
// entry e = row e / ncb, cell e % ncb): consecutive threads read consecutive
// cells of a node row and store consecutive 16-byte entries; kFill loads are
// in flight per thread before their stores. The caller synchronises the CTA
// afterwards.
__device__ __forceinline__ void fill_slab16(float4* __restrict__ slab, const TileCtx& C) {
    constexpr int kFill = 4;
    const int T = blockDim.x, total = C.slab_w * C.ncb;
    const int dr = T / C.ncb, dc = T - dr * C.ncb;
    int r = threadIdx.x / C.ncb, c = threadIdx.x - r * C.ncb;
    for (int e0 = threadIdx.x; e0 < total; e0 += kFill * T) {
        uint2 v[kFill];
        bool ok[kFill];
#pragma unroll
        for (int u = 0; u < kFill; ++u) {
            const int k = C.klo + r, cell = C.cell0 + c;
            ok[u] = e0 + u * T < total && k >= 0 && k < C.n_ls && cell < C.n_cells;
            v[u] = ok[u] ? __ldg(C.q16 + (long long)k * C.n_cells + cell) : make_uint2(0u, 0u);
            r += dr;
            c += dc;
            if (c >= C.ncb) {
                c -= C.ncb;
                ++r;
            }
        }
#pragma unroll
        for (int u = 0; u < kFill; ++u) {
            const int e = e0 + u * T;
            if (e < total) slab[e] = ok[u] ? unpack_quad(v[u], C.qdt) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
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
