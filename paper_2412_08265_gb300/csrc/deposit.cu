// deposit.cu -- SSP lookup, Doppler shift, resampling and per-spaxel sum
// (Sec. 3: every star's spectrum is taken from an SSP library by age and
// metallicity, shifted by its line-of-sight velocity, resampled onto the
// instrument's wavelength grid and added to the spaxel it falls in).
//
// K3 (k_setup, setup.cu) has turned each in-field particle, in sorted order,
// into a 32-byte record: its four mass-scaled bilinear corner weights, its
// SSP cell (the (ia, iz) cell whose four corner templates it interpolates)
// and the affine map t(j) = B + jA from output bin j to the fractional SSP
// node position.
//
// The templates are kept, for the deposit, as cell quads: for SSP cell c and
// node k, its four corner templates at k, stored node-major ([node][cell]) so
// that one 2-D TMA box holds a run of consecutive cells (an age band) over a
// run of nodes (FP32 quads; 16-bit quads are widened into the slab by the
// CTA's threads).
//
// K4 (k_deposit) is persistent: each CTA owns a contiguous, cost-balanced range
// of (wavelength tile, work item) pairs, a work item being <= chunk particles
// of one spaxel. For each tile and age band the CTA stages the band's quads
// over the tile's node range plus a Doppler halo in shared memory with TMA
// (TMA's zero fill outside the SSP range is the template's zero extension),
// and its warps accumulate whole items in registers in a fixed particle
// order. Particles are sorted by (spaxel, age band), so for band b each
// item's band-b particles are contiguous; band 0 writes the item's row and
// later bands add to it, in band order.
//
// Inner loop (one warp per particle, R rounds of 31 consecutive bins; lane l
// owns bin j0 + 31 r + l): with dt/dj = A in (1 - 1/31, 1] and the round's
// first bin at node position K0 + phi0, bin l sits at K0 + l + g with
// g = phi0 - l (1 - A) in (-1, 1). Lane l reads the quad at node K0 + l (one
// 16-byte shared load; an odd number of cells per node keeps the warp's 32
// loads free of bank conflicts), forms the mass-weighted template
// M = sum_c W_c T_c[K0 + l], and takes the neighbouring node's M from lane
// l - 1 or l + 1 with one shuffle; the bin value is M + |g| (M_neighbour - M).
// Lane 31 only supplies node K0 + 31. Other dt/dj, or Doppler shifts beyond
// the slab's halo, take a per-bin path.
//
// Spaxels with more than `chunk` particles are split into several items whose
// FP32 partial rows K5 (rows.cu) adds in item order, so the cube is bitwise
// reproducible. Each later age band continues the row the earlier bands left:
// the warp that owns the item in that band loads the row segment into its
// accumulators before its particles and stores it back after them (plain
// loads and stores, no atomics; one owner per row and band, bands separated
// by the CTA barrier, so the order of every addition is fixed).
#include "common.cuh"
#include "kernels.h"
#include "tile.cuh"

namespace rubix {

// ----------------------------------------------------------------------------
// K4: deposit.
// ----------------------------------------------------------------------------
// Shared memory: kDepHeader bytes (mbarrier, counters, job work table), then
// the slab: slab_w nodes x ncb cells of quads, node-major (quad of cell c at
// node k at slab[(k - klo) * ncb + c - cell0]). ncb is odd, so the 16-byte
// quads that 32 lanes read at consecutive nodes fall in distinct bank groups.

size_t deposit_smem_bytes(int ncb, int slab_w) { return kDepHeader + (size_t)ncb * slab_w * sizeof(float4); }

// Per-bin evaluation for the general path: does bin j's node pair lie in the slab?
__device__ __noinline__ bool bin_in_slab(const float4 g4, const TileCtx C, int j, int lane) {
    if (lane == 31 || j >= C.n_lambda) return true;
    const int c0_bi = __float_as_int(g4.x);
    if ((unsigned)(rec_c0(c0_bi) - C.cell0) >= (unsigned)C.ncb) return false;
    float f;
    const int k = node_pos(j, rec_bi(c0_bi), g4.y, g4.z, g4.w, f) - C.klo;
    return k >= 0 && k + 1 < C.slab_w;
}

// Spectrum value of one particle at bin j (0 for lane 31 and bins past the end),
// quads from the slab or, with use_slab false, from global memory.
__device__ __noinline__ float bin_value(const float4 w4, const float4 g4, const TileCtx C, int j, int lane,
                                        bool use_slab, const float4* __restrict__ slab,
                                        const float4* __restrict__ quad) {
    if (lane == 31 || j >= C.n_lambda) return 0.f;
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi);
    float f;
    const int k = node_pos(j, rec_bi(c0_bi), g4.y, g4.z, g4.w, f);
    float4 q0, q1;
    if (use_slab) {
        const int e = (k - C.klo) * C.ncb + (cell - C.cell0);
#if RUBIX_DEBUG
        dbg_check(e >= 0 && e + C.ncb < C.slab_w * C.ncb, C.err);
#endif
        const float4* p = slab + e;
        q0 = p[0];
        q1 = p[C.ncb];
    } else {
        q0 = quad_global(quad, C, cell, k);
        q1 = quad_global(quad, C, cell, k + 1);
    }
    const float m0 = quad_dot(w4, q0), m1 = quad_dot(w4, q1);
    return fmaf(f, m1 - m0, m0);
}

// The rounds of one particle on the fast path: q = its slab quad at node
// K0 + lane, f = frac(t(j0)), delta = 1 - dt/dj. acc[r] of lane l (l < 31) is
// output bin j0 + 31 r + l.
template <int R>
__device__ __forceinline__ void fast_rounds(const float4 w4, const float4* __restrict__ q, float f, float delta,
                                            int ncb, int lane, float lanef, float (&acc)[R]) {
    // round r: lane l reads node K0 + o_r + l, o_r = 31 r - (carries so far)
    const int s31 = 31 * ncb, s30 = 30 * ncb;
    const float nld = -lanef * delta;
    const float d31 = 31.f * delta;
    // rounds two at a time: the per-bin arithmetic in packed FP32x2
#pragma unroll
    for (int r = 0; r + 1 < R; r += 2) {
        const float4 Qa = *q;
        const float fa = f;
        f -= d31;
        bool carry = f < 0.f;
        f = carry ? f + 1.f : f;
        q += carry ? s30 : s31;
        const float4 Qb = *q;
        const float fb = f;
        f -= d31;
        carry = f < 0.f;
        f = carry ? f + 1.f : f;
        q += carry ? s30 : s31;
        const float Ma = quad_dot(w4, Qa), Mb = quad_dot(w4, Qb);
        // bin j0 + 31 r + l sits at node K0 + o_r + l + g, g = f - l delta in
        // (-1, 1); the neighbour node on g's side is lane l -+ 1's:
        // value = M + |g| (M_neighbour - M)
        const float2 g = __fadd2_rn(make_float2(fa, fb), make_float2(nld, nld));
        const float Xa = __shfl_sync(0xffffffffu, Ma, g.x < 0.f ? lane - 1 : lane + 1);
        const float Xb = __shfl_sync(0xffffffffu, Mb, g.y < 0.f ? lane - 1 : lane + 1);
        const float2 D = __fadd2_rn(make_float2(Xa, Xb), make_float2(-Ma, -Mb));
        const float2 v = __ffma2_rn(make_float2(fabsf(g.x), fabsf(g.y)), D, make_float2(Ma, Mb));
        const float2 a = __fadd2_rn(make_float2(acc[r], acc[r + 1]), v);
        acc[r] = a.x;
        acc[r + 1] = a.y;
    }
    if (R & 1) {
        const float M = quad_dot(w4, *q);
        const float g = f + nld;
        const float X = __shfl_sync(0xffffffffu, M, g < 0.f ? lane - 1 : lane + 1);
        acc[R - 1] += fmaf(fabsf(g), X - M, M);
    }
}

// General path (out of line; rare on the workloads here): each bin's node
// pair from the slab if every bin of the warp is inside it, else from the
// global quad array.
template <int R>
__device__ __forceinline__ void general_particle(const float4 w4, const float4 g4, const TileCtx& C,
                                                 const float4* __restrict__ slab, const float4* __restrict__ quad,
                                                 int lane, float (&acc)[R], unsigned long long* slow_count) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < R; ++i) ok = ok && bin_in_slab(g4, C, C.j0 + 31 * i + lane, lane);
    const bool use_slab = C.slab_w > 0 && __all_sync(0xffffffffu, ok);
    if (!use_slab && lane == 0 && slow_count) atomicAdd(slow_count, 1ull);
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] += bin_value(w4, g4, C, C.j0 + 31 * i + lane, lane, use_slab, slab, quad);
}

// Fast-path setup of one particle for this tile and band: the slab offset of
// its cell at node K0 (without the lane), frac(t(j0)) and 1 - dt/dj; false
// if it takes the general path (dt/dj outside (1 - 1/31, 1], a cell of
// another band, or a node of the rounds, K0 .. K0 + 31 R + EXTRA, outside the
// slab).
template <int R, int EXTRA = 0>
__device__ __forceinline__ bool fast_setup(const float4 g4, const TileCtx& C, int& base, float& f, float& delta) {
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi), bi = rec_bi(c0_bi);
    const int K0 = node_pos(C.j0, bi, g4.y, g4.z, g4.w, f);  // node position of the tile's first bin
    delta = (1.f - g4.z) - g4.w;                             // 1 - dt/dj (exact up to one rounding)
    const int kw = K0 - C.klo;
    const int cr = cell - C.cell0;
    base = kw * C.ncb + cr;
    return delta >= 0.f && delta * 31.f < 1.f && (unsigned)kw < (unsigned)(C.slab_w - 31 * R - EXTRA) &&
           (unsigned)cr < (unsigned)C.ncb;
}

// Adds one particle's spectrum to acc (setup by every lane; warp-uniform path).
template <int R>
__device__ __forceinline__ void deposit_particle(const float4 w4, const float4 g4, const TileCtx& C,
                                                 const float4* __restrict__ slab, const float4* __restrict__ quad,
                                                 int lane, float lanef, float (&acc)[R],
                                                 unsigned long long* slow_count) {
    int base;
    float f, delta;
    if (fast_setup<R>(g4, C, base, f, delta)) {
#if RUBIX_DEBUG
        dbg_check(dbg_rounds_in_slab(base, f, delta, C, lane, R, 31, 31, 0, 0), C.err);
#endif
        fast_rounds<R>(w4, slab + base + lane * C.ncb, f, delta, C.ncb, lane, lanef, acc);
    } else
        general_particle<R>(w4, g4, C, slab, quad, lane, acc, slow_count);
}

// ----------------------------------------------------------------------------
// Bin means (flux-conserving resampling). The record maps j to bin j's lower
// edge e_j = t(j) - A/2 (node units); bin j's value is the mean of the
// weighted template's linear interpolant M(t) over [e_j, e_{j+1}].
//
// Fast path (dt/dj = A = 1 - delta in (1 - 1/31, 1]): rounds of 30 bins.
// Lane l of a round owns edge l, at node K0 + l + g with g = f - l delta in
// (-1, 1), and bin l (l < 30) between edges l and l + 1. As in the centre
// path, lane l reads node K0 + l's quad, forms M there and takes the
// neighbouring node's M from lane l -+ 1, which gives the interpolant at its
// edge, L_l. The interval of bin l holds at most one node,
// K = K0 + l + (g >= 0), whose M is that neighbour's or the lane's own; with
// a the distance from edge l to K and b = A - a, the trapezoids on both sides
// of K give
//   mean = M_K / 2 + (a L_l + b L_{l+1}) / (2A),
// which also holds with no node inside (b < 0: the three points lie on one
// line). L_{l+1} is one more shuffle. A tile of 31 R bins is R rounds of 30
// bins and a last round of R bins, whose lanes above R + 1 read nothing: the
// rounds read nodes K0 .. K0 + 31 R + 1.
// ----------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void mean_rounds(const float4 w4, const float4* __restrict__ q, float f, float delta,
                                            int ncb, int lane, float lanef, float (&acc)[R + 1]) {
    // with the weights halved (M' = M/2, L' = L/2), and a L + b L_{l+1} =
    // a (L - L_{l+1}) + A L_{l+1}, the mean is M'_K + L'_{l+1} + (a/A)(L' - L'_{l+1})
    const float4 wh = make_float4(0.5f * w4.x, 0.5f * w4.y, 0.5f * w4.z, 0.5f * w4.w);
    const int s30 = 30 * ncb, s29 = 29 * ncb;
    const float nld = -lanef * delta;
    const float d30 = 30.f * delta;
    const float iA = 1.f / (1.f - delta);
    const int lp = lane + 1, lm = lane - 1;
    // rounds two at a time: the per-bin arithmetic in packed FP32x2
#pragma unroll
    for (int r = 0; r + 1 <= R; r += 2) {
        float4 Qa = *q;
        const float fa = f;
        f -= d30;
        bool carry = f < 0.f;
        f = carry ? f + 1.f : f;
        q += carry ? s29 : s30;
        float4 Qb = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r + 1 < R || lane <= R + 1) Qb = *q;
        const float fb = f;
        if (r + 2 <= R) {
            f -= d30;
            carry = f < 0.f;
            f = carry ? f + 1.f : f;
            q += carry ? s29 : s30;
        }
        const float2 M = make_float2(quad_dot(wh, Qa), quad_dot(wh, Qb));
        const float2 g = __fadd2_rn(make_float2(fa, fb), make_float2(nld, nld));
        const bool ua = g.x >= 0.f, ub = g.y >= 0.f;
        const float2 X = make_float2(__shfl_sync(0xffffffffu, M.x, ua ? lp : lm),
                                     __shfl_sync(0xffffffffu, M.y, ub ? lp : lm));
        const float2 L = __ffma2_rn(make_float2(fabsf(g.x), fabsf(g.y)), __fadd2_rn(X, make_float2(-M.x, -M.y)), M);
        const float2 Ln = make_float2(__shfl_down_sync(0xffffffffu, L.x, 1), __shfl_down_sync(0xffffffffu, L.y, 1));
        const float2 MK = make_float2(ua ? X.x : M.x, ub ? X.y : M.y);
        const float2 ai = __ffma2_rn(make_float2(-g.x, -g.y), make_float2(iA, iA),
                                     make_float2(ua ? iA : 0.f, ub ? iA : 0.f));
        const float2 v = __ffma2_rn(ai, __fadd2_rn(L, make_float2(-Ln.x, -Ln.y)), __fadd2_rn(MK, Ln));
        const float2 a = __fadd2_rn(make_float2(acc[r], acc[r + 1]), v);
        acc[r] = a.x;
        acc[r + 1] = a.y;
    }
    if (!(R & 1)) {
        // R + 1 rounds, odd: the last round (R bins) alone
        float4 Q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane <= R + 1) Q = *q;
        const float M = quad_dot(wh, Q);
        const float g = f + nld;
        const bool up = g >= 0.f;
        const float X = __shfl_sync(0xffffffffu, M, up ? lp : lm);
        const float L = fmaf(fabsf(g), X - M, M);
        const float Ln = __shfl_down_sync(0xffffffffu, L, 1);
        const float ai = fmaf(-g, iA, up ? iA : 0.f);
        acc[R] += fmaf(ai, L - Ln, (up ? X : M) + Ln);
    }
}

// General path of the bin means: bin j (owned = a bin of this tile held by
// this lane) integrates M segment by segment over [e_j, e_{j+1}], nodes from
// the slab or, with use_slab false, from global memory.
__device__ __noinline__ bool mean_in_slab(const float4 g4, const TileCtx C, int j, bool owned) {
    if (!owned || j >= C.n_lambda) return true;
    const int c0_bi = __float_as_int(g4.x);
    if ((unsigned)(rec_c0(c0_bi) - C.cell0) >= (unsigned)C.ncb) return false;
    float fa, fb;
    const int ka = node_pos(j, rec_bi(c0_bi), g4.y, g4.z, g4.w, fa) - C.klo;
    const int kb = node_pos(j + 1, rec_bi(c0_bi), g4.y, g4.z, g4.w, fb) - C.klo;
    return ka >= 0 && kb + 1 < C.slab_w;
}

__device__ __noinline__ float mean_value(const float4 w4, const float4 g4, const TileCtx C, int j, bool owned,
                                         bool use_slab, const float4* __restrict__ slab,
                                         const float4* __restrict__ quad) {
    if (!owned || j >= C.n_lambda) return 0.f;
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi);
    float fa, fb;
    const int ka = node_pos(j, rec_bi(c0_bi), g4.y, g4.z, g4.w, fa);
    const int kb = node_pos(j + 1, rec_bi(c0_bi), g4.y, g4.z, g4.w, fb);
    auto node = [&](int k) {
#if RUBIX_DEBUG
        if (use_slab)
            dbg_check((unsigned)((k - C.klo) * C.ncb + (cell - C.cell0)) < (unsigned)(C.slab_w * C.ncb), C.err);
#endif
        const float4 q = use_slab ? slab[(k - C.klo) * C.ncb + (cell - C.cell0)]
                                  : quad_global(quad, C, cell, k);
        return quad_dot(w4, q);
    };
    // segments [k, k + 1] outside [-1, n_ls] are zero
    const int k_first = max(ka, -1), k_last = min(kb, C.n_ls - 1);
    float s = 0.f;
    float m0 = node(k_first);
    for (int k = k_first; k <= k_last; ++k) {
        const float m1 = node(k + 1);
        const float u0 = (k == ka) ? fa : 0.f, u1 = (k == kb) ? fb : 1.f;
        s = fmaf(u1 - u0, fmaf(m1 - m0, 0.5f * (u0 + u1), m0), s);
        m0 = m1;
    }
    const float len = (float)(kb - ka) + (fb - fa);
    if (len > 0.f) return s / len;
    const float ma = node(ka);  // a bin narrower than FP32 resolves: the edge value
    return fmaf(fa, node(ka + 1) - ma, ma);
}

template <int R>
__device__ __forceinline__ void mean_general_particle(const float4 w4, const float4 g4, const TileCtx& C,
                                                      const float4* __restrict__ slab,
                                                      const float4* __restrict__ quad, int lane,
                                                      float (&acc)[R + 1], unsigned long long* slow_count) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i <= R; ++i) ok = ok && mean_in_slab(g4, C, C.j0 + 30 * i + lane, lane < (i < R ? 30 : R));
    const bool use_slab = C.slab_w > 0 && __all_sync(0xffffffffu, ok);
    if (!use_slab && lane == 0 && slow_count) atomicAdd(slow_count, 1ull);
#pragma unroll
    for (int i = 0; i <= R; ++i)
        acc[i] += mean_value(w4, g4, C, C.j0 + 30 * i + lane, lane < (i < R ? 30 : R), use_slab, slab, quad);
}

template <int R>
__device__ __forceinline__ void mean_particle(const float4 w4, const float4 g4, const TileCtx& C,
                                              const float4* __restrict__ slab, const float4* __restrict__ quad,
                                              int lane, float lanef, float (&acc)[R + 1],
                                              unsigned long long* slow_count) {
    int base;
    float f, delta;
    if (fast_setup<R, 1>(g4, C, base, f, delta)) {
#if RUBIX_DEBUG
        dbg_check(dbg_rounds_in_slab(base, f, delta, C, lane, R + 1, 30, R + 1, 0, 0), C.err);
#endif
        mean_rounds<R>(w4, slab + base + lane * C.ncb, f, delta, C.ncb, lane, lanef, acc);
    } else
        mean_general_particle<R>(w4, g4, C, slab, quad, lane, acc, slow_count);
}

// Per-tile cost of each job (in-field particles + cost_c0 per work item) and
// its exclusive prefix, read from the device-side counts of every job.
__global__ void k_job_cost(const DepositParams P, long long* job_cost) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    long long acc = 0;
    for (int j = 0; j < P.n_jobs; ++j) {
        const DepJob& J = P.jobs[j];
        job_cost[j] = acc;
        const long long n_in = J.seg_off[(long long)J.n_s * P.n_bands];
        const long long n_items = J.item_off[J.n_s];
        acc += n_in + (long long)P.cost_c0 * n_items;
    }
    job_cost[P.n_jobs] = acc;
}

constexpr int kJobChunk = 32;  // jobs per shared-memory work table

// One work item's particles [q0, q1) of the current band, accumulated in
// registers in sorted order onto the item's row dst (zero for band 0, the
// earlier bands' sum for later bands), then stored. MEAN: bin means (rounds
// of 30 bins, R + 1 of them), else centre samples (R rounds of 31).
template <int R, bool MEAN>
__device__ __forceinline__ void deposit_item(const DepositParams& P, const TileCtx& C, const float4* __restrict__ rec4,
                                             int q0, int q1, float* dst, int band, const float4* __restrict__ slab,
                                             int lane, float lanef) {
    constexpr int NR = MEAN ? R + 1 : R;
    float acc[NR];
    // band 0 starts the row from zero; later bands continue the row the
    // earlier bands left (loaded now, in flight while the first particle's
    // record and setup are prepared), so the row is written back with plain
    // stores and no atomics
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int j = MEAN ? C.j0 + 30 * r + lane : C.j0 + 31 * r + lane;
        const bool owned = MEAN ? lane < (r < R ? 30 : R) : lane < 31;
        acc[r] = (band > 0 && owned && j < P.n_lambda) ? dst[j] : 0.f;
    }
    // the next particle's record is pulled into L1 while the current one is
    // deposited (no registers held across the particle)
    if (q0 < q1) asm volatile("prefetch.global.L1 [%0];" ::"l"(rec4 + 2 * q0));
    for (int q = q0; q < q1; ++q) {
        if (q + 1 < q1) asm volatile("prefetch.global.L1 [%0];" ::"l"(rec4 + 2 * (q + 1)));
        const float4 w4 = rec4[2 * q], g4 = rec4[2 * q + 1];
        if constexpr (MEAN)
            mean_particle<R>(w4, g4, C, slab, P.quad, lane, lanef, acc, P.slow_count);
        else
            deposit_particle<R>(w4, g4, C, slab, P.quad, lane, lanef, acc, P.slow_count);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int j = MEAN ? C.j0 + 30 * r + lane : C.j0 + 31 * r + lane;
        const bool owned = MEAN ? lane < (r < R ? 30 : R) : lane < 31;
        if (owned && j < P.n_lambda) dst[j] = acc[r];
    }
}

template <int R, bool MEANS>
__global__ void __launch_bounds__(RUBIX_DEP_THREADS, RUBIX_DEP_CTAS) k_deposit(const __grid_constant__ DepositParams P,
                                                                   const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* s_next = reinterpret_cast<int*>(smem + 16);
    int* s_nv = reinterpret_cast<int*>(smem + 20);         // work items in the current table
    int* s_job = reinterpret_cast<int*>(smem + 64);        // [kJobChunk] job of table row k
    int* s_ia = s_job + kJobChunk;                         // [kJobChunk] its first item
    int* s_pre = s_ia + kJobChunk;                         // [kJobChunk + 1] prefix of item counts
    float4* slab = reinterpret_cast<float4*>(smem + kDepHeader);

    const int lane = threadIdx.x & 31;
    const float lanef = (float)lane;
    const int nb = P.n_bands;
    const long long* __restrict__ jc = P.job_cost;
    const long long C0 = P.cost_c0;
    const long long CT = jc[P.n_jobs];
    if (CT <= 0) return;
    const long long total = CT * P.n_tiles;
    const long long lo = total * blockIdx.x / gridDim.x;
    const long long hi = total * (blockIdx.x + 1) / gridDim.x;
    if (lo >= hi) return;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    TileCtx C;
    C.slab_w = P.slab_w;
    C.ncb = P.ncb;
    C.n_lambda = P.n_lambda;
    C.n_ls = P.n_ls;
    C.n_cells = P.n_cells;
    C.q16 = P.quad16;
    C.qdt = P.qdt;
#if RUBIX_DEBUG
    C.err = P.err;
#endif
    const uint32_t slab_bytes = (uint32_t)P.n_boxes * (uint32_t)P.box_w * (uint32_t)P.ncb * sizeof(float4);
    uint32_t phase = 0;

    for (long long t = lo / CT; t < P.n_tiles && t * CT < hi; ++t) {
        const long long a = max(lo - t * CT, 0ll), b = min(hi - t * CT, CT);
        if (a >= b) continue;
        // jobs overlapping the CTA's cost range [a, b) of this tile
        const int ja = upper_bound_ll(jc, P.n_jobs + 1, a) - 1;
        const int jb = min(upper_bound_ll(jc, P.n_jobs + 1, b - 1), P.n_jobs);
        C.klo = P.tile_klo[t];
        C.j0 = (int)t * P.tile_w;

      for (int cj = ja; cj < jb; cj += kJobChunk) {
        __syncthreads();  // every warp is done with the previous table
        if (threadIdx.x == 0) {
            int nv = 0, k = 0;
            s_pre[0] = 0;
            for (int j = cj; j < min(jb, cj + kJobChunk); ++j, ++k) {
                const DepJob& J = P.jobs[j];
                const long long ctj = jc[j + 1] - jc[j];
                const long long aj = max(a - jc[j], 0ll), bj = min(b - jc[j], ctj);
                const long long n_items = J.item_off[J.n_s];
                const int ia = (int)item_lower_bound(J.items, n_items, C0, aj);
                const int ib = (int)item_lower_bound(J.items, n_items, C0, bj);
                s_job[k] = j;
                s_ia[k] = ia;
                nv += max(ib - ia, 0);
                s_pre[k + 1] = nv;
            }
            for (; k < kJobChunk; ++k) s_pre[k + 1] = nv;
            *s_nv = nv;
        }

        for (int band = 0; band < nb; ++band) {
            C.cell0 = P.band_cell0[band];
            __syncthreads();  // all warps are done with the previous slab and rows
            if (threadIdx.x == 0) {
                *s_next = 0;
                if (C.slab_w > 0 && !C.qdt) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bar, slab_bytes);
                    for (int bx = 0; bx < P.n_boxes; ++bx)
                        tma_load_2d(slab + (size_t)bx * P.box_w * C.ncb, &tmap, bar, 4 * C.cell0,
                                    C.klo + bx * P.box_w);
                }
            }
            bool ok = true;
            if (C.slab_w > 0 && !C.qdt) {
                ok = mbar_wait_bounded(bar, phase, 4000000000ll);
                phase ^= 1u;
            } else if (C.slab_w > 0) {
                // 16-bit templates: every thread converts part of the slab
                fill_slab16(slab, C);
            }
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(P.err, kErrTmaTimeout);
                return;
            }

            const int nv = *s_nv;
            constexpr int G = RUBIX_DEP_GRAB;
            while (true) {
                int v0 = 0;
                if (lane == 0) v0 = atomicAdd(s_next, G);
                v0 = __shfl_sync(0xffffffffu, v0, 0);
                if (v0 >= nv) break;
                // lanes < G look up one work item each and its band segment
                int kk = 0, qb = 0, qe = 0, sp = 0, prow = -1;
                bool live = false;
                const int v = v0 + lane;
                if (lane < G && v < nv) {
                    while (s_pre[kk + 1] <= v) ++kk;  // table row holding work item v
                    const DepJob& J = P.jobs[s_job[kk]];
                    const Item I = J.items[s_ia[kk] + (v - s_pre[kk])];
                    sp = I.spaxel;
                    prow = I.part_row;
                    qb = I.begin;
                    qe = I.end;
                    if (prow >= J.part_cap || sp < 0 || sp >= J.n_s) {
                        atomicOr(P.err, kErrBadItem);
                    } else {
                        if (nb > 1) {
                            qb = max(qb, J.seg_off[(long long)sp * nb + band]);
                            qe = min(qe, J.seg_off[(long long)sp * nb + band + 1]);
                        }
                        // band 0 visits every item: it writes the row, zeros included
                        live = band == 0 || qb < qe;
                        // the item's first record, on its way to L1 before the warp reaches it
                        if (qb < qe)
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const float4*>(J.rec) + 2 * qb));
                    }
                }
                unsigned m = __ballot_sync(0xffffffffu, live);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const int k = __shfl_sync(0xffffffffu, kk, src);
                    const int q0 = __shfl_sync(0xffffffffu, qb, src);
                    const int q1 = __shfl_sync(0xffffffffu, qe, src);
                    const int s = __shfl_sync(0xffffffffu, sp, src);
                    const int pr = __shfl_sync(0xffffffffu, prow, src);
                    const DepJob& J = P.jobs[s_job[k]];
                    const float4* __restrict__ rec4 = reinterpret_cast<const float4*>(J.rec);
                    float* dst = (pr < 0) ? J.cube + (long long)s * J.pitch
                                          : J.partials + (long long)pr * P.n_lambda;
                    if (MEANS && J.resample)
                        deposit_item<R, true>(P, C, rec4, q0, q1, dst, band, slab, lane, lanef);
                    else
                        deposit_item<R, false>(P, C, rec4, q0, q1, dst, band, slab, lane, lanef);
                }
            }
        }
      }
    }
}

int launch_deposit(const DepositParams& P, const CUtensorMap* tmap, int n_ctas, int threads, size_t smem,
                   cudaStream_t st) {
    if (P.tile_w % 31 != 0) return -1;
    bool means = false;
    for (int j = 0; j < P.n_jobs && j < kMaxJobs; ++j) means = means || P.jobs[j].resample;
    void (*fn)(const DepositParams, const CUtensorMap) = nullptr;
    switch (P.tile_w / 31) {
#define RUBIX_DEP_R(r) \
    case r: fn = means ? k_deposit<r, true> : k_deposit<r, false>; break;
        RUBIX_DEP_R(1) RUBIX_DEP_R(2) RUBIX_DEP_R(3) RUBIX_DEP_R(4) RUBIX_DEP_R(5) RUBIX_DEP_R(6)
        RUBIX_DEP_R(7) RUBIX_DEP_R(8) RUBIX_DEP_R(9) RUBIX_DEP_R(10) RUBIX_DEP_R(11) RUBIX_DEP_R(12)
#if RUBIX_DEP_RMAX > 12
        RUBIX_DEP_R(13) RUBIX_DEP_R(14) RUBIX_DEP_R(15) RUBIX_DEP_R(16) RUBIX_DEP_R(17) RUBIX_DEP_R(18)
        RUBIX_DEP_R(19) RUBIX_DEP_R(20) RUBIX_DEP_R(21) RUBIX_DEP_R(22) RUBIX_DEP_R(23) RUBIX_DEP_R(24)
#endif
#undef RUBIX_DEP_R
        default: return -1;
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    if (P.n_jobs < 1 || P.n_jobs > kMaxJobs) return -1;
    k_job_cost<<<1, 32, 0, st>>>(P, P.job_cost);
    fn<<<n_ctas, threads, smem, st>>>(P, *tmap);
    return 2;  // job-cost prep + deposit
}

}  // namespace rubix
