// adjoint_tiles.cu -- the adjoint of the deposit (gradients through the
// pipeline, Abstract and Sec. 1) over the deposit's own decomposition.
//
// For particle p with unit-mass bilinear weights W_c(ta, tz), the spectrum at
// bin j is S_j = sum_c W_c lerp(T_c, t_j) and the loss sees it through
// G_j = dL/dcube0[s_p, j]. The gradient needs, per particle,
//   sm  = sum_j G_j S_j                      (dL/dm = flux_scale * sm)
//   sla = sum_j G_j dS_j/dta                 (chain rule to age outside)
//   slz = sum_j G_j dS_j/dtz                 (to Z outside)
//   sv  = sum_j G_j dS_j/dt * (t_j + ls0/dls) (times dt/dv / t_abs outside)
// dS/dta and dS/dtz are bilinear forms in the same four corners with weights
// a = (-(1-tz), 1-tz, -tz, tz) and b = (-(1-ta), -ta, 1-ta, ta). All three
// forms are linear in the corner templates, so the lanes accumulate per
// corner (G_j times the interpolated corner template, and G_j times the
// corner's slope times the bin position) and apply w, a and b once per
// particle and tile. The deposit's (tile, work item, age band) partition,
// quad slabs and 31-bin rounds carry over unchanged: lane l reads the quad at
// node K0 + o_r + l and the neighbouring node's quad from the slab. A warp
// reduction per (particle, tile) gives part[tile][particle]; K8 adds the
// tiles in tile order with a compensated FP32 sum.
#include "common.cuh"
#include "kernels.h"
#include "tile.cuh"
#include "twosum.cuh"

namespace rubix {

// ---------------------------------------------------------------------------
// Setup: unit-mass weights per sorted particle (zero when the spectrum misses
// every output bin, as in the forward).
// ---------------------------------------------------------------------------
__global__ void k_adj_setup(const AdjointParams P, const DepRec* __restrict__ rec, float4* __restrict__ wu) {
    const long long n_in = P.seg_off[(long long)P.n_s * P.n_bands];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_in;
         i += (long long)gridDim.x * blockDim.x) {
        const PartRec pr = P.prec[i];
        int ia, iz;
        float ta, tz, dta, dtz;
        ssp_cell(log10f(pr.age), P.ssp.la_nodes, P.ssp.n_age, ia, ta, dta);
        ssp_cell(log10f(pr.Z), P.ssp.lz_nodes, P.ssp.n_Z, iz, tz, dtz);
        const bool live = rec[i].a_hi > 0.f;
        wu[i] = live ? make_float4((1.f - ta) * (1.f - tz), ta * (1.f - tz), (1.f - ta) * tz, ta * tz)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

int launch_adjoint_setup(const AdjointParams& P, const DepRec* rec, float4* wu, cudaStream_t st) {
    if (P.n_in <= 0) return 0;
    long long nb = (P.n_in + 255) / 256;
    if (nb > 16ll * sm_count()) nb = 16ll * sm_count();
    k_adj_setup<<<(int)nb, 256, 0, st>>>(P, rec, wu);
    return 1;
}

// ---------------------------------------------------------------------------
// Per (particle, tile) sums.
// ---------------------------------------------------------------------------
struct AdjSums {
    float sm, sa, sz, sv;
};

// General path: bins of this tile one at a time, quads from the slab when
// every bin of the warp has its node pair there, else from global memory.
// It reads dL/dcube0 from the spaxel's row (grow) itself, so that the fast
// path's register copy never has to be kept in memory for this call.
template <int R>
__device__ __noinline__ AdjSums adj_general(const float4 w, const float4 g4, const TileCtx C, const float4* slab,
                                            const float4* quad, int lane, const float* __restrict__ grow,
                                            float ls0_over) {
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi), bi = rec_bi(c0_bi);
    bool ok = C.slab_w > 0 && (unsigned)(cell - C.cell0) < (unsigned)C.ncb;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = C.j0 + 31 * r + lane;
        if (lane < 31 && j < C.n_lambda) {
            float f;
            const int k = node_pos(j, bi, g4.y, g4.z, g4.w, f) - C.klo;
            ok = ok && k >= 0 && k + 1 < C.slab_w;
        }
    }
    const bool use_slab = __all_sync(0xffffffffu, ok);
    const float s01 = w.x + w.y, s23 = w.z + w.w, s02 = w.x + w.z, s13 = w.y + w.w;
    AdjSums S{0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = C.j0 + 31 * r + lane;
        if (lane == 31 || j >= C.n_lambda) continue;
        float f;
        const int k = node_pos(j, bi, g4.y, g4.z, g4.w, f);
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
        const float m0 = quad_dot(w, q0), m1 = quad_dot(w, q1);
        const float a0 = s01 * (q0.y - q0.x) + s23 * (q0.w - q0.z), a1 = s01 * (q1.y - q1.x) + s23 * (q1.w - q1.z);
        const float b0 = s02 * (q0.z - q0.x) + s13 * (q0.w - q0.y), b1 = s02 * (q1.z - q1.x) + s13 * (q1.w - q1.y);
        const float Gj = grow[j];
        S.sm = fmaf(Gj, fmaf(f, m1 - m0, m0), S.sm);
        S.sa = fmaf(Gj, fmaf(f, a1 - a0, a0), S.sa);
        S.sz = fmaf(Gj, fmaf(f, b1 - b0, b0), S.sz);
        S.sv = fmaf(Gj * (m1 - m0), ((float)k + f) + ls0_over, S.sv);
    }
    return S;
}

// Fast path. The three weighted forms are linear in the corner templates,
// so the rounds accumulate per corner c, in packed FP32x2 pairs (c = 0, 1 and
// 2, 3): U_c = sum_j G_j V_c(j), V_c(j) the corner template interpolated at
// bin j, and T_c = sum_j G_j u_j (T_c[hi] - T_c[lo]), the slope between the
// bracketing nodes times the bin's absolute position u_j = t_j + ls0/dls.
// Lane l reads node K0 + o_r + l's quad and the neighbouring node's (node
// K0 + o_r + l -+ 1, one more 16-byte load: as the four shuffles of lane
// l -+ 1's quad it replaces, four shared-memory wavefronts, conflict-free, as
// the lanes of each quarter-warp read at most eight consecutive nodes).
// Afterwards sm = w.U, sa = a.U, sz = b.U and sv = w.T.
template <int R>
__device__ __forceinline__ AdjSums adj_particle(const float4 w, const float4 g4, const TileCtx& C,
                                                const float4* __restrict__ slab, const float4* __restrict__ quad,
                                                int lane, float lanef, const float (&G)[R], const float* grow,
                                                float ls0_over) {
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi), bi = rec_bi(c0_bi);
    float f;
    const int K0 = node_pos(C.j0, bi, g4.y, g4.z, g4.w, f);
    const float delta = (1.f - g4.z) - g4.w;
    const int kw = K0 - C.klo;
    const int cr = cell - C.cell0;
    if (!(delta >= 0.f && delta * 31.f < 1.f && (unsigned)kw < (unsigned)(C.slab_w - 31 * R) &&
          (unsigned)cr < (unsigned)C.ncb))
        return adj_general<R>(w, g4, C, slab, quad, lane, grow, ls0_over);
#if RUBIX_DEBUG
    // each lane's node and the neighbour it reads (lane 0: node + 1, lane 31: node - 1)
    dbg_check(dbg_rounds_in_slab(kw * C.ncb + cr, f, delta, C, lane, R, 31, 31, lane > 0 ? -1 : 0, lane < 31 ? 1 : 0),
              C.err);
#endif
    const float4* q = slab + (kw + lane) * C.ncb + cr;
    const int s31 = 31 * C.ncb, s30 = 30 * C.ncb;
    const float nld = -lanef * delta;
    const float d31 = 31.f * delta;
    const float A = 1.f - delta;
    // absolute position of bin j0 + 31 r + l, advanced by 31 A per round
    float u = fmaf(lanef, A, ((float)K0 + f) + ls0_over);
    const float du = 31.f * A;
    float2 U01 = make_float2(0.f, 0.f), U23 = U01, T01 = U01, T23 = U01;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float4 Q = *q;
        const float g = f + nld;
        // lane 31 owns no bin (G = 0); it takes node - 1, so that every read
        // stays within nodes K0 .. K0 + 31 R of the slab
        const bool neg = g < 0.f || lane == 31;
        const float4 Xq = q[neg ? -C.ncb : C.ncb];
        const float2 X01 = make_float2(Xq.x, Xq.y);
        const float2 X23 = make_float2(Xq.z, Xq.w);
        const float2 Q01 = make_float2(Q.x, Q.y), Q23 = make_float2(Q.z, Q.w);
        const float2 D01 = __fadd2_rn(X01, make_float2(-Q.x, -Q.y));
        const float2 D23 = __fadd2_rn(X23, make_float2(-Q.z, -Q.w));
        const float ag = fabsf(g);
        const float2 ag2 = make_float2(ag, ag);
        const float Gj = G[r];  // 0 for lane 31 and bins past the end
        const float2 G2 = make_float2(Gj, Gj);
        U01 = __ffma2_rn(G2, __ffma2_rn(ag2, D01, Q01), U01);
        U23 = __ffma2_rn(G2, __ffma2_rn(ag2, D23, Q23), U23);
        const float gu = (neg ? -Gj : Gj) * u;  // D points from this node to the neighbour
        const float2 gu2 = make_float2(gu, gu);
        T01 = __ffma2_rn(gu2, D01, T01);
        T23 = __ffma2_rn(gu2, D23, T23);
        f -= d31;
        const bool carry = f < 0.f;
        f = carry ? f + 1.f : f;
        q += carry ? s30 : s31;
        u += du;
    }
    const float s01 = w.x + w.y, s23 = w.z + w.w, s02 = w.x + w.z, s13 = w.y + w.w;
    AdjSums S;
    S.sm = fmaf(w.x, U01.x, fmaf(w.y, U01.y, fmaf(w.z, U23.x, w.w * U23.y)));
    S.sa = fmaf(s01, U01.y - U01.x, s23 * (U23.y - U23.x));
    S.sz = fmaf(s02, U23.x - U01.x, s13 * (U23.y - U01.y));
    S.sv = fmaf(w.x, T01.x, fmaf(w.y, T01.y, fmaf(w.z, T23.x, w.w * T23.y)));
    return S;
}

// ---------------------------------------------------------------------------
// Bin means (resample = 1). With S_j the mean of the weighted interpolant over
// [e_j, e_{j+1}] (node units, width A) and the edges moving with v as
// t' = -(t + ls0/dls) / (c (1 + v/c)), differentiating the bounds gives
//   dS_j/dv = -1/(c (1 + v/c)) [ (L_{j+1} u_{j+1} - L_j u_j) / A - S_j ]
//           = -1/(c (1 + v/c)) [ u_j (L_{j+1} - L_j) / A + L_{j+1} - S_j ],
// L_j the interpolant at edge j and u_j = e_j + ls0/dls (u_{j+1} = u_j + A);
// sv sums G_j times the bracket, and sm, sa, sz sum G_j times the bin means
// of the three weighted interpolants (M, and the a- and b-weighted forms).
// ---------------------------------------------------------------------------
__device__ __noinline__ AdjSums adj_mean_bin(const float4 w, const float4 wa, const float4 wb, const float4 g4,
                                             const TileCtx C, int j, float Gj, bool use_slab, const float4* slab,
                                             const float4* quad, float ls0_over) {
    AdjSums S{0.f, 0.f, 0.f, 0.f};
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi), bi = rec_bi(c0_bi);
    float fa, fb;
    const int ka = node_pos(j, bi, g4.y, g4.z, g4.w, fa);
    const int kb = node_pos(j + 1, bi, g4.y, g4.z, g4.w, fb);
    auto node = [&](int k) {
#if RUBIX_DEBUG
        if (use_slab)
            dbg_check((unsigned)((k - C.klo) * C.ncb + (cell - C.cell0)) < (unsigned)(C.slab_w * C.ncb), C.err);
#endif
        return use_slab ? slab[(k - C.klo) * C.ncb + (cell - C.cell0)] : quad_global(quad, C, cell, k);
    };
    const float len = (float)(kb - ka) + (fb - fa);
    if (!(len > 0.f)) return S;
    const int k_first = max(ka, -1), k_last = min(kb, C.n_ls - 1);
    float im = 0.f, ia = 0.f, ib = 0.f;
    float4 q0 = node(k_first);
    float m0 = quad_dot(w, q0), a0 = quad_dot(wa, q0), b0 = quad_dot(wb, q0);
    for (int k = k_first; k <= k_last; ++k) {
        const float4 q1 = node(k + 1);
        const float m1 = quad_dot(w, q1), a1 = quad_dot(wa, q1), b1 = quad_dot(wb, q1);
        const float u0 = (k == ka) ? fa : 0.f, u1 = (k == kb) ? fb : 1.f;
        const float d = u1 - u0, mid = 0.5f * (u0 + u1);
        im = fmaf(d, fmaf(m1 - m0, mid, m0), im);
        ia = fmaf(d, fmaf(a1 - a0, mid, a0), ia);
        ib = fmaf(d, fmaf(b1 - b0, mid, b0), ib);
        m0 = m1;
        a0 = a1;
        b0 = b1;
    }
    const float inv = 1.f / len;
    const float4 qa0 = node(ka), qa1 = node(ka + 1), qb0 = node(kb), qb1 = node(kb + 1);
    const float ma = quad_dot(w, qa0), mb = quad_dot(w, qb0);
    const float La = fmaf(fa, quad_dot(w, qa1) - ma, ma), Lb = fmaf(fb, quad_dot(w, qb1) - mb, mb);
    const float Sm = im * inv;
    S.sm = Gj * Sm;
    S.sa = Gj * (ia * inv);
    S.sz = Gj * (ib * inv);
    const float u = ((float)ka + fa) + ls0_over;
    S.sv = Gj * fmaf(u * (Lb - La), inv, Lb - Sm);
    return S;
}

// General path of the bin means: bin j0 + 30 r + l on lane l (l < 30; the
// last round holds R bins), nodes from the slab when every bin of the warp
// has its nodes there, else from global memory.
template <int R>
__device__ __noinline__ AdjSums adj_mean_general(const float4 w, const float4 g4, const TileCtx C, const float4* slab,
                                                 const float4* quad, int lane, const float* __restrict__ grow,
                                                 float ls0_over) {
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi), bi = rec_bi(c0_bi);
    bool ok = C.slab_w > 0 && (unsigned)(cell - C.cell0) < (unsigned)C.ncb;
#pragma unroll
    for (int r = 0; r <= R; ++r) {
        const int j = C.j0 + 30 * r + lane;
        if (lane < (r < R ? 30 : R) && j < C.n_lambda) {
            float fa, fb;
            const int ka = node_pos(j, bi, g4.y, g4.z, g4.w, fa) - C.klo;
            const int kb = node_pos(j + 1, bi, g4.y, g4.z, g4.w, fb) - C.klo;
            ok = ok && ka >= 0 && kb + 1 < C.slab_w;
        }
    }
    const bool use_slab = __all_sync(0xffffffffu, ok);
    const float s01 = w.x + w.y, s23 = w.z + w.w, s02 = w.x + w.z, s13 = w.y + w.w;
    const float4 wa = make_float4(-s01, s01, -s23, s23), wb = make_float4(-s02, -s13, s02, s13);
    AdjSums S{0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r <= R; ++r) {
        const int j = C.j0 + 30 * r + lane;
        if (!(lane < (r < R ? 30 : R) && j < C.n_lambda)) continue;
        const AdjSums b = adj_mean_bin(w, wa, wb, g4, C, j, grow[j], use_slab, slab, quad, ls0_over);
        S.sm += b.sm;
        S.sa += b.sa;
        S.sz += b.sz;
        S.sv += b.sv;
    }
    return S;
}

// Fast path of the bin means: the forward's 30-bin rounds (edge l on lane l;
// see mean_rounds in deposit.cu), accumulated per corner as in adj_particle.
// Lane l interpolates the four corner templates at its edge (L), takes the
// next edge's (Ln) and the enclosed node's values, and adds G_j times twice
// the corner's bin mean (U) and G_j times the corner's share of the v bracket
// (T); the weights are applied once afterwards.
template <int R>
__device__ __forceinline__ AdjSums adj_mean_particle(const float4 w, const float4 g4, const TileCtx& C,
                                                     const float4* __restrict__ slab,
                                                     const float4* __restrict__ quad, int lane, float lanef,
                                                     const float (&G)[R + 1], const float* grow, float ls0_over) {
    const int c0_bi = __float_as_int(g4.x);
    const int cell = rec_c0(c0_bi), bi = rec_bi(c0_bi);
    float f;
    const int K0 = node_pos(C.j0, bi, g4.y, g4.z, g4.w, f);
    const float delta = (1.f - g4.z) - g4.w;
    const int kw = K0 - C.klo;
    const int cr = cell - C.cell0;
    if (!(delta >= 0.f && delta * 31.f < 1.f && (unsigned)kw < (unsigned)(C.slab_w - 31 * R - 1) &&
          (unsigned)cr < (unsigned)C.ncb))
        return adj_mean_general<R>(w, g4, C, slab, quad, lane, grow, ls0_over);
#if RUBIX_DEBUG
    dbg_check(dbg_rounds_in_slab(kw * C.ncb + cr, f, delta, C, lane, R + 1, 30, R + 1, 0, 0), C.err);
#endif
    const float4* q = slab + (kw + lane) * C.ncb + cr;
    const int s30 = 30 * C.ncb, s29 = 29 * C.ncb;
    const float nld = -lanef * delta;
    const float d30 = 30.f * delta;
    const float A = 1.f - delta;
    const float iA = 1.f / A;
    // absolute position of lane l's edge (node units + ls0/dls), 30 A further each round
    float u = fmaf(lanef, A, ((float)K0 + f) + ls0_over);
    const float du = 30.f * A;
    const float2 mhalf = make_float2(-0.5f, -0.5f);
    float2 U01 = make_float2(0.f, 0.f), U23 = U01, T01 = U01, T23 = U01;
#pragma unroll
    for (int r = 0; r <= R; ++r) {
        float4 Q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < R || lane <= R + 1) Q = *q;
        const float g = f + nld;
        const bool up = g >= 0.f;
        const int src = up ? lane + 1 : lane - 1;
        const float2 Q01 = make_float2(Q.x, Q.y), Q23 = make_float2(Q.z, Q.w);
        const float2 X01 = make_float2(__shfl_sync(0xffffffffu, Q.x, src), __shfl_sync(0xffffffffu, Q.y, src));
        const float2 X23 = make_float2(__shfl_sync(0xffffffffu, Q.z, src), __shfl_sync(0xffffffffu, Q.w, src));
        const float2 D01 = __fadd2_rn(X01, make_float2(-Q.x, -Q.y));
        const float2 D23 = __fadd2_rn(X23, make_float2(-Q.z, -Q.w));
        const float ag = fabsf(g);
        const float2 L01 = __ffma2_rn(make_float2(ag, ag), D01, Q01);
        const float2 L23 = __ffma2_rn(make_float2(ag, ag), D23, Q23);
        const float2 N01 = make_float2(__shfl_down_sync(0xffffffffu, L01.x, 1), __shfl_down_sync(0xffffffffu, L01.y, 1));
        const float2 N23 = make_float2(__shfl_down_sync(0xffffffffu, L23.x, 1), __shfl_down_sync(0xffffffffu, L23.y, 1));
        // the node between the edges (the neighbour if g >= 0)
        const float uf = up ? 1.f : 0.f;
        const float2 K01 = __ffma2_rn(make_float2(uf, uf), D01, Q01);
        const float2 K23 = __ffma2_rn(make_float2(uf, uf), D23, Q23);
        const float ai = fmaf(-g, iA, up ? iA : 0.f);  // a / A
        const float2 dd01 = __fadd2_rn(L01, make_float2(-N01.x, -N01.y));
        const float2 dd23 = __fadd2_rn(L23, make_float2(-N23.x, -N23.y));
        // twice the bin mean: M_K + L_{l+1} + (a/A)(L - L_{l+1})
        const float2 v01 = __ffma2_rn(make_float2(ai, ai), dd01, __fadd2_rn(K01, N01));
        const float2 v23 = __ffma2_rn(make_float2(ai, ai), dd23, __fadd2_rn(K23, N23));
        const float Gj = G[r];  // 0 for lanes that own no bin of the tile
        const float2 G2 = make_float2(Gj, Gj);
        U01 = __ffma2_rn(G2, v01, U01);
        U23 = __ffma2_rn(G2, v23, U23);
        // v bracket per corner: L_{l+1} - mean - u (L - L_{l+1}) / A
        const float gu = -Gj * u * iA;
        T01 = __ffma2_rn(G2, __ffma2_rn(mhalf, v01, N01), __ffma2_rn(make_float2(gu, gu), dd01, T01));
        T23 = __ffma2_rn(G2, __ffma2_rn(mhalf, v23, N23), __ffma2_rn(make_float2(gu, gu), dd23, T23));
        if (r < R) {
            f -= d30;
            const bool carry = f < 0.f;
            f = carry ? f + 1.f : f;
            q += carry ? s29 : s30;
            u += du;
        }
    }
    const float s01 = w.x + w.y, s23 = w.z + w.w, s02 = w.x + w.z, s13 = w.y + w.w;
    AdjSums S;
    S.sm = 0.5f * fmaf(w.x, U01.x, fmaf(w.y, U01.y, fmaf(w.z, U23.x, w.w * U23.y)));
    S.sa = 0.5f * fmaf(s01, U01.y - U01.x, s23 * (U23.y - U23.x));
    S.sz = 0.5f * fmaf(s02, U23.x - U01.x, s13 * (U23.y - U01.y));
    S.sv = fmaf(w.x, T01.x, fmaf(w.y, T01.y, fmaf(w.z, T23.x, w.w * T23.y)));
    return S;
}

template <int R, bool MEAN>
__global__ void __launch_bounds__(RUBIX_ADJ_THREADS, RUBIX_DEP_CTAS) k_adjoint_tiles(const __grid_constant__ AdjTileParams P,
                                                                         const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* s_next = reinterpret_cast<int*>(smem + 16);
    float4* slab = reinterpret_cast<float4*>(smem + kDepHeader);
    const int lane = threadIdx.x & 31;
    const float lanef = (float)lane;
    const int nb = P.n_bands;
    const long long n_items = P.item_off[P.n_s];
    const long long n_in = P.seg_off[(long long)P.n_s * nb];
    if (n_in > P.n_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(P.err, kErrBadItem);
        return;
    }
    const long long C0 = P.cost_c0;
    const long long CT = n_in + C0 * n_items;
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
    const float4* __restrict__ rec4 = reinterpret_cast<const float4*>(P.rec);

    for (long long t = lo / CT; t < P.n_tiles && t * CT < hi; ++t) {
        const long long a = max(lo - t * CT, 0ll), b = min(hi - t * CT, CT);
        if (a >= b) continue;
        const int ia = (int)item_lower_bound(P.items, n_items, C0, a);
        const int ib = (int)item_lower_bound(P.items, n_items, C0, b);
        const int nv = ib - ia;
        C.klo = P.tile_klo[t];
        C.j0 = (int)t * P.tile_w;
        float4* __restrict__ part = P.part + t * P.n_cap;
        for (int band = 0; band < nb; ++band) {
            C.cell0 = P.band_cell0[band];
            __syncthreads();  // all warps are done with the previous slab
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
            constexpr int GR = RUBIX_ADJ_GRAB;
            while (true) {
                int v0 = 0;
                if (lane == 0) v0 = atomicAdd(s_next, GR);
                v0 = __shfl_sync(0xffffffffu, v0, 0);
                if (v0 >= nv) break;
                int qb = 0, qe = 0, sp = 0;
                bool live = false;
                if (lane < GR && v0 + lane < nv) {
                    const Item I = P.items[ia + v0 + lane];
                    sp = I.spaxel;
                    if (sp < 0 || sp >= P.n_s) {
                        atomicOr(P.err, kErrBadItem);
                    } else {
                        qb = I.begin;
                        qe = I.end;
                        if (nb > 1) {
                            qb = max(qb, P.seg_off[(long long)sp * nb + band]);
                            qe = min(qe, P.seg_off[(long long)sp * nb + band + 1]);
                        }
                        live = qb < qe;
                        // the item's first weights and record, on their way to L1,
                        // and its tile slice of dL/dcube0 on its way to L2
                        if (live) {
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(P.wu + qb));
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(rec4 + 2 * qb + 1));
                            const float* gs = P.G0 + (long long)sp * P.n_lambda + C.j0;
                            const int nbin = min(P.tile_w + 1, P.n_lambda - C.j0);
#pragma unroll 1
                            for (int o = 0; o < nbin; o += 32)
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(gs + o));
                        }
                    }
                }
                unsigned m = __ballot_sync(0xffffffffu, live);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const int q0 = __shfl_sync(0xffffffffu, qb, src);
                    const int q1 = __shfl_sync(0xffffffffu, qe, src);
                    const int s = __shfl_sync(0xffffffffu, sp, src);
                    // this tile's slice of the spaxel's dL/dcube0 row, one bin per lane and round
                    constexpr int NR = MEAN ? R + 1 : R;
                    float G[NR];
                    const float* __restrict__ grow = P.G0 + (long long)s * P.n_lambda;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int j = MEAN ? C.j0 + 30 * r + lane : C.j0 + 31 * r + lane;
                        const bool owned = MEAN ? lane < (r < R ? 30 : R) : lane < 31;
                        G[r] = (owned && j < P.n_lambda) ? grow[j] : 0.f;
                    }
                    for (int q = q0; q < q1; ++q) {
                        if (q + 1 < q1) {
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(P.wu + q + 1));
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(rec4 + 2 * (q + 1) + 1));
                        }
                        AdjSums S;
                        if constexpr (MEAN)
                            S = adj_mean_particle<R>(P.wu[q], rec4[2 * q + 1], C, slab, P.quad, lane, lanef, G,
                                                     grow, P.ls0_over);
                        else
                            S = adj_particle<R>(P.wu[q], rec4[2 * q + 1], C, slab, P.quad, lane, lanef, G, grow,
                                                P.ls0_over);
                        // the four sums over the warp with 6 shuffles: halves of the
                        // warp trade pairs, quarters trade singles, then a butterfly
                        // over 8 lanes; lane 8 v ends with sum v (v = sm, sa, sz, sv)
                        const bool hi16 = lane >= 16, hi8 = (lane & 8) != 0;
                        const float r0 = __shfl_xor_sync(0xffffffffu, hi16 ? S.sm : S.sz, 16);
                        const float r1 = __shfl_xor_sync(0xffffffffu, hi16 ? S.sa : S.sv, 16);
                        const float b0 = (hi16 ? S.sz : S.sm) + r0, b1 = (hi16 ? S.sv : S.sa) + r1;
                        float c = (hi8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, hi8 ? b0 : b1, 8);
#pragma unroll
                        for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
#if RUBIX_DEBUG
                        dbg_check(q >= 0 && q < P.n_cap, P.err);
#endif
                        if ((lane & 7) == 0) reinterpret_cast<float*>(part + q)[lane >> 3] = c;
                    }
                }
            }
        }
    }
}

int launch_adjoint_tiles(const AdjTileParams& P, const CUtensorMap* tmap, int n_ctas, int threads, size_t smem,
                         cudaStream_t st) {
    if (P.tile_w % 31 != 0) return -1;
    void (*fn)(const AdjTileParams, const CUtensorMap) = nullptr;
    switch (P.tile_w / 31) {
#define RUBIX_ADJ_R(r) \
    case r: fn = P.resample ? k_adjoint_tiles<r, true> : k_adjoint_tiles<r, false>; break;
        RUBIX_ADJ_R(1) RUBIX_ADJ_R(2) RUBIX_ADJ_R(3) RUBIX_ADJ_R(4) RUBIX_ADJ_R(5) RUBIX_ADJ_R(6)
        RUBIX_ADJ_R(7) RUBIX_ADJ_R(8) RUBIX_ADJ_R(9) RUBIX_ADJ_R(10) RUBIX_ADJ_R(11) RUBIX_ADJ_R(12)
#if RUBIX_DEP_RMAX > 12
        RUBIX_ADJ_R(13) RUBIX_ADJ_R(14) RUBIX_ADJ_R(15) RUBIX_ADJ_R(16) RUBIX_ADJ_R(17) RUBIX_ADJ_R(18)
        RUBIX_ADJ_R(19) RUBIX_ADJ_R(20) RUBIX_ADJ_R(21) RUBIX_ADJ_R(22) RUBIX_ADJ_R(23) RUBIX_ADJ_R(24)
#endif
#undef RUBIX_ADJ_R
        default: return -1;
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    fn<<<n_ctas, threads, smem, st>>>(P, *tmap);
    return 1;
}

// ---------------------------------------------------------------------------
// K8: tiles summed in tile order (compensated FP32), chain rule, original order.
// ---------------------------------------------------------------------------
__global__ void k_adj_final(const AdjointParams P, const float4* __restrict__ part, int n_tiles, long long n_cap) {
    const long long n_in = P.seg_off[(long long)P.n_s * P.n_bands];
    const float ln10 = 2.302585092994046f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_in;
         i += (long long)gridDim.x * blockDim.x) {
        // the tiles' sums in tile order, compensated (two-sum) in FP32
        float sm = 0.f, sa = 0.f, sz = 0.f, sv = 0.f, em = 0.f, ea = 0.f, ez = 0.f, ev = 0.f;
        for (int t = 0; t < n_tiles; ++t) {
            const float4 v = part[t * n_cap + i];
            two_sum_add(sm, em, v.x);
            two_sum_add(sa, ea, v.y);
            two_sum_add(sz, ez, v.z);
            two_sum_add(sv, ev, v.w);
        }
        sm += em;
        sa += ea;
        sz += ez;
        sv += ev;
        const PartRec pr = P.prec[i];
        int ia, iz;
        float ta, tz, dta, dtz;
        ssp_cell(log10f(pr.age), P.ssp.la_nodes, P.ssp.n_age, ia, ta, dta);
        ssp_cell(log10f(pr.Z), P.ssp.lz_nodes, P.ssp.n_Z, iz, tz, dtz);
        // dt/dv = -(t + ls0/dls) / (c (1 + v/c)): the sums carry the (t + ls0/dls) factor
        const float q = -1.f / ((float)kC_kms + pr.v);  // = -1 / (c (1 + v/c))
        const float fs = (float)P.flux_scale;
        const float dm = fs * sm;
        const float dage = fs * pr.mass * dta * sa / (pr.age * ln10);
        const float dZ = fs * pr.mass * dtz * sz / (pr.Z * ln10);
        const float dv = fs * pr.mass * q * sv;
        const int p = P.perm[i];
        if (P.d_mass) P.d_mass[p] = dm;
        if (P.d_age) P.d_age[p] = dage;
        if (P.d_Z) P.d_Z[p] = dZ;
        if (P.d_v) P.d_v[p] = dv;
        if (P.contrib) {
            const float2 da = P.dv_dang ? P.dv_dang[p] : make_float2(0.f, 0.f);
            P.contrib[kGlobal * i] = (double)dv;
            P.contrib[kGlobal * i + 1] = (double)pr.mass * (double)dm;
            P.contrib[kGlobal * i + 2] = (double)dv * (double)da.x;
            P.contrib[kGlobal * i + 3] = (double)dv * (double)da.y;
        }
    }
}

int launch_adjoint_final(const AdjointParams& P, const float4* part, int n_tiles, long long n_cap, cudaStream_t st) {
    if (P.n_in <= 0) return 0;
    long long nb = (P.n_in + 255) / 256;
    if (nb > 16ll * sm_count()) nb = 16ll * sm_count();
    k_adj_final<<<(int)nb, 256, 0, st>>>(P, part, n_tiles, n_cap);
    return 1;
}

}  // namespace rubix
