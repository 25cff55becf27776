// setup.cu -- K3 of the deposit path (Sec. 3: each star's SSP lookup and
// Doppler shift, prepared once per particle): every in-field particle, in
// sorted order, becomes a 32-byte record (its four mass-scaled bilinear
// corner weights, its SSP cell and the affine map t(j) = B + jA from output
// bin j to the fractional SSP node position), and each spaxel's particles
// are cut into work items of at most `chunk` particles.
#include "common.cuh"
#include "kernels.h"

namespace rubix {

// ----------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2), about 48 significant bits. Products use the
// exact FMA residual, sums Knuth's two-sum; each operation is a handful of
// FP32 instructions instead of one FP64 instruction on this GPU's FP64 pipe,
// which runs at 1/64 of the FP32 rate (Dekker 1971; Shewchuk 1997).
// ----------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

// (the _rn intrinsics keep the compiler from contracting these products and
// sums into FMAs, which the error-free transformations must not see)
__device__ __forceinline__ DF df_norm(float hi, float lo) {  // |hi| >= |lo|
    const float s = __fadd_rn(hi, lo);
    return DF{s, __fsub_rn(lo, __fsub_rn(s, hi))};
}

__device__ __forceinline__ DF df_of(double x) {
    const float hi = (float)x;
    return DF{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float z = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    return df_norm(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}

__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    const float p = __fmul_rn(a.hi, b);
    const float e = fmaf(a.hi, b, -p);
    return df_norm(p, fmaf(a.lo, b, e));
}

// ----------------------------------------------------------------------------
// K3: per-particle setup (sorted order).
// ----------------------------------------------------------------------------
__global__ void k_setup(SetupParams P) {
    const long long n_in = P.seg_off[(long long)P.n_s * P.n_bands];
    if (n_in > P.n_cap) return;
    const int n_ls = P.ssp.n_ls;
    // t(j) = ((l0 + j dl) / dop - ls0) / dls = B + j A with dop = (1 + z)(1 + v/c).
    // With alpha_z = 1 / ((1 + z) dls) and g = (v/c) / (1 + v/c), so that
    // 1 / (1 + v/c) = 1 - g:
    //   A = A_z (1 - g),   A_z = dl alpha_z,
    //   B = B_z - L g,     L = l0 alpha_z,  B_z = L - ls0/dls,
    // (bin means: B - A/2, the bin's lower edge), the particle's part in
    // double-float from the FP64 constants below (converted once per thread).
    const DF Az = df_of(P.dl * P.alpha_z), L = df_of(P.l0 * P.alpha_z);
    const DF Bz = df_of(fma(P.l0, P.alpha_z, -P.ls0_dls)), invc = df_of(P.inv_c);
    const float t_lastj = (float)(P.resample ? P.n_lambda : P.n_lambda - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_in;
         i += (long long)gridDim.x * blockDim.x) {
        const PartRec pr = P.pin[P.perm[i]];
        const float m = pr.mass, age = pr.age, Z = pr.Z;
        int ia, iz;
        float ta, tz, dta, dtz;
        ssp_cell(log10f(age), P.ssp.la_nodes, P.ssp.n_age, ia, ta, dta);
        ssp_cell(log10f(Z), P.ssp.lz_nodes, P.ssp.n_Z, iz, tz, dtz);
        const float ms = (float)P.flux_scale * m;
        DepRec r;
        r.w[0] = ms * ((1.f - ta) * (1.f - tz));
        r.w[1] = ms * (ta * (1.f - tz));
        r.w[2] = ms * ((1.f - ta) * tz);
        r.w[3] = ms * (ta * tz);
        const int c0 = ia * max(P.ssp.n_Z - 1, 1) + iz;  // SSP cell of the four corners
        // b = v/c, q = 1 + b, g = b / q: one FP32 quotient and one correction
        // from the double-float residual b - g0 q (relative error ~2^-46)
        const DF b = df_mul_f(invc, pr.v);
        const DF q = df_add(DF{1.f, 0.f}, b);
        const float g0 = __fdiv_rn(b.hi, q.hi);
        const DF res = df_add(b, df_neg(df_mul_f(q, g0)));
        const DF g = df_norm(g0, __fdiv_rn(res.hi, q.hi));
        const DF A = df_add(Az, df_neg(df_mul(Az, g)));
        DF B = df_add(Bz, df_neg(df_mul(L, g)));
        if (P.resample) B = df_add(B, DF{-0.5f * A.hi, -0.5f * A.lo});
        const float t_last = fmaf(A.hi, t_lastj, B.hi);
        int bi = 0;
        float bf = 0.f, a_hi = 0.f, a_lo = 0.f;
        if (!(q.hi > 0.f) || !(B.hi < (float)n_ls) || !(t_last >= -1.f) || !(B.hi > -32768.f)) {
            // the spectrum misses every output bin (a_hi = 0 marks the record)
            r.w[0] = r.w[1] = r.w[2] = r.w[3] = 0.f;
        } else {
            // B = bi + bf, bf in [0, 1] rounded once; A = a_hi + a_lo with
            // a_hi of 11 significant bits, so that j a_hi is exact in FP32
            const float fb = floorf(B.hi);
            bi = (int)fb;
            bf = __fadd_rn(__fsub_rn(B.hi, fb), B.lo);
            if (bf < 0.f) {
                bf += 1.f;
                --bi;
            }
            a_hi = __uint_as_float(__float_as_uint(A.hi) & ~((1u << 13) - 1u));
            a_lo = __fadd_rn(__fsub_rn(A.hi, a_hi), A.lo);
        }
        r.c0_bi = (c0 << 16) | (bi & 0xffff);
        r.bf = bf;
        r.a_hi = a_hi;
        r.a_lo = a_lo;
        P.rec[i] = r;
        P.prec[i] = pr;
    }
}

int launch_setup(const SetupParams& P, long long n_total, cudaStream_t st) {
    if (n_total <= 0) return 0;
    long long nb = (n_total + 255) / 256;
    if (nb > 16ll * sm_count()) nb = 16ll * sm_count();
    k_setup<<<(int)nb, 256, 0, st>>>(P);
    return 1;
}

// ----------------------------------------------------------------------------
// Work items: one per <= chunk particles of a spaxel (all age bands). Empty
// spaxels get no item: k_zero_empty writes their rows.
// ----------------------------------------------------------------------------
__global__ void k_item_counts(ItemParams P) {
    const int nb = P.n_bands;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= P.n_s; s += gridDim.x * blockDim.x) {
        if (s == P.n_s) { P.n_items[s] = 0; P.n_parts[s] = 0; continue; }
        const int cnt = P.seg_off[(long long)(s + 1) * nb] - P.seg_off[(long long)s * nb];
        const int ni = (cnt + P.chunk - 1) / P.chunk;
        P.n_items[s] = ni;
        P.n_parts[s] = ni > 1 ? ni : 0;
    }
}

__global__ void k_item_fill(ItemParams P) {
    const int nb = P.n_bands;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.n_s; s += gridDim.x * blockDim.x) {
        const int base = P.item_off[s], ni = P.item_off[s + 1] - base;
        const bool split = P.part_off[s + 1] > P.part_off[s];
        const int b0 = P.seg_off[(long long)s * nb], e0 = P.seg_off[(long long)(s + 1) * nb];
        for (int i = 0; i < ni; ++i) {
            if ((long long)base + i >= P.item_cap) { atomicOr(P.err, kErrBadItem); return; }
            Item it;
            it.spaxel = s;
            it.begin = b0 + i * P.chunk;
            it.end = min(b0 + (i + 1) * P.chunk, e0);
            it.part_row = split ? P.part_off[s] + i : -1;
            P.items[base + i] = it;
        }
    }
}

int launch_items(const ItemParams& P, cudaStream_t st) {
    int nb = (P.n_s + 1 + 255) / 256;
    if (nb > 4096) nb = 4096;
    k_item_counts<<<nb, 256, 0, st>>>(P);
    int l = 1;
    l += launch_exclusive_scan(P.n_items, P.item_off, P.n_s + 1, P.scan_scratch, st);
    l += launch_exclusive_scan(P.n_parts, P.part_off, P.n_s + 1, P.scan_scratch, st);
    k_item_fill<<<nb, 256, 0, st>>>(P);
    return l + 1;
}

}  // namespace rubix
