// adjoint.cu -- gradients through the pipeline (Abstract and Sec. 1: the
// forward model is differentiable end to end), written by hand instead of by
// autodiff.
//
// Given G0 = dL/d(cube before PSF/LSF) (the caller of these kernels forms it
// by applying the transposed LSF and PSF to dL/dcube; both are symmetric
// zero-padded convolutions, so each is its own transpose), K7 gives, for each
// in-field particle p in spaxel s, with V_c(j) the resampled corner template c
// at bin j and w_c the bilinear weights:
//   dL/dm    = fs * sum_j G0[s,j] sum_c w_c V_c(j)
//   dL/dlog10 age = fs m dta * sum_j G0 [(1-tz)(V10-V00) + tz(V11-V01)]
//   dL/dlog10 Z   = fs m dtz * sum_j G0 [(1-ta)(V01-V00) + ta(V11-V10)]
//   dL/dv    = fs m * sum_j G0 (M(k+1) - M(k)) dt/dv,
//              M(k) = sum_c w_c T_c[k], dt/dv = -(lambda_rest/dls) / (c (1 + v/c)),
// with the derivative of each piecewise-linear interpolant taken in the
// half-open cell holding the point (clamped coordinates give 0). One warp per
// particle, lanes over wavelength, fixed-order warp reduction. K8 sums the
// per-particle contributions to the shared (global) parameters in FP64 in a
// fixed order.
#include "common.cuh"
#include "kernels.h"

namespace rubix {

template <typename T>
__device__ __forceinline__ float tplg(const T* __restrict__ tpl, int pitch, int n_ls, int row, int k) {
    return (k >= 0 && k < n_ls) ? TplTraits<T>::ld(tpl + (long long)row * pitch + k) : 0.f;
}

template <typename T>
__global__ void __launch_bounds__(256) k_adjoint(const AdjointParams P, const DepRec* __restrict__ rec) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n_in = P.seg_off[(long long)P.n_s * P.n_bands];
    const T* __restrict__ tpl = reinterpret_cast<const T*>(P.ssp.tpl);
    const int pitch = P.ssp.pitch, n_ls = P.ssp.n_ls;
    const int da = (P.ssp.n_age > 1) ? P.ssp.n_Z : 0;
    const int dz = (P.ssp.n_Z > 1) ? 1 : 0;
    const float ls0_over = (float)(P.ssp.ls0 / P.ssp.dls);
    const float ln10 = 2.302585092994046f;
    for (long long i = gw; i < n_in; i += nw) {
        const PartRec pr = P.prec[i];
        const int s = P.sorted_keys[i] / P.n_bands;
        const int p = P.perm[i];
        int ia, iz;
        float ta, tz, dta, dtz;
        ssp_cell(log10f(pr.age), P.ssp.la_nodes, P.ssp.n_age, ia, ta, dta);
        ssp_cell(log10f(pr.Z), P.ssp.lz_nodes, P.ssp.n_Z, iz, tz, dtz);
        const float w0 = (1.f - ta) * (1.f - tz), w1 = ta * (1.f - tz), w2 = (1.f - ta) * tz, w3 = ta * tz;
        const int c0 = ia * P.ssp.n_Z + iz;
        const int r0 = c0, r1 = c0 + da, r2 = c0 + dz, r3 = c0 + da + dz;
        const float4 g4 = reinterpret_cast<const float4*>(rec)[2 * i + 1];
        const int c0_bi = __float_as_int(g4.x);
        const int bi = rec_bi(c0_bi);
        const float bf = g4.y, a_hi = g4.z, a_lo = g4.w;
        const bool live = a_hi > 0.f;   // zero only for particles whose spectrum misses every bin
        const float q = (float)(-1.0 / (kC_kms * (1.0 + (double)pr.v / kC_kms)));
        const float* __restrict__ g = P.G0 + (long long)s * P.n_lambda;
        float sm = 0.f, sla = 0.f, slz = 0.f, sv = 0.f;
        if (live) {
            for (int j = lane; j < P.n_lambda; j += 32) {
                const float jf = (float)j;
                const float pp = jf * a_hi;
                const float pi = floorf(pp);
                const float sx = (pp - pi) + fmaf(jf, a_lo, bf);
                const float fl = floorf(sx);
                const float f = sx - fl;
                const int k = bi + (int)pi + (int)fl;
                const float a0 = tplg(tpl, pitch, n_ls, r0, k), b0 = tplg(tpl, pitch, n_ls, r0, k + 1);
                const float a1 = tplg(tpl, pitch, n_ls, r1, k), b1 = tplg(tpl, pitch, n_ls, r1, k + 1);
                const float a2 = tplg(tpl, pitch, n_ls, r2, k), b2 = tplg(tpl, pitch, n_ls, r2, k + 1);
                const float a3 = tplg(tpl, pitch, n_ls, r3, k), b3 = tplg(tpl, pitch, n_ls, r3, k + 1);
                const float V0 = fmaf(f, b0 - a0, a0), V1 = fmaf(f, b1 - a1, a1);
                const float V2 = fmaf(f, b2 - a2, a2), V3 = fmaf(f, b3 - a3, a3);
                const float Sj = w0 * V0 + w1 * V1 + w2 * V2 + w3 * V3;
                const float ga = (1.f - tz) * (V1 - V0) + tz * (V3 - V2);
                const float gz = (1.f - ta) * (V2 - V0) + ta * (V3 - V1);
                const float Mk = w0 * a0 + w1 * a1 + w2 * a2 + w3 * a3;
                const float Mk1 = w0 * b0 + w1 * b1 + w2 * b2 + w3 * b3;
                const float tabs = ((float)k + f) + ls0_over;   // lambda_rest / dls
                const float gj = g[j];
                sm = fmaf(gj, Sj, sm);
                sla = fmaf(gj, ga, sla);
                slz = fmaf(gj, gz, slz);
                sv = fmaf(gj * (Mk1 - Mk), q * tabs, sv);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sm += __shfl_xor_sync(0xffffffffu, sm, o);
            sla += __shfl_xor_sync(0xffffffffu, sla, o);
            slz += __shfl_xor_sync(0xffffffffu, slz, o);
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
        }
        if (lane == 0) {
            const float fs = (float)P.flux_scale;
            const float dm = fs * sm;
            const float dage = fs * pr.mass * dta * sla / (pr.age * ln10);
            const float dZ = fs * pr.mass * dtz * slz / (pr.Z * ln10);
            const float dv = fs * pr.mass * sv;
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
}

// The adjoint reads the forward's records (bin -> node map) for consistency.
int launch_adjoint_rec(const AdjointParams& P, const DepRec* rec, cudaStream_t st) {
    if (P.n_in <= 0) return 0;
    long long warps = P.n_in;
    long long nb = (warps * 32 + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    switch (P.ssp.dtype) {
        case 0: k_adjoint<float><<<(int)nb, 256, 0, st>>>(P, rec); break;
        case 1: k_adjoint<__nv_bfloat16><<<(int)nb, 256, 0, st>>>(P, rec); break;
        case 2: k_adjoint<__half><<<(int)nb, 256, 0, st>>>(P, rec); break;
        default: return -1;
    }
    return 1;
}

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
    if (nb > 152 * 8) nb = 152 * 8;
    k_zero4<<<(int)nb, 256, 0, st>>>(a, b, c, d, n);
    return 1;
}

// K8: fixed-order FP64 reduction of contrib[n][kGlobal] -> out[kGlobal]
// (each block sums a contiguous range, then one thread adds the blocks in order).
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

__global__ void k_reduce_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a[kGlobal];
        for (int c = 0; c < kGlobal; ++c) a[c] = 0.0;
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < kGlobal; ++c) a[c] += part[kGlobal * i + c];
        for (int c = 0; c < kGlobal; ++c) out[c] = a[c];
    }
}

int launch_reduce_global(const double* contrib, const int* n_in_dev, double* out, double* scratch, cudaStream_t st) {
    k_reduce_partial<<<kRedBlocks, 256, 0, st>>>(contrib, n_in_dev, scratch);
    k_reduce_final<<<1, 32, 0, st>>>(scratch, kRedBlocks, out);
    return 2;
}

}  // namespace rubix
