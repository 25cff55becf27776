// psf_lsf.cu -- observational effects (Sec. 3: "we apply a point-spread
// function (PSF) and line-spread function (LSF) convolution and add realistic
// noise"; Sec. 4: both Gaussian).
//
// The 3-D kernel is separable, g(dy) g(dx) h(dj), with zero padding on every
// axis, so the PSF and LSF are applied as three 1-D stencils:
//   pass 1 (k_lsf_psfx): one CTA per (wavelength chunk, x chunk, row y) loads
//     the row segment with its halos into shared memory, applies the LSF along
//     wavelength and then the PSF along x, and writes an intermediate cube;
//   pass 2 (k_psfy_noise): each thread owns one (x, wavelength) column of a
//     y-chunk and applies the PSF along y, then optional Philox noise.
// Both passes read and write along wavelength (the fastest axis), so every
// global access is coalesced.
#include "common.cuh"
#include "kernels.h"

namespace rubix {

constexpr int kLC = 64;   // wavelength bins per CTA in pass 1
constexpr int kXC = 64;   // spaxels along x per CTA in pass 1

__global__ void __launch_bounds__(256) k_lsf_psfx(const ConvParams P, const float* __restrict__ in,
                                                  float* __restrict__ out) {
    extern __shared__ float sm[];
    const int rl = P.rl, rp = P.rp;
    const int W_in = kLC + 2 * rl;
    const int XW = kXC + 2 * rp;
    float* s_in = sm;                  // [XW][W_in]
    float* s_mid = sm + XW * W_in;     // [XW][kLC]
    const int j0 = blockIdx.x * kLC;
    const int x0 = blockIdx.y * kXC;
    const int y = blockIdx.z;
    const int nx = P.nx, nl = P.n_lambda;
    const long long row = (long long)y * nx;
    for (int e = threadIdx.x; e < XW * W_in; e += blockDim.x) {
        const int xi = e / W_in, l = e - xi * W_in;
        const int x = x0 - rp + xi, j = j0 - rl + l;
        s_in[e] = (x >= 0 && x < nx && j >= 0 && j < nl) ? in[(row + x) * nl + j] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < XW * kLC; e += blockDim.x) {
        const int xi = e / kLC, l = e - xi * kLC;
        const float* src = s_in + xi * W_in + l;
        float acc = 0.f;
        for (int d = 0; d <= 2 * rl; ++d) acc = fmaf(P.gl[d], src[d], acc);
        s_mid[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kXC * kLC; e += blockDim.x) {
        const int xi = e / kLC, l = e - xi * kLC;
        const int x = x0 + xi, j = j0 + l;
        if (x >= nx || j >= nl) continue;
        const float* src = s_mid + xi * kLC + l;
        float acc = 0.f;
        for (int d = 0; d <= 2 * rp; ++d) acc = fmaf(P.gp[d], src[d * kLC], acc);
        out[(row + x) * nl + j] = acc;
    }
}

constexpr int kYC = 32;  // rows per thread in pass 2

__global__ void __launch_bounds__(256) k_psfy_noise(const ConvParams P, const float* __restrict__ in,
                                                    float* __restrict__ out) {
    const long long plane = (long long)P.nx * P.n_lambda;  // one y row of the cube
    const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (col >= plane) return;
    const int y0 = blockIdx.y * kYC;
    const int y1 = min(y0 + kYC, P.ny);
    const int rp = P.rp;
    for (int y = y0; y < y1; ++y) {
        float acc = 0.f;
        for (int d = -rp; d <= rp; ++d) {
            const int yy = y + d;
            if (yy < 0 || yy >= P.ny) continue;
            acc = fmaf(P.gp[d + rp], in[(long long)yy * plane + col], acc);
        }
        const long long idx = (long long)y * plane + col;
        if (P.noise_inv_s2n > 0.f) {
            U4 c;
            c.x = (uint32_t)idx;
            c.y = (uint32_t)((unsigned long long)idx >> 32);
            c.z = 0u;
            c.w = 0u;
            const U4 r = philox4x32_10(c, P.seed_lo, P.seed_hi);
            const float u1 = (float)((r.x >> 8) + 1u) * (1.0f / 16777216.0f);   // (0, 1]
            const float u2 = (float)(r.y >> 8) * (1.0f / 16777216.0f);          // [0, 1)
            const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
            acc = fmaf(fabsf(acc) * P.noise_inv_s2n, z, acc);
        }
        out[idx] = acc;
    }
}

int launch_psf_lsf(const ConvParams& P, const float* in, float* tmp, float* out, cudaStream_t st) {
    const int XW = kXC + 2 * P.rp;
    const size_t smem = (size_t)XW * (kLC + 2 * P.rl + kLC) * sizeof(float);
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_lsf_psfx, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_done = true;
    }
    dim3 g1((P.n_lambda + kLC - 1) / kLC, (P.nx + kXC - 1) / kXC, P.ny);
    k_lsf_psfx<<<g1, 256, smem, st>>>(P, in, tmp);
    const long long plane = (long long)P.nx * P.n_lambda;
    dim3 g2((unsigned)((plane + 255) / 256), (P.ny + kYC - 1) / kYC);
    k_psfy_noise<<<g2, 256, 0, st>>>(P, tmp, out);
    return 2;
}

}  // namespace rubix
