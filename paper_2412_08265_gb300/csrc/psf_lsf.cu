// psf_lsf.cu -- observational effects (Sec. 3: the cube is convolved with the
// instrument's point-spread and line-spread functions and noise is added;
// Sec. 4: both functions are Gaussian).
//
// The 3-D kernel is separable, g(dy) g(dx) h(dj), with zero padding on every
// axis. For the radii of the instruments used here a single fused pass
// (k_psf_lsf_fused, below) reads the cube once and writes it once. Other radii
// take two passes through an intermediate cube:
//   pass 1 (k_lsf_psfx): one CTA per (wavelength chunk, x chunk, row y) loads
//     the row segment with its halos into shared memory, applies the LSF along
//     wavelength and then the PSF along x, and writes an intermediate cube;
//   pass 2 (k_psfy_noise): each thread owns one (x, wavelength) column of a
//     y-chunk and applies the PSF along y, then optional Philox noise.
// All global accesses run along wavelength (the fastest axis): coalesced.
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


// ----------------------------------------------------------------------------
// Fused single pass for the common radii (compile-time rp, rl): one CTA owns an
// (x block of kFX spaxels, wavelength chunk of kFL = 32 bins, y band of kFY
// rows) and streams the input rows of its band, plus rp halo rows, through a
// cp.async pipeline (zero fill outside the cube). For each input row: PSF along
// x into shared memory (each warp its own output columns, over the tile's
// bins and the LSF halo; lanes run along wavelength), then LSF along
// wavelength; the value of input row y_in is added, with weight
// gp[m], to the register accumulator of output row y_in - rp + m (the 2 rp + 1
// accumulators of each owned (x, wavelength) rotate with the row, the loop
// being unrolled by 2 rp + 1 so their indices are static). After row y_in the
// accumulator of output row y_in - rp is complete: noise is added and it is
// written once. The cube is read once (plus halos) and written once.
// ----------------------------------------------------------------------------
#ifndef RUBIX_PSF_STAGES
#define RUBIX_PSF_STAGES 3      // input rows in flight (cp.async pipeline depth)
#endif
#ifndef RUBIX_PSF_FX
#define RUBIX_PSF_FX 32         // spaxels along x per CTA (a multiple of 8)
#endif
#ifndef RUBIX_PSF_FY
#define RUBIX_PSF_FY 50         // output rows along y per CTA
#endif
constexpr int kFX = RUBIX_PSF_FX, kFL = 32, kFY = RUBIX_PSF_FY;  // kFL must equal the warp width
constexpr int kFThreads = 256;
constexpr int kFWarps = kFThreads / 32;
constexpr int kFXW = kFX / kFWarps;          // output x rows owned by each warp
constexpr int kFStages = RUBIX_PSF_STAGES;

template <int RP, int RL>
constexpr size_t fused_smem_bytes() {
    return sizeof(float) * ((size_t)kFStages * (kFX + 2 * RP) * (kFL + 2 * RL) + (size_t)kFX * (kFL + 2 * RL));
}

__device__ __forceinline__ float add_noise(float v, long long idx, const ConvParams& P) {
    U4 c;
    c.x = (uint32_t)idx;
    c.y = (uint32_t)((unsigned long long)idx >> 32);
    c.z = 0u;
    c.w = 0u;
    const U4 r = philox4x32_10(c, P.seed_lo, P.seed_hi);
    const float u1 = (float)((r.x >> 8) + 1u) * (1.0f / 16777216.0f);  // (0, 1]
    const float u2 = (float)(r.y >> 8) * (1.0f / 16777216.0f);         // [0, 1)
    const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    return fmaf(fabsf(v) * P.noise_inv_s2n, z, v);
}

template <int RP, int RL>
__global__ void __launch_bounds__(kFThreads) k_psf_lsf_fused(const ConvParams P, const float* __restrict__ in,
                                                             float* __restrict__ out) {
    constexpr int XW = kFX + 2 * RP, LW = kFL + 2 * RL, NR = 2 * RP + 1;
    extern __shared__ float sm[];
    float* s_in = sm;                        // [kFStages][XW][LW]
    float* s_x = s_in + kFStages * XW * LW;  // [kFX][LW]   PSF-x output (row xo written and read by its warp)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * kFL;
    const int x0 = blockIdx.y * kFX;
    const int y0 = blockIdx.z * kFY;
    const int y1 = min(y0 + kFY, P.ny);
    const int nx = P.nx, ny = P.ny, nl = P.n_lambda;
    const int n_rows = (y1 - y0) + 2 * RP;   // input rows y0 - RP .. y1 + RP - 1
    float gl[2 * RL + 1], gp[NR];
#pragma unroll
    for (int d = 0; d <= 2 * RL; ++d) gl[d] = P.gl[d];
#pragma unroll
    for (int d = 0; d < NR; ++d) gp[d] = P.gp[d];

    auto load_row = [&](int i, int buf) {
        const int y = y0 - RP + i;
        float* dst = s_in + buf * XW * LW;
        const bool yok = (y >= 0 && y < ny);
        for (int xi = warp; xi < XW; xi += kFWarps) {
            const int x = x0 - RP + xi;
            const bool xok = yok && x >= 0 && x < nx;
            const float* row = in + ((long long)(xok ? y : 0) * nx + (xok ? x : 0)) * nl;
#pragma unroll
            for (int l = lane; l < LW; l += 32) {
                const int j = j0 - RL + l;
                const bool ok = xok && j >= 0 && j < nl;
                cp_async4(dst + xi * LW + l, ok ? row + j : in, ok);
            }
        }
        cp_async_commit();
    };

    float acc[kFXW][NR];
#pragma unroll
    for (int k = 0; k < kFXW; ++k)
#pragma unroll
        for (int m = 0; m < NR; ++m) acc[k][m] = 0.f;

    for (int k = 0; k < kFStages - 1; ++k) {
        if (k < n_rows) load_row(k, k);
        else cp_async_commit();
    }
    int buf = 0;
    const int j = j0 + lane;
    for (int ib = 0; ib < n_rows; ib += NR) {
#pragma unroll
        for (int ph = 0; ph < NR; ++ph) {   // input row i = ib + ph; accumulator of row y_in - RP + m is (ph + m) % NR
            const int i = ib + ph;
            if (i < n_rows) {
                const int ahead = i + kFStages - 1;
                int abuf = buf + kFStages - 1;
                if (abuf >= kFStages) abuf -= kFStages;
                if (ahead < n_rows) load_row(ahead, abuf);  // that buffer was read in iteration i - 1
                else cp_async_commit();
                cp_async_wait<kFStages - 1>();
                __syncthreads();  // row i landed
                const float* src = s_in + buf * XW * LW;
                if (++buf == kFStages) buf = 0;
#pragma unroll
                for (int k = 0; k < kFXW; ++k) {
                    const int xo = warp + k * kFWarps;
                    for (int l = lane; l < LW; l += 32) {
                        const float* c = src + xo * LW + l;
                        float a = 0.f;
#pragma unroll
                        for (int d = 0; d < NR; ++d) a = fmaf(gp[d], c[d * LW], a);
                        s_x[xo * LW + l] = a;
                    }
                }
                __syncthreads();  // every warp is done with row i's input buffer
                const int y_done = y0 + i - 2 * RP;  // output row completed by this input row
#pragma unroll
                for (int k = 0; k < kFXW; ++k) {
                    const int xi = warp + k * kFWarps;
                    const float* r = s_x + xi * LW + lane;
                    float v = 0.f;
#pragma unroll
                    for (int d = 0; d <= 2 * RL; ++d) v = fmaf(gl[d], r[d], v);
#pragma unroll
                    for (int m = 0; m < NR; ++m) acc[k][(ph + m) % NR] = fmaf(gp[m], v, acc[k][(ph + m) % NR]);
                    // accumulator (ph + 0) % NR holds output row y_in - RP = y_done: complete
                    float& done = acc[k][ph % NR];
                    const int x = x0 + xi;
                    if (y_done >= y0 && x < nx && j < nl) {
                        const long long idx = ((long long)y_done * nx + x) * nl + j;
                        out[idx] = (P.noise_inv_s2n > 0.f) ? add_noise(done, idx, P) : done;
                    }
                    done = 0.f;
                }
            }
        }
    }
}

template <int RP, int RL>
static bool launch_fused(const ConvParams& P, const float* in, float* out, cudaStream_t st) {
    constexpr size_t smem = fused_smem_bytes<RP, RL>();
    static_assert(smem <= 200 * 1024, "fused PSF/LSF tile does not fit shared memory");
    // per launch: the attribute belongs to the current device
    if (cudaFuncSetAttribute(k_psf_lsf_fused<RP, RL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return false;
    dim3 g((P.n_lambda + kFL - 1) / kFL, (P.nx + kFX - 1) / kFX, (P.ny + kFY - 1) / kFY);
    k_psf_lsf_fused<RP, RL><<<g, kFThreads, smem, st>>>(P, in, out);
    return true;
}

// Radii with a fused instantiation: the PSF of FWHM 1.5 spaxels (rp = 3) and
// LSFs of sigma 1.2 A on 1.25 A or 3 A bins (rl = 4, 2), plus neighbours.
#define RUBIX_FUSED_RADII(X) X(3, 4) X(3, 2) X(3, 0) X(0, 4) X(0, 2) X(2, 4) X(4, 4) X(3, 3) X(3, 5)

static bool try_fused(const ConvParams& P, const float* in, float* out, cudaStream_t st) {
#define RUBIX_FUSED_CASE(RP_, RL_) \
    if (P.rp == RP_ && P.rl == RL_) return launch_fused<RP_, RL_>(P, in, out, st);
    RUBIX_FUSED_RADII(RUBIX_FUSED_CASE)
#undef RUBIX_FUSED_CASE
    return false;
}


// ----------------------------------------------------------------------------
// TMA variant of the fused pass for a cube whose rows are 16-byte aligned (the
// deposit's own pitched cube). One CTA owns kTX = 8 spaxels along x (one per
// warp) x kTY rows along y x kTL = kTB - 2 RLa bins. Each input row arrives
// as one 3-D TMA box (kTB = 128 bins from j0 - RLa, spaxels x0 - rp ..
// x0 + kTX + rp; zero fill outside the cube is the zero padding) in a
// kTS-stage mbarrier ring. Warp w owns output column x0 + w and lane q the
// box's bins 4q .. 4q + 3:
//   PSF along x: the lane's 4 bins of column w from the box's columns
//     w .. w + 2 rp, into the warp's own row of px (so every bin the LSF
//     needs, halo included, is computed once, by the warp that reads it);
//   LSF along wavelength from the warp's px row (lanes RLa/4 .. 31 - RLa/4,
//     whose bins are the tile's), then the rotating PSF-y register
//     accumulators.
// One CTA barrier per input row (every warp is done with the stage before it
// is refilled); px is private to its warp. The terms of each output are
// summed in the order of the cp.async kernel (PSF x, LSF, PSF y; each over
// its taps in order), so the cube is bitwise the same.
// ----------------------------------------------------------------------------
#ifndef RUBIX_PSF_TY
#define RUBIX_PSF_TY 150
#endif
#ifndef RUBIX_PSF_TSTAGES
#define RUBIX_PSF_TSTAGES 4
#endif
#ifndef RUBIX_PSF_TMINB
#define RUBIX_PSF_TMINB 4       // CTAs per SM the register budget is sized for
#endif
constexpr int kTB = 128, kTX = 8, kTThreads = 256, kTWarps = kTThreads / 32;
constexpr int kTY = RUBIX_PSF_TY, kTS = RUBIX_PSF_TSTAGES;
static_assert(kTX == kTWarps, "one output column per warp");

template <int RP, int RL>
struct TmaGeo {
    static constexpr int RLa = (RL + 3) / 4 * 4;  // wavelength halo rounded up to 16 bytes
    static constexpr int LW = kTB;                // box: bins
    static constexpr int TL = kTB - 2 * RLa;      // output bins per tile
    static constexpr int XW = kTX + 2 * RP;       // box: spaxels along x
    static constexpr int NV = 1 + RLa / 2;        // 16-byte loads per lane for 4 LSF outputs
    static constexpr int stage_floats = LW * XW;  // 512-byte rows: stages stay 128-byte aligned
    static constexpr size_t smem = 128 + (size_t)kTS * stage_floats * 4 + (size_t)kTX * kTB * 4;
};

template <int RP, int RL>
__global__ void __launch_bounds__(kTThreads, RUBIX_PSF_TMINB) k_psf_lsf_tma(const __grid_constant__ ConvParams P,
                                                           const __grid_constant__ CUtensorMap in_map,
                                                           float* __restrict__ out) {
    using G = TmaGeo<RP, RL>;
    constexpr int NR = 2 * RP + 1;
    constexpr int Q0 = G::RLa / 4, Q1 = 32 - G::RLa / 4;  // lanes whose bins are the tile's
    extern __shared__ __align__(1024) float smt[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smt);
    float* stages = smt + 32;  // 128 bytes in
    float* px = stages + kTS * G::stage_floats;  // [kTX][kTB] PSF-x output, one row per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * G::TL, x0 = blockIdx.y * kTX, y0 = blockIdx.z * kTY;
    const int y1 = min(y0 + kTY, P.ny);
    const int nx = P.nx, nl = P.n_lambda;
    const int n_rows = (y1 - y0) + 2 * RP;  // input rows y0 - RP .. y1 + RP - 1
    float gl[2 * RL + 1], gp[NR];
#pragma unroll
    for (int d = 0; d <= 2 * RL; ++d) gl[d] = P.gl[d];
#pragma unroll
    for (int d = 0; d < NR; ++d) gp[d] = P.gp[d];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int i) {  // input row i into stage i % kTS (thread 0)
        const int s = i % kTS;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[s], (uint32_t)(G::LW * G::XW * 4));
        tma_load_3d(stages + s * G::stage_floats, &in_map, &bars[s], j0 - G::RLa, x0 - RP, y0 - RP + i);
    };
    if (threadIdx.x == 0)
        for (int i = 0; i < min(kTS, n_rows); ++i) issue(i);

    float acc[NR][4];
#pragma unroll
    for (int m = 0; m < NR; ++m)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[m][u] = 0.f;
    float* prow = px + warp * kTB;
    const bool owns = lane >= Q0 && lane < Q1;
    const int x = x0 + warp;
    const int jl = j0 - G::RLa + 4 * lane;  // cube bin of the lane's first box bin

    for (int ib = 0; ib < n_rows; ib += NR) {
#pragma unroll
        for (int ph = 0; ph < NR; ++ph) {  // accumulator of output row y_in - RP + m is (ph + m) % NR
            const int i = ib + ph;
            if (i < n_rows) {
                const int s = i % kTS;
                const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((i / kTS) & 1), 2000000000ll);
                if (ok) {
                    // PSF along x: box columns warp .. warp + 2 RP, bins 4 lane .. 4 lane + 3
                    const float* src = stages + s * G::stage_floats + warp * G::LW + 4 * lane;
                    float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int d = 0; d < NR; ++d) {
                        const float4 c = *reinterpret_cast<const float4*>(src + d * G::LW);
                        a[0] = fmaf(gp[d], c.x, a[0]);
                        a[1] = fmaf(gp[d], c.y, a[1]);
                        a[2] = fmaf(gp[d], c.z, a[2]);
                        a[3] = fmaf(gp[d], c.w, a[3]);
                    }
                    *reinterpret_cast<float4*>(prow + 4 * lane) = make_float4(a[0], a[1], a[2], a[3]);
                }
                if (__syncthreads_or(!ok)) {
                    // a load did not complete in time: record it, let the copies in
                    // flight land (bounded), and stop
                    if (threadIdx.x == 0) {
                        if (P.err) atomicOr(P.err, kErrTmaTimeout);
                        for (int r = i; r < min(i + kTS, n_rows); ++r)
                            mbar_wait_bounded(&bars[r % kTS], (uint32_t)((r / kTS) & 1), 200000000ll);
                    }
                    return;
                }
                // every warp is done with stage s (and the barrier made this
                // warp's px row visible to its lanes): refill it
                if (threadIdx.x == 0 && i + kTS < n_rows) issue(i + kTS);
                const int y_done = y0 + i - 2 * RP;  // output row completed by this input row
                if (owns) {
                    // LSF along wavelength from px: bins 4 lane - RLa .. 4 lane + 3 + RLa
                    const float4* r4 = reinterpret_cast<const float4*>(prow + 4 * lane - G::RLa);
                    float v[4 * G::NV];
#pragma unroll
                    for (int c = 0; c < G::NV; ++c) {
                        const float4 t = r4[c];
                        v[4 * c] = t.x;
                        v[4 * c + 1] = t.y;
                        v[4 * c + 2] = t.z;
                        v[4 * c + 3] = t.w;
                    }
                    float o[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float b = 0.f;
#pragma unroll
                        for (int d = 0; d <= 2 * RL; ++d) b = fmaf(gl[d], v[u + d + G::RLa - RL], b);
                        o[u] = b;
                    }
#pragma unroll
                    for (int m = 0; m < NR; ++m)
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[(ph + m) % NR][u] = fmaf(gp[m], o[u], acc[(ph + m) % NR][u]);
                    float* done = acc[ph % NR];
                    if (y_done >= y0 && x < nx) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = jl + u;
                            if (j < nl) {
                                const long long idx = ((long long)y_done * nx + x) * nl + j;
                                out[idx] = (P.noise_inv_s2n > 0.f) ? add_noise(done[u], idx, P) : done[u];
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) done[u] = 0.f;
                }
                __syncwarp();  // the warp's px row is rewritten by the next input row
            }
        }
    }
}

// Radii with a TMA instantiation (the wavelength halo of at most 8 bins).
#define RUBIX_TMA_RADII(X) X(3, 4) X(3, 2) X(3, 0) X(0, 4) X(0, 2) X(2, 4) X(4, 4) X(3, 3) X(3, 5)

bool conv_tma_box(int rp, int rl, unsigned box[2]) {
#define RUBIX_TMA_BOX(RP_, RL_)                    \
    if (rp == RP_ && rl == RL_) {                  \
        box[0] = (unsigned)TmaGeo<RP_, RL_>::LW;   \
        box[1] = (unsigned)TmaGeo<RP_, RL_>::XW;   \
        return true;                               \
    }
    RUBIX_TMA_RADII(RUBIX_TMA_BOX)
#undef RUBIX_TMA_BOX
    return false;
}

template <int RP, int RL>
static bool launch_tma(const ConvParams& P, const CUtensorMap* map, float* out, cudaStream_t st) {
    constexpr size_t smem = TmaGeo<RP, RL>::smem;
    static_assert(smem <= 200 * 1024, "TMA PSF/LSF tile does not fit shared memory");
    if (cudaFuncSetAttribute(k_psf_lsf_tma<RP, RL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return false;
    constexpr int TL = TmaGeo<RP, RL>::TL;
    dim3 g((P.n_lambda + TL - 1) / TL, (P.nx + kTX - 1) / kTX, (P.ny + kTY - 1) / kTY);
    k_psf_lsf_tma<RP, RL><<<g, kTThreads, smem, st>>>(P, *map, out);
    return true;
}

static bool try_tma(const ConvParams& P, const CUtensorMap* map, float* out, cudaStream_t st) {
#define RUBIX_TMA_CASE(RP_, RL_) \
    if (P.rp == RP_ && P.rl == RL_) return launch_tma<RP_, RL_>(P, map, out, st);
    RUBIX_TMA_RADII(RUBIX_TMA_CASE)
#undef RUBIX_TMA_CASE
    return false;
}

bool psf_lsf_needs_tmp(int rp, int rl) {
#define RUBIX_FUSED_HAS(RP_, RL_) \
    if (rp == RP_ && rl == RL_) return false;
    RUBIX_FUSED_RADII(RUBIX_FUSED_HAS)
#undef RUBIX_FUSED_HAS
    return true;
}

int launch_psf_lsf(const ConvParams& P, const float* in, int in_pitch, const CUtensorMap* in_map, float* tmp,
                   float* out, cudaStream_t st) {
    if (in_map && try_tma(P, in_map, out, st)) return 1;
    if (in_pitch != P.n_lambda) return -1;  // the cp.async kernels read dense rows
    if (try_fused(P, in, out, st)) return 1;
    // generic radii: two passes through an intermediate cube
    const int XW = kXC + 2 * P.rp;
    const size_t smem = (size_t)XW * (kLC + 2 * P.rl + kLC) * sizeof(float);
    cudaFuncSetAttribute(k_lsf_psfx, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    dim3 g1((P.n_lambda + kLC - 1) / kLC, (P.nx + kXC - 1) / kXC, P.ny);
    k_lsf_psfx<<<g1, 256, smem, st>>>(P, in, tmp);
    const long long plane = (long long)P.nx * P.n_lambda;
    dim3 g2((unsigned)((plane + 255) / 256), (P.ny + kYC - 1) / kYC);
    k_psfy_noise<<<g2, 256, 0, st>>>(P, tmp, out);
    return 2;
}

}  // namespace rubix
