// engine.cu -- host side of the forward model: SSP state + deposit tiling,
// per-galaxy plans, and the enqueue sequence of one forward (see engine.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

namespace rubix {

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
static thread_local std::string g_err;

rubix_status fail(rubix_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}
void set_last_error(const char* msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? RUBIX_ERR_OOM : RUBIX_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    } while (0)

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------
namespace {

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled_t get_encode_tiled() {
    static PFN_encodeTiled_t fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled_t>(p);
    });
    return fn;
}

// Round-to-nearest-even FP32 -> BF16 (bit manipulation; NaN kept quiet).
uint16_t f32_to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

void gauss_kernel(double sigma, int r, float* out) {
    std::vector<double> k(2 * r + 1);
    double s = 0.0;
    for (int d = -r; d <= r; ++d) {
        k[d + r] = std::exp(-(double)d * d / (2.0 * sigma * sigma));
        s += k[d + r];
    }
    for (int d = -r; d <= r; ++d) out[d + r] = (float)(k[d + r] / s);
}

int kernel_radius(double sigma, int r) {
    if (r > 0) return r;
    if (!(sigma > 0.0)) return 0;
    return (int)std::ceil(4.0 * sigma);
}

template <typename T>
cudaError_t dalloc_sync(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

}  // namespace

int sm_count() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev >= 64) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }
    int n = __atomic_load_n(&cache[dev], __ATOMIC_RELAXED);
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        __atomic_store_n(&cache[dev], n, __ATOMIC_RELAXED);
    }
    return n;
}

// ----------------------------------------------------------------------------
// validation
// ----------------------------------------------------------------------------
rubix_status validate_ssp(const rubix_ssp_grid* ssp) {
    if (!ssp) return fail(RUBIX_ERR_INVALID_ARG, "ssp is NULL");
    if (ssp->n_age < 1 || ssp->n_Z < 1 || ssp->n_lambda < 2 || ssp->n_lambda > 16384)
        return fail(RUBIX_ERR_INVALID_ARG, "SSP sizes out of range (n_age, n_Z >= 1, 2 <= n_lambda <= 16384)");
    if ((long long)ssp->n_age * ssp->n_Z > 65535) return fail(RUBIX_ERR_INVALID_ARG, "more than 65535 templates");
    if (!ssp->log10_age_nodes || !ssp->log10_Z_nodes || !ssp->spectra)
        return fail(RUBIX_ERR_INVALID_ARG, "SSP arrays must be non-NULL host pointers");
    for (int i = 1; i < ssp->n_age; ++i)
        if (!(ssp->log10_age_nodes[i] > ssp->log10_age_nodes[i - 1]))
            return fail(RUBIX_ERR_INVALID_ARG, "age nodes not strictly increasing");
    for (int i = 1; i < ssp->n_Z; ++i)
        if (!(ssp->log10_Z_nodes[i] > ssp->log10_Z_nodes[i - 1]))
            return fail(RUBIX_ERR_INVALID_ARG, "Z nodes not strictly increasing");
    if (!(ssp->dlambda > 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "SSP dlambda must be > 0");
    if (ssp->storage_dtype < 0 || ssp->storage_dtype > 2) return fail(RUBIX_ERR_INVALID_ARG, "bad storage_dtype");
    return RUBIX_OK;
}

rubix_status validate_telescope(const rubix_telescope* tel, double ssp_dlambda) {
    if (!tel) return fail(RUBIX_ERR_INVALID_ARG, "telescope is NULL");
    if (tel->nx < 1 || tel->ny < 1 || tel->ny > 65535 || (long long)tel->nx * tel->ny >= (1ll << 24))
        return fail(RUBIX_ERR_INVALID_ARG, "nx, ny out of range (ny <= 65535, nx*ny < 2^24)");
    if (!(tel->spaxel_size > 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "spaxel_size must be > 0");
    if (tel->n_lambda < 1 || tel->n_lambda > 8192) return fail(RUBIX_ERR_INVALID_ARG, "n_lambda must be in [1, 8192]");
    if (!(tel->dlambda > 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "dlambda must be > 0");
    if (!(tel->psf_fwhm >= 0.0) || !(tel->lsf_sigma >= 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "negative PSF/LSF width");
    if (!(tel->z_cosmo > -1.0)) return fail(RUBIX_ERR_INVALID_ARG, "z_cosmo must be > -1");
    if (tel->resample != 0 && tel->resample != 1) return fail(RUBIX_ERR_INVALID_ARG, "resample must be 0 or 1");
    if (!(tel->row_lo == 0 && tel->row_hi == 0) && !(tel->row_lo >= 0 && tel->row_lo < tel->row_hi && tel->row_hi <= tel->ny))
        return fail(RUBIX_ERR_INVALID_ARG, "row window must satisfy 0 <= row_lo < row_hi <= ny (or 0, 0 for all rows)");
    if (tel->dlambda / ((1.0 + tel->z_cosmo) * ssp_dlambda) > 3.0)
        return fail(RUBIX_ERR_INVALID_ARG, "instrument bins wider than 3 SSP steps are not supported");
    const double sp = tel->psf_fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const double sl = tel->lsf_sigma / tel->dlambda;
    if ((sp > 0.0 && kernel_radius(sp, tel->psf_radius) > kMaxRadius) ||
        (sl > 0.0 && kernel_radius(sl, tel->lsf_radius) > kMaxRadius))
        return fail(RUBIX_ERR_INVALID_ARG, "PSF/LSF radius > 64");
    return RUBIX_OK;
}

rubix_status check_particles(const rubix_particles* p) {
    if (!p) return fail(RUBIX_ERR_INVALID_ARG, "particles is NULL");
    if (p->n < 0 || p->n > (1ll << 30)) return fail(RUBIX_ERR_INVALID_ARG, "n out of range");
    if (p->n == 0) return RUBIX_OK;
    if (!p->x || !p->y || !p->mass || !p->age || !p->Z) return fail(RUBIX_ERR_INVALID_ARG, "x, y, mass, age, Z required");
    if (p->preprojected) {
        if (!p->v_los) return fail(RUBIX_ERR_INVALID_ARG, "v_los required when preprojected");
    } else {
        if (!p->z || !p->vy || !p->vz) return fail(RUBIX_ERR_INVALID_ARG, "z, vy, vz required when not preprojected");
        if (!p->vx && p->azimuth != 0.0) return fail(RUBIX_ERR_INVALID_ARG, "vx required when azimuth != 0");
    }
    return RUBIX_OK;
}

void orientation_matrix(double inclination, double azimuth, double position_angle, double R[9], double Di[3],
                        double Da[2]) {
    const double ca = std::cos(azimuth), sa = std::sin(azimuth);
    const double ci = std::cos(inclination), si = std::sin(inclination);
    const double cq = std::cos(position_angle), sq = std::sin(position_angle);
    const double cisa = ci * sa, cica = ci * ca;
    R[0] = cq * ca - sq * cisa;
    R[1] = -(cq * sa) - sq * cica;
    R[2] = sq * si;
    R[3] = sq * ca + cq * cisa;
    R[4] = cq * cica - sq * sa;
    R[5] = -(cq * si);
    R[6] = si * sa;
    R[7] = si * ca;
    R[8] = ci;
    Di[0] = cisa;
    Di[1] = cica;
    Di[2] = -si;
    Da[0] = si * ca;
    Da[1] = -(si * sa);
}

int window_rows(const rubix_telescope* tel) { return (tel->row_hi > 0) ? tel->row_hi - tel->row_lo : tel->ny; }

bool same_wavelength_grid(const SspState& S, const rubix_telescope* tel) {
    return tel->n_lambda == S.n_lambda && tel->lambda0 == S.lambda0 && tel->dlambda == S.dlambda &&
           tel->z_cosmo == S.z_cosmo;
}

// ----------------------------------------------------------------------------
// SSP state
// ----------------------------------------------------------------------------
void ssp_state_destroy(SspState* S) {
    if (!S) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    void* ptrs[] = {S->d_quad, S->d_quad16, S->d_la, S->d_lz, S->d_tile_klo, S->d_err, S->d_slow};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    cudaSetDevice(prev);
    delete S;
}

rubix_status ssp_state_create(const rubix_ssp_grid* ssp, const rubix_telescope* tel, SspState** out) {
    *out = nullptr;
    rubix_status st = validate_ssp(ssp);
    if (st != RUBIX_OK) return st;
    st = validate_telescope(tel, ssp->dlambda);
    if (st != RUBIX_OK) return st;
    SspState* h = new SspState();
    auto bail = [&](rubix_status s) {
        ssp_state_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(RUBIX_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->n_lambda = tel->n_lambda;
    h->lambda0 = tel->lambda0;
    h->dlambda = tel->dlambda;
    h->z_cosmo = tel->z_cosmo;

    // ---- SSP grid: sizes and node vectors (the templates go to the device as
    // cell quads, below) ----
    SspDev& S = h->ssp;
    S.dtype = ssp->storage_dtype;
    S.n_age = ssp->n_age;
    S.n_Z = ssp->n_Z;
    S.n_t = ssp->n_age * ssp->n_Z;
    S.n_ls = ssp->n_lambda;
    S.ls0 = ssp->lambda0;
    S.dls = ssp->dlambda;
    {
        std::vector<float> la(S.n_age), lz(S.n_Z);
        for (int i = 0; i < S.n_age; ++i) la[i] = (float)ssp->log10_age_nodes[i];
        for (int i = 0; i < S.n_Z; ++i) lz[i] = (float)ssp->log10_Z_nodes[i];
        if (dalloc_sync(&h->d_la, S.n_age) || dalloc_sync(&h->d_lz, S.n_Z) || dalloc_sync(&h->d_err, 4) ||
            dalloc_sync(&h->d_slow, 1))
            return bail(fail(RUBIX_ERR_OOM, "SSP state alloc"));
        cudaMemcpy(h->d_la, la.data(), la.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(h->d_lz, lz.data(), lz.size() * 4, cudaMemcpyHostToDevice);
        cudaMemset(h->d_err, 0, 16);
        cudaMemset(h->d_slow, 0, 8);
        S.la_nodes = h->d_la;
        S.lz_nodes = h->d_lz;
    }

    // ---- cell quads: for SSP cell (ia, iz) and node k, the four bilinear
    // corners (ia,iz) (ia+1,iz) (ia,iz+1) (ia+1,iz+1), node-major
    // [n_ls][n_cells], in the storage dtype: a float4 of FP32 values, or an
    // 8-byte uint2 of BF16 / FP16 bit patterns (x = corner 0 | corner 1 << 16,
    // y = corner 2 | corner 3 << 16) that the kernels widen to FP32 exactly ----
    h->cz = std::max(S.n_Z - 1, 1);
    const int ca = std::max(S.n_age - 1, 1);
    h->n_cells = ca * h->cz;
    h->qdt = (S.dtype == RUBIX_F32) ? 0 : (S.dtype == RUBIX_BF16 ? 1 : 2);
    {
        const int da = (S.n_age > 1) ? 1 : 0, dz = (S.n_Z > 1) ? 1 : 0;
        auto tpl = [&](int ia, int iz, int k) { return (float)ssp->spectra[((size_t)ia * S.n_Z + iz) * S.n_ls + k]; };
        auto bits16 = [&](float f) -> uint32_t {
            if (S.dtype == RUBIX_BF16) return f32_to_bf16(f);
            const __half hv = __float2half_rn(f);
            uint16_t b;
            std::memcpy(&b, &hv, 2);
            return b;
        };
        const size_t nq = (size_t)S.n_ls * h->n_cells;
        if (h->qdt == 0) {
            std::vector<float4> q(nq);
            for (int ia = 0; ia < ca; ++ia)
                for (int iz = 0; iz < h->cz; ++iz) {
                    const int c = ia * h->cz + iz;
                    for (int k = 0; k < S.n_ls; ++k)
                        q[(size_t)k * h->n_cells + c] = make_float4(tpl(ia, iz, k), tpl(ia + da, iz, k),
                                                                    tpl(ia, iz + dz, k), tpl(ia + da, iz + dz, k));
                }
            if (dalloc_sync(&h->d_quad, q.size())) return bail(fail(RUBIX_ERR_OOM, "quad alloc"));
            if (cudaMemcpy(h->d_quad, q.data(), q.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(RUBIX_ERR_CUDA, "quad copy"));
        } else {
            std::vector<uint2> q(nq);
            for (int ia = 0; ia < ca; ++ia)
                for (int iz = 0; iz < h->cz; ++iz) {
                    const int c = ia * h->cz + iz;
                    for (int k = 0; k < S.n_ls; ++k) {
                        uint2 v;
                        v.x = bits16(tpl(ia, iz, k)) | (bits16(tpl(ia + da, iz, k)) << 16);
                        v.y = bits16(tpl(ia, iz + dz, k)) | (bits16(tpl(ia + da, iz + dz, k)) << 16);
                        q[(size_t)k * h->n_cells + c] = v;
                    }
                }
            if (dalloc_sync(&h->d_quad16, q.size())) return bail(fail(RUBIX_ERR_OOM, "quad alloc"));
            if (cudaMemcpy(h->d_quad16, q.data(), q.size() * sizeof(uint2), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(RUBIX_ERR_CUDA, "quad copy"));
        }
    }

    // ---- deposit tiling: wavelength tiles and the quad slab staged per tile
    // and age band. A band's slab holds ncb cells (odd) x slab_w nodes: the
    // tile's R rounds of 31 bins plus a Doppler halo of +-RUBIX_DEP_VHALO.
    // Among the band sizes that fit, take the one with the lowest estimated
    // cost per particle: n_tiles * (per-particle setup + R rounds + bands). ----
    const double A0 = tel->dlambda / ((1.0 + tel->z_cosmo) * S.dls);
    const double v_halo = RUBIX_DEP_VHALO;
    const double lam_max = (tel->lambda0 + (tel->n_lambda - 1) * tel->dlambda) / (1.0 + tel->z_cosmo);
    const int shift = (int)std::ceil(lam_max / S.dls * (v_halo / kC_kms) / (1.0 - v_halo / kC_kms));
    long long budget = (long long)h->smem_optin - kDepHeader;
    if (RUBIX_DEP_CTAS > 1) {
        int per_sm = 0;
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
        budget = std::min<long long>(budget, per_sm / RUBIX_DEP_CTAS - 1024 - kDepHeader);  // 1 KB reserved per CTA
    }
    struct Geo { int apb, bands, ncb, box_w, n_boxes, slab_w, R; double cost; };
    Geo best{0, 0, 0, 0, 0, 0, 0, 1e300};
    const bool fast_A = A0 <= 1.0 && A0 > 1.0 - 1.0 / 31.0;
    for (int apb = ca; apb >= 1; --apb) {
        const int bands = (ca + apb - 1) / apb;
        if (bands > kMaxBands) break;
        if (RUBIX_DEP_BANDS > 0 && bands != std::min(RUBIX_DEP_BANDS, ca)) continue;
        int ncb = apb * h->cz;
        ncb += (ncb % 2 == 0) ? 1 : 0;
        if (4 * ncb > 256) continue;  // TMA box: at most 256 elements per dimension
        const long long wmax = budget / ((long long)ncb * (long long)sizeof(float4));
        if (wmax < 64) continue;
        // each box lands 128-byte aligned in shared memory (TMA destination
        // rule): box_w * ncb * 16 bytes a multiple of 128, i.e. box_w % 8 == 0
        const int n_boxes = (int)((wmax + 255) / 256);
        const int box_w = (int)(wmax / n_boxes) / 8 * 8;
        const int slab_w = n_boxes * box_w;
        int R = 0;
        for (int r = RUBIX_DEP_RMAX; r >= 1; --r)
            if (31 * r + 1 + 2 * shift + 2 <= slab_w) { R = r; break; }
        if (R == 0) continue;
        if (!fast_A) R = std::min(R, 2);
        const int n_tiles = (tel->n_lambda + 31 * R - 1) / (31 * R);
        const double cost = n_tiles * (40.0 + 15.0 * R + 6.0 * bands);
        if (cost < best.cost) best = Geo{apb, bands, ncb, box_w, n_boxes, slab_w, R, cost};
    }
    if (best.R == 0) {
        // no slab fits (very wide Doppler halo): global-memory path only. ncb
        // = 0 fails every kernel's "cell inside the slab" test, so that no
        // particle takes a fast path into the (absent) slab.
        best = Geo{ca, 1, 0, 0, 0, 0, 1, 0.0};
    }
    h->apb = best.apb;
    h->n_bands = best.bands;
    h->ncb = best.ncb;
    h->box_w = best.box_w;
    h->n_boxes = best.n_boxes;
    h->slab_w = best.slab_w;
    for (int b = 0; b < kMaxBands; ++b) h->band_cell0[b] = std::min(b * best.apb, ca - 1) * h->cz;
    h->tile_w = 31 * best.R;
    h->n_tiles = (tel->n_lambda + h->tile_w - 1) / h->tile_w;
    std::vector<int> klo(h->n_tiles, 0);
    for (int t = 0; t < h->n_tiles; ++t) {
        // nodes the tile's fast path reads: K0 .. K0 + 31 R with K0 within
        // +-shift of the zero-velocity position t00 of its first bin
        const int j0 = t * h->tile_w;
        const double t00 = ((tel->lambda0 + j0 * tel->dlambda) / (1.0 + tel->z_cosmo) - S.ls0) / S.dls;
        const double need = 2.0 * shift + h->tile_w + 3.0;
        const double k = std::floor(t00 - shift - 1.0 - 0.5 * (h->slab_w - need));
        klo[t] = (int)std::max(-1e6, std::min(k, 1e6));
    }
    if (dalloc_sync(&h->d_tile_klo, h->n_tiles)) return bail(fail(RUBIX_ERR_OOM, "tile alloc"));
    cudaMemcpy(h->d_tile_klo, klo.data(), klo.size() * 4, cudaMemcpyHostToDevice);
    static_assert(kDepHeader % 128 == 0, "slab must start 128-byte aligned");
    if ((h->box_w * h->ncb * (int)sizeof(float4)) % 128 != 0)
        return bail(fail(RUBIX_ERR_CUDA, "internal: TMA box of %d x %d quads is not 128-byte aligned", h->box_w, h->ncb));
    h->dep_smem = deposit_smem_bytes(h->ncb, h->slab_w);
    h->dep_ctas = h->n_sm * RUBIX_DEP_CTAS;
    if (h->slab_w > 0 && h->qdt == 0) {
        PFN_encodeTiled_t enc = get_encode_tiled();
        if (!enc) return bail(fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"));
        // 2-D view of the quads: x = 4 floats per cell (innermost), y = node
        cuuint64_t gdim[2] = {(cuuint64_t)4 * h->n_cells, (cuuint64_t)S.n_ls};
        cuuint64_t gstr[1] = {(cuuint64_t)h->n_cells * sizeof(float4)};
        cuuint32_t box[2] = {(cuuint32_t)(4 * h->ncb), (cuuint32_t)h->box_w};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&h->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->d_quad, gdim, gstr, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return bail(fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r));
    }
    if (cudaDeviceSynchronize() != cudaSuccess)
        return bail(fail(RUBIX_ERR_CUDA, "SSP state: %s", cudaGetErrorString(cudaGetLastError())));
    *out = h;
    return RUBIX_OK;
}

// ----------------------------------------------------------------------------
// plans
// ----------------------------------------------------------------------------
namespace {

struct Buf {
    void** ptr;
    size_t bytes;
};

// Every device buffer of a plan for n particles, with its size.
std::vector<Buf> plan_buffers(Plan* P, const SspState& S, int n_s, int n_lambda, long long n, bool with_out,
                              bool with_grad, bool need_tmp, bool staging, int pitch0) {
    const size_t N = (size_t)std::max(n, 1ll);
    const long long item_cap = (long long)n_s + n / S.chunk + 2;
    const long long part_cap = 2 * (n / S.chunk) + 2;
    const size_t cube = (size_t)n_s * n_lambda * sizeof(float);
    std::vector<Buf> v;
    if (staging)
        v = {{(void**)&P->d_x, 4 * N},    {(void**)&P->d_y, 4 * N},    {(void**)&P->d_z, 4 * N},
             {(void**)&P->d_vx, 4 * N},   {(void**)&P->d_vy, 4 * N},   {(void**)&P->d_vz, 4 * N},
             {(void**)&P->d_vlos, 4 * N},
             {(void**)&P->d_mass, 4 * N}, {(void**)&P->d_age, 4 * N}, {(void**)&P->d_Z, 4 * N}};
    const std::vector<Buf> rest = {
        {(void**)&P->d_key, 4 * N},
        {(void**)&P->d_keys_tmp, 4 * N}, {(void**)&P->d_vals_tmp, 4 * N}, {(void**)&P->d_skeys, 4 * N},
        {(void**)&P->d_perm, 4 * N}, {(void**)&P->d_pin, 16 * N},
        {(void**)&P->d_sort_scratch, 4 * sort_scratch_ints((long long)N)},
        {(void**)&P->d_items, sizeof(Item) * (size_t)item_cap}, {(void**)&P->d_rec, sizeof(DepRec) * N},
        {(void**)&P->d_prec, sizeof(PartRec) * N},
        {(void**)&P->d_partials, 4 * (size_t)part_cap * n_lambda},
        {(void**)&P->d_seg_off, 4 * ((size_t)n_s * S.n_bands + 2)}, {(void**)&P->d_n_items, 4 * ((size_t)n_s + 1)},
        {(void**)&P->d_n_parts, 4 * ((size_t)n_s + 1)}, {(void**)&P->d_item_off, 4 * ((size_t)n_s + 1)},
        {(void**)&P->d_part_off, 4 * ((size_t)n_s + 1)},
        {(void**)&P->d_scan_scratch, 4 * (scan_scratch_ints(n_s + 1) + 16)},
        {(void**)&P->d_cube0, (size_t)n_s * std::max(pitch0, n_lambda) * sizeof(float)},
        {(void**)&P->d_job_cost, 8 * (size_t)(kMaxJobs + 1)},
    };
    v.insert(v.end(), rest.begin(), rest.end());
    // with gradients d_tmp also holds the loss gradient in pitched rows, so that
    // the transposed PSF/LSF reads it through a TMA map like the forward
    if (need_tmp || with_grad)
        v.push_back({(void**)&P->d_tmp, with_grad ? (size_t)n_s * std::max(pitch0, n_lambda) * sizeof(float) : cube});
    if (with_out) v.push_back({(void**)&P->d_out, cube});
    if (with_grad) {
        v.push_back({(void**)&P->d_contrib, 8 * kGlobal * N});
        v.push_back({(void**)&P->d_dvda, 8 * N});
        v.push_back({(void**)&P->d_red, 8 * 1024});
        v.push_back({(void**)&P->d_wu, 16 * N});
        v.push_back({(void**)&P->d_adjpart, 16 * N * (size_t)std::max(S.n_tiles, 1)});
    }
    return v;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int conv_radius_psf(const rubix_telescope* tel) {
    const double sp = tel->psf_fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    return sp > 0.0 ? kernel_radius(sp, tel->psf_radius) : 0;
}
// Row stride of the pre-convolution cube: 16-byte rows when the PSF/LSF radii
// have a TMA kernel (it loads rows with 3-D TMA boxes), else dense.
int cube0_pitch(int rp, int rl, int n_lambda) {
    unsigned box[2];
    return conv_tma_box(rp, rl, box) ? (n_lambda + 3) / 4 * 4 : n_lambda;
}

int conv_radius_lsf(const rubix_telescope* tel) {
    const double sl = tel->lsf_sigma / tel->dlambda;
    return sl > 0.0 ? kernel_radius(sl, tel->lsf_radius) : 0;
}

}  // namespace

bool conv_params(const rubix_telescope* tel, int rows, ConvParams* C) {
    C->nx = tel->nx;
    C->ny = rows;
    C->n_lambda = tel->n_lambda;
    const double sp = tel->psf_fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    const double sl = tel->lsf_sigma / tel->dlambda;
    C->rp = conv_radius_psf(tel);
    C->rl = conv_radius_lsf(tel);
    if (sp > 0.0) gauss_kernel(sp, C->rp, C->gp); else C->gp[0] = 1.f;
    if (sl > 0.0) gauss_kernel(sl, C->rl, C->gl); else C->gl[0] = 1.f;
    C->noise_inv_s2n = 0.f;
    return (sp > 0.0) || (sl > 0.0);
}

size_t plan_bytes(const SspState& S, const rubix_telescope* tel, long long n, bool with_out, bool with_grad,
                  bool staging) {
    Plan tmp;
    const int rp = conv_radius_psf(tel), rl = conv_radius_lsf(tel);
    const bool need_tmp = psf_lsf_needs_tmp(rp, rl);
    size_t total = 0;
    for (const Buf& b : plan_buffers(&tmp, S, tel->nx * window_rows(tel), tel->n_lambda, n, with_out, with_grad, need_tmp,
                                     staging, cube0_pitch(rp, rl, tel->n_lambda)))
        total += round256(b.bytes);
    return total;
}

void plan_release(Plan* P) {
    if (!P->S) return;
    const bool need_tmp = true;
    for (const Buf& b : plan_buffers(P, *P->S, P->n_s, P->tel.n_lambda, P->cap, true, true, need_tmp, true, P->pitch0)) {
        if (*b.ptr) {
            if (P->alloc.async) cudaFreeAsync(*b.ptr, P->alloc.stream);
            else cudaFree(*b.ptr);
        }
        *b.ptr = nullptr;
    }
    P->bytes = 0;
    P->cap = 0;
}

// Host-side fault injection for tests: RUBIX_FAULT_ALLOC_AT=k makes the k-th
// buffer allocation of every plan fail as if the device were out of memory
// (nothing is run on the GPU; the plan's other buffers are released).
static int fault_alloc_at() {
    const char* e = std::getenv("RUBIX_FAULT_ALLOC_AT");
    return e ? std::atoi(e) : 0;
}

rubix_status plan_init(Plan* P, const SspState* S, const rubix_telescope* tel, long long n, Alloc a, bool with_out,
                       bool with_grad) {
    rubix_status st = validate_telescope(tel, S->ssp.dls);
    if (st != RUBIX_OK) return st;
    if (!same_wavelength_grid(*S, tel))
        return fail(RUBIX_ERR_INVALID_ARG, "telescope wavelength grid differs from the SSP state's");
    if (n < 0 || n > (1ll << 30)) return fail(RUBIX_ERR_INVALID_ARG, "particle count out of range");
    P->S = S;
    P->alloc = a;
    P->tel = *tel;
    if (P->tel.flux_scale == 0.0) P->tel.flux_scale = 1.0;
    P->rows = window_rows(tel);
    P->row_lo = (tel->row_hi > 0) ? tel->row_lo : 0;
    P->n_s = tel->nx * P->rows;
    P->x_lo = (-0.5 * (double)tel->nx) * tel->spaxel_size;
    P->y_lo = (-0.5 * (double)tel->ny) * tel->spaxel_size;
    P->inv_size = 1.0 / tel->spaxel_size;
    ConvParams& C = P->conv;
    P->need_conv = conv_params(tel, P->rows, &C);
    C.err = S->d_err;
    P->pitch0 = cube0_pitch(C.rp, C.rl, tel->n_lambda);
    P->has_conv_map = false;
    P->has_grad_map = false;
    P->cap = std::max(n, 1ll);
    P->item_cap = (long long)P->n_s + P->cap / S->chunk + 2;
    P->part_cap = 2 * (P->cap / S->chunk) + 2;
    const bool need_tmp = psf_lsf_needs_tmp(C.rp, C.rl);
    P->bytes = 0;
    const int fail_at = fault_alloc_at();
    int idx = 0;
    for (const Buf& b :
         plan_buffers(P, *S, P->n_s, tel->n_lambda, P->cap, with_out, with_grad, need_tmp, a.staging, P->pitch0)) {
        cudaError_t e;
        if (++idx == fail_at) e = cudaErrorMemoryAllocation;
        else if (!a.async) e = cudaMalloc(b.ptr, round256(b.bytes));
        else if (a.pool) e = cudaMallocFromPoolAsync(b.ptr, round256(b.bytes), a.pool, a.stream);
        else e = cudaMallocAsync(b.ptr, round256(b.bytes), a.stream);
        if (e != cudaSuccess) {
            *b.ptr = nullptr;
            cudaGetLastError();
            plan_release(P);
            return fail(RUBIX_ERR_OOM, "plan allocation of %zu bytes failed: %s", b.bytes, cudaGetErrorString(e));
        }
        P->bytes += round256(b.bytes);
    }
    unsigned box[2];
    if (P->pitch0 != tel->n_lambda && conv_tma_box(C.rp, C.rl, box)) {
        // 3-D view of the pre-convolution cube: x = bin (n_lambda of each
        // pitched row), y = spaxel x, z = spaxel y; zero fill outside
        PFN_encodeTiled_t enc = get_encode_tiled();
        if (!enc) {
            plan_release(P);
            return fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        }
        cuuint64_t gdim[3] = {(cuuint64_t)tel->n_lambda, (cuuint64_t)tel->nx, (cuuint64_t)P->rows};
        cuuint64_t gstr[2] = {(cuuint64_t)P->pitch0 * 4, (cuuint64_t)P->pitch0 * 4 * (cuuint64_t)tel->nx};
        cuuint32_t bx[3] = {box[0], box[1], 1};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&P->conv_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P->d_cube0, gdim, gstr, bx, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            plan_release(P);
            return fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled (PSF/LSF) failed (%d)", (int)r);
        }
        P->has_conv_map = true;
        if (with_grad && P->d_tmp) {
            // the same view of d_tmp: the loss gradient, copied into pitched rows by the backward
            r = enc(&P->grad_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P->d_tmp, gdim, gstr, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                plan_release(P);
                return fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled (PSF/LSF gradient) failed (%d)", (int)r);
            }
            P->has_grad_map = true;
        }
    }
    return RUBIX_OK;
}

rubix_status plan_grow(Plan* P, long long n) {
    if (P->alloc.async) return fail(RUBIX_ERR_INVALID_ARG, "stream-ordered plans do not grow");
    const bool with_out = P->d_out != nullptr, with_grad = P->d_contrib != nullptr;
    const SspState* S = P->S;
    const rubix_telescope tel = P->tel;
    CK(cudaDeviceSynchronize());
    plan_release(P);
    return plan_init(P, S, &tel, n + n / 8, P->alloc, with_out, with_grad);
}

// ----------------------------------------------------------------------------
// forward, in enqueued parts
// ----------------------------------------------------------------------------
namespace {

// Host inputs are copied into the plan's staging buffers; device inputs are
// read in place. arrs[] follows rubix_particles' field order.
rubix_status stage_particles(Plan& P, const rubix_particles* p, const float** arrs, cudaStream_t st) {
    const long long n = p->n;
    const float* src[10] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->v_los, p->mass, p->age, p->Z};
    float* dst[10] = {P.d_x, P.d_y, P.d_z, P.d_vx, P.d_vy, P.d_vz, P.d_vlos, P.d_mass, P.d_age, P.d_Z};
    for (int i = 0; i < 10; ++i) {
        arrs[i] = nullptr;
        if (!src[i] || n == 0) continue;
        if (p->on_device) {
            arrs[i] = src[i];
        } else if (!p->preprojected || i < 2 || i > 5) {
            // host arrays the call reads (the 3-D ones only for 3-D input)
            if (!dst[i]) return fail(RUBIX_ERR_INVALID_ARG, "host particle arrays need a plan with staging buffers");
            CK(cudaMemcpyAsync(dst[i], src[i], (size_t)n * 4, cudaMemcpyHostToDevice, st));
            arrs[i] = dst[i];
        }
    }
    if (p->preprojected) arrs[2] = arrs[3] = arrs[4] = arrs[5] = nullptr;
    else arrs[6] = nullptr;
    return RUBIX_OK;
}

AssignParams assign_params(const Plan& P, const rubix_particles* p, const float* const* arrs) {
    AssignParams A{};
    A.n = p->n;
    A.x = arrs[0];
    A.y = arrs[1];
    A.z = arrs[2];
    A.vx = arrs[3];
    A.vy = arrs[4];
    A.vz = arrs[5];
    A.v_los = arrs[6];
    A.preprojected = p->preprojected ? 1 : 0;
    orientation_matrix(p->inclination, p->azimuth, p->position_angle, A.R, A.Di, A.Da);
    A.x_lo = P.x_lo;
    A.y_lo = P.y_lo;
    A.inv_size = P.inv_size;
    A.nx = P.tel.nx;
    A.ny = P.tel.ny;
    A.row_lo = P.row_lo;
    A.rows = P.rows;
    A.n_bands = 1;
    return A;
}

}  // namespace

rubix_status enqueue_keys(Plan& P, const rubix_particles* p, int* keys_out, cudaStream_t st) {
    if (p->n > P.cap) return fail(RUBIX_ERR_INVALID_ARG, "more particles than the plan holds");
    if (p->n == 0) return RUBIX_OK;
    const float* arrs[10];
    rubix_status s = stage_particles(P, p, arrs, st);
    if (s != RUBIX_OK) return s;
    AssignParams A = assign_params(P, p, arrs);
    A.key = keys_out;
    A.pin_out = nullptr;
    launch_assign(A, st);
    CK(cudaGetLastError());
    return RUBIX_OK;
}

rubix_status enqueue_pre(Plan& P, const rubix_particles* p, cudaStream_t st, cudaEvent_t* ev) {
    NvtxRange nvtx("rubix: assign, sort, setup, items");
    const SspState& S = *P.S;
    if (p->n > P.cap) return fail(RUBIX_ERR_INVALID_ARG, "more particles than the plan holds");
    const long long n = p->n;
    const float* arrs[10];
    rubix_status s = stage_particles(P, p, arrs, st);
    if (s != RUBIX_OK) return s;
    P.launches = 0;
    P.dep_launches = 0;
    if (n > 0) {
        AssignParams A = assign_params(P, p, arrs);
        A.key = P.d_key;
        A.pin_out = P.d_pin;
        A.mass = arrs[7];
        A.Zm = arrs[9];
        A.dv_dang = P.d_dvda;  // null unless the plan keeps backward state
        A.age = arrs[8];
        A.la_nodes = S.d_la;
        A.n_age = S.ssp.n_age;
        A.apb = S.apb;
        A.n_bands = S.n_bands;
        P.launches += launch_assign(A, st);
        P.launches += launch_sort_by_key(P.d_key, n, P.n_s * S.n_bands + 1, P.d_keys_tmp, P.d_vals_tmp, P.d_skeys,
                                         P.d_perm, P.d_seg_off, P.d_sort_scratch, st);
    } else {
        CK(cudaMemsetAsync(P.d_seg_off, 0, ((size_t)P.n_s * S.n_bands + 2) * sizeof(int), st));
    }
    if (ev) cudaEventRecord(ev[1], st);
    SetupParams SP{};
    SP.ssp = S.ssp;
    SP.perm = P.d_perm;
    SP.seg_off = P.d_seg_off;
    SP.n_s = P.n_s;
    SP.n_bands = S.n_bands;
    SP.pin = P.d_pin;
    SP.l0 = P.tel.lambda0;
    SP.dl = P.tel.dlambda;
    SP.z_cosmo = P.tel.z_cosmo;
    SP.inv_c = 1.0 / kC_kms;
    SP.alpha_z = 1.0 / ((1.0 + P.tel.z_cosmo) * S.ssp.dls);
    SP.ls0_dls = S.ssp.ls0 / S.ssp.dls;
    SP.flux_scale = P.tel.flux_scale;
    SP.n_lambda = P.tel.n_lambda;
    SP.resample = P.tel.resample;
    SP.rec = P.d_rec;
    SP.prec = P.d_prec;
    SP.n_cap = P.cap;
    P.launches += launch_setup(SP, n, st);
    ItemParams IP{};
    IP.seg_off = P.d_seg_off;
    IP.n_s = P.n_s;
    IP.n_bands = S.n_bands;
    IP.chunk = S.chunk;
    IP.n_items = P.d_n_items;
    IP.n_parts = P.d_n_parts;
    IP.item_off = P.d_item_off;
    IP.part_off = P.d_part_off;
    IP.items = P.d_items;
    IP.item_cap = P.item_cap;
    IP.scan_scratch = P.d_scan_scratch;
    IP.err = S.d_err;
    P.launches += launch_items(IP, st);
    P.last_n = n;
    CK(cudaGetLastError());
    return RUBIX_OK;
}

float* deposit_target(const Plan& P, float* out, bool noise) { return (P.need_conv || noise) ? P.d_cube0 : out; }

DepJob plan_job(const Plan& P, float* target) {
    DepJob J{};
    J.rec = P.d_rec;
    J.items = P.d_items;
    J.item_off = P.d_item_off;
    J.seg_off = P.d_seg_off;
    J.cube = target;
    J.partials = P.d_partials;
    J.part_cap = P.part_cap;
    J.n_s = P.n_s;
    J.pitch = (target == P.d_cube0) ? P.pitch0 : P.tel.n_lambda;
    J.resample = P.tel.resample;
    return J;
}

int enqueue_deposit(const SspState& S, const DepJob* jobs, int n_jobs, long long* d_job_cost, cudaStream_t st) {
    NvtxRange nvtx("rubix: deposit");
    if (n_jobs < 1 || n_jobs > kMaxJobs) return -1;
    DepositParams DP{};
    DP.quad = S.d_quad;
    DP.quad16 = S.d_quad16;
    DP.qdt = S.qdt;
    DP.n_cells = S.n_cells;
    DP.n_ls = S.ssp.n_ls;
    for (int j = 0; j < n_jobs; ++j) DP.jobs[j] = jobs[j];
    DP.n_jobs = n_jobs;
    DP.job_cost = d_job_cost;
    DP.n_bands = S.n_bands;
    for (int b = 0; b < kMaxBands; ++b) DP.band_cell0[b] = S.band_cell0[b];
    DP.n_lambda = S.n_lambda;
    DP.tile_w = S.tile_w;
    DP.n_tiles = S.n_tiles;
    DP.tile_klo = S.d_tile_klo;
    DP.slab_w = S.slab_w;
    DP.ncb = S.ncb;
    DP.box_w = S.box_w;
    DP.n_boxes = S.n_boxes;
    DP.cost_c0 = S.cost_c0;
    DP.err = S.d_err;
    DP.slow_count = S.d_slow;
    return launch_deposit(DP, &S.tmap, S.dep_ctas, S.dep_threads, S.dep_smem, st);
}

int enqueue_post(Plan& P, float* target, float* out, uint64_t noise_seed, float noise_s2n, cudaStream_t st,
                 cudaEvent_t* ev) {
    NvtxRange nvtx("rubix: rows, PSF/LSF, noise");
    const int pitch = target == P.d_cube0 ? P.pitch0 : P.tel.n_lambda;
    int l = launch_zero_empty(P.d_seg_off, P.n_s, P.S->n_bands, target, pitch, P.tel.n_lambda, st);
    // d_n_parts (scanned into d_part_off by the item stage) is free here: the
    // combine's list of split spaxels
    l += launch_combine(P.d_part_off, P.n_s, P.tel.n_lambda, P.d_partials, target, pitch, P.d_n_parts, st);
    if (ev) cudaEventRecord(ev[4], st);
    const bool noise = noise_s2n > 0.f;
    if (P.need_conv || noise) {
        ConvParams C = P.conv;
        C.noise_inv_s2n = noise ? 1.0f / noise_s2n : 0.f;
        C.seed_lo = (uint32_t)noise_seed;
        C.seed_hi = (uint32_t)(noise_seed >> 32);
        l += launch_psf_lsf(C, P.d_cube0, P.pitch0, P.has_conv_map ? &P.conv_map : nullptr, P.d_tmp, out, st);
    }
    return l;
}

}  // namespace rubix
