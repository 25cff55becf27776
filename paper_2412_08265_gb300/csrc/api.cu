// api.cu -- the C ABI (include/rubix.h): handle life cycle, validation,
// device memory, TMA descriptors and the forward/backward launch sequences.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rubix.h"
#include "common.cuh"
#include "kernels.h"

using namespace rubix;

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
static thread_local std::string g_err;

static rubix_status fail(rubix_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? RUBIX_ERR_OOM : RUBIX_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

extern "C" const char* rubix_last_error_message(void) { return g_err.c_str(); }

namespace rubix {
void set_last_error(const char* msg) { g_err = msg; }
}
extern "C" const char* rubix_version(void) { return "rubix-gb300 0.1 (sm_103a)"; }

// ----------------------------------------------------------------------------
// handle
// ----------------------------------------------------------------------------
namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

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

}  // namespace

struct rubix_cube {
    int device = 0;
    int n_sm = 0;
    // SSP on device
    SspDev ssp{};
    void* d_tpl = nullptr;
    float* d_la = nullptr;
    float* d_lz = nullptr;
    int elem = 4;
    // telescope
    rubix_telescope tel{};
    int n_s = 0;
    double x_lo = 0, y_lo = 0, inv_size = 0;
    ConvParams conv{};
    bool need_conv = false;
    // deposit geometry
    int tile_w = 32, n_tiles = 0, slab_w = 0, box_rows = 0, n_boxes = 0, n_rows_alloc = 0;
    size_t dep_smem = 0;
    int* d_tile_klo = nullptr;
    CUtensorMap tmap{};
    int dep_ctas = 0, dep_threads = RUBIX_DEP_THREADS;
    int n_bands = 1, apb = 1;           // age bands of the template grid (sort key = spaxel * n_bands + band)
    int band_row0[kMaxBands] = {};
    int chunk = RUBIX_DEP_CHUNK, cost_c0 = 2;
    // scratch
    long long cap = 0;
    long long item_cap = 0, part_cap = 0;
    float *d_x = nullptr, *d_y = nullptr, *d_z = nullptr, *d_vy = nullptr, *d_vz = nullptr, *d_vlos = nullptr;
    float *d_mass = nullptr, *d_age = nullptr, *d_Z = nullptr;
    int *d_key = nullptr, *d_keys_tmp = nullptr, *d_vals_tmp = nullptr, *d_skeys = nullptr, *d_perm = nullptr;
    double* d_v = nullptr;
    int* d_sort_scratch = nullptr;
    int *d_seg_off = nullptr, *d_n_items = nullptr, *d_n_parts = nullptr, *d_item_off = nullptr,
        *d_part_off = nullptr, *d_scan_scratch = nullptr;
    Item* d_items = nullptr;
    DepRec* d_rec = nullptr;
    PartRec* d_prec = nullptr;
    float* d_partials = nullptr;
    float *d_cube0 = nullptr, *d_tmp = nullptr, *d_out = nullptr;
    unsigned* d_err = nullptr;
    unsigned long long* d_slow = nullptr;
    double *d_contrib = nullptr, *d_red = nullptr;
    // state of the last forward
    bool have_forward = false, forward_noise = false;
    long long last_n = 0;
    int launches = 0, dep_launches = 0;
    bool prof = false;
    // profiling: a ring of event sets, one set per forward since profiling was enabled
    static constexpr int kRing = 256;
    std::vector<cudaEvent_t> ring;   // kRing * 7 events, created on first enable
    int ring_next = 0, ring_count = 0;
    cudaEvent_t* ev = nullptr;       // event set of the forward being enqueued
};

static void free_scratch(rubix_cube* h) {
    void* ptrs[] = {h->d_x, h->d_y, h->d_z, h->d_vy, h->d_vz, h->d_vlos, h->d_mass, h->d_age, h->d_Z,
                    h->d_key, h->d_keys_tmp, h->d_vals_tmp, h->d_skeys, h->d_perm, h->d_v, h->d_sort_scratch,
                    h->d_items, h->d_rec, h->d_prec, h->d_partials, h->d_contrib};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->d_x = h->d_y = h->d_z = h->d_vy = h->d_vz = h->d_vlos = h->d_mass = h->d_age = h->d_Z = nullptr;
    h->d_key = h->d_keys_tmp = h->d_vals_tmp = h->d_skeys = h->d_perm = nullptr;
    h->d_v = nullptr;
    h->d_sort_scratch = nullptr;
    h->d_items = nullptr;
    h->d_rec = nullptr;
    h->d_prec = nullptr;
    h->d_partials = nullptr;
    h->d_contrib = nullptr;
    h->cap = 0;
}

static rubix_status alloc_scratch(rubix_cube* h, long long n) {
    free_scratch(h);
    if (n < 1) n = 1;
    const size_t N = (size_t)n;
    CK(dalloc(&h->d_x, N));
    CK(dalloc(&h->d_y, N));
    CK(dalloc(&h->d_z, N));
    CK(dalloc(&h->d_vy, N));
    CK(dalloc(&h->d_vz, N));
    CK(dalloc(&h->d_vlos, N));
    CK(dalloc(&h->d_mass, N));
    CK(dalloc(&h->d_age, N));
    CK(dalloc(&h->d_Z, N));
    CK(dalloc(&h->d_key, N));
    CK(dalloc(&h->d_keys_tmp, N));
    CK(dalloc(&h->d_vals_tmp, N));
    CK(dalloc(&h->d_skeys, N));
    CK(dalloc(&h->d_perm, N));
    CK(dalloc(&h->d_v, N));
    CK(dalloc(&h->d_sort_scratch, sort_scratch_ints(n)));
    h->item_cap = (long long)h->n_s + n / h->chunk + 2;
    h->part_cap = 2 * (n / h->chunk) + 2;
    CK(dalloc(&h->d_items, (size_t)h->item_cap));
    CK(dalloc(&h->d_rec, N));
    CK(dalloc(&h->d_prec, N));
    CK(dalloc(&h->d_partials, (size_t)h->part_cap * h->tel.n_lambda));
    CK(dalloc(&h->d_contrib, 2 * N));
    h->cap = n;
    return RUBIX_OK;
}

static void destroy(rubix_cube* h) {
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    free_scratch(h);
    void* ptrs[] = {h->d_tpl, h->d_la, h->d_lz, h->d_tile_klo, h->d_seg_off, h->d_n_items, h->d_n_parts,
                    h->d_item_off, h->d_part_off, h->d_scan_scratch, h->d_cube0, h->d_tmp, h->d_out,
                    h->d_err, h->d_slow, h->d_red};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& e : h->ring)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(prev);
    delete h;
}

// Round-to-nearest-even FP32 -> BF16 (bit manipulation; NaN kept quiet).
static uint16_t f32_to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static void gauss_kernel(double sigma, int r, float* out) {
    std::vector<double> k(2 * r + 1);
    double s = 0.0;
    for (int d = -r; d <= r; ++d) {
        k[d + r] = std::exp(-(double)d * d / (2.0 * sigma * sigma));
        s += k[d + r];
    }
    for (int d = -r; d <= r; ++d) out[d + r] = (float)(k[d + r] / s);
}

static int kernel_radius(double sigma, int r) {
    if (r > 0) return r;
    if (!(sigma > 0.0)) return 0;
    return (int)std::ceil(4.0 * sigma);
}

extern "C" rubix_status rubix_cube_create(const rubix_ssp_grid* ssp, const rubix_telescope* tel,
                                          int64_t max_particles, rubix_cube_t** out) {
    if (!out) return fail(RUBIX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ssp || !tel) return fail(RUBIX_ERR_INVALID_ARG, "ssp or telescope is NULL");
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
    if (tel->nx < 1 || tel->ny < 1 || tel->ny > 65535 || (long long)tel->nx * tel->ny >= (1ll << 24))
        return fail(RUBIX_ERR_INVALID_ARG, "nx, ny out of range (ny <= 65535, nx*ny < 2^24)");
    if (!(tel->spaxel_size > 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "spaxel_size must be > 0");
    if (tel->n_lambda < 1 || tel->n_lambda > 8192) return fail(RUBIX_ERR_INVALID_ARG, "n_lambda must be in [1, 8192]");
    if (!(tel->dlambda > 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "dlambda must be > 0");
    if (!(tel->psf_fwhm >= 0.0) || !(tel->lsf_sigma >= 0.0)) return fail(RUBIX_ERR_INVALID_ARG, "negative PSF/LSF width");
    if (!(tel->z_cosmo > -1.0)) return fail(RUBIX_ERR_INVALID_ARG, "z_cosmo must be > -1");
    const double A0 = tel->dlambda / ((1.0 + tel->z_cosmo) * ssp->dlambda);
    if (A0 > 3.0) return fail(RUBIX_ERR_INVALID_ARG, "instrument bins wider than 3 SSP steps are not supported");
    if (max_particles < 0 || max_particles > (1ll << 30)) return fail(RUBIX_ERR_INVALID_ARG, "max_particles out of range");

    rubix_cube* h = new rubix_cube();
    rubix_status st = RUBIX_OK;
    auto bail = [&](rubix_status s) {
        destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(RUBIX_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);

    // ---- SSP grid to device ----
    SspDev& S = h->ssp;
    S.dtype = ssp->storage_dtype;
    h->elem = (S.dtype == RUBIX_F32) ? 4 : 2;
    S.n_age = ssp->n_age;
    S.n_Z = ssp->n_Z;
    S.n_t = ssp->n_age * ssp->n_Z;
    S.n_ls = ssp->n_lambda;
    S.pitch = (ssp->n_lambda + 7) / 8 * 8;
    S.ls0 = ssp->lambda0;
    S.dls = ssp->dlambda;
    {
        const size_t cnt = (size_t)S.n_t * S.pitch;
        std::vector<unsigned char> host(cnt * h->elem, 0);
        for (int c = 0; c < S.n_t; ++c)
            for (int k = 0; k < S.n_ls; ++k) {
                const double v = ssp->spectra[(size_t)c * S.n_ls + k];
                const float f = (float)v;
                const size_t o = (size_t)c * S.pitch + k;
                if (S.dtype == RUBIX_F32) {
                    std::memcpy(&host[o * 4], &f, 4);
                } else if (S.dtype == RUBIX_BF16) {
                    uint16_t b = f32_to_bf16(f);
                    std::memcpy(&host[o * 2], &b, 2);
                } else {
                    __half hv = __float2half_rn(f);
                    std::memcpy(&host[o * 2], &hv, 2);
                }
            }
        if (cudaMalloc(&h->d_tpl, host.size()) != cudaSuccess) return bail(fail(RUBIX_ERR_OOM, "SSP alloc"));
        if (cudaMemcpy(h->d_tpl, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(RUBIX_ERR_CUDA, "SSP copy"));
        std::vector<float> la(S.n_age), lz(S.n_Z);
        for (int i = 0; i < S.n_age; ++i) la[i] = (float)ssp->log10_age_nodes[i];
        for (int i = 0; i < S.n_Z; ++i) lz[i] = (float)ssp->log10_Z_nodes[i];
        if (dalloc(&h->d_la, S.n_age) || dalloc(&h->d_lz, S.n_Z)) return bail(fail(RUBIX_ERR_OOM, "node alloc"));
        cudaMemcpy(h->d_la, la.data(), la.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(h->d_lz, lz.data(), lz.size() * 4, cudaMemcpyHostToDevice);
        S.tpl = h->d_tpl;
        S.la_nodes = h->d_la;
        S.lz_nodes = h->d_lz;
    }

    // ---- telescope ----
    h->tel = *tel;
    if (h->tel.flux_scale == 0.0) h->tel.flux_scale = 1.0;
    h->n_s = tel->nx * tel->ny;
    h->x_lo = (-0.5 * (double)tel->nx) * tel->spaxel_size;
    h->y_lo = (-0.5 * (double)tel->ny) * tel->spaxel_size;
    h->inv_size = 1.0 / tel->spaxel_size;
    {
        ConvParams& C = h->conv;
        C.nx = tel->nx;
        C.ny = tel->ny;
        C.n_lambda = tel->n_lambda;
        const double sp = tel->psf_fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
        const double sl = tel->lsf_sigma / tel->dlambda;
        C.rp = (sp > 0.0) ? kernel_radius(sp, tel->psf_radius) : 0;
        C.rl = (sl > 0.0) ? kernel_radius(sl, tel->lsf_radius) : 0;
        if (C.rp > kMaxRadius || C.rl > kMaxRadius) return bail(fail(RUBIX_ERR_INVALID_ARG, "PSF/LSF radius > 64"));
        if (sp > 0.0) gauss_kernel(sp, C.rp, C.gp); else C.gp[0] = 1.f;
        if (sl > 0.0) gauss_kernel(sl, C.rl, C.gl); else C.gl[0] = 1.f;
        h->need_conv = (sp > 0.0) || (sl > 0.0);
    }

    // ---- deposit geometry: wavelength tiles and the SSP slab staged per tile ----
    {
        // The slab holds one age band of templates x (tile nodes + Doppler halo).
        // A tile is R rounds of 31 bins; choose the fewest bands that give R >= 5
        // (the per-particle setup is shared by R rounds).
        const int align = 16 / h->elem;  // TMA: 16-byte aligned innermost coordinate and extent
        const double v_halo = RUBIX_DEP_VHALO;
        const double lam_max = (tel->lambda0 + (tel->n_lambda - 1) * tel->dlambda) / (1.0 + tel->z_cosmo);
        const double shift = lam_max / S.dls * (v_halo / kC_kms) / (1.0 - v_halo / kC_kms);
        const int cells = std::max(S.n_age - 1, 1);
        struct Geo { int bands, apb, box_rows, n_boxes, rows_alloc, R; long long wcap; };
        Geo best{0, 0, 0, 0, 0, 0, 0}, widest{0, 0, 0, 0, 0, 0, -1};
        for (int nb = 1; nb <= kMaxBands; ++nb) {
            if (nb > 1 && S.n_age < 3) break;
            const int apb = (cells + nb - 1) / nb;
            if (nb > 1 && (nb - 1) * apb >= cells) continue;  // a band would be empty
            const int cols = (S.n_age >= 2) ? std::min(apb + 1, S.n_age) : 1;
            const int rows = cols * S.n_Z;
            const int n_boxes = (rows + 255) / 256;
            const int box_rows = ((rows + n_boxes - 1) / n_boxes + 7) / 8 * 8;
            const int rows_alloc = n_boxes * box_rows;
            long long wcap = ((long long)smem_optin - 128) / ((long long)rows_alloc * h->elem);
            wcap = std::min<long long>(wcap, 256);
            wcap -= wcap % align;
            int R = 0;
            for (int r = 6; r >= 1; --r) {
                const double span = std::max(31.0 * r + 1.0, (31.0 * r - 1.0) * A0 * (1.0 + v_halo / kC_kms) + 2.0);
                const double need = span + 2.0 * shift + (align - 1);
                if (need <= (double)wcap) { R = r; break; }
            }
            if (R > best.R) best = Geo{nb, apb, box_rows, n_boxes, rows_alloc, R, wcap};
            if (wcap > widest.wcap) widest = Geo{nb, apb, box_rows, n_boxes, rows_alloc, 1, wcap};
            if (best.R >= RUBIX_DEP_MIN_R) break;
        }
        if (best.R == 0) {
            // not even 31 bins fit with the full halo: widest slab, 31-bin tiles,
            // smaller halo; if a tile does not fit at all, global-memory path only
            best = widest;
            if (std::max(32.0, 30.0 * A0 + 2.0) + (align - 1) > (double)best.wcap) best.wcap = 0;
        }
        const long long wcap = best.wcap;
        const int R = best.R;
        h->n_bands = best.bands;
        h->apb = best.apb;
        h->n_boxes = best.n_boxes;
        h->box_rows = best.box_rows;
        h->n_rows_alloc = best.rows_alloc;
        for (int b = 0; b < kMaxBands; ++b) h->band_row0[b] = std::min(b * best.apb, std::max(S.n_age - 1, 0)) * S.n_Z;
        h->tile_w = 31 * R;
        h->n_tiles = (tel->n_lambda + h->tile_w - 1) / h->tile_w;
        h->slab_w = (int)wcap;
        std::vector<int> klo(h->n_tiles, 0);
        for (int t = 0; t < h->n_tiles; ++t) {
            const int j0 = t * h->tile_w;
            const double t00 = ((tel->lambda0 + j0 * tel->dlambda) / (1.0 + tel->z_cosmo) - S.ls0) / S.dls;
            const double span0 = std::max(31.0 * R + 1.0, (h->tile_w - 1) * A0 + 2.0);
            long long k = (long long)std::floor(t00 + 0.5 * span0 - 0.5 * h->slab_w);
            long long ka = k >= 0 ? (k / align) * align : -(((-k) + align - 1) / align) * align;
            if (ka < -(1ll << 20)) ka = -(1ll << 20);
            if (ka > (1ll << 20)) ka = (1ll << 20);
            klo[t] = (int)ka;
        }
        if (dalloc(&h->d_tile_klo, h->n_tiles)) return bail(fail(RUBIX_ERR_OOM, "tile alloc"));
        cudaMemcpy(h->d_tile_klo, klo.data(), klo.size() * 4, cudaMemcpyHostToDevice);
        h->dep_smem = deposit_smem_bytes(h->n_rows_alloc, std::max(h->slab_w, 0), h->elem);
        h->dep_ctas = h->n_sm;
        if (h->slab_w > 0) {
            PFN_encodeTiled_t enc = get_encode_tiled();
            if (!enc) return bail(fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"));
            const CUtensorMapDataType dt = (S.dtype == RUBIX_F32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                         : (S.dtype == RUBIX_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
            cuuint64_t gdim[2] = {(cuuint64_t)S.n_ls, (cuuint64_t)S.n_t};
            cuuint64_t gstr[1] = {(cuuint64_t)S.pitch * h->elem};
            cuuint32_t box[2] = {(cuuint32_t)h->slab_w, (cuuint32_t)h->box_rows};
            cuuint32_t es[2] = {1, 1};
            CUresult r = enc(&h->tmap, dt, 2, h->d_tpl, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return bail(fail(RUBIX_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r));
        }
    }

    // ---- fixed-size device buffers ----
    const size_t cube_n = (size_t)h->n_s * tel->n_lambda;
    if (dalloc(&h->d_seg_off, (size_t)h->n_s * h->n_bands + 2) || dalloc(&h->d_n_items, h->n_s + 1) || dalloc(&h->d_n_parts, h->n_s + 1) ||
        dalloc(&h->d_item_off, h->n_s + 1) || dalloc(&h->d_part_off, h->n_s + 1) ||
        dalloc(&h->d_scan_scratch, scan_scratch_ints(h->n_s + 1) + 16) || dalloc(&h->d_cube0, cube_n) ||
        dalloc(&h->d_tmp, cube_n) || dalloc(&h->d_err, 4) || dalloc(&h->d_slow, 1) || dalloc(&h->d_red, 1024))
        return bail(fail(RUBIX_ERR_OOM, "buffer allocation failed"));
    cudaMemset(h->d_err, 0, 16);
    cudaMemset(h->d_slow, 0, 8);
    st = alloc_scratch(h, std::max<int64_t>(max_particles, 1));
    if (st != RUBIX_OK) return bail(st);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(RUBIX_ERR_CUDA, "create: %s", cudaGetErrorString(cudaGetLastError())));
    *out = h;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_destroy(rubix_cube_t* h) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    destroy(h);
    return RUBIX_OK;
}

// ----------------------------------------------------------------------------
// forward
// ----------------------------------------------------------------------------
static rubix_status check_particles(const rubix_particles* p) {
    if (!p) return fail(RUBIX_ERR_INVALID_ARG, "particles is NULL");
    if (p->n < 0 || p->n > (1ll << 30)) return fail(RUBIX_ERR_INVALID_ARG, "n out of range");
    if (p->n == 0) return RUBIX_OK;
    if (!p->x || !p->y || !p->mass || !p->age || !p->Z) return fail(RUBIX_ERR_INVALID_ARG, "x, y, mass, age, Z required");
    if (p->preprojected) {
        if (!p->v_los) return fail(RUBIX_ERR_INVALID_ARG, "v_los required when preprojected");
    } else {
        if (!p->z || !p->vy || !p->vz) return fail(RUBIX_ERR_INVALID_ARG, "z, vy, vz required when not preprojected");
    }
    return RUBIX_OK;
}

static inline void rec_ev(rubix_cube* h, int i, cudaStream_t st) {
    if (h->prof && h->ev) cudaEventRecord(h->ev[i], st);
}

// Enqueue assign + sort for particles already on the device; returns launches.
static rubix_status run_assign_sort(rubix_cube* h, const rubix_particles* p, const float* const* arrs,
                                    cudaStream_t st) {
    AssignParams A{};
    A.n = p->n;
    A.x = arrs[0];
    A.y = arrs[1];
    A.z = arrs[2];
    A.vy = arrs[4];
    A.vz = arrs[5];
    A.v_los = arrs[6];
    A.preprojected = p->preprojected ? 1 : 0;
    A.cos_i = std::cos(p->inclination);
    A.sin_i = std::sin(p->inclination);
    A.x_lo = h->x_lo;
    A.y_lo = h->y_lo;
    A.inv_size = h->inv_size;
    A.nx = h->tel.nx;
    A.ny = h->tel.ny;
    A.key = h->d_key;
    A.v_out = h->d_v;
    A.age = arrs[8];
    A.la_nodes = h->d_la;
    A.n_age = h->ssp.n_age;
    A.apb = h->apb;
    A.n_bands = h->n_bands;
    h->launches += launch_assign(A, st);
    h->launches += launch_sort_by_key(h->d_key, p->n, h->n_s * h->n_bands + 1, h->d_keys_tmp, h->d_vals_tmp, h->d_skeys,
                                      h->d_perm, h->d_seg_off, h->d_sort_scratch, st);
    return RUBIX_OK;
}

static rubix_status stage_particles(rubix_cube* h, const rubix_particles* p, const float** arrs, cudaStream_t st) {
    const float* src[10] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->v_los, p->mass, p->age, p->Z};
    float* dst[10] = {h->d_x, h->d_y, h->d_z, nullptr, h->d_vy, h->d_vz, h->d_vlos, h->d_mass, h->d_age, h->d_Z};
    for (int i = 0; i < 10; ++i) {
        arrs[i] = nullptr;
        if (!src[i]) continue;
        if (p->on_device) {
            arrs[i] = src[i];
        } else if (dst[i]) {
            CK(cudaMemcpyAsync(dst[i], src[i], (size_t)p->n * 4, cudaMemcpyHostToDevice, st));
            arrs[i] = dst[i];
        }
    }
    if (p->preprojected) arrs[2] = arrs[4] = arrs[5] = nullptr;
    else arrs[6] = nullptr;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_forward(rubix_cube_t* h, const rubix_particles* p, uint64_t noise_seed,
                                           float noise_s2n, float* cube_out, int32_t cube_on_device, void* stream) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    if (!cube_out) return fail(RUBIX_ERR_INVALID_ARG, "cube_out is NULL");
    rubix_status s = check_particles(p);
    if (s != RUBIX_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    if (p->n > h->cap) {
        CK(cudaDeviceSynchronize());
        s = alloc_scratch(h, p->n + p->n / 8);
        if (s != RUBIX_OK) return s;
    }
    h->launches = 0;
    h->dep_launches = 0;
    const long long n = p->n;
    const size_t cube_n = (size_t)h->n_s * h->tel.n_lambda;
    const bool noise = noise_s2n > 0.f;
    float* out = cube_out;
    if (!cube_on_device) {
        if (!h->d_out) CK(dalloc(&h->d_out, cube_n));
        out = h->d_out;
    }
    if (h->prof) {
        h->ev = &h->ring[(size_t)h->ring_next * 7];
        h->ring_next = (h->ring_next + 1) % rubix_cube::kRing;
        h->ring_count = std::min(h->ring_count + 1, rubix_cube::kRing);
    }
    rec_ev(h, 0, st);
    CK(cudaMemsetAsync(h->d_slow, 0, 8, st));
    const float* arrs[10];
    s = stage_particles(h, p, arrs, st);
    if (s != RUBIX_OK) return s;
    if (n > 0) {
        s = run_assign_sort(h, p, arrs, st);
        if (s != RUBIX_OK) return s;
    } else {
        CK(cudaMemsetAsync(h->d_seg_off, 0, ((size_t)h->n_s * h->n_bands + 2) * sizeof(int), st));
    }
    rec_ev(h, 1, st);
    SetupParams SP{};
    SP.ssp = h->ssp;
    SP.perm = h->d_perm;
    SP.seg_off = h->d_seg_off;
    SP.n_s = h->n_s;
    SP.n_bands = h->n_bands;
    SP.mass = arrs[7];
    SP.age = arrs[8];
    SP.Z = arrs[9];
    SP.v = h->d_v;
    SP.l0 = h->tel.lambda0;
    SP.dl = h->tel.dlambda;
    SP.z_cosmo = h->tel.z_cosmo;
    SP.flux_scale = h->tel.flux_scale;
    SP.n_lambda = h->tel.n_lambda;
    SP.rec = h->d_rec;
    SP.prec = h->d_prec;
    SP.n_cap = h->cap;
    h->launches += launch_setup(SP, n, st);
    ItemParams IP{};
    IP.seg_off = h->d_seg_off;
    IP.n_s = h->n_s;
    IP.n_bands = h->n_bands;
    IP.chunk = h->chunk;
    IP.n_items = h->d_n_items;
    IP.n_parts = h->d_n_parts;
    IP.item_off = h->d_item_off;
    IP.part_off = h->d_part_off;
    IP.items = h->d_items;
    IP.item_cap = h->item_cap;
    IP.scan_scratch = h->d_scan_scratch;
    IP.err = h->d_err;
    h->launches += launch_items(IP, st);
    rec_ev(h, 2, st);
    float* dep_target = (h->need_conv || noise) ? h->d_cube0 : out;
    DepositParams DP{};
    DP.ssp = h->ssp;
    DP.rec = h->d_rec;
    DP.items = h->d_items;
    DP.item_off = h->d_item_off;
    DP.seg_off = h->d_seg_off;
    DP.n_s = h->n_s;
    DP.n_bands = h->n_bands;
    for (int b = 0; b < kMaxBands; ++b) DP.band_row0[b] = h->band_row0[b];
    DP.n_lambda = h->tel.n_lambda;
    DP.tile_w = h->tile_w;
    DP.n_tiles = h->n_tiles;
    DP.tile_klo = h->d_tile_klo;
    DP.slab_w = h->slab_w;
    DP.box_rows = h->box_rows;
    DP.n_boxes = h->n_boxes;
    DP.cost_c0 = h->cost_c0;
    DP.cube = dep_target;
    DP.partials = h->d_partials;
    DP.part_cap = h->part_cap;
    DP.err = h->d_err;
    DP.slow_count = h->d_slow;
    int l = launch_deposit(DP, &h->tmap, h->dep_ctas, h->dep_threads, h->dep_smem, st);
    if (l < 0) return fail(RUBIX_ERR_CUDA, "deposit launch configuration failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->launches += l;
    h->dep_launches += l;
    rec_ev(h, 3, st);
    h->launches += launch_combine(h->d_part_off, h->n_s, h->tel.n_lambda, h->d_partials, dep_target, st);
    rec_ev(h, 4, st);
    if (h->need_conv || noise) {
        ConvParams C = h->conv;
        C.noise_inv_s2n = noise ? 1.0f / noise_s2n : 0.f;
        C.seed_lo = (uint32_t)noise_seed;
        C.seed_hi = (uint32_t)(noise_seed >> 32);
        h->launches += launch_psf_lsf(C, h->d_cube0, h->d_tmp, out, st);
    }
    rec_ev(h, 5, st);
    CK(cudaGetLastError());
    h->have_forward = true;
    h->forward_noise = noise;
    h->last_n = n;
    if (!cube_on_device) {
        CK(cudaMemcpyAsync(cube_out, out, cube_n * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        unsigned err = 0;
        CK(cudaMemcpy(&err, h->d_err, 4, cudaMemcpyDeviceToHost));
        if (err) return fail(RUBIX_ERR_DEVICE, "device error word 0x%x", err);
    }
    rec_ev(h, 6, st);
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_spaxel_keys(rubix_cube_t* h, const rubix_particles* p, int32_t* keys_out,
                                               void* stream) {
    if (!h || !keys_out) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    rubix_status s = check_particles(p);
    if (s != RUBIX_OK) return s;
    CK(cudaSetDevice(h->device));
    if (p->n > h->cap) {
        CK(cudaDeviceSynchronize());
        s = alloc_scratch(h, p->n);
        if (s != RUBIX_OK) return s;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float* arrs[10];
    s = stage_particles(h, p, arrs, st);
    if (s != RUBIX_OK) return s;
    AssignParams A{};
    A.n = p->n;
    A.x = arrs[0];
    A.y = arrs[1];
    A.z = arrs[2];
    A.vy = arrs[4];
    A.vz = arrs[5];
    A.v_los = arrs[6];
    A.preprojected = p->preprojected ? 1 : 0;
    A.cos_i = std::cos(p->inclination);
    A.sin_i = std::sin(p->inclination);
    A.x_lo = h->x_lo;
    A.y_lo = h->y_lo;
    A.inv_size = h->inv_size;
    A.nx = h->tel.nx;
    A.ny = h->tel.ny;
    A.key = keys_out;
    A.v_out = nullptr;
    launch_assign(A, st);
    CK(cudaGetLastError());
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_sorted(rubix_cube_t* h, int32_t* perm_out, int32_t* seg_off_out, void* stream) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_forward) return fail(RUBIX_ERR_INVALID_ARG, "no forward has run on this handle");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    if (perm_out && h->last_n > 0)
        CK(cudaMemcpyAsync(perm_out, h->d_perm, (size_t)h->last_n * 4, cudaMemcpyDeviceToDevice, st));
    if (seg_off_out) {
        // spaxel boundaries are every n_bands-th entry of the (spaxel, band) offsets
        CK(cudaMemcpy2DAsync(seg_off_out, 4, h->d_seg_off, 4 * (size_t)h->n_bands, 4, (size_t)h->n_s + 1,
                             cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(seg_off_out + h->n_s + 1, h->d_seg_off + (size_t)h->n_s * h->n_bands + 1, 4,
                           cudaMemcpyDeviceToDevice, st));
    }
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_set_profiling(rubix_cube_t* h, int32_t enable) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    CK(cudaSetDevice(h->device));
    if (enable && h->ring.empty()) {
        h->ring.assign((size_t)rubix_cube::kRing * 7, nullptr);
        for (auto& e : h->ring) CK(cudaEventCreate(&e));
    }
    h->prof = enable != 0;
    h->ring_next = 0;
    h->ring_count = 0;
    h->ev = nullptr;
    return RUBIX_OK;
}

// Stage times of one profiled forward (event set `ev`).
static rubix_status stage_ms(cudaEvent_t* ev, float t[6]) {
    CK(cudaEventSynchronize(ev[5]));
    const int a[6] = {0, 1, 2, 3, 4, 0};
    const int b[6] = {1, 2, 3, 4, 5, 5};
    for (int i = 0; i < 6; ++i) CK(cudaEventElapsedTime(&t[i], ev[a[i]], ev[b[i]]));
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_stage_times(rubix_cube_t* h, float* ms, int32_t* n_inout) {
    if (!h || !ms || !n_inout) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    if (!h->prof || !h->ev) return fail(RUBIX_ERR_INVALID_ARG, "no profiled forward");
    CK(cudaSetDevice(h->device));
    float t[6];
    rubix_status s = stage_ms(h->ev, t);
    if (s != RUBIX_OK) return s;
    const int n = std::min<int>(*n_inout, 6);
    for (int i = 0; i < n; ++i) ms[i] = t[i];
    *n_inout = n;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_profile_history(rubix_cube_t* h, int32_t stage, float* ms, int32_t* n_inout) {
    if (!h || !ms || !n_inout) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    if (stage < 0 || stage > 5) return fail(RUBIX_ERR_INVALID_ARG, "stage must be in [0, 5]");
    CK(cudaSetDevice(h->device));
    const int cnt = std::min<int>(h->ring_count, *n_inout);
    const int first = (h->ring_next - h->ring_count + rubix_cube::kRing) % rubix_cube::kRing;
    for (int i = 0; i < cnt; ++i) {
        float t[6];
        rubix_status s = stage_ms(&h->ring[(size_t)((first + i) % rubix_cube::kRing) * 7], t);
        if (s != RUBIX_OK) return s;
        ms[i] = t[stage];
    }
    *n_inout = cnt;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_stats(rubix_cube_t* h, int64_t* stats, int32_t* n_inout) {
    if (!h || !stats || !n_inout) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    int n_in = 0;
    unsigned long long slow = 0;
    unsigned err = 0;
    if (h->have_forward)
        CK(cudaMemcpy(&n_in, h->d_seg_off + (size_t)h->n_s * h->n_bands, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&slow, h->d_slow, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&err, h->d_err, 4, cudaMemcpyDeviceToHost));
    int64_t v[9] = {n_in, (int64_t)n_in * h->tel.n_lambda, (int64_t)slow, h->dep_launches, h->launches,
                    (int64_t)err, h->tile_w, h->slab_w, h->n_bands};
    const int n = std::min<int>(*n_inout, 9);
    for (int i = 0; i < n; ++i) stats[i] = v[i];
    *n_inout = n;
    return RUBIX_OK;
}

// ----------------------------------------------------------------------------
// backward
// ----------------------------------------------------------------------------
extern "C" rubix_status rubix_cube_backward(rubix_cube_t* h, const float* dL_dcube, float* d_mass, float* d_age,
                                            float* d_Z, float* d_vlos, double* d_global, void* stream) {
    if (!h || !dL_dcube) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_forward) return fail(RUBIX_ERR_INVALID_ARG, "backward needs a forward on this handle first");
    if (h->forward_noise) return fail(RUBIX_ERR_INVALID_ARG, "backward of a noisy forward is not defined");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const float* G0 = dL_dcube;
    if (h->need_conv) {
        ConvParams C = h->conv;
        C.noise_inv_s2n = 0.f;
        launch_psf_lsf(C, dL_dcube, h->d_tmp, h->d_cube0, st);
        G0 = h->d_cube0;
    }
    launch_zero_grads(d_mass, d_age, d_Z, d_vlos, h->last_n, st);
    AdjointParams P{};
    P.ssp = h->ssp;
    P.prec = h->d_prec;
    P.perm = h->d_perm;
    P.seg_off = h->d_seg_off;
    P.sorted_keys = h->d_skeys;
    P.n_s = h->n_s;
    P.n_bands = h->n_bands;
    P.n_lambda = h->tel.n_lambda;
    P.l0 = h->tel.lambda0;
    P.dl = h->tel.dlambda;
    P.z_cosmo = h->tel.z_cosmo;
    P.flux_scale = h->tel.flux_scale;
    P.G0 = G0;
    P.d_mass = d_mass;
    P.d_age = d_age;
    P.d_Z = d_Z;
    P.d_v = d_vlos;
    P.contrib = d_global ? h->d_contrib : nullptr;
    P.n_in = h->last_n;  // upper bound; the kernel reads the in-field count on the device
    launch_adjoint_rec(P, h->d_rec, st);
    if (d_global)
        launch_reduce_global(h->d_contrib, h->d_seg_off + (size_t)h->n_s * h->n_bands, d_global, h->d_red, st);
    CK(cudaGetLastError());
    return RUBIX_OK;
}
