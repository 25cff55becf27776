// api.cu -- the C ABI of include/rubix.h for single-galaxy handles: a handle
// is an SSP state (device templates + deposit tiling) and one plan (telescope
// + device buffers); forward = pre (stage, keys, sort, setup, work items) ->
// deposit (one job) -> post (combine of split spaxels, PSF/LSF/noise).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/rubix.h"
#include "engine.h"

using namespace rubix;

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? RUBIX_ERR_OOM : RUBIX_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    } while (0)

extern "C" const char* rubix_last_error_message(void) { return last_error(); }
extern "C" const char* rubix_version(void) { return "rubix-gb300 0.2 (sm_103a)"; }

struct rubix_cube {
    SspState* S = nullptr;
    Plan P;
    bool prof = false;
    // profiling: a ring of event sets, one set per forward since profiling was enabled
    static constexpr int kRing = 256;
    std::vector<cudaEvent_t> ring;  // kRing * 7 events, created on first enable
    int ring_next = 0, ring_count = 0;
    cudaEvent_t* ev = nullptr;      // event set of the forward being enqueued
};

static void destroy(rubix_cube* h) {
    if (!h) return;
    if (h->S) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(h->S->device);
        plan_release(&h->P);
        for (auto& e : h->ring)
            if (e) cudaEventDestroy(e);
        cudaSetDevice(prev);
        ssp_state_destroy(h->S);
    }
    delete h;
}

extern "C" rubix_status rubix_cube_create(const rubix_ssp_grid* ssp, const rubix_telescope* tel,
                                          int64_t max_particles, rubix_cube_t** out) {
    if (!out) return fail(RUBIX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ssp || !tel) return fail(RUBIX_ERR_INVALID_ARG, "ssp or telescope is NULL");
    if (max_particles < 0 || max_particles > (1ll << 30)) return fail(RUBIX_ERR_INVALID_ARG, "max_particles out of range");
    rubix_cube* h = new rubix_cube();
    rubix_status st = ssp_state_create(ssp, tel, &h->S);
    if (st == RUBIX_OK) st = plan_init(&h->P, h->S, tel, std::max<int64_t>(max_particles, 1), Alloc{}, false, true);
    if (st == RUBIX_OK && cudaDeviceSynchronize() != cudaSuccess)
        st = fail(RUBIX_ERR_CUDA, "create: %s", cudaGetErrorString(cudaGetLastError()));
    if (st != RUBIX_OK) {
        destroy(h);
        return st;
    }
    *out = h;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_destroy(rubix_cube_t* h) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    cudaSetDevice(h->S->device);
    cudaDeviceSynchronize();
    destroy(h);
    return RUBIX_OK;
}

static inline void rec_ev(rubix_cube* h, int i, cudaStream_t st) {
    if (h->prof && h->ev) cudaEventRecord(h->ev[i], st);
}

extern "C" rubix_status rubix_cube_forward(rubix_cube_t* h, const rubix_particles* p, uint64_t noise_seed,
                                           float noise_s2n, float* cube_out, int32_t cube_on_device, void* stream) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    if (!cube_out) return fail(RUBIX_ERR_INVALID_ARG, "cube_out is NULL");
    rubix_status s = check_particles(p);
    if (s != RUBIX_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SspState& S = *h->S;
    Plan& P = h->P;
    CK(cudaSetDevice(S.device));
    if (p->n > P.cap) {
        s = plan_grow(&P, p->n);
        if (s != RUBIX_OK) return s;
    }
    const size_t cube_n = (size_t)P.n_s * P.tel.n_lambda;
    const bool noise = noise_s2n > 0.f;
    float* out = cube_out;
    if (!cube_on_device) {
        if (!P.d_out) {
            CK(cudaMalloc(&P.d_out, cube_n * sizeof(float)));
            P.bytes += cube_n * sizeof(float);
        }
        out = P.d_out;
    }
    if (h->prof) {
        h->ev = &h->ring[(size_t)h->ring_next * 7];
        h->ring_next = (h->ring_next + 1) % rubix_cube::kRing;
        h->ring_count = std::min(h->ring_count + 1, rubix_cube::kRing);
    }
    rec_ev(h, 0, st);
    CK(cudaMemsetAsync(S.d_slow, 0, 8, st));
    s = enqueue_pre(P, p, st, h->prof ? h->ev : nullptr);
    if (s != RUBIX_OK) return s;
    rec_ev(h, 2, st);
    float* target = deposit_target(P, out, noise);
    const DepJob job = plan_job(P, target);
    const int l = enqueue_deposit(S, &job, 1, P.d_job_cost, st);
    if (l < 0) return fail(RUBIX_ERR_CUDA, "deposit launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    P.launches += l;
    P.dep_launches = 1;
    rec_ev(h, 3, st);
    P.launches += enqueue_post(P, target, out, noise_seed, noise_s2n, st, h->prof ? h->ev : nullptr);
    rec_ev(h, 5, st);
    CK(cudaGetLastError());
    P.have_forward = true;
    P.forward_noise = noise;
    P.forward_tag += 1;
    if (!cube_on_device) {
        CK(cudaMemcpyAsync(cube_out, out, cube_n * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        unsigned err = 0;
        CK(cudaMemcpy(&err, S.d_err, 4, cudaMemcpyDeviceToHost));
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
    CK(cudaSetDevice(h->S->device));
    if (p->n > h->P.cap) {
        s = plan_grow(&h->P, p->n);
        if (s != RUBIX_OK) return s;
    }
    return enqueue_keys(h->P, p, keys_out, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" rubix_status rubix_cube_sorted(rubix_cube_t* h, int32_t* perm_out, int32_t* seg_off_out, void* stream) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    const Plan& P = h->P;
    if (!P.have_forward) return fail(RUBIX_ERR_INVALID_ARG, "no forward has run on this handle");
    const int nb = h->S->n_bands;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->S->device));
    if (perm_out && P.last_n > 0)
        CK(cudaMemcpyAsync(perm_out, P.d_perm, (size_t)P.last_n * 4, cudaMemcpyDeviceToDevice, st));
    if (seg_off_out) {
        // spaxel boundaries are every n_bands-th entry of the (spaxel, band) offsets
        CK(cudaMemcpy2DAsync(seg_off_out, 4, P.d_seg_off, 4 * (size_t)nb, 4, (size_t)P.n_s + 1,
                             cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(seg_off_out + P.n_s + 1, P.d_seg_off + (size_t)P.n_s * nb + 1, 4,
                           cudaMemcpyDeviceToDevice, st));
    }
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_set_profiling(rubix_cube_t* h, int32_t enable) {
    if (!h) return fail(RUBIX_ERR_INVALID_ARG, "NULL handle");
    CK(cudaSetDevice(h->S->device));
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
    CK(cudaSetDevice(h->S->device));
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
    CK(cudaSetDevice(h->S->device));
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
    const SspState& S = *h->S;
    const Plan& P = h->P;
    CK(cudaSetDevice(S.device));
    CK(cudaDeviceSynchronize());
    int n_in = 0;
    unsigned long long slow = 0;
    unsigned err = 0;
    if (P.have_forward) CK(cudaMemcpy(&n_in, P.d_seg_off + (size_t)P.n_s * S.n_bands, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&slow, S.d_slow, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&err, S.d_err, 4, cudaMemcpyDeviceToHost));
    int64_t v[9] = {n_in, (int64_t)n_in * P.tel.n_lambda, (int64_t)slow, P.dep_launches, P.launches,
                    (int64_t)err, S.tile_w, S.slab_w, S.n_bands};
    const int n = std::min<int>(*n_inout, 9);
    for (int i = 0; i < n; ++i) stats[i] = v[i];
    *n_inout = n;
    return RUBIX_OK;
}

// ----------------------------------------------------------------------------
// PSF + LSF of a given device cube
// ----------------------------------------------------------------------------
extern "C" rubix_status rubix_convolve(const rubix_telescope* tel, const float* cube_in, float* cube_out,
                                       int32_t n_rows, void* stream) {
    if (!tel || !cube_in || !cube_out) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    if (cube_in == cube_out) return fail(RUBIX_ERR_INVALID_ARG, "cube_in and cube_out must be distinct");
    if (n_rows < 1 || tel->nx < 1 || (long long)tel->nx * n_rows >= (1ll << 24) || tel->n_lambda < 1 ||
        tel->n_lambda > 8192 || !(tel->dlambda > 0.0) || !(tel->psf_fwhm >= 0.0) || !(tel->lsf_sigma >= 0.0))
        return fail(RUBIX_ERR_INVALID_ARG, "cube or telescope sizes out of range");
    ConvParams C{};
    const bool conv = conv_params(tel, n_rows, &C);
    if (C.rp > kMaxRadius || C.rl > kMaxRadius) return fail(RUBIX_ERR_INVALID_ARG, "PSF/LSF radius > 64");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)n_rows * tel->nx * tel->n_lambda * sizeof(float);
    if (!conv) {
        CK(cudaMemcpyAsync(cube_out, cube_in, bytes, cudaMemcpyDeviceToDevice, st));
        return RUBIX_OK;
    }
    unsigned* d_err = nullptr;
    float* tmp = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&d_err), 16, st));
    CK(cudaMemsetAsync(d_err, 0, 16, st));
    C.err = d_err;
    if (psf_lsf_needs_tmp(C.rp, C.rl)) {
        const cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), bytes, st);
        if (e != cudaSuccess) {
            cudaFreeAsync(d_err, st);
            return fail(RUBIX_ERR_OOM, "rubix_convolve scratch: %s", cudaGetErrorString(e));
        }
    }
    const int l = launch_psf_lsf(C, cube_in, tel->n_lambda, nullptr, tmp, cube_out, st);
    if (tmp) cudaFreeAsync(tmp, st);
    cudaFreeAsync(d_err, st);
    if (l < 0) return fail(RUBIX_ERR_CUDA, "PSF/LSF launch failed");
    CK(cudaGetLastError());
    return RUBIX_OK;
}

// ----------------------------------------------------------------------------
// backward
// ----------------------------------------------------------------------------
extern "C" rubix_status rubix_cube_forward_tag(rubix_cube_t* h, uint64_t* tag) {
    if (!h || !tag) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    *tag = h->P.have_forward ? h->P.forward_tag : 0;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_cube_backward(rubix_cube_t* h, uint64_t forward_tag, const float* dL_dcube,
                                            float* d_mass, float* d_age, float* d_Z, float* d_vlos,
                                            double* d_global, void* stream) {
    NvtxRange nvtx("rubix: backward");
    if (!h || !dL_dcube) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    const SspState& S = *h->S;
    Plan& P = h->P;
    if (!P.have_forward) return fail(RUBIX_ERR_INVALID_ARG, "backward needs a forward on this handle first");
    if (forward_tag != P.forward_tag)
        return fail(RUBIX_ERR_INVALID_ARG,
                    "backward for forward %llu, but the handle holds the state of forward %llu (a later forward "
                    "replaced it)",
                    (unsigned long long)forward_tag, (unsigned long long)P.forward_tag);
    if (P.forward_noise) return fail(RUBIX_ERR_INVALID_ARG, "backward of a noisy forward is not defined");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(S.device));
    const float* G0 = dL_dcube;
    if (P.need_conv) {
        // the PSF and LSF kernels are symmetric: their adjoint is the same convolution
        ConvParams C = P.conv;
        C.noise_inv_s2n = 0.f;
        int lc;
        if (P.has_grad_map) {
            // the gradient into pitched rows, then the TMA kernel, as in the forward
            CK(cudaMemcpy2DAsync(P.d_tmp, (size_t)P.pitch0 * sizeof(float), dL_dcube,
                                 (size_t)P.tel.n_lambda * sizeof(float), (size_t)P.tel.n_lambda * sizeof(float),
                                 (size_t)P.n_s, cudaMemcpyDeviceToDevice, st));
            lc = launch_psf_lsf(C, P.d_tmp, P.pitch0, &P.grad_map, nullptr, P.d_cube0, st);
        } else {
            lc = launch_psf_lsf(C, dL_dcube, P.tel.n_lambda, nullptr, P.d_tmp, P.d_cube0, st);
        }
        if (lc < 0) return fail(RUBIX_ERR_CUDA, "PSF/LSF transpose launch failed");
        G0 = P.d_cube0;
    }
    launch_zero_grads(d_mass, d_age, d_Z, d_vlos, P.last_n, st);
    AdjointParams A{};
    A.ssp = S.ssp;
    A.prec = P.d_prec;
    A.perm = P.d_perm;
    A.seg_off = P.d_seg_off;
    A.sorted_keys = P.d_skeys;
    A.n_s = P.n_s;
    A.n_bands = S.n_bands;
    A.n_lambda = P.tel.n_lambda;
    A.l0 = P.tel.lambda0;
    A.dl = P.tel.dlambda;
    A.z_cosmo = P.tel.z_cosmo;
    A.flux_scale = P.tel.flux_scale;
    A.G0 = G0;
    A.d_mass = d_mass;
    A.d_age = d_age;
    A.d_Z = d_Z;
    A.d_v = d_vlos;
    A.contrib = d_global ? P.d_contrib : nullptr;
    A.dv_dang = P.d_dvda;
    A.n_in = P.last_n;  // upper bound; the kernel reads the in-field count on the device
    // over the deposit's (tile, work item, age band) decomposition and slabs
    launch_adjoint_setup(A, P.d_rec, P.d_wu, st);
    AdjTileParams T{};
    T.quad = S.d_quad;
    T.quad16 = S.d_quad16;
    T.qdt = S.qdt;
    T.n_cells = S.n_cells;
    T.n_ls = S.ssp.n_ls;
    T.rec = P.d_rec;
    T.wu = P.d_wu;
    T.items = P.d_items;
    T.item_off = P.d_item_off;
    T.seg_off = P.d_seg_off;
    T.n_s = P.n_s;
    T.n_bands = S.n_bands;
    for (int b = 0; b < kMaxBands; ++b) T.band_cell0[b] = S.band_cell0[b];
    T.G0 = G0;
    T.part = P.d_adjpart;
    T.n_cap = P.cap;
    T.n_lambda = P.tel.n_lambda;
    T.tile_w = S.tile_w;
    T.n_tiles = S.n_tiles;
    T.tile_klo = S.d_tile_klo;
    T.slab_w = S.slab_w;
    T.ncb = S.ncb;
    T.box_w = S.box_w;
    T.n_boxes = S.n_boxes;
    T.cost_c0 = S.cost_c0;
    T.ls0_over = (float)(S.ssp.ls0 / S.ssp.dls);
    T.resample = P.tel.resample;
    T.err = S.d_err;
    if (launch_adjoint_tiles(T, &S.tmap, S.dep_ctas, RUBIX_ADJ_THREADS, S.dep_smem, st) < 0)
        return fail(RUBIX_ERR_CUDA, "adjoint launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    launch_adjoint_final(A, P.d_adjpart, S.n_tiles, P.cap, st);
    if (d_global)
        launch_reduce_global(P.d_contrib, P.d_seg_off + (size_t)P.n_s * S.n_bands, d_global, P.d_red, st);
    CK(cudaGetLastError());
    return RUBIX_OK;
}
