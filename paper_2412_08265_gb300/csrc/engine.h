// engine.h -- host-side engine shared by the C-ABI handle (api.cu) and the
// request server (serve.cu): the SSP grid resident on a device with the
// deposit tiling of one output wavelength grid, and per-galaxy plans holding
// the device buffers of one forward model.
#pragma once

#include <cstddef>
#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rubix.h"
#include "common.cuh"
#include "kernels.h"

namespace rubix {

// NVTX range over a host stage (enqueue time; a profiler that records NVTX
// shows the stages of a forward, backward or serving batch by name).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Thread-local message behind rubix_last_error_message(); fail() sets it and
// returns `st`.
rubix_status fail(rubix_status st, const char* fmt, ...);
void set_last_error(const char* msg);

// SSP templates on one device + the deposit tiling for one output wavelength
// grid (n_lambda, lambda0, dlambda, z_cosmo): the cell quads the deposit and
// adjoint read (the storage dtype's values), wavelength tiles,
// the age bands and width of the shared-memory quad slab, and its TMA
// descriptor.
struct SspState {
    int device = 0, n_sm = 0, smem_optin = 0;
    SspDev ssp{};
    float4* d_quad = nullptr;   // [n_ls][n_cells] cell quads, FP32 templates
    uint2* d_quad16 = nullptr;  // [n_ls][n_cells] cell quads, BF16 / FP16 templates (qdt 1 / 2)
    int qdt = 0;
    int n_cells = 0, cz = 1;    // cells = max(n_age-1,1) * cz, cz = max(n_Z-1,1)
    float* d_la = nullptr;
    float* d_lz = nullptr;
    int n_lambda = 0;
    double lambda0 = 0, dlambda = 0, z_cosmo = 0;
    int tile_w = 31, n_tiles = 0, slab_w = 0, ncb = 1, box_w = 0, n_boxes = 0;
    int n_bands = 1, apb = 1;
    int band_cell0[kMaxBands] = {};
    size_t dep_smem = 0;
    int* d_tile_klo = nullptr;
    CUtensorMap tmap{};
    int dep_ctas = 0, dep_threads = RUBIX_DEP_THREADS, chunk = RUBIX_DEP_CHUNK, cost_c0 = RUBIX_DEP_COSTC0;
    unsigned* d_err = nullptr;              // device error word (kernel bit flags)
    unsigned long long* d_slow = nullptr;   // (particle, tile) pairs on the global-memory path
};

rubix_status validate_ssp(const rubix_ssp_grid* ssp);
rubix_status validate_telescope(const rubix_telescope* tel, double ssp_dlambda);
rubix_status ssp_state_create(const rubix_ssp_grid* ssp, const rubix_telescope* wavelength_grid, SspState** out);
void ssp_state_destroy(SspState* S);
bool same_wavelength_grid(const SspState& S, const rubix_telescope* tel);
// Spaxel rows the telescope's row window models (ny without a window).
int window_rows(const rubix_telescope* tel);
// PSF/LSF parameters of a telescope for a cube of `rows` spaxel rows (kernel
// radii and normalised Gaussian weights, no noise); false if the telescope
// has neither a PSF nor an LSF.
bool conv_params(const rubix_telescope* tel, int rows, ConvParams* C);
// Particle descriptor checks shared by every entry point (arrays present, n in range).
rubix_status check_particles(const rubix_particles* p);
// Orientation R = Rz(position_angle) Rx(inclination) Rz(azimuth), row-major,
// each element rounded as the header's reading states, and the coefficients
// of dv_los/d(inclination) (Di, on vx, vy, vz) and dv_los/d(azimuth) (Da, on vx, vy).
void orientation_matrix(double inclination, double azimuth, double position_angle, double R[9], double Di[3],
                        double Da[2]);

// Where a plan's device buffers come from: cudaMalloc, or stream-ordered
// allocation on `stream` from `pool` (the server, which must not synchronise).
// staging = false leaves out the particle staging buffers (inputs that are
// already on the device).
struct Alloc {
    bool async = false;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    bool staging = true;
};

// One galaxy's forward model on the device: its telescope (spatial grid,
// PSF/LSF) and every scratch and cube buffer, sized for up to `cap` particles.
struct Plan {
    const SspState* S = nullptr;
    rubix_telescope tel{};
    int n_s = 0;                            // spaxels of the modelled rows: nx * rows
    int rows = 0, row_lo = 0;               // the telescope's row window (all ny rows: 0, ny)
    double x_lo = 0, y_lo = 0, inv_size = 0;
    ConvParams conv{};
    bool need_conv = false;
    long long cap = 0, item_cap = 0, part_cap = 0;
    float *d_x = nullptr, *d_y = nullptr, *d_z = nullptr, *d_vx = nullptr, *d_vy = nullptr, *d_vz = nullptr,
          *d_vlos = nullptr;
    float *d_mass = nullptr, *d_age = nullptr, *d_Z = nullptr;
    int *d_key = nullptr, *d_keys_tmp = nullptr, *d_vals_tmp = nullptr, *d_skeys = nullptr, *d_perm = nullptr;
    PartRec* d_pin = nullptr;  // [cap] (mass, age, Z, v_los) in original order, written by the assign
    int* d_sort_scratch = nullptr;
    int *d_seg_off = nullptr, *d_n_items = nullptr, *d_n_parts = nullptr, *d_item_off = nullptr;
    int *d_part_off = nullptr, *d_scan_scratch = nullptr;
    Item* d_items = nullptr;
    DepRec* d_rec = nullptr;
    PartRec* d_prec = nullptr;
    float* d_partials = nullptr;
    float *d_cube0 = nullptr, *d_tmp = nullptr, *d_out = nullptr;
    int pitch0 = 0;                         // row stride of d_cube0 (16-byte rows for the TMA PSF/LSF)
    CUtensorMap conv_map{};                 // 3-D TMA map of d_cube0 for the PSF/LSF kernel
    bool has_conv_map = false;
    CUtensorMap grad_map{};                 // the same view of d_tmp (backward: pitched loss gradient)
    bool has_grad_map = false;
    long long* d_job_cost = nullptr;        // deposit launch scratch [kMaxJobs + 1]
    double *d_contrib = nullptr, *d_red = nullptr;
    float2* d_dvda = nullptr;               // backward: dv_los/d(inclination, azimuth) per particle [cap]
    float4* d_wu = nullptr;                 // backward: unit-mass weights [cap]
    float4* d_adjpart = nullptr;            // backward: per (tile, particle) sums [n_tiles][cap]
    Alloc alloc;
    size_t bytes = 0;                       // device bytes held by the plan
    // state of the last forward
    bool have_forward = false, forward_noise = false;
    uint64_t forward_tag = 0;               // tag of the last forward (1, 2, ...)
    long long last_n = 0;
    int launches = 0, dep_launches = 0;
};

// Device bytes plan_init would take for n particles (with_out: plus a device
// cube for host output; with_grad: plus backward scratch).
size_t plan_bytes(const SspState& S, const rubix_telescope* tel, long long n, bool with_out, bool with_grad,
                  bool staging = true);
rubix_status plan_init(Plan* P, const SspState* S, const rubix_telescope* tel, long long max_particles, Alloc a,
                       bool with_out, bool with_grad);
rubix_status plan_grow(Plan* P, long long n);  // synchronous plans only
void plan_release(Plan* P);                    // async plans: frees stream-ordered on a.stream

// Forward in three enqueued parts (all on `st`): stage particles, assign keys,
// sort, per-particle setup and work items; the (possibly batched) deposit; and
// the combine of split spaxels + PSF/LSF/noise into `out`.
// `ev` (optional, profiling): enqueue_pre records ev[1] after the sort,
// enqueue_post records ev[4] after the combine.
rubix_status enqueue_pre(Plan& P, const rubix_particles* p, cudaStream_t st, cudaEvent_t* ev = nullptr);
// Plain spaxel keys (no age band) of p into keys_out (device, [p->n]).
rubix_status enqueue_keys(Plan& P, const rubix_particles* p, int* keys_out, cudaStream_t st);
float* deposit_target(const Plan& P, float* out, bool noise);
DepJob plan_job(const Plan& P, float* target);
int enqueue_deposit(const SspState& S, const DepJob* jobs, int n_jobs, long long* d_job_cost, cudaStream_t st);
int enqueue_post(Plan& P, float* target, float* out, uint64_t noise_seed, float noise_s2n, cudaStream_t st,
                 cudaEvent_t* ev = nullptr);
const char* last_error();

}  // namespace rubix
