// kernels.h -- internal launch interface between the C-ABI layer and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rubix {

struct DepRec;
struct PartRec;
struct Item;

constexpr int kMaxBands = 32;

// Streaming multiprocessors of the current device (cached per device); grid
// caps of the grid-stride kernels are multiples of it.
int sm_count();

// Deposit launch shape: threads per CTA (one CTA per SM: the SSP slab fills
// shared memory; 896 threads leave 72 registers per thread).
#ifndef RUBIX_DEP_THREADS
#define RUBIX_DEP_THREADS 896
#endif
// Deposit CTAs resident per SM (each gets 1/RUBIX_DEP_CTAS of the shared memory).
#ifndef RUBIX_DEP_CTAS
#define RUBIX_DEP_CTAS 1
#endif
// Deposit geometry: particles per work item, the line-of-sight speed (km/s)
// the shared-memory slab's Doppler halo covers, the most 31-bin rounds per
// wavelength tile, and a fixed number of age bands (0 = chosen by the cost
// estimate).
#ifndef RUBIX_DEP_CHUNK
#define RUBIX_DEP_CHUNK 256
#endif
#ifndef RUBIX_DEP_VHALO
#define RUBIX_DEP_VHALO 800.0
#endif
#ifndef RUBIX_DEP_RMAX
#define RUBIX_DEP_RMAX 12
#endif
#ifndef RUBIX_DEP_BANDS
#define RUBIX_DEP_BANDS 0
#endif
// Cost of a work item in particle units, for the static split of the
// (tile, item) cost space over CTAs.
#ifndef RUBIX_DEP_COSTC0
#define RUBIX_DEP_COSTC0 4
#endif
// Work items a warp claims at once (its first lanes look them up together),
// in the deposit and in the adjoint.
#ifndef RUBIX_DEP_GRAB
#define RUBIX_DEP_GRAB 4
#endif
#ifndef RUBIX_ADJ_GRAB
#define RUBIX_ADJ_GRAB 2
#endif
// Threads of an adjoint CTA (one per SM, the deposit's slab geometry).
#ifndef RUBIX_ADJ_THREADS
#define RUBIX_ADJ_THREADS 768
#endif

// K1 parameters. The sort key is spaxel * n_bands + age band (n_bands <= 1:
// the plain spaxel key); particles outside the field get nx*ny*n_bands.
struct AssignParams {
    long long n;
    const float *x, *y, *z, *vx, *vy, *vz, *v_los;  // vx nullable (treated as 0)
    int preprojected;
    double R[9];      // orientation, row-major: x' = (R0 x + R1 y) + R2 z, ..., v_los = (R6 vx + R7 vy) + R8 vz
    double Di[3];     // dv_los/d(inclination) = Di . (vx, vy, vz)
    double Da[2];     // dv_los/d(azimuth) = Da . (vx, vy)
    float2* dv_dang;  // [n] original order (nullable): (dv_los/d inclination, dv_los/d azimuth)
    double x_lo, y_lo, inv_size;
    int nx, ny;
    int row_lo, rows; // row window: spaxel rows [row_lo, row_lo + rows) are kept (rows <= 0: all ny)
    int* key;         // [n]
    // [n] original order (nullable): (mass, age, Z, line-of-sight velocity),
    // one 16-byte record per particle, so that the setup gathers one record
    // per particle in sorted order instead of four arrays
    PartRec* pin_out;
    const float *mass, *Zm;
    // age bands (optional; the age also goes into pin_out)
    const float* age;
    const float* la_nodes;
    int n_age, apb, n_bands;
};

int launch_assign(const AssignParams& P, cudaStream_t st);
size_t scan_scratch_ints(long long n);
int launch_exclusive_scan(const int* in, int* out, long long n, int* scratch, cudaStream_t st);
size_t sort_scratch_ints(long long n);
// Stable sort of keys in [0, n_keys); seg_off gets n_keys + 1 entries.
int launch_sort_by_key(const int* keys, long long n, int n_keys, int* keys_tmp, int* vals_tmp, int* keys_out,
                       int* perm_out, int* seg_off, int* scratch, cudaStream_t st);

// SSP grid as seen by the kernels (the templates themselves as cell quads).
struct SspDev {
    int dtype;              // 0 f32, 1 bf16, 2 f16
    int n_age, n_Z, n_t, n_ls;
    const float* la_nodes;  // [n_age]
    const float* lz_nodes;  // [n_Z]
    double ls0, dls;
};

// K3: per-particle setup in sorted order + work items.
struct SetupParams {
    SspDev ssp;
    const int* perm;         // sorted position -> particle index
    const int* seg_off;      // [n_s * n_bands + 2]
    int n_s, n_bands;
    const PartRec* pin;      // [n] original order: (mass, age, Z, v_los) per particle
    double l0, dl, z_cosmo, flux_scale;
    double inv_c;            // 1 / c in km/s
    double alpha_z;          // 1 / ((1 + z_cosmo) dls)
    double ls0_dls;          // ls0 / dls
    int n_lambda;
    int resample;            // 0: records map bin centres, 1: bin lower edges (bin means)
    DepRec* rec;             // [n_in]
    PartRec* prec;           // [n_in]
    long long n_cap;         // capacity of rec / prec
};
int launch_setup(const SetupParams& P, long long n_total, cudaStream_t st);

struct ItemParams {
    const int* seg_off;      // [n_s * n_bands + 2]
    int n_s, n_bands;
    int chunk;               // max particles per item
    int* n_items;            // [n_s + 1] scratch
    int* n_parts;            // [n_s + 1] scratch
    int* item_off;           // [n_s + 1]
    int* part_off;           // [n_s + 1]
    Item* items;             // capacity item_cap
    long long item_cap;
    int* scan_scratch;
    unsigned* err;
};
int launch_items(const ItemParams& P, cudaStream_t st);

// K4: deposit. One launch deposits up to kMaxJobs galaxies (jobs) that share
// the SSP grid and the output wavelength grid.
constexpr int kMaxJobs = 64;
constexpr int kDepHeader = 1024;  // deposit shared-memory header (barrier, counters, job table)
struct DepJob {
    const DepRec* rec;
    const Item* items;
    const int* item_off;     // [n_s + 1]: total items at [n_s]
    const int* seg_off;      // [n_s * n_bands + 2]: in-field particles at [n_s * n_bands]
    float* cube;             // [n_s][pitch] (the first n_lambda of each row)
    float* partials;         // [part_cap][n_lambda]
    long long part_cap;
    int n_s;
    int pitch;               // cube row stride in floats (>= n_lambda)
    int resample;            // 1: bin means (records hold the bins' lower edges)
};
struct DepositParams {
    const float4* quad;      // [n_ls][n_cells] SSP cell quads (the four bilinear corners per node), FP32
    const uint2* quad16;     // the same as 16-bit values (qdt 1: BF16, 2: FP16; quad is then null)
    int qdt;
    int n_cells, n_ls;
    DepJob jobs[kMaxJobs];
    int n_jobs;
    long long* job_cost;     // [n_jobs + 1] device scratch: exclusive prefix of the jobs' per-tile cost
    int n_bands;
    int band_cell0[kMaxBands];  // first cell of each age band's slab
    int n_lambda;
    int tile_w;              // output bins per tile = 31 * rounds (1..12)
    int n_tiles;
    const int* tile_klo;     // [n_tiles] first SSP node of each tile's slab
    int slab_w;              // nodes per slab (0 = no slab: global path only)
    int ncb;                 // cells per slab node (odd)
    int box_w, n_boxes;      // TMA boxes of box_w nodes covering the slab
    int cost_c0;             // per-item cost in particle units
    unsigned* err;
    unsigned long long* slow_count;
};
int launch_deposit(const DepositParams& P, const CUtensorMap* tmap, int n_ctas, int threads, size_t smem,
                   cudaStream_t st);
size_t deposit_smem_bytes(int ncb, int slab_w);

// Zero rows of the spaxels without particles (no work item covers them).
int launch_zero_empty(const int* seg_off, int n_s, int nb, float* cube, int pitch, int n_lambda, cudaStream_t st);

// K5: combine partial rows of split spaxels in a fixed order: FP32 for at most
// kCombineF32Rows rows, a compensated FP32 sum (two-sum) above. list: n_s + 1
// ints of scratch (the split spaxels and their count).
constexpr int kCombineF32Rows = 4;
int launch_combine(const int* part_off, int n_s, int n_lambda, const float* partials, float* cube, int pitch,
                   int* list, cudaStream_t st);

// K6: PSF + LSF (+ noise).
constexpr int kMaxRadius = 64;
struct ConvParams {
    int nx, ny, n_lambda;
    int rp, rl;                  // radii (0 = identity)
    float gp[2 * kMaxRadius + 1];
    float gl[2 * kMaxRadius + 1];
    float noise_inv_s2n;         // 0 = no noise
    uint32_t seed_lo, seed_hi;
    unsigned* err;               // device error word (bounded waits of the TMA kernel)
};
// `in` rows have stride in_pitch floats; `out` is dense ([ny][nx][n_lambda]).
// in_map (nullable): a 3-D TMA map of `in` (x = wavelength over n_lambda, y = x
// spaxel, z = y spaxel; zero fill outside) from conv_tma_map; with it the
// instrument radii take the TMA kernel.
int launch_psf_lsf(const ConvParams& P, const float* in, int in_pitch, const CUtensorMap* in_map, float* tmp,
                   float* out, cudaStream_t st);
// Box the TMA kernel loads for these radii: {wavelength, x}; false if the
// radii have no TMA instantiation.
bool conv_tma_box(int rp, int rl, unsigned box[2]);
// True if launch_psf_lsf needs the intermediate cube `tmp` for these radii.
bool psf_lsf_needs_tmp(int rp, int rl);

// K7/K8: adjoint.
struct AdjointParams {
    SspDev ssp;
    const PartRec* prec;       // [n_in] sorted order
    const int* perm;           // sorted position -> particle index
    const int* seg_off;        // [n_s * n_bands + 2]
    const int* sorted_keys;    // [n] key per sorted position (spaxel * n_bands + band)
    int n_s, n_bands, n_lambda;
    double l0, dl, z_cosmo, flux_scale;
    const float* G0;           // [n_s][n_lambda] dL/dcube0
    float *d_mass, *d_age, *d_Z, *d_v;   // original order, nullable
    double* contrib;           // [n_in][kGlobal] per sorted particle: dL/dv, m*dL/dm, dL/dv * dv/d(incl), dL/dv * dv/d(azim)
    const float2* dv_dang;     // [n] original order: dv_los/d(inclination), dv_los/d(azimuth)
    long long n_in;            // upper bound (grid sizing)
};

// Adjoint over the deposit's (wavelength tile, work item, age band)
// decomposition: per (tile, particle) the four sums
//   part = (sum_j G S, sum_j G dS/dta', sum_j G dS/dtz', sum_j G dS/dt * t_abs)
// over the tile's bins (unit mass), from the same shared-memory quad slabs.
struct AdjTileParams {
    const float4* quad;
    const uint2* quad16;        // 16-bit quads (qdt 1: BF16, 2: FP16; quad is then null)
    int qdt;
    int n_cells, n_ls;
    const DepRec* rec;          // [n_in] forward records (sorted order)
    const float4* wu;           // [n_in] unit-mass bilinear weights (0: spectrum misses every bin)
    const Item* items;
    const int* item_off;        // [n_s + 1]
    const int* seg_off;         // [n_s * n_bands + 2]
    int n_s, n_bands;
    int band_cell0[kMaxBands];
    const float* G0;            // [n_s][n_lambda] dL/d(cube before PSF/LSF)
    float4* part;               // [n_tiles][n_cap]
    long long n_cap;
    int n_lambda, tile_w, n_tiles;
    const int* tile_klo;
    int slab_w, ncb, box_w, n_boxes;
    int cost_c0;
    float ls0_over;             // ls0 / dls: node index -> rest wavelength / dls
    int resample;               // 1: bin means (records hold the bins' lower edges)
    unsigned* err;
};
int launch_adjoint_tiles(const AdjTileParams& P, const CUtensorMap* tmap, int n_ctas, int threads, size_t smem,
                         cudaStream_t st);
// Unit-mass bilinear weights per sorted particle (K7 setup).
int launch_adjoint_setup(const AdjointParams& P, const DepRec* rec, float4* wu, cudaStream_t st);
// Sum of the tiles' parts in FP64 (tile order) and the chain rule to
// dL/d(mass, age, Z, v_los) in original order (+ contributions to global sums).
int launch_adjoint_final(const AdjointParams& P, const float4* part, int n_tiles, long long n_cap, cudaStream_t st);
int launch_zero_grads(float* a, float* b, float* c, float* d, long long n, cudaStream_t st);
// Gradients of the shared parameters: dL/dv_sys, dL/dln(M), dL/d(inclination), dL/d(azimuth).
constexpr int kGlobal = 4;
int launch_reduce_global(const double* contrib, const int* n_in_dev, double* out, double* scratch, cudaStream_t st);

}  // namespace rubix
