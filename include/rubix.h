/*
 * rubix.h -- C ABI of the GB300 (sm_103a) particle -> IFU data-cube forward
 * model of RUBIX (arXiv 2412.08265). Every step of the pipeline runs in the
 * library's own CUDA kernels; callers pass plain host or device pointers.
 *
 * The pipeline (Sec. 3 "RUBIX Codebase" of the paper):
 *   orient the galaxy in the field of view -> assign particles to spaxels ->
 *   look each star's spectrum up in an SSP library -> Doppler shift by the
 *   line-of-sight velocity -> resample onto the telescope wavelength grid ->
 *   sum the spectra in each spaxel -> convolve with a Gaussian PSF and LSF
 *   (Sec. 4) -> add noise.  Gradients through the pipeline (Abstract, Sec. 1)
 *   are provided by rubix_cube_backward.
 *
 * Readings of the steps the paper leaves unspecified (all implemented exactly
 * this way by the library):
 *   - Orientation: the galaxy frame is turned by the azimuth a about its own
 *     z axis, inclined by i about x, then turned by the position angle q about
 *     the line of sight: R = Rz(q) Rx(i) Rz(a), with (c = cos, s = sin, host
 *     libm, FP64, each product and sum rounded once in the order written)
 *       R00 = cq ca - sq (ci sa)   R01 = -(cq sa) - sq (ci ca)   R02 = sq si
 *       R10 = sq ca + cq (ci sa)   R11 = cq (ci ca) - sq sa      R12 = -(cq si)
 *       R20 = si sa                R21 = si ca                   R22 = ci
 *     x' = (R00 x + R01 y) + R02 z, y' likewise, v_los = (R20 vx + R21 vy) + R22 vz,
 *     no FMA. With a = q = 0: x' = x, y' = y cos i - z sin i,
 *     v_los = vy sin i + vz cos i. (The library decides each key from an FP32
 *     evaluation with an error bound and falls back to this FP64 expression
 *     near spaxel edges, so keys are those of the FP64 expression; v_los,
 *     which decides no integer, is evaluated in FP32 with FMA, within a few
 *     FP32 ulps of the expression.)
 *   - Spaxels: nx*ny squares of side spaxel_size centred on (0, 0), half-open;
 *     x_lo = (-0.5*nx)*size, u = (x' - x_lo) * (1/size) in FP64, ix = floor(u).
 *     Particles outside the field are dropped.
 *   - SSP lookup: bilinear in (log10 age/Gyr, log10 Z), clamped at the grid.
 *   - Doppler + resampling: rest wavelength of output bin j is
 *     (lambda0 + j*dlambda) / ((1 + z_cosmo)(1 + v_los/c)); the template is
 *     linearly interpolated there, and is zero outside its wavelength range.
 *     With rubix_telescope.resample = 1 the bin takes instead the mean of that
 *     interpolant over the bin [lambda_j - dlambda/2, lambda_j + dlambda/2]
 *     mapped to the rest frame (flux-conserving rebinning).
 *   - Spectrum of a particle = flux_scale * mass * interpolated template.
 *   - PSF: 2-D Gaussian, sigma = FWHM / (2 sqrt(2 ln 2)) spaxels; LSF: 1-D
 *     Gaussian, sigma = lsf_sigma / dlambda bins; both sampled at integer
 *     offsets up to r = ceil(4 sigma), normalised to 1, zero padded, PSF first.
 *   - Noise: cube + |cube| / S2N * N(0, 1), N(0,1) from Philox4x32-10 keyed by
 *     the seed, counter = voxel index, Box-Muller.
 *
 * Conventions
 *   - Every call returns a rubix_status; rubix_last_error_message() gives a
 *     thread-local description of the last failure. No exception crosses the ABI.
 *   - The caller owns every buffer it passes. Handles own their device copies
 *     of the SSP grid, their scratch space and the state kept for backward.
 *   - A handle is not thread safe: use one handle per host thread / stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work is enqueued on it; calls return without waiting unless
 *     they must return host data.
 *   - Cube layout: float32 [ny][nx][n_lambda], wavelength fastest.
 */
#ifndef RUBIX_H
#define RUBIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rubix_status;
#define RUBIX_OK 0
#define RUBIX_ERR_INVALID_ARG 1
#define RUBIX_ERR_OOM 2
#define RUBIX_ERR_CUDA 3
#define RUBIX_ERR_TIMEOUT 4
#define RUBIX_ERR_REJECTED 5
#define RUBIX_ERR_CANCELLED 6
#define RUBIX_ERR_NOT_READY 7
#define RUBIX_ERR_UNSUPPORTED 8
#define RUBIX_ERR_DEVICE 9 /* a kernel reported an internal error (e.g. a bounded wait expired) */

/* Storage type of the SSP templates on the device (arithmetic is FP32). */
#define RUBIX_F32 0
#define RUBIX_BF16 1
#define RUBIX_F16 2

/* SSP library (Sec. 3: star spectra are looked up in a simple stellar
 * population library).
 * All pointers are HOST pointers, read during rubix_cube_create only. */
typedef struct rubix_ssp_grid {
    int32_t n_age, n_Z, n_lambda;   /* grid sizes, each >= 1; n_lambda >= 2 */
    const double *log10_age_nodes;  /* [n_age], strictly increasing, log10(age / Gyr) */
    const double *log10_Z_nodes;    /* [n_Z], strictly increasing, log10(Z) */
    double lambda0, dlambda;        /* template wavelengths lambda0 + k*dlambda, Angstrom */
    const double *spectra;          /* [n_age][n_Z][n_lambda], luminosity per unit mass */
    int32_t storage_dtype;          /* RUBIX_F32 | RUBIX_BF16 | RUBIX_F16 */
} rubix_ssp_grid;

/* Telescope / IFU (Sec. 3: the instrument's spatial and spectral grids and its
 * responses; Sec. 4: Gaussian PSF and LSF). */
typedef struct rubix_telescope {
    int32_t nx, ny;                 /* spaxels, each >= 1, nx*ny < 2^24 */
    double spaxel_size;             /* kpc, > 0 */
    int32_t n_lambda;               /* output bins, >= 1 */
    double lambda0, dlambda;        /* bin centres lambda0 + j*dlambda, Angstrom, dlambda > 0 */
    double psf_fwhm;                /* spaxels; 0 = no PSF */
    double lsf_sigma;               /* Angstrom; 0 = no LSF */
    int32_t psf_radius, lsf_radius; /* kernel radii; <= 0 means ceil(4 sigma); each <= 64 */
    double z_cosmo;                 /* cosmological redshift of the galaxy (usually 0) */
    double flux_scale;              /* multiplies every spectrum (e.g. 1/(4 pi d_L^2)); 1 = none */
    int32_t resample;               /* Sec. 3 "additional resampling" onto the output grid:
                                     * 0 = the shifted template at each bin centre (linear
                                     * interpolation between template nodes);
                                     * 1 = its mean over each bin [lambda_j - dlambda/2,
                                     * lambda_j + dlambda/2] (flux-conserving rebinning). */
    int32_t row_lo, row_hi;         /* row window: only spaxel rows [row_lo, row_hi) of the
                                     * ny-row field are modelled (0, 0 = all rows). Spaxel keys
                                     * are computed on the whole field, so a row-sharded galaxy
                                     * (each shard its own rows) gets bitwise the unsharded
                                     * assignment; particles of other rows are dropped. The
                                     * cube then has row_hi - row_lo rows, PSF and LSF see zero
                                     * padding at its edges, noise is keyed by the window's own
                                     * voxel index. */
} rubix_telescope;

/* Star particles (Sec. 3: input handler fields), float32 structure of arrays.
 * preprojected = 1: x, y are sky-plane positions (kpc) and v_los (km/s) is
 *                   given; z, vx, vy, vz are ignored (may be NULL).
 * preprojected = 0: x, y, z (kpc) and vx, vy, vz (km/s) are 3-D; the galaxy
 *                   is oriented by `azimuth`, `inclination` and
 *                   `position_angle` (radians, see Orientation above); vx may
 *                   be NULL when azimuth = 0.
 * mass: Msun; age: Gyr (> 0); Z: metal mass fraction (> 0).
 * on_device = 1: all pointers are device pointers; 0: host pointers (copied
 * to the device inside the call; pinned memory makes the copy asynchronous). */
typedef struct rubix_particles {
    int64_t n;
    const float *x, *y, *z, *vx, *vy, *vz, *v_los;
    const float *mass, *age, *Z;
    int32_t on_device;
    int32_t preprojected;
    double inclination;
    double azimuth, position_angle;
} rubix_particles;

typedef struct rubix_cube rubix_cube_t;
typedef struct rubix_server rubix_server_t;

/* Create a forward-model handle for one SSP grid and one telescope.
 * Copies the SSP grid to the device in its storage dtype (rows padded to 16 B)
 * and reserves scratch for up to `max_particles` particles (grown on demand).
 * Errors: INVALID_ARG (bad sizes, non-increasing nodes, NULL pointers),
 * OOM, CUDA. On error *out is NULL. Uses the current CUDA device. */
rubix_status rubix_cube_create(const rubix_ssp_grid *ssp, const rubix_telescope *tel,
                               int64_t max_particles, rubix_cube_t **out);

/* Forward model (Sec. 3 pipeline): particles -> cube_out [ny][nx][n_lambda].
 * cube_out is a device pointer if cube_on_device = 1, else a host pointer
 * (the call then waits for the device-to-host copy; with page-locked memory
 * the copy runs at the host link's rate, ~190 GB/s on GB300). noise_s2n <= 0 turns the
 * noise off; noise_seed selects the Philox stream. Deterministic: the same
 * inputs give bitwise the same cube. The sorted particle order and setup of
 * this call are kept for rubix_cube_backward.
 * Errors: INVALID_ARG, OOM (scratch growth), CUDA, DEVICE. */
rubix_status rubix_cube_forward(rubix_cube_t *h, const rubix_particles *p, uint64_t noise_seed,
                                float noise_s2n, float *cube_out, int32_t cube_on_device,
                                void *stream);

/* Tag of the most recent successful rubix_cube_forward on this handle: 1 for
 * the first forward, one more for each later one (0 before any). The
 * backward state a handle keeps (sorted particles, per-particle setup)
 * belongs to that forward only; rubix_cube_backward checks the tag. */
rubix_status rubix_cube_forward_tag(rubix_cube_t *h, uint64_t *tag);

/* Adjoint of the most recent noiseless forward on this handle (gradients
 * through the pipeline, Abstract / Sec. 1). forward_tag must be that
 * forward's tag (rubix_cube_forward_tag, read after the forward): a backward
 * meant for an earlier forward -- whose particles the handle no longer holds
 * -- is refused with INVALID_ARG instead of differentiating the wrong
 * particles. dL_dcube: device pointer, float32
 * [ny][nx][n_lambda]. Outputs (device pointers, float32 [n], original particle
 * order, any may be NULL): dL/dmass, dL/dage (per Gyr), dL/dZ, dL/dv_los
 * (per km/s). Out-of-field particles get 0. d_global (device, nullable,
 * float64[4]), gradients of parameters every particle shares: [0] = dL/dv_sys
 * (a systemic velocity added to every particle) = sum of dL/dv_los; [1] =
 * dL/dln(M) for a global mass scale = sum of mass * dL/dmass; [2] =
 * dL/d(inclination) = sum of dL/dv_los * dv_los/di; [3] = dL/d(azimuth)
 * likewise (positions carry no gradient, so the position angle has none and
 * preprojected input gives 0 for [2] and [3]); each summed in FP64 in a fixed
 * order.
 * Errors: INVALID_ARG (no forward yet, a tag other than the most recent
 * forward's, or the forward used noise), CUDA. */
rubix_status rubix_cube_backward(rubix_cube_t *h, uint64_t forward_tag, const float *dL_dcube,
                                 float *d_mass, float *d_age, float *d_Z, float *d_vlos,
                                 double *d_global, void *stream);

rubix_status rubix_cube_destroy(rubix_cube_t *h);

/* Spaxel assignment only (orientation + key, bit-exact definition above):
 * keys_out (device int32 [n]) gets iy*nx + ix, or nx*ny for particles outside
 * (with a row window: (iy - row_lo)*nx + ix, or nx*(row_hi - row_lo) for
 * particles outside the window). */
rubix_status rubix_cube_spaxel_keys(rubix_cube_t *h, const rubix_particles *p, int32_t *keys_out,
                                    void *stream);

/* Copy the sort result of the most recent forward (device pointers):
 * perm_out int32 [n]: particle indices ordered by spaxel key, then by the
 * SSP age band the deposit kernel uses for that handle (stats[8] bands; one
 * band = plain spaxel order), then by index;
 * seg_off_out int32 [nx*ny + 2]: first sorted position of each spaxel key,
 * then n. Either may be NULL. */
rubix_status rubix_cube_sorted(rubix_cube_t *h, int32_t *perm_out, int32_t *seg_off_out,
                               void *stream);

/* Per-stage device times (milliseconds) of the most recent forward, measured
 * with CUDA events on the forward's stream when profiling is on. Order:
 * [0] assign+sort, [1] particle setup + work list, [2] deposit, [3] combine,
 * [4] PSF+LSF+noise, [5] whole forward. Waits for the forward to finish.
 * n_inout: capacity in, number written out. */
rubix_status rubix_cube_set_profiling(rubix_cube_t *h, int32_t enable);
rubix_status rubix_cube_stage_times(rubix_cube_t *h, float *ms, int32_t *n_inout);

/* Time of one stage (index as above) for every forward enqueued since
 * profiling was last enabled (at most 256, oldest first), without waiting
 * between forwards while they are enqueued; waits for them here. */
rubix_status rubix_cube_profile_history(rubix_cube_t *h, int32_t stage, float *ms, int32_t *n_inout);

/* Counters of the most recent forward (waits for it): [0] particles in the
 * field, [1] deposits = in-field particles * n_lambda, [2] (particle, tile)
 * pairs on the global-memory path (Doppler shift beyond the slab halo),
 * [3] deposit launches, [4] kernels launched by the forward, [5] device error
 * word (0 = none; bits: 1 a bounded wait on a slab load expired, 2 a work
 * item pointed outside its buffers, 4 an index check of the bounds-checking
 * build failed), [6] output bins per wavelength tile, [7] SSP nodes per
 * shared-memory slab row, [8] age bands of the template grid.
 * n_inout: capacity in, number written out. */
rubix_status rubix_cube_stats(rubix_cube_t *h, int64_t *stats, int32_t *n_inout);

/* Spaxel assignment + stable sort by spaxel that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory themselves -- for instance when another
 * allocator (a framework's caching allocator, a pool sized at start-up) owns
 * the device's memory budget, or when the call runs in a latency-critical
 * loop where cudaMalloc/cudaFree would synchronise the device.
 * The stable sort of the particles by spaxel key (the key of
 * rubix_cube_spaxel_keys): perm_out (device int32 [n]) lists particle indices
 * by key, ties by index; seg_off_out (device int32 [nx*ny + 2]) gives the
 * first sorted position of each key, then n (entry nx*ny = particles in the
 * field). (rubix_cube_sorted orders each spaxel's particles by SSP age band
 * first; its segment offsets are the same.) Particles must be device pointers (on_device = 1); only
 * x, y (and z when preprojected = 0) are read; the telescope's row window is
 * not applied (the whole field is sorted). Scratch lives in one fixed
 * device array inside the library (about 4.3 MB, held on every device that
 * loads the library until exit). Limits: n <= 262144 and nx*ny <= 262143;
 * larger problems return RUBIX_ERR_INVALID_ARG with a message (and
 * RUBIX_ERR_UNSUPPORTED if the sort's scratch ever outgrew the array). The first call
 * on a device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture. All calls
 * share the array: calls whose work overlaps on the GPU (other streams or
 * threads without ordering) race and give wrong results. */
rubix_status rubix_spaxel_sort_noalloc(const rubix_particles *p, const rubix_telescope *tel,
                                       int32_t *perm_out, int32_t *seg_off_out, void *stream);

/* PSF then LSF of a telescope (Sec. 4: Gaussian responses; the readings above)
 * applied to a device cube: cube_in and cube_out are float32
 * [n_rows][nx][n_lambda] (dense, distinct buffers), zero padded at the cube's
 * borders, no noise; the telescope's row window is not used (n_rows gives the
 * cube's rows). This is the convolution rubix_cube_forward applies after the
 * deposit, bit for bit, so a row-sharded galaxy can convolve each shard's rows
 * together with r_psf halo rows taken from its neighbours (Sec. 4's
 * multi-device runs). May allocate scratch on `stream` for radii without a
 * fused kernel. Errors: INVALID_ARG, CUDA, OOM. */
rubix_status rubix_convolve(const rubix_telescope *tel, const float *cube_in, float *cube_out, int32_t n_rows,
                            void *stream);

/* Measured FP32 FMA throughput of the current device (no counterpart in the
 * paper: the denominator of the deposit kernel's FP32 roofline, measured on
 * the machine and at the clocks the deposit runs at). Runs eight independent
 * chains of FFMA (packed = 0) or packed FFMA2 (packed = 1) in every thread of
 * four 512-thread blocks per SM for about a millisecond, on the legacy
 * default stream, and synchronises. Outputs (host pointers, the last two
 * nullable): flops_per_s (2 per FMA); FMAs per clock per SM; the SM clock in
 * MHz during the run (clock64 against the global timer).
 * Errors: INVALID_ARG, CUDA. */
rubix_status rubix_measure_fp32_peak(int32_t packed, double *flops_per_s, double *fma_per_clk_per_sm,
                                     double *sm_mhz);

/* ---------------------------------------------------------------------------
 * Serving: many galaxies through one resident SSP grid.
 *
 * The paper motivates fast forward modelling for large simulation suites and
 * inference loops (Sec. 1, Sec. 5) but defines no server; this is the
 * library's request interface for that use. A server owns one device copy of
 * the SSP grid, tiled for one output wavelength grid, and a host thread that
 * runs a continuous-batching loop:
 *   - admission: a request is admitted when a slot is free and its device
 *     footprint (every scratch and cube buffer of its forward model) fits in
 *     hbm_budget_bytes next to the requests already on the GPU; the queue is
 *     FIFO, so a large request is never starved by smaller ones behind it;
 *   - each admitted request stages, assigns, sorts and sets up its particles
 *     on its own stream while earlier requests deposit;
 *   - requests whose setup is enqueued are deposited together: one deposit
 *     launch covers up to max_batch galaxies (<= 64) of different particle
 *     counts and cube sizes, sharing each shared-memory template slab; a
 *     launch takes requests in queue order while its estimated work stays
 *     within that of its first request (or a floor of about 2e9 deposits), so
 *     small requests share launches without waiting behind a larger one;
 *   - the combine, PSF, LSF and noise of each request then run on its stream.
 * The work decomposition of a request never depends on the others, so its
 * cube is bitwise the same alone, in any mix, and from rubix_cube_forward.
 * Device memory comes from a stream-ordered pool owned by the server, so the
 * loop never synchronises the device.
 * ------------------------------------------------------------------------- */

/* Create a server on the current device. wavelength_grid gives the output
 * wavelength grid every request must use (n_lambda, lambda0, dlambda,
 * z_cosmo are read). hbm_budget_bytes bounds the summed footprints of the
 * admitted requests (the SSP grid is outside it). max_slots (1..256): requests
 * on the GPU at once. max_batch (1..64): galaxies per deposit launch; 1 gives
 * one galaxy per launch. */
rubix_status rubix_serve_create(const rubix_ssp_grid *ssp, const rubix_telescope *wavelength_grid,
                                size_t hbm_budget_bytes, int32_t max_slots, int32_t max_batch,
                                rubix_server_t **out);

/* Queue one forward model; returns at once with a ticket. Particle arrays and
 * cube_out (float32 [ny][nx][n_lambda], device if cube_on_device else host)
 * belong to the caller and must stay valid until the request is finished.
 * Host particle arrays are copied when the request is admitted; device ones
 * are read in place. noise_seed / noise_s2n as in rubix_cube_forward.
 * RUBIX_ERR_REJECTED: the request's footprint alone exceeds the budget.
 * RUBIX_ERR_INVALID_ARG: bad arguments, or a wavelength grid other than the
 * server's. */
rubix_status rubix_serve_submit(rubix_server_t *srv, const rubix_telescope *tel, const rubix_particles *p,
                                uint64_t noise_seed, float noise_s2n, float *cube_out, int32_t cube_on_device,
                                uint64_t *ticket);

/* Device bytes a request would hold while on the GPU (what admission counts
 * against hbm_budget_bytes), without submitting it. */
rubix_status rubix_serve_footprint(rubix_server_t *srv, const rubix_telescope *tel, const rubix_particles *p,
                                   int32_t cube_on_device, size_t *bytes);

/* Status of a request without waiting: RUBIX_OK (finished; latency_s, if not
 * NULL, gets submit-to-completion seconds), RUBIX_ERR_NOT_READY (queued or on
 * the GPU), or the error that ended it (RUBIX_ERR_CANCELLED, ..._OOM, ...).
 * An unknown ticket gives RUBIX_ERR_INVALID_ARG. */
rubix_status rubix_serve_poll(rubix_server_t *srv, uint64_t ticket, double *latency_s);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; returns as
 * rubix_serve_poll, with RUBIX_ERR_TIMEOUT if the time ran out first. */
rubix_status rubix_serve_wait(rubix_server_t *srv, uint64_t ticket, double timeout_s);

/* Cancel a queued request: RUBIX_OK, and it will never touch its buffers.
 * A request already on the GPU cannot be cancelled: RUBIX_ERR_NOT_READY (it
 * completes normally). A finished request returns its final status. */
rubix_status rubix_serve_cancel(rubix_server_t *srv, uint64_t ticket);

/* Server counters: [0] submitted, [1] finished OK, [2] rejected, [3] cancelled,
 * [4] failed, [5] deposit launches, [6] largest batch, [7] device bytes in use
 * by admitted requests, [8] peak of [7], [9] requests on the GPU now,
 * [10] queued now. n_inout: capacity in, number written out. */
rubix_status rubix_serve_stats(rubix_server_t *srv, int64_t *stats, int32_t *n_inout);

/* Finish every admitted request, cancel the queued ones, stop the loop and
 * free the server. */
rubix_status rubix_serve_destroy(rubix_server_t *srv);

/* Self-test of failure detection (no counterpart in the paper). Every wait in
 * the library's kernels is bounded: when it runs out it sets a bit in the
 * device error word (reported as RUBIX_ERR_DEVICE) and the kernel returns.
 * This call launches one 32-thread kernel on the current device that waits on
 * a shared-memory barrier nothing completes, with that bounded wait and a
 * limit of limit_s seconds (0 < limit_s <= 10), and waits for it: *timed_out
 * is 1 when the wait gave up and the kernel returned. The device stays usable. */
rubix_status rubix_selftest_bounded_wait(double limit_s, int32_t *timed_out);

/* Thread-local message for the last non-OK status returned on this thread. */
const char *rubix_last_error_message(void);

/* Library version string. */
const char *rubix_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RUBIX_H */
