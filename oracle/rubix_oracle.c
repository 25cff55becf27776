/*
 * rubix_oracle.c -- plain FP64 CPU oracle of the particle -> IFU data-cube
 * forward model (RUBIX, arXiv 2412.08265, Sec. 3 "RUBIX Codebase") and of its
 * gradient.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or constant generator with the CUDA library; the two meet only in the
 * seeded synthetic inputs.
 *
 * The paper (Sec. 3) lists the pipeline steps in order: orient the galaxy in
 * the field of view, assign particles to IFU spaxels, look each star's
 * spectrum up in an SSP library, Doppler shift it by its line-of-sight
 * velocity, resample onto the telescope's wavelength grid, sum the spectra in
 * each spaxel, convolve with a PSF and an LSF (both Gaussian, Sec. 4), add
 * noise. The paper gives no formulas for these steps; each function below
 * states the reading it implements. Everything is evaluated straight from its
 * definition in FP64, one particle and one wavelength bin at a time, with no
 * blocking or fusion. Threads (pthreads) only split independent output rows;
 * each output value is summed in the same order whatever the thread count.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC -pthread
 * (no FMA contraction: the spaxel keys below must be rounded op by op).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C_KMS 299792.458 /* speed of light, km/s */

/* ---------------------------------------------------------------------- */
/* a1: orientation (Sec. 3: the galaxy is rotated into the field of view   */
/* as its configuration says). Reading: three rotations of the galaxy      */
/* frame, first by the azimuth a about its own z axis, then by the         */
/* inclination i about x, then by the position angle q about the line of   */
/* sight z:  R = Rz(q) Rx(i) Rz(a),  Rz(t) = [[c,-s,0],[s,c,0],[0,0,1]],    */
/* Rx(t) = [[1,0,0],[0,c,-s],[0,s,c]].  x' = (R r)_x, y' = (R r)_y,         */
/* v_los = (R v)_z. With ca = cos a, sa = sin a, ci, si, cq, sq likewise:  */
/*   R00 = cq ca - sq (ci sa)     R01 = -(cq sa) - sq (ci ca)   R02 = sq si */
/*   R10 = sq ca + cq (ci sa)     R11 = cq (ci ca) - sq sa      R12 = -(cq si) */
/*   R20 = si sa                  R21 = si ca                   R22 = ci    */
/* each product and sum rounded once in FP64 in the order written, and     */
/*   x' = (R00 x + R01 y) + R02 z   (likewise y', v_los), no FMA.           */
/* With a = q = 0 this is x' = x, y' = y cos i - z sin i,                  */
/* v_los = vy sin i + vz cos i. The derivatives of v_los that the global   */
/* gradients need (positions have none, reading R12):                      */
/*   dv/di = (ci sa) vx + (ci ca) vy - si vz,  dv/da = si (ca vx - sa vy). */
/* vx may be NULL when a = 0 (its coefficients are then zero).             */
/* ---------------------------------------------------------------------- */
static void or_rotation(double incl, double azim, double pa, double R[9])
{
    double ca = cos(azim), sa = sin(azim), ci = cos(incl), si = sin(incl);
    double cq = cos(pa), sq = sin(pa);
    R[0] = cq * ca - sq * (ci * sa);
    R[1] = -(cq * sa) - sq * (ci * ca);
    R[2] = sq * si;
    R[3] = sq * ca + cq * (ci * sa);
    R[4] = cq * (ci * ca) - sq * sa;
    R[5] = -(cq * si);
    R[6] = si * sa;
    R[7] = si * ca;
    R[8] = ci;
}

int or_orient(int64_t n, const float *x, const float *y, const float *z, const float *vx,
              const float *vy, const float *vz, const float *vlos, int preprojected,
              double incl, double azim, double pa, double *xp, double *yp, double *v,
              double *dv_di, double *dv_da)
{
    double R[9];
    or_rotation(incl, azim, pa, R);
    double ca = cos(azim), sa = sin(azim), ci = cos(incl), si = sin(incl);
    for (int64_t p = 0; p < n; ++p) {
        if (preprojected) {
            xp[p] = (double)x[p];
            yp[p] = (double)y[p];
            v[p] = (double)vlos[p];
            if (dv_di) dv_di[p] = 0.0;
            if (dv_da) dv_da[p] = 0.0;
            continue;
        }
        double X = (double)x[p], Y = (double)y[p], Z = (double)z[p];
        double VX = vx ? (double)vx[p] : 0.0, VY = (double)vy[p], VZ = (double)vz[p];
        xp[p] = (R[0] * X + R[1] * Y) + R[2] * Z;
        yp[p] = (R[3] * X + R[4] * Y) + R[5] * Z;
        v[p] = (R[6] * VX + R[7] * VY) + R[8] * VZ;
        if (dv_di) dv_di[p] = ((ci * sa) * VX + (ci * ca) * VY) - si * VZ;
        if (dv_da) dv_da[p] = si * (ca * VX - sa * VY);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* a2: spaxel assignment (Sec. 3: each particle goes to one IFU spaxel).  */
/* Reading: a square grid of nx*ny spaxels of side `size`,                 */
/* centred on the origin; spaxel (ix, iy) is the half-open square          */
/* [x_lo + ix*size, x_lo + (ix+1)*size) x [...). Key = iy*nx + ix; a       */
/* particle outside the field (or NaN) gets key nx*ny and is dropped.      */
/* Rounding: x_lo = (-0.5*nx)*size, s = 1/size, u = (x' - x_lo)*s, each    */
/* op rounded to nearest in FP64; ix = floor(u) for 0 <= u < nx.           */
/* ---------------------------------------------------------------------- */
int or_spaxel_keys(int64_t n, const double *xp, const double *yp, int nx, int ny,
                   double size, int32_t *key)
{
    double x_lo = (-0.5 * (double)nx) * size;
    double y_lo = (-0.5 * (double)ny) * size;
    double s = 1.0 / size;
    for (int64_t p = 0; p < n; ++p) {
        double dx = xp[p] - x_lo;
        double dy = yp[p] - y_lo;
        double u = dx * s;
        double w = dy * s;
        if (u >= 0.0 && u < (double)nx && w >= 0.0 && w < (double)ny)
            key[p] = (int32_t)w * nx + (int32_t)u;
        else
            key[p] = nx * ny;
    }
    return 0;
}

/* a3: stable counting sort of particles by key (plain definition of "the */
/* particles of spaxel s, in index order").  seg_off has n_keys+1 entries. */
int or_stable_sort(int64_t n, const int32_t *key, int32_t n_keys, int32_t *perm,
                   int64_t *seg_off)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n_keys + 1, sizeof(int64_t));
    if (!cnt) return 1;
    for (int64_t p = 0; p < n; ++p) cnt[key[p]]++;
    seg_off[0] = 0;
    for (int32_t s = 0; s < n_keys; ++s) seg_off[s + 1] = seg_off[s] + cnt[s];
    for (int32_t s = 0; s < n_keys; ++s) cnt[s] = seg_off[s];
    for (int64_t p = 0; p < n; ++p) perm[cnt[key[p]]++] = (int32_t)p;
    free(cnt);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* a4: SSP lookup (Sec. 3: a star's spectrum comes from an SSP library by */
/* age and metallicity). Reading: bilinear in (log10 age, log10 Z)         */
/* between the four templates around the particle; outside the node range  */
/* the coordinate is clamped to the end node. The cell is the half-open    */
/* interval [node_i, node_i+1) holding the coordinate.                     */
/* Returns 1 if the coordinate is strictly inside the node range (its      */
/* derivative is then 1/(node_i+1 - node_i)), 0 if clamped.                */
/* ---------------------------------------------------------------------- */
static int or_cell(double q, const double *nodes, int n, int *i_out, double *t_out,
                   double *dt_dq)
{
    if (n < 2) { *i_out = 0; *t_out = 0.0; *dt_dq = 0.0; return 0; }
    if (!(q > nodes[0])) { *i_out = 0; *t_out = 0.0; *dt_dq = 0.0; return 0; }
    if (q >= nodes[n - 1]) { *i_out = n - 2; *t_out = 1.0; *dt_dq = 0.0; return 0; }
    int i = 0;
    while (i + 1 < n - 1 && nodes[i + 1] <= q) ++i;
    double h = nodes[i + 1] - nodes[i];
    *i_out = i;
    *t_out = (q - nodes[i]) / h;
    *dt_dq = 1.0 / h;
    return 1;
}

typedef struct {
    int n_age, n_Z, n_ls;
    const double *la_nodes, *lz_nodes;
    double ls0, dls;
    const double *spectra; /* [n_age][n_Z][n_ls] */
} or_ssp;

typedef struct {
    int nx, ny, n_l;
    double l0, dl, z_cosmo, flux_scale;
    int resample; /* 0: value at the bin centre; 1: mean over the bin (flux-conserving) */
} or_tel;

/* Template value with zero extension outside the SSP wavelength range. */
static double or_T(const or_ssp *S, int ia, int iz, int64_t k)
{
    if (k < 0 || k >= S->n_ls) return 0.0;
    return S->spectra[((int64_t)ia * S->n_Z + iz) * S->n_ls + k];
}

/* Per-particle quantities shared by the spectrum and its derivatives. */
typedef struct {
    int ia, iz, ia1, iz1;
    double ta, tz, dta, dtz;      /* interpolation coords and d/d(log10) */
    double w[4];                  /* corner weights 00, 10, 01, 11 */
    double dop;                   /* (1 + z_cosmo)(1 + v/c) */
} or_part;

static void or_particle_setup(const or_ssp *S, const or_tel *T, double age, double Z,
                              double v, or_part *P)
{
    double la = log10(age), lz = log10(Z);
    or_cell(la, S->la_nodes, S->n_age, &P->ia, &P->ta, &P->dta);
    or_cell(lz, S->lz_nodes, S->n_Z, &P->iz, &P->tz, &P->dtz);
    P->ia1 = (P->ia + 1 < S->n_age) ? P->ia + 1 : P->ia;
    P->iz1 = (P->iz + 1 < S->n_Z) ? P->iz + 1 : P->iz;
    P->w[0] = (1.0 - P->ta) * (1.0 - P->tz);
    P->w[1] = P->ta * (1.0 - P->tz);
    P->w[2] = (1.0 - P->ta) * P->tz;
    P->w[3] = P->ta * P->tz;
    P->dop = (1.0 + T->z_cosmo) * (1.0 + v / OR_C_KMS);
}

/* ---------------------------------------------------------------------- */
/* a5: Doppler shift + resampling (Sec. 3). Reading: non-relativistic      */
/* shift, observed = rest * (1 + z_cosmo)(1 + v/c); the template is        */
/* sampled at the rest-frame wavelength of each output bin centre,         */
/*   lambda_j = l0 + j*dl,  lambda_rest = lambda_j / dop,                  */
/*   t = (lambda_rest - ls0)/dls,  k = floor(t),  f = t - k,               */
/* by linear interpolation between nodes k and k+1 (templates are zero     */
/* outside the SSP range). Corner c's resampled template is               */
/*   V_c(j) = (1-f) T_c[k] + f T_c[k+1].                                   */
/* ---------------------------------------------------------------------- */
static void or_bin_position(const or_ssp *S, const or_tel *T, const or_part *P, int j,
                            int64_t *k, double *f, double *lrest)
{
    double lam = T->l0 + (double)j * T->dl;
    double lr = lam / P->dop;
    double t = (lr - S->ls0) / S->dls;
    double fk = floor(t);
    *k = (int64_t)fk;
    *f = t - fk;
    *lrest = lr;
}

static void or_corner_values(const or_ssp *S, const or_part *P, int64_t k, double f,
                             double V[4], double Tk[4], double Tk1[4])
{
    int ia[4] = {P->ia, P->ia1, P->ia, P->ia1};
    int iz[4] = {P->iz, P->iz, P->iz1, P->iz1};
    for (int c = 0; c < 4; ++c) {
        Tk[c] = or_T(S, ia[c], iz[c], k);
        Tk1[c] = or_T(S, ia[c], iz[c], k + 1);
        V[c] = (1.0 - f) * Tk[c] + f * Tk1[c];
    }
}

/* ---------------------------------------------------------------------- */
/* a5, flux-conserving alternative (resample = 1; the paper names only an  */
/* "additional resampling", Sec. 3). Reading: output bin j covers the      */
/* observed interval [lambda_j - dl/2, lambda_j + dl/2], and its value is  */
/* the mean of the shifted spectrum over that interval. With the shift a  */
/* plain scaling of wavelength, this is the mean of the rest-frame         */
/* template over [ta, tb] (node units),                                    */
/*   ta = ((lambda_j - dl/2)/dop - ls0)/dls,  tb = ((lambda_j + dl/2)/dop - ls0)/dls, */
/* where the template between nodes is the same zero-extended linear       */
/* interpolant as above. Summed over the bins, value x width then equals   */
/* the integral of the shifted spectrum over the grid: flux is conserved.  */
/* ---------------------------------------------------------------------- */

/* Weighted template sum_c wc[c] T_c[k] at one node (zero outside). */
static double or_node_mix(const or_ssp *S, const or_part *P, const double wc[4], int64_t k)
{
    int ia[4] = {P->ia, P->ia1, P->ia, P->ia1};
    int iz[4] = {P->iz, P->iz, P->iz1, P->iz1};
    double s = 0.0;
    for (int c = 0; c < 4; ++c) s += wc[c] * or_T(S, ia[c], iz[c], k);
    return s;
}

/* Linear interpolant of the weighted template at node position t. */
static double or_mix_at(const or_ssp *S, const or_part *P, const double wc[4], double t)
{
    double fk = floor(t);
    int64_t k = (int64_t)fk;
    double f = t - fk;
    double m0 = or_node_mix(S, P, wc, k), m1 = or_node_mix(S, P, wc, k + 1);
    return (1.0 - f) * m0 + f * m1;
}

/* Rest-frame node positions of the two edges of output bin j. */
static void or_bin_edges(const or_ssp *S, const or_tel *T, const or_part *P, int j,
                         double *ta, double *tb, double *lra, double *lrb)
{
    double la = T->l0 + ((double)j - 0.5) * T->dl;
    double lb = T->l0 + ((double)j + 0.5) * T->dl;
    *lra = la / P->dop;
    *lrb = lb / P->dop;
    *ta = (*lra - S->ls0) / S->dls;
    *tb = (*lrb - S->ls0) / S->dls;
}

/* Mean of the weighted template's interpolant over [ta, tb]: the integral  */
/* segment by segment (the midpoint value of a linear piece times its      */
/* length is its exact integral), divided by tb - ta. Segments [k, k+1]     */
/* with k < -1 or k >= n_ls are zero and skipped.                          */
static double or_mix_mean(const or_ssp *S, const or_part *P, const double wc[4], double ta,
                          double tb)
{
    double k_lo = floor(ta), k_hi = floor(tb);
    if (k_lo < -1.0) k_lo = -1.0;
    if (k_hi > (double)S->n_ls - 1.0) k_hi = (double)S->n_ls - 1.0;
    double s = 0.0;
    for (double kd = k_lo; kd <= k_hi; kd += 1.0) {
        int64_t k = (int64_t)kd;
        double u0 = ta > kd ? ta : kd, u1 = tb < kd + 1.0 ? tb : kd + 1.0;
        if (!(u1 > u0)) continue;
        double m0 = or_node_mix(S, P, wc, k), m1 = or_node_mix(S, P, wc, k + 1);
        double mid = 0.5 * (u0 + u1) - kd;
        s += (u1 - u0) * (m0 + (m1 - m0) * mid);
    }
    return s / (tb - ta);
}

/* Spectrum of one particle on the output grid (a4 + a5 + mass scaling):  */
/*   S_p(j) = flux_scale * m_p * sum_c w_c V_c(j),                         */
/* V_c(j) the corner template at bin j's centre (resample = 0) or its mean */
/* over bin j (resample = 1).                                              */
int or_particle_spectrum(const or_ssp *S, const or_tel *T, double mass, double age,
                         double Z, double v, double *out)
{
    or_part P;
    or_particle_setup(S, T, age, Z, v, &P);
    if (T->resample) {
        for (int j = 0; j < T->n_l; ++j) {
            double ta, tb, lra, lrb;
            or_bin_edges(S, T, &P, j, &ta, &tb, &lra, &lrb);
            out[j] = T->flux_scale * mass * or_mix_mean(S, &P, P.w, ta, tb);
        }
        return 0;
    }
    for (int j = 0; j < T->n_l; ++j) {
        int64_t k; double f, lr, V[4], a[4], b[4];
        or_bin_position(S, T, &P, j, &k, &f, &lr);
        or_corner_values(S, &P, k, f, V, a, b);
        double s = 0.0;
        for (int c = 0; c < 4; ++c) s += P.w[c] * V[c];
        out[j] = T->flux_scale * mass * s;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* a6: per-spaxel sum (Sec. 3: the spectra of a spaxel's stars are added) */
/*  cube0[s][j] = sum over particles p with key_p = s, in                  */
/* increasing p, of S_p(j).  Only spaxels with mask[s] != 0 are computed   */
/* (mask may be NULL = all); the others are left at zero.                  */
/* ---------------------------------------------------------------------- */
typedef struct {
    const or_ssp *S; const or_tel *T;
    int64_t n; const int32_t *key; const double *v;
    const float *mass, *age, *Z;
    const uint8_t *mask;
    double *cube;
    int row0, row1; /* spaxel rows iy in [row0, row1) */
} or_dep_job;

static void *or_deposit_worker(void *arg)
{
    or_dep_job *J = (or_dep_job *)arg;
    const or_tel *T = J->T;
    int ns = T->nx * T->ny;
    double *spec = (double *)malloc(sizeof(double) * (size_t)T->n_l);
    if (!spec) return (void *)1;
    for (int64_t p = 0; p < J->n; ++p) {
        int s = J->key[p];
        if (s < 0 || s >= ns) continue;
        int iy = s / T->nx;
        if (iy < J->row0 || iy >= J->row1) continue;
        if (J->mask && !J->mask[s]) continue;
        or_particle_spectrum(J->S, T, (double)J->mass[p], (double)J->age[p],
                             (double)J->Z[p], J->v[p], spec);
        double *row = J->cube + (int64_t)s * T->n_l;
        for (int j = 0; j < T->n_l; ++j) row[j] += spec[j];
    }
    free(spec);
    return NULL;
}

static int or_run_rows(void *(*fn)(void *), void *jobs, size_t job_size, int ny, int n_threads,
                       void (*set_rows)(void *, int, int))
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > ny) n_threads = ny > 0 ? ny : 1;
    pthread_t th[256];
    if (n_threads > 256) n_threads = 256;
    for (int t = 0; t < n_threads; ++t) {
        void *job = (char *)jobs + (size_t)t * job_size;
        set_rows(job, (int)((int64_t)ny * t / n_threads), (int)((int64_t)ny * (t + 1) / n_threads));
    }
    if (n_threads == 1) return fn(jobs) != NULL;
    int err = 0;
    for (int t = 0; t < n_threads; ++t)
        if (pthread_create(&th[t], NULL, fn, (char *)jobs + (size_t)t * job_size)) err = 1;
    for (int t = 0; t < n_threads; ++t) {
        void *r = NULL;
        pthread_join(th[t], &r);
        if (r) err = 1;
    }
    return err;
}

static void or_dep_rows(void *j, int r0, int r1) { ((or_dep_job *)j)->row0 = r0; ((or_dep_job *)j)->row1 = r1; }

int or_deposit(int64_t n, const int32_t *key, const double *v, const float *mass,
               const float *age, const float *Z,
               int n_age, int n_Z, int n_ls, const double *la_nodes, const double *lz_nodes,
               double ls0, double dls, const double *spectra,
               int nx, int ny, int n_l, double l0, double dl, double z_cosmo, double flux_scale,
               int resample, const uint8_t *mask, int n_threads, double *cube)
{
    or_ssp S = {n_age, n_Z, n_ls, la_nodes, lz_nodes, ls0, dls, spectra};
    or_tel T = {nx, ny, n_l, l0, dl, z_cosmo, flux_scale, resample};
    memset(cube, 0, sizeof(double) * (size_t)nx * ny * n_l);
    or_dep_job jobs[256];
    if (n_threads > 256) n_threads = 256;
    if (n_threads < 1) n_threads = 1;
    for (int t = 0; t < n_threads; ++t) {
        or_dep_job J = {&S, &T, n, key, v, mass, age, Z, mask, cube, 0, 0};
        jobs[t] = J;
    }
    return or_run_rows(or_deposit_worker, jobs, sizeof(or_dep_job), ny, n_threads, or_dep_rows);
}

/* ---------------------------------------------------------------------- */
/* a7/a8: Gaussian PSF and LSF (Sec. 4: both instrument responses are     */
/* Gaussian).                                                              */
/* Reading: a discrete kernel sampled at integer offsets d, |d| <= r,      */
/* g(d) proportional to exp(-d^2 / (2 sigma^2)), normalised to sum 1; PSF  */
/* sigma = FWHM / (2 sqrt(2 ln 2)) spaxels and 2-D kernel g(dy) g(dx); LSF */
/* sigma in bins = sigma_A / dl; r <= 0 means ceil(4 sigma). Both are      */
/* "same"-size convolutions with zero padding, PSF first, then LSF.       */
/* ---------------------------------------------------------------------- */
int or_gauss_kernel(double sigma, int radius, double *k)
{
    double sum = 0.0;
    for (int d = -radius; d <= radius; ++d) {
        double e = exp(-((double)d * (double)d) / (2.0 * sigma * sigma));
        k[d + radius] = e;
        sum += e;
    }
    for (int d = -radius; d <= radius; ++d) k[d + radius] /= sum;
    return 0;
}

int or_kernel_radius(double sigma, int radius)
{
    if (radius > 0) return radius;
    if (!(sigma > 0.0)) return 0;
    return (int)ceil(4.0 * sigma);
}

typedef struct {
    int nx, ny, n_l, r; const double *k; const double *in; double *out; int row0, row1;
} or_conv_job;
static void or_conv_rows(void *j, int r0, int r1) { ((or_conv_job *)j)->row0 = r0; ((or_conv_job *)j)->row1 = r1; }

/* PSF: out[y][x][j] = sum_{dy,dx} g(dy) g(dx) in[y+dy][x+dx][j]. */
static void *or_psf_worker(void *arg)
{
    or_conv_job *J = (or_conv_job *)arg;
    int r = J->r;
    for (int y = J->row0; y < J->row1; ++y)
        for (int x = 0; x < J->nx; ++x)
            for (int j = 0; j < J->n_l; ++j) {
                double acc = 0.0;
                for (int dy = -r; dy <= r; ++dy) {
                    int yy = y + dy;
                    if (yy < 0 || yy >= J->ny) continue;
                    for (int dx = -r; dx <= r; ++dx) {
                        int xx = x + dx;
                        if (xx < 0 || xx >= J->nx) continue;
                        acc += J->k[dy + r] * J->k[dx + r] *
                               J->in[((int64_t)yy * J->nx + xx) * J->n_l + j];
                    }
                }
                J->out[((int64_t)y * J->nx + x) * J->n_l + j] = acc;
            }
    return NULL;
}

/* LSF: out[y][x][j] = sum_d h(d) in[y][x][j+d]. */
static void *or_lsf_worker(void *arg)
{
    or_conv_job *J = (or_conv_job *)arg;
    int r = J->r;
    for (int y = J->row0; y < J->row1; ++y)
        for (int x = 0; x < J->nx; ++x) {
            const double *row = J->in + ((int64_t)y * J->nx + x) * J->n_l;
            double *o = J->out + ((int64_t)y * J->nx + x) * J->n_l;
            for (int j = 0; j < J->n_l; ++j) {
                double acc = 0.0;
                for (int d = -r; d <= r; ++d) {
                    int jj = j + d;
                    if (jj < 0 || jj >= J->n_l) continue;
                    acc += J->k[d + r] * row[jj];
                }
                o[j] = acc;
            }
        }
    return NULL;
}

static int or_conv(void *(*fn)(void *), int nx, int ny, int n_l, double sigma, int radius,
                   const double *in, double *out, int n_threads)
{
    int r = or_kernel_radius(sigma, radius);
    if (!(sigma > 0.0)) { /* no convolution: identity */
        memcpy(out, in, sizeof(double) * (size_t)nx * ny * n_l);
        return 0;
    }
    double *k = (double *)malloc(sizeof(double) * (size_t)(2 * r + 1));
    if (!k) return 1;
    or_gauss_kernel(sigma, r, k);
    or_conv_job jobs[256];
    if (n_threads > 256) n_threads = 256;
    if (n_threads < 1) n_threads = 1;
    for (int t = 0; t < n_threads; ++t) {
        or_conv_job J = {nx, ny, n_l, r, k, in, out, 0, 0};
        jobs[t] = J;
    }
    int err = or_run_rows(fn, jobs, sizeof(or_conv_job), ny, n_threads, or_conv_rows);
    free(k);
    return err;
}

int or_psf(int nx, int ny, int n_l, double fwhm, int radius, const double *in, double *out,
           int n_threads)
{
    double sigma = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    return or_conv(or_psf_worker, nx, ny, n_l, sigma, radius, in, out, n_threads);
}

int or_lsf(int nx, int ny, int n_l, double sigma_A, double dl, int radius, const double *in,
           double *out, int n_threads)
{
    return or_conv(or_lsf_worker, nx, ny, n_l, sigma_A / dl, radius, in, out, n_threads);
}

/* Final (PSF then LSF) cube values for listed spaxels only, straight from */
/* the definition: out[i][j] = sum_{dy,dx,d} h(d) g(dy) g(dx)               */
/*                              cube0[y+dy][x+dx][j+d].                     */
int or_psf_lsf_at(int nx, int ny, int n_l, double fwhm, int psf_radius, double sigma_A,
                  double dl, int lsf_radius, const double *cube0, int n_sel,
                  const int32_t *sel_spaxels, double *out)
{
    double sp = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    double sl = sigma_A / dl;
    int rp = (sp > 0.0) ? or_kernel_radius(sp, psf_radius) : 0;
    int rl = (sl > 0.0) ? or_kernel_radius(sl, lsf_radius) : 0;
    double g[256], h[256];
    if (rp > 127 || rl > 127) return 1;
    if (sp > 0.0) or_gauss_kernel(sp, rp, g); else g[0] = 1.0;
    if (sl > 0.0) or_gauss_kernel(sl, rl, h); else h[0] = 1.0;
    for (int i = 0; i < n_sel; ++i) {
        int s = sel_spaxels[i];
        int y = s / nx, x = s % nx;
        for (int j = 0; j < n_l; ++j) {
            double acc = 0.0;
            for (int d = -rl; d <= rl; ++d) {
                int jj = j + d;
                if (jj < 0 || jj >= n_l) continue;
                double a2 = 0.0;
                for (int dy = -rp; dy <= rp; ++dy) {
                    int yy = y + dy;
                    if (yy < 0 || yy >= ny) continue;
                    for (int dx = -rp; dx <= rp; ++dx) {
                        int xx = x + dx;
                        if (xx < 0 || xx >= nx) continue;
                        a2 += g[dy + rp] * g[dx + rp] * cube0[((int64_t)yy * nx + xx) * n_l + jj];
                    }
                }
                acc += h[d + rl] * a2;
            }
            out[(int64_t)i * n_l + j] = acc;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* a10: analytic gradient (Sec. 1/Abstract: gradients through the whole    */
/* pipeline). Given G0 = dL/d(cube0), the gradient of the loss with        */
/* respect to the pre-convolution cube (the caller forms it by applying    */
/* the transposed LSF and PSF to dL/dcube), for each in-field particle:    */
/*   dL/dm   = fs * sum_j G0[s][j] * sum_c w_c V_c(j)                      */
/*   dL/dla  = fs m dta * sum_j G0 [(1-tz)(V10-V00) + tz(V11-V01)]         */
/*   dL/dlz  = fs m dtz * sum_j G0 [(1-ta)(V01-V00) + ta(V11-V10)]         */
/*   dL/dv   = fs m * sum_j G0 * (M(k+1) - M(k)) * dt/dv,                  */
/*             M(k) = sum_c w_c T_c[k],  dt/dv = -lambda_rest/(dls c dop') */
/*             with dop' = 1 + v/c;                                        */
/*   dL/dage = dL/dla / (age ln 10),  dL/dZ = dL/dlz / (Z ln 10).          */
/* The derivative of each piecewise-linear interpolant is taken in the     */
/* half-open cell holding the point; clamped coordinates give 0.           */
/* Out-of-field particles get 0. Outputs are FP64.                         */
/* ---------------------------------------------------------------------- */
typedef struct {
    const or_ssp *S; const or_tel *T; int64_t p0, p1;
    const int32_t *key; const double *v; const float *mass, *age, *Z;
    const double *G0; double *dm, *dage, *dZ, *dv;
} or_grad_job;

static void *or_grad_worker(void *arg)
{
    or_grad_job *J = (or_grad_job *)arg;
    const or_ssp *S = J->S; const or_tel *T = J->T;
    int ns = T->nx * T->ny;
    const double ln10 = log(10.0);
    for (int64_t p = J->p0; p < J->p1; ++p) {
        int s = J->key[p];
        J->dm[p] = J->dage[p] = J->dZ[p] = J->dv[p] = 0.0;
        if (s < 0 || s >= ns) continue;
        or_part P;
        double m = (double)J->mass[p], age = (double)J->age[p], Zp = (double)J->Z[p];
        or_particle_setup(S, T, age, Zp, J->v[p], &P);
        const double *g = J->G0 + (int64_t)s * T->n_l;
        double sm = 0.0, sla = 0.0, slz = 0.0, sv = 0.0;
        double vfac = 1.0 + J->v[p] / OR_C_KMS;
        if (T->resample) {
            /* bin means: S_j is linear in the corner means R_c; d/dv moves   */
            /* both edges, d/dtb of the integral is the interpolant at tb     */
            static const double e[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
            for (int j = 0; j < T->n_l; ++j) {
                double ta, tb, lra, lrb, R[4];
                or_bin_edges(S, T, &P, j, &ta, &tb, &lra, &lrb);
                for (int c = 0; c < 4; ++c) R[c] = or_mix_mean(S, &P, e[c], ta, tb);
                double Sj = 0.0;
                for (int c = 0; c < 4; ++c) Sj += P.w[c] * R[c];
                double ga = (1.0 - P.tz) * (R[1] - R[0]) + P.tz * (R[3] - R[2]);
                double gz = (1.0 - P.ta) * (R[2] - R[0]) + P.ta * (R[3] - R[1]);
                double dta = -lra / (S->dls * OR_C_KMS * vfac);
                double dtb = -lrb / (S->dls * OR_C_KMS * vfac);
                double w = tb - ta;
                double dS = (or_mix_at(S, &P, P.w, tb) * dtb - or_mix_at(S, &P, P.w, ta) * dta) / w
                            - Sj * (dtb - dta) / w;
                sm += g[j] * Sj;
                sla += g[j] * ga;
                slz += g[j] * gz;
                sv += g[j] * dS;
            }
        }
        if (!T->resample)
        for (int j = 0; j < T->n_l; ++j) {
            int64_t k; double f, lr, V[4], a[4], b[4];
            or_bin_position(S, T, &P, j, &k, &f, &lr);
            or_corner_values(S, &P, k, f, V, a, b);
            double Sj = 0.0, Mk = 0.0, Mk1 = 0.0;
            for (int c = 0; c < 4; ++c) { Sj += P.w[c] * V[c]; Mk += P.w[c] * a[c]; Mk1 += P.w[c] * b[c]; }
            double ga = (1.0 - P.tz) * (V[1] - V[0]) + P.tz * (V[3] - V[2]);
            double gz = (1.0 - P.ta) * (V[2] - V[0]) + P.ta * (V[3] - V[1]);
            double dtdv = -lr / (S->dls * OR_C_KMS * vfac);
            sm += g[j] * Sj;
            sla += g[j] * ga;
            slz += g[j] * gz;
            sv += g[j] * (Mk1 - Mk) * dtdv;
        }
        double fs = T->flux_scale;
        J->dm[p] = fs * sm;
        J->dage[p] = fs * m * P.dta * sla / (age * ln10);
        J->dZ[p] = fs * m * P.dtz * slz / (Zp * ln10);
        J->dv[p] = fs * m * sv;
    }
    return NULL;
}

int or_gradient(int64_t n, const int32_t *key, const double *v, const float *mass,
                const float *age, const float *Z,
                int n_age, int n_Z, int n_ls, const double *la_nodes, const double *lz_nodes,
                double ls0, double dls, const double *spectra,
                int nx, int ny, int n_l, double l0, double dl, double z_cosmo, double flux_scale,
                int resample, const double *G0, int n_threads, double *dm, double *dage, double *dZ,
                double *dv)
{
    or_ssp S = {n_age, n_Z, n_ls, la_nodes, lz_nodes, ls0, dls, spectra};
    or_tel T = {nx, ny, n_l, l0, dl, z_cosmo, flux_scale, resample};
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    or_grad_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < n_threads; ++t) {
        or_grad_job J = {&S, &T, n * t / n_threads, n * (t + 1) / n_threads, key, v, mass, age, Z,
                         G0, dm, dage, dZ, dv};
        jobs[t] = J;
    }
    if (n_threads == 1) { or_grad_worker(&jobs[0]); return 0; }
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, or_grad_worker, &jobs[t]);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    return 0;
}
