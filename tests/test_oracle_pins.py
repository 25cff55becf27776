"""Pins of the FP64 oracle against closed forms, invariants, library routines and
brute force (CPU only). Each test names the step of the pipeline (Sec. 3 of the
paper) and the reading it checks. A mistake anywhere in the oracle (a dropped
term, a wrong sign or index, a transposed operand) fails at least one of these.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2412_08265_gb300 import synth
import _brute as brute


def tiny_ssp(seed=7):
    return synth.ssp_grid(4, 3, 80, 4000.0, 4158.0, seed=seed)  # dlambda_s = 2 A


def tiny_tel(**kw):
    d = dict(nx=6, ny=5, spaxel_size=0.5, n_lambda=64, lambda0=4010.0, dlambda=2.1,
             psf_fwhm=1.5, lsf_sigma=2.5)
    d.update(kw)
    return synth.Telescope(**d)


def tiny_particles(n=40, seed=3, spread=1.8, vmax=300.0):
    rng = np.random.default_rng(seed)
    f = lambda a: np.asarray(a, dtype=np.float32)
    return synth.Particles(
        x=f(rng.uniform(-spread, spread, n)), y=f(rng.uniform(-spread, spread, n)),
        mass=f(np.exp(rng.normal(np.log(1e5), 0.5, n))),
        age=f(np.exp(rng.uniform(np.log(0.05), np.log(20.0), n))),   # includes clamped ages
        Z=f(np.exp(rng.uniform(np.log(5e-5), np.log(0.06), n))),     # includes clamped Z
        v_los=f(rng.uniform(-vmax, vmax, n)), preprojected=True)


# --------------------------------------------------------------------------
# a1 orientation
# --------------------------------------------------------------------------
def test_orientation_identity_and_edge_on():
    p = synth.disk_3d(500, 11, inclination=0.0)
    xp, yp, v = oracle.orient(p)
    assert np.array_equal(xp, p.x.astype(np.float64))
    assert np.array_equal(yp, p.y.astype(np.float64))
    assert np.array_equal(v, p.vz.astype(np.float64))
    p.inclination = math.pi / 2
    xp, yp, v = oracle.orient(p)
    # edge-on: the line of sight is the old y axis; y' = -z
    np.testing.assert_allclose(yp, -p.z.astype(np.float64), atol=1e-14)
    np.testing.assert_allclose(v, p.vy.astype(np.float64), atol=1e-12)


def test_orientation_is_a_rotation():
    """|(y', z')| is preserved: the projected y and the line-of-sight velocity come
    from a proper rotation (checked through the velocity, the norm of (vy, vz))."""
    p = synth.disk_3d(300, 12, inclination=0.7)
    _, yp, v = oracle.orient(p)
    ci, si = math.cos(0.7), math.sin(0.7)
    vy = p.vy.astype(np.float64); vz = p.vz.astype(np.float64)
    v_perp = vy * ci - vz * si
    np.testing.assert_allclose(v * v + v_perp * v_perp, vy * vy + vz * vz, rtol=1e-12)
    y = p.y.astype(np.float64); z = p.z.astype(np.float64)
    z_rot = y * si + z * ci
    np.testing.assert_allclose(yp * yp + z_rot * z_rot, y * y + z * z, rtol=1e-12, atol=1e-14)


def test_orientation_euler_angles_match_scipy():
    """R = Rz(position angle) Rx(inclination) Rz(azimuth) against scipy's
    extrinsic z-x-z Euler rotation, for random angles."""
    rng = np.random.default_rng(4)
    for k in range(6):
        p = synth.disk_3d(200, 40 + k, inclination=float(rng.uniform(0, math.pi)),
                          azimuth=float(rng.uniform(-math.pi, math.pi)),
                          position_angle=float(rng.uniform(-math.pi, math.pi)))
        got = oracle.orient(p)
        ref = brute.projected(p)
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


def test_orientation_inclination_only_is_bitwise_the_plain_formula():
    """Azimuth and position angle 0: x' = x, y' = y cos i - z sin i and
    v_los = vy sin i + vz cos i, each operation rounded once (bitwise)."""
    p = synth.disk_3d(1000, 13, inclination=0.83)
    xp, yp, v = oracle.orient(p)
    ci, si = math.cos(0.83), math.sin(0.83)
    f = lambda a: a.astype(np.float64)
    assert np.array_equal(xp, f(p.x))
    assert np.array_equal(yp, f(p.y) * ci - f(p.z) * si)
    assert np.array_equal(v, f(p.vy) * si + f(p.vz) * ci)


def test_position_angle_turns_the_sky_plane():
    """The position angle rotates (x', y') about the line of sight and leaves
    v_los bitwise unchanged."""
    p = synth.disk_3d(500, 14, inclination=0.6, azimuth=0.3)
    x0, y0, v0 = oracle.orient(p)
    q = 1.1
    p.position_angle = q
    x1, y1, v1 = oracle.orient(p)
    assert np.array_equal(v0, v1)
    np.testing.assert_allclose(x1, math.cos(q) * x0 - math.sin(q) * y0, atol=1e-12)
    np.testing.assert_allclose(y1, math.sin(q) * x0 + math.cos(q) * y0, atol=1e-12)


def test_orientation_velocity_derivatives():
    """dv_los/d(inclination) and dv_los/d(azimuth) against central differences."""
    p = synth.disk_3d(300, 15, inclination=0.9, azimuth=-0.4, position_angle=0.2)
    _, _, v, di, da = oracle.orient(p, derivatives=True)
    h = 1e-6
    for name, d in (("inclination", di), ("azimuth", da)):
        x0 = getattr(p, name)
        setattr(p, name, x0 + h)
        vp = oracle.orient(p)[2]
        setattr(p, name, x0 - h)
        vm = oracle.orient(p)[2]
        setattr(p, name, x0)
        np.testing.assert_allclose(d, (vp - vm) / (2 * h), rtol=0, atol=1e-6 * np.abs(d).max())
    pp = tiny_particles(n=10)
    _, _, _, di, da = oracle.orient(pp, derivatives=True)
    assert not di.any() and not da.any()


# --------------------------------------------------------------------------
# a2 spaxel keys (reading C1/C3: half-open spaxels, FoV centred on 0)
# --------------------------------------------------------------------------
def test_spaxel_keys_edges():
    tel = synth.Telescope(nx=4, ny=3, spaxel_size=0.5, n_lambda=1, lambda0=5000.0, dlambda=1.0)
    # x_lo = -1.0, x_hi = 1.0; y_lo = -0.75, y_hi = 0.75
    xs = np.array([-1.0, -0.5, 0.0, 0.5, 0.99999, 1.0, -1.0000001, 0.25, 0.0, 0.0, np.nan])
    ys = np.array([-0.75, 0.0, 0.25, 0.74, 0.0, 0.0, 0.0, -0.25, 0.75, -0.7500001, 0.0])
    key = oracle.spaxel_keys(xs, ys, tel)
    expect = [0 * 4 + 0, 1 * 4 + 1, 2 * 4 + 2, 2 * 4 + 3, 1 * 4 + 3, 12, 12, 1 * 4 + 2, 12, 12, 12]
    assert key.tolist() == expect


def test_spaxel_keys_vs_exact_rationals():
    p = synth.disk_projected(3000, 5)
    tel = synth.Telescope(nx=25, ny=25, spaxel_size=0.5, n_lambda=1, lambda0=5000.0, dlambda=1.0)
    xp, yp, _ = oracle.orient(p)
    key = oracle.spaxel_keys(xp, yp, tel)
    n_checked = 0
    for i in range(p.n):
        ex = brute.exact_spaxel(xp[i], yp[i], tel)
        if ex is None:
            # exactly outside unless within rounding of the border
            assert key[i] == tel.nx * tel.ny or abs(abs(xp[i]) - 6.25) < 1e-9 or abs(abs(yp[i]) - 6.25) < 1e-9
            continue
        ix, iy, u, w = ex
        near = min(abs(float(u) - round(float(u))), abs(float(w) - round(float(w)))) < 1e-9
        if not near:
            assert key[i] == iy * tel.nx + ix
            n_checked += 1
    assert n_checked > 1500


NEAR_EDGE_ANGLES = [(0.83, 0.0, 0.61), (1.3, -2.4, 0.61), (0.3, 1.1, -1.2), (1.2, 0.4, 2.5)]


@pytest.mark.parametrize("angles", NEAR_EDGE_ANGLES)
def test_near_edge_particles_resolve_one_ulp_of_the_rotation(angles):
    """The near-edge inputs of the GPU key test (tests/_edges.py): the test's
    own projection is the oracle's bit for bit, every constructed x' or y'
    lies within 3 FP64 ulps of a key edge, and a one-ulp change of any
    in-plane element of R (R00, R01, R10, R11) moves some of them to another
    spaxel -- so a GPU host that rounds R differently cannot pass."""
    import _edges as edges
    tel = synth.serving_telescope(73)
    i, a, q = angles
    x, y, z = edges.near_edge_particles(tel, i, a, q, n_edges=64, seed=1)
    n = len(x)
    assert n > 1000
    zero = np.zeros(n, np.float32)
    p = synth.Particles(x=x, y=y, z=z, vx=zero, vy=zero, vz=zero, mass=np.full(n, 1e5, np.float32),
                        age=np.ones(n, np.float32), Z=np.full(n, 0.01, np.float32), preprojected=False,
                        inclination=i, azimuth=a, position_angle=q)
    xp, yp, _ = oracle.orient(p)
    R = edges.rotation(i, a, q)
    ex, ey = edges.project(R, x, y, z)
    assert np.array_equal(xp, ex) and np.array_equal(yp, ey)
    key = oracle.spaxel_keys(xp, yp, tel)
    assert np.array_equal(key, edges.keys(ex, ey, tel))
    size = tel.spaxel_size
    d = [np.abs(c - (lo + np.round((c - lo) / size) * size)) for c, lo in
         ((xp, (-0.5 * tel.nx) * size), (yp, (-0.5 * tel.ny) * size))]
    assert float(np.minimum(d[0], d[1]).max()) < 1e-14
    for idx in (0, 1, 3, 4):
        for direction in (math.inf, -math.inf):
            px, py = edges.project(edges.perturbed(R, idx, direction), x, y, z)
            assert (edges.keys(px, py, tel) != key).sum() > 0, (idx, direction)


def test_stable_sort_matches_numpy_stable_argsort():
    rng = np.random.default_rng(0)
    key = rng.integers(0, 37, 5000).astype(np.int32)
    perm, seg = oracle.stable_sort(key, 37)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert np.array_equal(seg, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=37))]))


# --------------------------------------------------------------------------
# a4/a5 spectrum (readings C4/C5)
# --------------------------------------------------------------------------
def _one(x, y, mass, age, Z, v):
    f = lambda a: np.array([a], dtype=np.float32)
    return synth.Particles(x=f(x), y=f(y), mass=f(mass), age=f(age), Z=f(Z), v_los=f(v),
                           preprojected=True)


def test_single_particle_is_shifted_scaled_template():
    """(i) one particle reproduces m * T(lambda / (1 + v/c)) at every bin (np.interp)."""
    ssp = tiny_ssp()
    tel = tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0)
    for v in (0.0, 137.0, -451.5, 2900.0):
        p = _one(0.1, -0.2, 3.5e4, 1.7, 0.003, v)
        cube = oracle.forward(p, ssp, tel, n_threads=1)
        key = oracle.spaxel_keys(*oracle.orient(p)[:2], tel)[0]
        row = cube.reshape(-1, tel.n_lambda)[key]
        expect = brute.particle_spectrum(ssp, tel, float(p.mass[0]), float(p.age[0]),
                                         float(p.Z[0]), float(p.v_los[0]))
        np.testing.assert_allclose(row, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
        others = np.delete(cube.reshape(-1, tel.n_lambda), key, axis=0)
        assert not others.any()


def test_grid_node_particle_gives_exact_template():
    """(iii) v = 0, particle on an (age, Z) node, instrument grid = SSP grid."""
    Zf = float(np.float32(2.0 ** -10))
    la = np.array([-1.0, 0.0, 1.0])
    lz = np.array([-4.0, math.log10(Zf), -1.0])
    rng = np.random.default_rng(1)
    spectra = rng.uniform(0.1, 1.0, (3, 3, 50))
    ssp = synth.SSPGrid(la, lz, 4000.0, 2.0, spectra)
    tel = synth.Telescope(nx=2, ny=2, spaxel_size=1.0, n_lambda=50, lambda0=4000.0, dlambda=2.0,
                          psf_fwhm=0.0, lsf_sigma=0.0)
    p = _one(0.5, 0.5, 3.0, 1.0, Zf, 0.0)
    cube = oracle.forward(p, ssp, tel, n_threads=1)
    assert np.array_equal(cube[1, 1], float(np.float32(3.0)) * spectra[1, 1])


def test_bilinear_midpoint_is_average_of_corners():
    la = np.array([-1.0, 0.0, 1.0])
    lz = np.array([-3.0, -2.0])
    rng = np.random.default_rng(2)
    spectra = rng.uniform(0.1, 1.0, (3, 2, 30))
    ssp = synth.SSPGrid(la, lz, 4000.0, 2.0, spectra)
    tel = synth.Telescope(nx=1, ny=1, spaxel_size=1.0, n_lambda=30, lambda0=4000.0, dlambda=2.0,
                          psf_fwhm=0.0, lsf_sigma=0.0)
    age = float(np.float32(10 ** 0.5)); Z = float(np.float32(10 ** -2.5))
    p = _one(0.0, 0.0, 1.0, age, Z, 0.0)
    cube = oracle.forward(p, ssp, tel, n_threads=1)
    ta = (math.log10(age) - 0.0) / 1.0
    tz = (math.log10(Z) + 3.0) / 1.0
    expect = ((1 - ta) * (1 - tz) * spectra[1, 0] + ta * (1 - tz) * spectra[2, 0]
              + (1 - ta) * tz * spectra[1, 1] + ta * tz * spectra[2, 1])
    np.testing.assert_allclose(cube[0, 0], expect, rtol=1e-13)
    assert abs(ta - 0.5) < 1e-6 and abs(tz - 0.5) < 1e-6


def test_clamping_outside_nodes():
    ssp = tiny_ssp()
    tel = tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0, nx=1, ny=1, spaxel_size=10.0)
    young = oracle.forward(_one(0, 0, 1.0, 1e-4, 1e-7, 0.0), ssp, tel, n_threads=1)
    lo = oracle.forward(_one(0, 0, 1.0, 10 ** ssp.log10_age_nodes[0], 10 ** ssp.log10_Z_nodes[0], 0.0),
                        ssp, tel, n_threads=1)
    np.testing.assert_allclose(young, lo, rtol=1e-6)  # FP32 node rounding only


def test_mass_linearity_and_additivity():
    ssp, tel = tiny_ssp(), tiny_tel()
    p = tiny_particles()
    c1 = oracle.forward(p, ssp, tel, n_threads=1)
    p2 = p.subset(np.arange(p.n)); p2.mass = (p.mass * np.float32(2.0)).astype(np.float32)
    c2 = oracle.forward(p2, ssp, tel, n_threads=1)
    np.testing.assert_allclose(c2, 2.0 * c1, rtol=1e-14, atol=0)
    a = p.subset(np.arange(0, 20)); b = p.subset(np.arange(20, p.n))
    np.testing.assert_allclose(oracle.forward(a, ssp, tel, 1) + oracle.forward(b, ssp, tel, 1), c1,
                               rtol=1e-12, atol=1e-12 * c1.max())


# --------------------------------------------------------------------------
# a6 deposit vs brute force (v), threads do not change values
# --------------------------------------------------------------------------
def test_deposit_matches_brute_force():
    ssp, tel = tiny_ssp(), tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0)
    p = tiny_particles(n=60)
    parts = oracle.forward_parts(p, ssp, tel, n_threads=1)
    bf = brute.cube0(p, ssp, tel)
    np.testing.assert_allclose(parts["cube0"], bf, rtol=1e-11, atol=1e-11 * bf.max())
    assert (bf.reshape(-1, tel.n_lambda).sum(1) > 0).sum() >= 10


def test_redshift_and_flux_scale_match_brute_force():
    """A galaxy at cosmological redshift z with a flux scale (distance
    dimming): rest wavelength lambda_j / ((1 + z)(1 + v/c)), spectrum times
    flux_scale; and flux_scale enters linearly."""
    ssp = tiny_ssp()
    tel = tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0, z_cosmo=0.03, flux_scale=2.5e-3)
    p = tiny_particles(n=60)
    got = oracle.forward_parts(p, ssp, tel, n_threads=2)["cube0"]
    bf = brute.cube0(p, ssp, tel)
    np.testing.assert_allclose(got, bf, rtol=1e-11, atol=1e-11 * bf.max())
    one = oracle.forward_parts(p, ssp, tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0, z_cosmo=0.03), n_threads=2)["cube0"]
    np.testing.assert_allclose(got, 2.5e-3 * one, rtol=1e-13, atol=0)
    # the redshift moves the spectrum: z = 0 differs
    z0 = oracle.forward_parts(p, ssp, tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0), n_threads=2)["cube0"]
    assert np.abs(z0 - one).max() > 1e-3 * np.abs(one).max()


# --------------------------------------------------------------------------
# a5, flux-conserving alternative (reading R14): each output bin takes the
# mean of the shifted spectrum over [lambda_j - dl/2, lambda_j + dl/2]
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dl", [0.7, 2.1, 5.3])
def test_bin_mean_matches_brute_force(dl):
    """Bins finer than, about equal to and coarser than the template spacing
    (2 A): the oracle's segment sums against break-point trapezoids."""
    ssp = tiny_ssp()
    n_l = int(150 / dl)
    tel = tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0, dlambda=dl, n_lambda=n_l, lambda0=4003.0,
                   z_cosmo=0.004, flux_scale=0.8, resample=1)
    p = tiny_particles(n=30, vmax=900.0)
    got = oracle.forward_parts(p, ssp, tel, n_threads=2)["cube0"]
    bf = brute.cube0(p, ssp, tel)
    np.testing.assert_allclose(got, bf, rtol=1e-11, atol=1e-11 * bf.max())
    # the bin mean is not the centre sample
    lin = oracle.forward_parts(p, ssp, tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0, dlambda=dl, n_lambda=n_l,
                                                lambda0=4003.0, z_cosmo=0.004, flux_scale=0.8),
                               n_threads=2)["cube0"]
    assert np.abs(lin - got).max() > 1e-4 * np.abs(got).max()


@pytest.mark.parametrize("dl", [0.9, 2.0, 3.7])
def test_bin_mean_conserves_flux(dl):
    """Closed form: with the output grid covering the shifted template's whole
    support, sum_j S_j dl = fs m dop dls sum_k T[k] (each node's hat function
    has unit area in node units), whatever the bin width and shift."""
    ssp = tiny_ssp()
    for v in (0.0, -310.0, 1234.5):
        dop = 1.01 * (1.0 + float(np.float32(v)) / oracle.C_KMS)
        lo = (ssp.lambda0 - 2 * ssp.dlambda) * dop - 3 * dl
        hi = (ssp.lambda0 + (ssp.n_lambda + 1) * ssp.dlambda) * dop + 3 * dl
        tel = tiny_tel(nx=1, ny=1, psf_fwhm=0.0, lsf_sigma=0.0, dlambda=dl, lambda0=lo,
                       n_lambda=int((hi - lo) / dl) + 1, z_cosmo=0.01, flux_scale=1.7, resample=1)
        p = _one(0.0, 0.0, 2.5e4, 0.8, 0.004, v)
        row = oracle.forward_parts(p, ssp, tel, n_threads=1)["cube0"].reshape(-1)
        _, T_ext = brute.interpolated_template(ssp, float(p.age[0]), float(p.Z[0]))
        expect = 1.7 * float(p.mass[0]) * dop * ssp.dlambda * T_ext.sum()
        assert abs(row.sum() * dl - expect) <= 1e-12 * expect


def test_bin_mean_of_linear_template_is_centre_value():
    """A template linear in wavelength: away from its ends the bin mean equals
    the centre sample (the mean of a linear function over an interval is its
    midpoint value), so resample = 1 and resample = 0 agree there."""
    ssp = tiny_ssp()
    lam = ssp.lambda0 + ssp.dlambda * np.arange(ssp.n_lambda)
    slope = np.linspace(0.5, 2.0, ssp.n_age * ssp.n_Z).reshape(ssp.n_age, ssp.n_Z, 1)
    ssp.spectra = (1.0 + slope * (lam - 4000.0) / 100.0) * np.ones((ssp.n_age, ssp.n_Z, 1))
    kw = dict(nx=1, ny=1, psf_fwhm=0.0, lsf_sigma=0.0, lambda0=4020.0, dlambda=2.3, n_lambda=40)
    p = _one(0.0, 0.0, 1.0e4, 2.2, 0.0011, 217.0)
    a = oracle.forward_parts(p, ssp, tiny_tel(resample=1, **kw), n_threads=1)["cube0"].reshape(-1)
    b = oracle.forward_parts(p, ssp, tiny_tel(**kw), n_threads=1)["cube0"].reshape(-1)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_threads_do_not_change_values():
    ssp, tel = tiny_ssp(), tiny_tel()
    p = tiny_particles(n=200)
    a = oracle.forward(p, ssp, tel, n_threads=1)
    b = oracle.forward(p, ssp, tel, n_threads=5)
    assert np.array_equal(a, b)


def test_inclined_galaxy_matches_brute_force():
    ssp = tiny_ssp()
    tel = tiny_tel(nx=5, ny=5, spaxel_size=1.5)
    p = synth.disk_3d(40, 9, inclination=1.1)
    got = oracle.forward(p, ssp, tel, n_threads=2)
    bf = brute.psf_lsf(brute.cube0(p, ssp, tel), tel)
    np.testing.assert_allclose(got, bf, rtol=1e-10, atol=1e-11 * bf.max())


# --------------------------------------------------------------------------
# a7/a8 PSF and LSF (reading C8)
# --------------------------------------------------------------------------
def test_full_pipeline_matches_brute_force():
    ssp, tel = tiny_ssp(), tiny_tel()
    p = tiny_particles(n=50)
    got = oracle.forward(p, ssp, tel, n_threads=3)
    bf = brute.psf_lsf(brute.cube0(p, ssp, tel), tel)
    np.testing.assert_allclose(got, bf, rtol=1e-10, atol=1e-11 * bf.max())


def test_kernel_widths_and_normalisation():
    s = 1.5 / (2 * math.sqrt(2 * math.log(2)))
    assert oracle.kernel_radius(s, 0) == 3
    assert oracle.kernel_radius(1.2 / 1.25, 0) == 4
    assert oracle.kernel_radius(1.2 / 3.0, 0) == 2
    k = oracle.gauss_kernel(s, 3)
    assert abs(k.sum() - 1.0) < 1e-15
    d = np.arange(-3, 4)
    # ratio of neighbouring taps fixes sigma: k(1)/k(0) = exp(-1/(2 sigma^2))
    assert abs(k[4] / k[3] - math.exp(-1.0 / (2 * s * s))) < 1e-14
    assert np.allclose(k, k[::-1], rtol=0, atol=0)
    assert abs((k * d).sum()) < 1e-16


def test_point_source_psf_is_the_kernel():
    tel = synth.Telescope(nx=11, ny=11, spaxel_size=1.0, n_lambda=3, lambda0=5000.0, dlambda=1.0,
                          psf_fwhm=1.5, lsf_sigma=0.0)
    cube = np.zeros((11, 11, 3)); cube[5, 5, 1] = 2.0
    out = oracle.psf(cube, tel, n_threads=1)
    s = 1.5 / (2 * math.sqrt(2 * math.log(2)))
    g = brute.gauss_weights(s, 3)
    np.testing.assert_allclose(out[2:9, 2:9, 1], 2.0 * np.outer(g, g), rtol=1e-14)
    assert out[:, :, 0].sum() == 0 and abs(out.sum() - 2.0) < 1e-14


def test_gaussian_line_widths_add_in_quadrature():
    """(iv) a Gaussian line of sigma_in bins through the LSF has
    sigma_out^2 = sigma_in^2 + sigma_lsf^2 (continuous limit; the discrete,
    4-sigma-truncated kernel changes this by < 2e-4 relative)."""
    n = 401
    tel = synth.Telescope(nx=1, ny=1, spaxel_size=1.0, n_lambda=n, lambda0=5000.0, dlambda=1.25,
                          psf_fwhm=0.0, lsf_sigma=1.2)
    j = np.arange(n); s_in = 3.0
    line = np.exp(-0.5 * ((j - 200.0) / s_in) ** 2)[None, None, :]
    out = oracle.lsf(line, tel, n_threads=1)[0, 0]
    var = lambda y: ((j - 200.0) ** 2 * y).sum() / y.sum()
    s_l = 1.2 / 1.25
    assert abs(var(out) - (var(line[0, 0]) + s_l ** 2)) / (s_in ** 2 + s_l ** 2) < 2e-4
    # exact discrete statement: variances of normalised sequences add
    h = oracle.gauss_kernel(s_l, 0)
    dh = np.arange(-(len(h) // 2), len(h) // 2 + 1)
    var_h = (dh * dh * h).sum()
    assert abs(var(out) - (var(line[0, 0]) + var_h)) < 1e-10
    assert abs(out.sum() - line.sum()) < 1e-10


def test_flux_conserved_through_psf_and_lsf():
    """(ii) with all flux more than r from the borders, PSF and LSF keep the total."""
    ssp = tiny_ssp()
    tel = tiny_tel(nx=12, ny=12, spaxel_size=0.5, n_lambda=120, lambda0=4010.0, dlambda=1.0)
    p = tiny_particles(n=30, spread=1.2, vmax=50.0)
    parts = oracle.forward_parts(p, ssp, tel, n_threads=2)
    c0 = parts["cube0"]
    # keep flux more than the LSF radius (10 bins) from the spectral borders
    inner = c0.copy()
    inner[:, :, :12] = 0; inner[:, :, -12:] = 0
    assert c0[:, :2].sum() == 0 and c0[:, -2:].sum() == 0   # and > r_psf from the x borders
    out = oracle.lsf(oracle.psf(inner, tel, 1), tel, 1)
    assert abs(out.sum() - inner.sum()) <= 1e-12 * inner.sum()
    # and the deposit conserves every particle's spectrum total
    per = sum(brute.particle_spectrum(ssp, tel, float(p.mass[i]), float(p.age[i]), float(p.Z[i]),
                                      float(p.v_los[i])).sum() for i in range(p.n)
              if parts["key"][i] < tel.nx * tel.ny)
    assert abs(c0.sum() - per) <= 1e-11 * per


def test_psf_lsf_at_matches_full_convolution():
    ssp, tel = tiny_ssp(), tiny_tel()
    p = tiny_particles(n=80)
    parts = oracle.forward_parts(p, ssp, tel, n_threads=2)
    sel = np.array([0, 7, 13, 29], dtype=np.int32)
    got = oracle.psf_lsf_at(parts["cube0"], tel, sel)
    full = parts["cube"].reshape(-1, tel.n_lambda)[sel]
    np.testing.assert_allclose(got, full, rtol=1e-12, atol=1e-13 * full.max())


def test_masked_deposit_equals_full_on_mask():
    ssp, tel = tiny_ssp(), tiny_tel()
    p = tiny_particles(n=80)
    xp, yp, v = oracle.orient(p)
    key = oracle.spaxel_keys(xp, yp, tel)
    full = oracle.deposit(key, v, p, ssp, tel, n_threads=1)
    mask = np.zeros(tel.nx * tel.ny, np.uint8); mask[[3, 4, 17]] = 1
    part = oracle.deposit(key, v, p, ssp, tel, mask=mask, n_threads=2)
    f = full.reshape(-1, tel.n_lambda); g = part.reshape(-1, tel.n_lambda)
    assert np.array_equal(f[mask == 1], g[mask == 1])
    assert not g[mask == 0].any()


# --------------------------------------------------------------------------
# a10 gradient vs central finite differences of the FP64 forward (C12)
# --------------------------------------------------------------------------
def _loss_and_G(p, ssp, tel, target):
    cube = oracle.forward(p, ssp, tel, n_threads=1)
    r = cube - target
    return 0.5 * float((r * r).sum()), r


def _G0(G, tel):
    # transposed LSF then transposed PSF; both kernels are symmetric with zero
    # padding, so each transpose is the same convolution
    return oracle.psf(oracle.lsf(G, tel, 1), tel, 1)


@pytest.mark.parametrize("seed,resample", [(0, 0), (1, 0), (2, 1), (3, 1)])
def test_gradient_matches_central_differences(seed, resample):
    ssp = tiny_ssp()
    tel = tiny_tel(nx=5, ny=4, n_lambda=48, resample=resample)
    p = tiny_particles(n=25, seed=seed, spread=1.1)
    p.age = np.clip(p.age, 0.15, 12.0).astype(np.float32)   # stay inside the node range
    p.Z = np.clip(p.Z, 2e-4, 0.035).astype(np.float32)
    rng = np.random.default_rng(100 + seed)
    target = oracle.forward(p, ssp, tel, 1) * (1 + 0.2 * rng.standard_normal((tel.ny, tel.nx, tel.n_lambda)))
    L0, G = _loss_and_G(p, ssp, tel, target)
    parts = oracle.forward_parts(p, ssp, tel, 1)
    dm, dage, dZ, dv = oracle.gradient(parts["key"], parts["v"], p, ssp, tel, _G0(G, tel), 1)
    ns = tel.nx * tel.ny
    checked = 0
    for i in range(p.n):
        if parts["key"][i] >= ns:
            assert dm[i] == dage[i] == dZ[i] == dv[i] == 0.0
            continue
        for name, grad, rel in (("mass", dm, 1e-4), ("age", dage, 1e-4), ("Z", dZ, 1e-4),
                                ("v_los", dv, 1e-4)):
            arr = getattr(p, name)
            x0 = float(arr[i])
            h = max(abs(x0) * rel, 1e-3 if name == "v_los" else 0.0)
            hi = np.float32(x0 + h); lo = np.float32(x0 - h)
            q = p.subset(np.arange(p.n)); getattr(q, name)[i] = hi
            Lp, _ = _loss_and_G(q, ssp, tel, target)
            getattr(q, name)[i] = lo
            Lm, _ = _loss_and_G(q, ssp, tel, target)
            fd = (Lp - Lm) / (float(hi) - float(lo))
            scale = max(abs(fd), abs(grad[i]), 1e-300)
            # kinks (a node crossed inside [lo, hi]) make the FD one-sided: skip those
            if name in ("age", "Z"):
                nodes = ssp.log10_age_nodes if name == "age" else ssp.log10_Z_nodes
                if any(math.log10(float(lo)) <= nd <= math.log10(float(hi)) for nd in nodes):
                    continue
            # central differences with h = 1e-4 |x| agree to 1e-6 (measured worst 5e-7)
            assert abs(fd - grad[i]) <= 1e-6 * scale + 1e-12 * abs(L0), (name, i, fd, grad[i])
            checked += 1
    assert checked >= 40


@pytest.mark.parametrize("resample", [0, 1])
def test_orientation_gradients_match_central_differences(resample):
    """Gradients of the shared orientation angles, dL/d(angle) =
    sum_p dL/dv_p dv_p/d(angle) (positions carry none, R12), against central
    differences of the FP64 loss, with a step that moves no particle to
    another spaxel."""
    ssp = tiny_ssp()
    tel = tiny_tel(nx=5, ny=4, n_lambda=48, resample=resample)
    p = synth.disk_3d(30, 17, inclination=0.7, azimuth=0.5, position_angle=0.3, r_scale=0.8)
    p.age = np.clip(p.age, 0.15, 12.0).astype(np.float32)
    p.Z = np.clip(p.Z, 2e-4, 0.035).astype(np.float32)
    rng = np.random.default_rng(23)
    target = oracle.forward(p, ssp, tel, 1) * (1 + 0.2 * rng.standard_normal((tel.ny, tel.nx, tel.n_lambda)))
    L0, G = _loss_and_G(p, ssp, tel, target)
    parts = oracle.forward_parts(p, ssp, tel, 1)
    assert (parts["key"] < tel.nx * tel.ny).sum() >= 10
    _, _, _, dv = oracle.gradient(parts["key"], parts["v"], p, ssp, tel, _G0(G, tel), 1)
    _, _, _, di, da = oracle.orient(p, derivatives=True)
    h = 1e-6
    for name, dd in (("inclination", di), ("azimuth", da)):
        pred = float((dv * dd).sum())
        x0 = getattr(p, name)
        Ls = []
        for x in (x0 + h, x0 - h):
            setattr(p, name, x)
            key = oracle.spaxel_keys(*oracle.orient(p)[:2], tel)
            assert np.array_equal(key, parts["key"])
            Ls.append(_loss_and_G(p, ssp, tel, target)[0])
        setattr(p, name, x0)
        fd = (Ls[0] - Ls[1]) / (2 * h)
        assert abs(fd - pred) <= 1e-5 * max(abs(fd), abs(pred)) + 1e-9 * abs(L0), (name, fd, pred)
        assert abs(pred) > 1e-6 * abs(L0)


def test_mass_gradient_closed_form():
    """dL/dm for L = <G, cube(m)> is the spectrum per unit mass dotted with G0."""
    ssp, tel = tiny_ssp(), tiny_tel(psf_fwhm=0.0, lsf_sigma=0.0)
    p = tiny_particles(n=12)
    parts = oracle.forward_parts(p, ssp, tel, 1)
    rng = np.random.default_rng(5)
    G = rng.standard_normal(parts["cube0"].shape)
    dm, *_ = oracle.gradient(parts["key"], parts["v"], p, ssp, tel, G, 1)
    for i in range(p.n):
        k = parts["key"][i]
        if k >= tel.nx * tel.ny:
            continue
        s1 = brute.particle_spectrum(ssp, tel, 1.0, float(p.age[i]), float(p.Z[i]), float(p.v_los[i]))
        assert abs(dm[i] - (G.reshape(-1, tel.n_lambda)[k] * s1).sum()) < 1e-10 * np.abs(s1).sum()


# --------------------------------------------------------------------------
# seeded random configurations: the whole forward model against the brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(12))
def test_random_configurations_match_brute_force(seed):
    """Random SSP grids, telescopes (bin width, redshift, flux scale, resampling
    mode, PSF/LSF) and oriented 3-D or projected galaxies: the oracle's cube
    against the independent brute force."""
    rng = np.random.default_rng(1000 + seed)
    n_age, n_Z = int(rng.integers(2, 6)), int(rng.integers(1, 5))
    n_ls = int(rng.integers(40, 120))
    ls_lo = float(rng.uniform(3900.0, 4100.0))
    ssp = synth.ssp_grid(n_age, n_Z, n_ls, ls_lo, ls_lo + float(rng.uniform(1.0, 3.0)) * n_ls, seed=seed)
    dls = ssp.dlambda
    dl = float(dls * rng.uniform(0.4, 2.5))
    n_l = int(rng.integers(8, 60))
    tel = synth.Telescope(nx=int(rng.integers(2, 7)), ny=int(rng.integers(2, 7)),
                          spaxel_size=float(rng.uniform(0.3, 1.2)), n_lambda=n_l,
                          lambda0=float(ls_lo + rng.uniform(0.0, 0.5) * n_ls * dls), dlambda=dl,
                          psf_fwhm=float(rng.choice([0.0, 1.3, 2.2])), lsf_sigma=float(rng.choice([0.0, 1.1 * dl])),
                          z_cosmo=float(rng.choice([0.0, 0.002, 0.01])), flux_scale=float(rng.uniform(0.5, 2.0)),
                          resample=int(rng.integers(0, 2)))
    if seed % 2:
        p = synth.disk_3d(30, seed, inclination=float(rng.uniform(0, np.pi)), r_scale=0.8,
                          azimuth=float(rng.uniform(-np.pi, np.pi)), position_angle=float(rng.uniform(-np.pi, np.pi)))
    else:
        p = tiny_particles(n=30, seed=seed, spread=0.5 * tel.spaxel_size * max(tel.nx, tel.ny))
    got = oracle.forward(p, ssp, tel, n_threads=2)
    bf = brute.psf_lsf(brute.cube0(p, ssp, tel), tel)
    scale = max(float(np.abs(bf).max()), 1e-300)
    np.testing.assert_allclose(got, bf, rtol=0, atol=1e-10 * scale)
