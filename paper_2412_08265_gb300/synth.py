"""Seeded synthetic inputs: star-particle tables, SSP template grids, telescopes.

This module only draws input data. It contains none of the forward model's
arithmetic (no spaxel assignment, interpolation, Doppler shift, deposit or
convolution), so both the CUDA path and the FP64 oracle can consume the same
inputs without sharing any of the method's code.

The paper's own inputs (IllustrisTNG/TNG50 star particles and the MaStar
CB19 SSP library, Sec. 4 "Qualitative Analysis") are not available; these
generators stand in for them with galaxies and templates of the same shape:

* disk: exponential surface density (scale radius 3 kpc), exponential
  vertical profile (scale height 0.3 kpc), rotation 200 km/s * tanh(R/2 kpc),
  isotropic dispersion 50 km/s;
* bulge: Hernquist profile (scale 1 kpc), isotropic, dispersion 150 km/s;
* ages log-uniform on [0.1, 13.5] Gyr, metallicity log-uniform on
  [1e-4, 0.04], masses lognormal (median 1e5 Msun, sigma_ln 0.5);
* SSP templates on log-spaced (age, Z) nodes: three blackbody-like continua
  whose temperatures fall with age, times 20 Gaussian absorption lines whose
  depths vary smoothly with (age, Z).

All generators use numpy's PCG64 with an explicit seed, except
:func:`disk_3d_device`, which draws on a CUDA device with torch's generator.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

C_KMS = 299792.458


# --------------------------------------------------------------------------
# data containers
# --------------------------------------------------------------------------
@dataclass
class Particles:
    """Star-particle table (structure of arrays, float32).

    When ``preprojected`` is True, ``x``/``y`` are sky-plane coordinates in kpc
    and ``v_los`` is the line-of-sight velocity in km/s; ``z``/``vx``/``vy``/
    ``vz`` are unused. Otherwise ``x, y, z`` and ``vx, vy, vz`` are 3-D and the
    galaxy frame is turned by ``azimuth`` about its own z axis, inclined by
    ``inclination`` about x and turned by ``position_angle`` about the line of
    sight (radians; R = Rz(position_angle) Rx(inclination) Rz(azimuth)).
    """

    x: np.ndarray
    y: np.ndarray
    mass: np.ndarray
    age: np.ndarray
    Z: np.ndarray
    v_los: np.ndarray | None = None
    z: np.ndarray | None = None
    vx: np.ndarray | None = None
    vy: np.ndarray | None = None
    vz: np.ndarray | None = None
    preprojected: bool = True
    inclination: float = 0.0
    azimuth: float = 0.0
    position_angle: float = 0.0

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, idx: np.ndarray) -> "Particles":
        def take(a):
            return None if a is None else np.ascontiguousarray(a[idx])
        return Particles(x=take(self.x), y=take(self.y), mass=take(self.mass),
                         age=take(self.age), Z=take(self.Z), v_los=take(self.v_los),
                         z=take(self.z), vx=take(self.vx), vy=take(self.vy),
                         vz=take(self.vz), preprojected=self.preprojected,
                         inclination=self.inclination, azimuth=self.azimuth,
                         position_angle=self.position_angle)


@dataclass
class SSPGrid:
    """SSP library on an (age, Z, wavelength) grid.

    ``spectra[ia, iz, k]`` is the luminosity per unit mass (arbitrary units,
    normalised so the grid maximum is 1) at wavelength ``lambda0 + k*dlambda``.
    """

    log10_age_nodes: np.ndarray  # float64 [n_age], log10(age / Gyr)
    log10_Z_nodes: np.ndarray    # float64 [n_Z]
    lambda0: float
    dlambda: float
    spectra: np.ndarray          # float64 [n_age, n_Z, n_lambda]

    @property
    def n_age(self) -> int:
        return int(self.spectra.shape[0])

    @property
    def n_Z(self) -> int:
        return int(self.spectra.shape[1])

    @property
    def n_lambda(self) -> int:
        return int(self.spectra.shape[2])


@dataclass
class Telescope:
    """IFU geometry and instrument response.

    Spaxels are ``spaxel_size`` kpc squares tiling an ``nx`` x ``ny`` field of
    view centred on the origin. Output wavelength bins have centres
    ``lambda0 + j*dlambda`` (j = 0..n_lambda-1). The PSF is a Gaussian of
    FWHM ``psf_fwhm`` spaxels and the LSF a Gaussian of standard deviation
    ``lsf_sigma`` Angstrom; a radius <= 0 means ceil(4 sigma). ``resample``
    0 takes each bin's value at its centre (linear interpolation), 1 the mean
    over the bin ``[lambda_j - dlambda/2, lambda_j + dlambda/2]``
    (flux-conserving rebinning). ``row_lo``, ``row_hi`` select a window of
    spaxel rows to model (0, 0: all rows), as a row-sharded galaxy does.
    """

    nx: int
    ny: int
    spaxel_size: float
    n_lambda: int
    lambda0: float
    dlambda: float
    psf_fwhm: float = 1.5
    lsf_sigma: float = 1.2
    psf_radius: int = 0
    lsf_radius: int = 0
    z_cosmo: float = 0.0
    flux_scale: float = 1.0
    resample: int = 0
    row_lo: int = 0
    row_hi: int = 0


# --------------------------------------------------------------------------
# particles
# --------------------------------------------------------------------------
def _stellar_pops(rng: np.random.Generator, n: int):
    age = np.exp(rng.uniform(math.log(0.1), math.log(13.5), n))
    Z = np.exp(rng.uniform(math.log(1e-4), math.log(0.04), n))
    mass = np.exp(rng.normal(math.log(1e5), 0.5, n))
    return (age.astype(np.float32), Z.astype(np.float32), mass.astype(np.float32))


def disk_projected(n: int, seed: int, r_scale: float = 3.0, v_circ: float = 200.0,
                   r_turn: float = 2.0, sigma_v: float = 50.0,
                   incl_deg_for_vlos: float = 45.0) -> Particles:
    """Face-on exponential disk with line-of-sight velocities.

    Positions are face-on; ``v_los = v_circ tanh(R/r_turn) sin(i) cos(phi) +
    N(0, sigma_v)`` with i = ``incl_deg_for_vlos``. R follows the exponential
    surface density (Gamma(2, r_scale)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    R = rng.gamma(2.0, r_scale, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    x = (R * np.cos(phi)).astype(np.float32)
    y = (R * np.sin(phi)).astype(np.float32)
    vlos = (v_circ * np.tanh(R / r_turn) * math.sin(math.radians(incl_deg_for_vlos))
            * np.cos(phi) + rng.normal(0.0, sigma_v, n)).astype(np.float32)
    age, Z, mass = _stellar_pops(rng, n)
    return Particles(x=x, y=y, mass=mass, age=age, Z=Z, v_los=vlos, preprojected=True)


def bulge_plus_disk_projected(n: int, seed: int, bulge_frac: float = 0.3,
                              a_bulge: float = 1.0, sigma_bulge: float = 150.0) -> Particles:
    """Projected Hernquist bulge (fraction ``bulge_frac``) plus the disk above."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = int(round(bulge_frac * n))
    nd = n - nb
    d = disk_projected(nd, seed + 1000003)
    u = rng.uniform(0.0, 1.0, nb)
    su = np.sqrt(u)
    r = a_bulge * su / np.maximum(1.0 - su, 1e-12)
    cth = rng.uniform(-1.0, 1.0, nb)
    ph = rng.uniform(0.0, 2.0 * math.pi, nb)
    sth = np.sqrt(1.0 - cth * cth)
    xb = (r * sth * np.cos(ph)).astype(np.float32)
    yb = (r * sth * np.sin(ph)).astype(np.float32)
    vb = rng.normal(0.0, sigma_bulge, nb).astype(np.float32)
    age, Z, mass = _stellar_pops(rng, nb)
    return Particles(x=np.concatenate([xb, d.x]), y=np.concatenate([yb, d.y]),
                     mass=np.concatenate([mass, d.mass]), age=np.concatenate([age, d.age]),
                     Z=np.concatenate([Z, d.Z]), v_los=np.concatenate([vb, d.v_los]),
                     preprojected=True)


def disk_3d(n: int, seed: int, inclination: float, r_scale: float = 3.0,
            h_scale: float = 0.3, v_circ: float = 200.0, r_turn: float = 2.0,
            sigma_v: float = 50.0, azimuth: float = 0.0, position_angle: float = 0.0) -> Particles:
    """3-D rotating exponential disk in the x-y plane, to be inclined by the library."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = rng.gamma(2.0, r_scale, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    zz = rng.laplace(0.0, h_scale, n)
    vphi = v_circ * np.tanh(R / r_turn)
    vx = -vphi * np.sin(phi) + rng.normal(0.0, sigma_v, n)
    vy = vphi * np.cos(phi) + rng.normal(0.0, sigma_v, n)
    vz = rng.normal(0.0, sigma_v, n)
    age, Z, mass = _stellar_pops(rng, n)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Particles(x=f32(R * np.cos(phi)), y=f32(R * np.sin(phi)), z=f32(zz),
                     vx=f32(vx), vy=f32(vy), vz=f32(vz), mass=mass, age=age, Z=Z,
                     preprojected=False, inclination=float(inclination), azimuth=float(azimuth),
                     position_angle=float(position_angle))


# --------------------------------------------------------------------------
# SSP grid
# --------------------------------------------------------------------------
_HC_OVER_K = 1.438776877e8  # Angstrom * Kelvin


def ssp_grid(n_age: int, n_Z: int, n_lambda: int, lambda_lo: float, lambda_hi: float,
             seed: int = 12345, n_lines: int = 20) -> SSPGrid:
    """Smooth synthetic SSP grid on log-spaced (age, Z) nodes.

    Each template is ``sum_i c_i(Z) B(lambda, T_i(age))`` with three
    blackbody-like terms, ``T_i = T_i0 (age/0.1 Gyr)^(-gamma_i)``, multiplied by
    ``prod_l (1 - d_l(age, Z) exp(-(lambda - mu_l)^2 / (2 w_l^2)))``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    la = np.linspace(math.log10(0.1), math.log10(13.5), n_age)
    lz = np.linspace(math.log10(1e-4), math.log10(0.04), n_Z)
    lam = lambda_lo + np.arange(n_lambda, dtype=np.float64) * ((lambda_hi - lambda_lo) / (n_lambda - 1))
    T0 = np.array([3.0e4, 1.0e4, 5.0e3])
    gam = np.array([0.35, 0.2, 0.1]) * (1.0 + 0.1 * rng.uniform(-1, 1, 3))
    zn = (lz - lz[0]) / max(lz[-1] - lz[0], 1e-30) if n_Z > 1 else np.zeros(1)
    an = (la - la[0]) / max(la[-1] - la[0], 1e-30) if n_age > 1 else np.zeros(1)
    c0 = np.array([1.0, 0.6, 0.4]) * (1.0 + 0.2 * rng.uniform(-1, 1, 3))
    cz = rng.uniform(-0.5, 0.5, 3)
    mu = rng.uniform(lambda_lo + 20.0, lambda_hi - 20.0, n_lines)
    w = rng.uniform(1.5, 6.0, n_lines)
    d0 = rng.uniform(0.2, 0.8, n_lines)
    da = rng.uniform(-0.5, 0.5, n_lines)
    dz = rng.uniform(-0.5, 0.5, n_lines)
    spectra = np.empty((n_age, n_Z, n_lambda), dtype=np.float64)
    for ia in range(n_age):
        age = 10.0 ** la[ia]
        Ti = T0 * (age / 0.1) ** (-gam)
        bb = []
        for i in range(3):
            x = _HC_OVER_K / (lam * Ti[i])
            b = lam ** -5.0 / np.expm1(np.minimum(x, 700.0))
            bb.append(b / b.max())
        for iz in range(n_Z):
            cont = sum(c0[i] * (1.0 + cz[i] * (zn[iz] - 0.5)) * bb[i] for i in range(3))
            depth = np.clip(d0 * (1.0 + da * (an[ia] - 0.5) + dz * (zn[iz] - 0.5)), 0.0, 0.9)
            absn = np.ones_like(lam)
            for l in range(n_lines):
                absn *= 1.0 - depth[l] * np.exp(-0.5 * ((lam - mu[l]) / w[l]) ** 2)
            spectra[ia, iz] = cont * absn
    spectra /= spectra.max()
    return SSPGrid(log10_age_nodes=la, log10_Z_nodes=lz, lambda0=float(lambda_lo),
                   dlambda=float((lambda_hi - lambda_lo) / (n_lambda - 1)), spectra=spectra)


# --------------------------------------------------------------------------
# named workloads (shapes of the paper's runs, Sec. 4)
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    particles: Particles
    ssp: SSPGrid
    telescope: Telescope
    template_dtype: str = "f32"
    extra: dict = field(default_factory=dict)


def small_galaxy(n: int = 10_000, seed: int = 0) -> Workload:
    """1e4-particle disk, 12x6x2000 SSP (3600-7400 A), 25x25 spaxels of 0.5 kpc,
    1000 bins of 3 A on 4000-7000 A, PSF FWHM 1.5 spaxels, LSF sigma 1.2 A."""
    return Workload("small-disk-1e4p-25x25x1000", disk_projected(n, seed),
                    ssp_grid(12, 6, 2000, 3600.0, 7400.0),
                    Telescope(nx=25, ny=25, spaxel_size=0.5, n_lambda=1000,
                              lambda0=4001.5, dlambda=3.0))


def _muse_like_ssp() -> SSPGrid:
    return ssp_grid(50, 10, 3721, 4700.0, 9450.0)


def mid_galaxy(n: int = 1_000_000, seed: int = 1) -> Workload:
    """1e6-particle disk, 50x10x3721 FP32 SSP, 150x150 spaxels of 0.2 kpc,
    3721 bins of 1.25 A from 4750 A."""
    return Workload("mid-disk-1e6p-150x150x3721-f32", disk_projected(n, seed), _muse_like_ssp(),
                    Telescope(nx=150, ny=150, spaxel_size=0.2, n_lambda=3721,
                              lambda0=4750.0, dlambda=1.25))


def large_galaxy(n: int = 20_000_000, seed: int = 2) -> Workload:
    """2e7 particles, 30% Hernquist bulge + disk, BF16 templates,
    300x300 spaxels of 0.1 kpc x 3721 bins."""
    return Workload("large-bulge-disk-2e7p-300x300x3721-bf16",
                    bulge_plus_disk_projected(n, seed), _muse_like_ssp(),
                    Telescope(nx=300, ny=300, spaxel_size=0.1, n_lambda=3721,
                              lambda0=4750.0, dlambda=1.25), template_dtype="bf16")


def perturbed_target(p: Particles, seed: int = 4242, rel_sigma: float = 0.1,
                     dv: float = 20.0) -> Particles:
    """Particles whose ages and metallicities are scaled by (1 + N(0, rel_sigma))
    and whose velocities are shifted by ``dv`` km/s (the target galaxy of the
    differentiable workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = p.n
    age = (p.age * (1.0 + rng.normal(0.0, rel_sigma, n))).astype(np.float32)
    Z = (p.Z * (1.0 + rng.normal(0.0, rel_sigma, n))).astype(np.float32)
    age = np.clip(age, 1e-3, None).astype(np.float32)
    Z = np.clip(Z, 1e-6, None).astype(np.float32)
    return Particles(x=p.x, y=p.y, mass=p.mass, age=age, Z=Z,
                     v_los=(p.v_los + np.float32(dv)).astype(np.float32), preprojected=True)


def serving_requests(n_requests: int, seed: int = 4, n_min: float = 1e4, n_max: float = 2e7,
                     side_min: int = 40, side_max: int = 300, rate_hz: float = 1.0,
                     scale_n: float = 1.0):
    """Request stream: Poisson arrival times, particle counts log-uniform on
    [n_min, n_max] (times ``scale_n``), square cubes with side uniform on
    [side_min, side_max] spaxels of 0.2 kpc x 3721 bins, inclination uniform on
    [0, 90] degrees. Returns a list of dicts (arrival_s, n, side, inclination,
    seed); particles are drawn lazily with :func:`disk_3d`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_requests)) * scale_n
    sides = rng.integers(side_min, side_max + 1, n_requests)
    incl = rng.uniform(0.0, 0.5 * math.pi, n_requests)
    return [dict(arrival_s=float(t[i]), n=max(1, int(ns[i])), side=int(sides[i]),
                 inclination=float(incl[i]), seed=int(10_000 + i)) for i in range(n_requests)]


def serving_telescope(side: int) -> Telescope:
    return Telescope(nx=side, ny=side, spaxel_size=0.2, n_lambda=3721, lambda0=4750.0,
                     dlambda=1.25)


def disk_3d_device(n: int, seed: int, device, r_scale: float = 3.0, h_scale: float = 0.3,
                   v_circ: float = 200.0, r_turn: float = 2.0, sigma_v: float = 50.0) -> dict:
    """The distributions of :func:`disk_3d`, drawn on a CUDA device with torch's
    Philox generator (for request streams too large to draw on the host).
    Returns a dict of float32 device tensors x, y, z, vx, vy, vz, mass, age, Z;
    a prefix of length m is itself a sample of m particles."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f = dict(device=device, dtype=torch.float32, generator=g)
    u = lambda: torch.rand(n, **f).clamp_min_(1e-12)
    R = -r_scale * (torch.log(u()) + torch.log(u()))  # Gamma(2, r_scale)
    phi = (2.0 * math.pi) * torch.rand(n, **f)
    s = torch.rand(n, **f) - 0.5                        # Laplace(0, h_scale) by inversion
    zz = -h_scale * torch.sign(s) * torch.log1p(-2.0 * s.abs()).clamp_max(0.0)
    vphi = v_circ * torch.tanh(R / r_turn)
    vx = -vphi * torch.sin(phi) + sigma_v * torch.randn(n, **f)
    vy = vphi * torch.cos(phi) + sigma_v * torch.randn(n, **f)
    vz = sigma_v * torch.randn(n, **f)
    age = torch.exp(math.log(0.1) + (math.log(13.5) - math.log(0.1)) * torch.rand(n, **f))
    Z = torch.exp(math.log(1e-4) + (math.log(0.04) - math.log(1e-4)) * torch.rand(n, **f))
    mass = torch.exp(math.log(1e5) + 0.5 * torch.randn(n, **f))
    return dict(x=R * torch.cos(phi), y=R * torch.sin(phi), z=zz, vx=vx, vy=vy, vz=vz, mass=mass, age=age, Z=Z)
