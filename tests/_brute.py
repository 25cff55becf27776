"""Independent brute-force restatement of the forward model for tiny inputs.

Used only to pin the FP64 C oracle. It is written differently on purpose:
spaxel membership by exact rational arithmetic, bilinear interpolation by
scipy's RegularGridInterpolator, Doppler resampling by numpy.interp on the
zero-extended template, per-voxel sums by an explicit membership test, and the
PSF/LSF by scipy.ndimage.convolve with zero padding. The kernel weights are
written out from the Gaussian formula here, independently of the oracle.
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np
from scipy.interpolate import RegularGridInterpolator
from scipy.ndimage import convolve

C_KMS = 299792.458


def exact_spaxel(xp: float, yp: float, tel):
    """Spaxel (ix, iy) by exact rational arithmetic, None if outside."""
    size = Fraction(tel.spaxel_size)
    x_lo = -Fraction(tel.nx) * size / 2
    y_lo = -Fraction(tel.ny) * size / 2
    u = (Fraction(xp) - x_lo) / size
    w = (Fraction(yp) - y_lo) / size
    if 0 <= u < tel.nx and 0 <= w < tel.ny:
        return int(math.floor(u)), int(math.floor(w)), u, w
    return None


def rotation(p):
    """Rotation matrix of the orientation: scipy's extrinsic z-x-z Euler
    rotation (azimuth about z, then inclination about x, then the position
    angle about z)."""
    from scipy.spatial.transform import Rotation
    return Rotation.from_euler("zxz", [getattr(p, "azimuth", 0.0), p.inclination,
                                       getattr(p, "position_angle", 0.0)]).as_matrix()


def projected(p):
    if p.preprojected:
        return (p.x.astype(np.float64), p.y.astype(np.float64), p.v_los.astype(np.float64))
    R = rotation(p)
    r = np.stack([p.x, p.y, p.z]).astype(np.float64)
    vx = np.zeros(p.n) if p.vx is None else p.vx.astype(np.float64)
    vel = np.stack([vx, p.vy.astype(np.float64), p.vz.astype(np.float64)])
    rp, vp = R @ r, R @ vel
    return rp[0], rp[1], vp[2]


def interpolated_template(ssp, age, Z, spectra=None):
    """Template at (age, Z), bilinear in (log age, log Z) and clamped, with one
    zero node appended on either side: (rest wavelengths, values)."""
    sp = ssp.spectra if spectra is None else spectra
    la = np.clip(math.log10(age), ssp.log10_age_nodes[0], ssp.log10_age_nodes[-1])
    lz = np.clip(math.log10(Z), ssp.log10_Z_nodes[0], ssp.log10_Z_nodes[-1])
    interp = RegularGridInterpolator((ssp.log10_age_nodes, ssp.log10_Z_nodes), sp, method="linear")
    T = interp([[la, lz]])[0]
    lam_s = ssp.lambda0 + ssp.dlambda * np.arange(-1, ssp.n_lambda + 1)
    return lam_s, np.concatenate([[0.0], T, [0.0]])


def particle_spectrum(ssp, tel, mass, age, Z, v, spectra=None):
    """m * T_interp(lambda_j / dop), linear in wavelength (np.interp), or with
    ``tel.resample`` = 1 the mean of that curve over each output bin."""
    lam_s, T_ext = interpolated_template(ssp, age, Z, spectra)
    dop = (1.0 + tel.z_cosmo) * (1.0 + v / C_KMS)
    if getattr(tel, "resample", 0):
        return tel.flux_scale * mass * bin_means(lam_s, T_ext, tel, dop)
    lam = tel.lambda0 + tel.dlambda * np.arange(tel.n_lambda)
    return tel.flux_scale * mass * np.interp(lam / dop, lam_s, T_ext, left=0.0, right=0.0)


def bin_means(lam_s, T_ext, tel, dop):
    """Mean of the piecewise-linear curve (lam_s, T_ext) over each output bin's
    rest-frame interval: trapezoid rule with every curve node inside the
    interval taken as a break point (exact for a piecewise-linear curve)."""
    out = np.empty(tel.n_lambda)
    for j in range(tel.n_lambda):
        a = (tel.lambda0 + (j - 0.5) * tel.dlambda) / dop
        b = (tel.lambda0 + (j + 0.5) * tel.dlambda) / dop
        pts = np.concatenate([[a], lam_s[(lam_s > a) & (lam_s < b)], [b]])
        vals = np.interp(pts, lam_s, T_ext, left=0.0, right=0.0)
        out[j] = np.trapezoid(vals, pts) / (b - a)
    return out


def cube0(p, ssp, tel, spectra=None):
    xp, yp, v = projected(p)
    spec = [particle_spectrum(ssp, tel, float(p.mass[i]), float(p.age[i]), float(p.Z[i]), v[i],
                              spectra) for i in range(p.n)]
    where = [exact_spaxel(xp[i], yp[i], tel) for i in range(p.n)]
    cube = np.zeros((tel.ny, tel.nx, tel.n_lambda))
    for iy in range(tel.ny):
        for ix in range(tel.nx):
            for i in range(p.n):
                if where[i] is not None and where[i][0] == ix and where[i][1] == iy:
                    cube[iy, ix] += spec[i]
    return cube


def gauss_weights(sigma: float, radius: int):
    d = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-0.5 * (d / sigma) ** 2)
    return g / g.sum()


def psf_lsf(cube, tel):
    out = cube
    if tel.psf_fwhm > 0:
        s = tel.psf_fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        r = tel.psf_radius if tel.psf_radius > 0 else math.ceil(4 * s)
        g = gauss_weights(s, r)
        k = np.outer(g, g)[:, :, None]
        out = convolve(out, k, mode="constant", cval=0.0)
    if tel.lsf_sigma > 0:
        s = tel.lsf_sigma / tel.dlambda
        r = tel.lsf_radius if tel.lsf_radius > 0 else math.ceil(4 * s)
        h = gauss_weights(s, r)[None, None, :]
        out = convolve(out, h, mode="constant", cval=0.0)
    return out
