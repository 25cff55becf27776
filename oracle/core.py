"""ctypes wrapper of the FP64 C oracle (``rubix_oracle.c``). Test infrastructure only.

Each function mirrors one step of the pipeline of Sec. 3 of the paper
(orient -> assign spaxels -> SSP lookup + Doppler + resample -> per-spaxel sum
-> PSF -> LSF); the C source states the reading of each step.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

C_KMS = 299792.458
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rubix_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_OUT)
    return _lib


def _p(a, dtype):
    if a is None:
        return None
    assert a.dtype == dtype and a.flags.c_contiguous, (a.dtype, dtype)
    return a.ctypes.data_as(C.c_void_p)


def _nthreads(n_threads):
    if n_threads is None:
        return os.cpu_count() or 1
    return max(1, int(n_threads))


def orient(p, derivatives=False):
    """a1: projected positions (x', y') and line-of-sight velocity, FP64; with
    ``derivatives`` also dv_los/d(inclination) and dv_los/d(azimuth)."""
    lib = _load()
    n = p.n
    xp = np.empty(n); yp = np.empty(n); v = np.empty(n)
    di = np.empty(n) if derivatives else None
    da = np.empty(n) if derivatives else None
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    lib.or_orient(C.c_int64(n), _p(f32(p.x), np.float32), _p(f32(p.y), np.float32),
                  _p(f32(p.z), np.float32), _p(f32(getattr(p, "vx", None)), np.float32),
                  _p(f32(p.vy), np.float32), _p(f32(p.vz), np.float32),
                  _p(f32(p.v_los), np.float32), C.c_int(1 if p.preprojected else 0),
                  C.c_double(p.inclination), C.c_double(getattr(p, "azimuth", 0.0)),
                  C.c_double(getattr(p, "position_angle", 0.0)), _p(xp, np.float64),
                  _p(yp, np.float64), _p(v, np.float64), _p(di, np.float64), _p(da, np.float64))
    if derivatives:
        return xp, yp, v, di, da
    return xp, yp, v


def spaxel_keys(xp, yp, tel):
    """a2: spaxel key per particle (nx*ny = outside the field)."""
    lib = _load()
    n = xp.shape[0]
    key = np.empty(n, dtype=np.int32)
    lib.or_spaxel_keys(C.c_int64(n), _p(np.ascontiguousarray(xp), np.float64),
                       _p(np.ascontiguousarray(yp), np.float64), C.c_int(tel.nx), C.c_int(tel.ny),
                       C.c_double(tel.spaxel_size), _p(key, np.int32))
    return key


def stable_sort(key, n_keys):
    """a3: stable permutation by key and segment offsets (n_keys + 1 entries)."""
    lib = _load()
    n = key.shape[0]
    perm = np.empty(n, dtype=np.int32)
    seg = np.empty(n_keys + 1, dtype=np.int64)
    rc = lib.or_stable_sort(C.c_int64(n), _p(key, np.int32), C.c_int32(n_keys), _p(perm, np.int32),
                            _p(seg, np.int64))
    assert rc == 0
    return perm, seg


def _ssp_args(ssp, spectra=None):
    sp = np.ascontiguousarray(ssp.spectra if spectra is None else spectra, dtype=np.float64)
    la = np.ascontiguousarray(ssp.log10_age_nodes, dtype=np.float64)
    lz = np.ascontiguousarray(ssp.log10_Z_nodes, dtype=np.float64)
    keep = (sp, la, lz)
    args = [C.c_int(sp.shape[0]), C.c_int(sp.shape[1]), C.c_int(sp.shape[2]),
            _p(la, np.float64), _p(lz, np.float64), C.c_double(ssp.lambda0),
            C.c_double(ssp.dlambda), _p(sp, np.float64)]
    return args, keep


def _tel_args(tel):
    return [C.c_int(tel.nx), C.c_int(tel.ny), C.c_int(tel.n_lambda), C.c_double(tel.lambda0),
            C.c_double(tel.dlambda), C.c_double(tel.z_cosmo), C.c_double(tel.flux_scale),
            C.c_int(int(getattr(tel, "resample", 0)))]


def deposit(key, v, p, ssp, tel, mask=None, n_threads=None, spectra=None):
    """a4-a6: pre-convolution cube [ny, nx, n_lambda] in FP64.

    ``mask`` (uint8 [ny*nx]) restricts the computation to selected spaxels;
    ``spectra`` overrides the SSP templates (e.g. BF16-rounded copies)."""
    lib = _load()
    cube = np.empty((tel.ny, tel.nx, tel.n_lambda), dtype=np.float64)
    sargs, keep = _ssp_args(ssp, spectra)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    mass, age, Z = f32(p.mass), f32(p.age), f32(p.Z)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rc = lib.or_deposit(C.c_int64(p.n), _p(np.ascontiguousarray(key, dtype=np.int32), np.int32),
                        _p(np.ascontiguousarray(v, dtype=np.float64), np.float64),
                        _p(mass, np.float32), _p(age, np.float32), _p(Z, np.float32), *sargs,
                        *_tel_args(tel), _p(m, np.uint8), C.c_int(_nthreads(n_threads)),
                        _p(cube, np.float64))
    assert rc == 0
    return cube


def psf(cube, tel, n_threads=None):
    """a7: Gaussian PSF, zero padding."""
    lib = _load()
    out = np.empty_like(cube)
    rc = lib.or_psf(C.c_int(tel.nx), C.c_int(tel.ny), C.c_int(tel.n_lambda),
                    C.c_double(tel.psf_fwhm), C.c_int(tel.psf_radius),
                    _p(np.ascontiguousarray(cube), np.float64), _p(out, np.float64),
                    C.c_int(_nthreads(n_threads)))
    assert rc == 0
    return out


def lsf(cube, tel, n_threads=None):
    """a8: Gaussian LSF along wavelength, zero padding."""
    lib = _load()
    out = np.empty_like(cube)
    rc = lib.or_lsf(C.c_int(tel.nx), C.c_int(tel.ny), C.c_int(tel.n_lambda),
                    C.c_double(tel.lsf_sigma), C.c_double(tel.dlambda), C.c_int(tel.lsf_radius),
                    _p(np.ascontiguousarray(cube), np.float64), _p(out, np.float64),
                    C.c_int(_nthreads(n_threads)))
    assert rc == 0
    return out


def psf_lsf_at(cube0, tel, spaxels):
    """Final (PSF then LSF) cube rows at the listed spaxels, from the definition."""
    lib = _load()
    sel = np.ascontiguousarray(spaxels, dtype=np.int32)
    out = np.empty((sel.shape[0], tel.n_lambda), dtype=np.float64)
    rc = lib.or_psf_lsf_at(C.c_int(tel.nx), C.c_int(tel.ny), C.c_int(tel.n_lambda),
                           C.c_double(tel.psf_fwhm), C.c_int(tel.psf_radius),
                           C.c_double(tel.lsf_sigma), C.c_double(tel.dlambda),
                           C.c_int(tel.lsf_radius), _p(np.ascontiguousarray(cube0), np.float64),
                           C.c_int(sel.shape[0]), _p(sel, np.int32), _p(out, np.float64))
    assert rc == 0
    return out


def gradient(key, v, p, ssp, tel, G0, n_threads=None, spectra=None):
    """a10: per-particle dL/d(mass, age, Z, v_los) given G0 = dL/d(cube0)."""
    lib = _load()
    n = p.n
    outs = [np.empty(n) for _ in range(4)]
    sargs, keep = _ssp_args(ssp, spectra)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    mass, age, Z = f32(p.mass), f32(p.age), f32(p.Z)
    rc = lib.or_gradient(C.c_int64(n), _p(np.ascontiguousarray(key, dtype=np.int32), np.int32),
                         _p(np.ascontiguousarray(v, dtype=np.float64), np.float64),
                         _p(mass, np.float32), _p(age, np.float32), _p(Z, np.float32), *sargs,
                         *_tel_args(tel), _p(np.ascontiguousarray(G0, dtype=np.float64), np.float64),
                         C.c_int(_nthreads(n_threads)), *[_p(o, np.float64) for o in outs])
    assert rc == 0
    return tuple(outs)


def gauss_kernel(sigma, radius):
    lib = _load()
    r = kernel_radius(sigma, radius)
    k = np.empty(2 * r + 1)
    lib.or_gauss_kernel(C.c_double(sigma), C.c_int(r), _p(k, np.float64))
    return k


def kernel_radius(sigma, radius):
    lib = _load()
    return int(lib.or_kernel_radius(C.c_double(sigma), C.c_int(radius)))


def forward_parts(p, ssp, tel, n_threads=None, spectra=None, mask=None):
    """Run a1..a8 and return every intermediate (FP64)."""
    xp, yp, v = orient(p)
    key = spaxel_keys(xp, yp, tel)
    cube0 = deposit(key, v, p, ssp, tel, mask=mask, n_threads=n_threads, spectra=spectra)
    cube1 = psf(cube0, tel, n_threads) if tel.psf_fwhm > 0 else cube0
    cube2 = lsf(cube1, tel, n_threads) if tel.lsf_sigma > 0 else cube1
    return dict(xp=xp, yp=yp, v=v, key=key, cube0=cube0, cube1=cube1, cube=cube2)


def forward(p, ssp, tel, n_threads=None, spectra=None):
    """The noiseless FP64 cube [ny, nx, n_lambda]."""
    return forward_parts(p, ssp, tel, n_threads, spectra)["cube"]
