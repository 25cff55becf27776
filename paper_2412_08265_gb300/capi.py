"""ctypes binding of the C ABI declared in include/rubix.h (argument marshalling only).

The Python functions carry the C names (``rubix_cube_create``,
``rubix_cube_forward`` ...) and take the same arguments; every step of the
computation runs in the library's CUDA kernels. The library must have been
built (``paper_2412_08265_gb300.build.build()``); loading fails loudly
otherwise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librubix.so")

RUBIX_OK = 0
RUBIX_ERR_INVALID_ARG = 1
RUBIX_ERR_OOM = 2
RUBIX_ERR_CUDA = 3
RUBIX_ERR_TIMEOUT = 4
RUBIX_ERR_REJECTED = 5
RUBIX_ERR_CANCELLED = 6
RUBIX_ERR_NOT_READY = 7
RUBIX_ERR_UNSUPPORTED = 8
RUBIX_ERR_DEVICE = 9

RUBIX_F32, RUBIX_BF16, RUBIX_F16 = 0, 1, 2
DTYPES = {"f32": RUBIX_F32, "bf16": RUBIX_BF16, "f16": RUBIX_F16}

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


class rubix_ssp_grid(C.Structure):
    _fields_ = [("n_age", C.c_int32), ("n_Z", C.c_int32), ("n_lambda", C.c_int32),
                ("log10_age_nodes", C.c_void_p), ("log10_Z_nodes", C.c_void_p),
                ("lambda0", C.c_double), ("dlambda", C.c_double), ("spectra", C.c_void_p),
                ("storage_dtype", C.c_int32)]


class rubix_telescope(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("spaxel_size", C.c_double),
                ("n_lambda", C.c_int32), ("lambda0", C.c_double), ("dlambda", C.c_double),
                ("psf_fwhm", C.c_double), ("lsf_sigma", C.c_double), ("psf_radius", C.c_int32),
                ("lsf_radius", C.c_int32), ("z_cosmo", C.c_double), ("flux_scale", C.c_double),
                ("resample", C.c_int32), ("row_lo", C.c_int32), ("row_hi", C.c_int32)]


class rubix_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p), ("v_los", C.c_void_p),
                ("mass", C.c_void_p), ("age", C.c_void_p), ("Z", C.c_void_p),
                ("on_device", C.c_int32), ("preprojected", C.c_int32), ("inclination", C.c_double),
                ("azimuth", C.c_double), ("position_angle", C.c_double)]


class RubixError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rubix status {status}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_SIGS = {
    "rubix_cube_create": (C.c_int32, [C.POINTER(rubix_ssp_grid), C.POINTER(rubix_telescope), C.c_int64,
                                      C.POINTER(C.c_void_p)]),
    "rubix_cube_forward": (C.c_int32, [C.c_void_p, C.POINTER(rubix_particles), C.c_uint64, C.c_float,
                                       C.c_void_p, C.c_int32, C.c_void_p]),
    "rubix_cube_forward_tag": (C.c_int32, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "rubix_cube_backward": (C.c_int32, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rubix_cube_destroy": (C.c_int32, [C.c_void_p]),
    "rubix_cube_spaxel_keys": (C.c_int32, [C.c_void_p, C.POINTER(rubix_particles), C.c_void_p, C.c_void_p]),
    "rubix_cube_sorted": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rubix_cube_set_profiling": (C.c_int32, [C.c_void_p, C.c_int32]),
    "rubix_cube_stage_times": (C.c_int32, [C.c_void_p, _fp, C.POINTER(C.c_int32)]),
    "rubix_cube_profile_history": (C.c_int32, [C.c_void_p, C.c_int32, _fp, C.POINTER(C.c_int32)]),
    "rubix_cube_stats": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "rubix_spaxel_sort_noalloc": (C.c_int32, [C.POINTER(rubix_particles), C.POINTER(rubix_telescope),
                                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "rubix_serve_create": (C.c_int32, [C.POINTER(rubix_ssp_grid), C.POINTER(rubix_telescope), C.c_size_t,
                                       C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "rubix_serve_submit": (C.c_int32, [C.c_void_p, C.POINTER(rubix_telescope), C.POINTER(rubix_particles),
                                       C.c_uint64, C.c_float, C.c_void_p, C.c_int32, C.POINTER(C.c_uint64)]),
    "rubix_serve_footprint": (C.c_int32, [C.c_void_p, C.POINTER(rubix_telescope), C.POINTER(rubix_particles),
                                          C.c_int32, C.POINTER(C.c_size_t)]),
    "rubix_serve_poll": (C.c_int32, [C.c_void_p, C.c_uint64, C.POINTER(C.c_double)]),
    "rubix_serve_wait": (C.c_int32, [C.c_void_p, C.c_uint64, C.c_double]),
    "rubix_serve_cancel": (C.c_int32, [C.c_void_p, C.c_uint64]),
    "rubix_serve_stats": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "rubix_serve_destroy": (C.c_int32, [C.c_void_p]),
    "rubix_selftest_bounded_wait": (C.c_int32, [C.c_double, C.POINTER(C.c_int32)]),
    "rubix_measure_fp32_peak": (C.c_int32, [C.c_int32, _dp, _dp, _dp]),
    "rubix_convolve": (C.c_int32, [C.POINTER(rubix_telescope), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "rubix_last_error_message": (C.c_char_p, []),
    "rubix_version": (C.c_char_p, []),
}


def load(path: str | None = None):
    """Load librubix.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} is missing "
                                   "(run paper_2412_08265_gb300.build.build())")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS.keys())


def check(status: int):
    if status != RUBIX_OK:
        msg = load().rubix_last_error_message()
        raise RubixError(status, msg.decode() if msg else "")
    return status


def _call(name, *args):
    return check(getattr(load(), name)(*args))


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------
def rubix_cube_create(ssp: rubix_ssp_grid, tel: rubix_telescope, max_particles: int) -> int:
    h = C.c_void_p()
    _call("rubix_cube_create", C.byref(ssp), C.byref(tel), C.c_int64(max_particles), C.byref(h))
    return h.value


def rubix_cube_forward(h: int, p: rubix_particles, noise_seed: int, noise_s2n: float, cube_out: int,
                       cube_on_device: int, stream: int) -> None:
    _call("rubix_cube_forward", C.c_void_p(h), C.byref(p), C.c_uint64(noise_seed), C.c_float(noise_s2n),
          C.c_void_p(cube_out), C.c_int32(cube_on_device), C.c_void_p(stream))


def rubix_cube_forward_tag(h: int) -> int:
    t = C.c_uint64()
    _call("rubix_cube_forward_tag", C.c_void_p(h), C.byref(t))
    return int(t.value)


def rubix_cube_backward(h: int, forward_tag: int, dL_dcube: int, d_mass: int, d_age: int, d_Z: int,
                        d_vlos: int, d_global: int, stream: int) -> None:
    _call("rubix_cube_backward", C.c_void_p(h), C.c_uint64(forward_tag), C.c_void_p(dL_dcube),
          C.c_void_p(d_mass), C.c_void_p(d_age), C.c_void_p(d_Z), C.c_void_p(d_vlos), C.c_void_p(d_global),
          C.c_void_p(stream))


def rubix_cube_destroy(h: int) -> None:
    _call("rubix_cube_destroy", C.c_void_p(h))


def rubix_cube_spaxel_keys(h: int, p: rubix_particles, keys_out: int, stream: int) -> None:
    _call("rubix_cube_spaxel_keys", C.c_void_p(h), C.byref(p), C.c_void_p(keys_out), C.c_void_p(stream))


def rubix_cube_sorted(h: int, perm_out: int, seg_off_out: int, stream: int) -> None:
    _call("rubix_cube_sorted", C.c_void_p(h), C.c_void_p(perm_out), C.c_void_p(seg_off_out),
          C.c_void_p(stream))


def rubix_cube_set_profiling(h: int, enable: bool) -> None:
    _call("rubix_cube_set_profiling", C.c_void_p(h), C.c_int32(1 if enable else 0))


def rubix_cube_stage_times(h: int) -> list[float]:
    buf = (C.c_float * 8)()
    n = C.c_int32(8)
    _call("rubix_cube_stage_times", C.c_void_p(h), buf, C.byref(n))
    return [float(buf[i]) for i in range(n.value)]


def rubix_cube_profile_history(h: int, stage: int) -> list[float]:
    buf = (C.c_float * 256)()
    n = C.c_int32(256)
    _call("rubix_cube_profile_history", C.c_void_p(h), C.c_int32(stage), buf, C.byref(n))
    return [float(buf[i]) for i in range(n.value)]


def rubix_cube_stats(h: int) -> list[int]:
    buf = (C.c_int64 * 16)()
    n = C.c_int32(16)
    _call("rubix_cube_stats", C.c_void_p(h), buf, C.byref(n))
    return [int(buf[i]) for i in range(n.value)]


def rubix_spaxel_sort_noalloc(p: rubix_particles, tel: rubix_telescope, perm_out: int, seg_off_out: int,
                              stream: int) -> None:
    """Spaxel sort for callers that may not allocate device memory (their
    memory budget belongs to another allocator, or cudaMalloc's device
    synchronisation is not acceptable where they call it): scratch lives in a
    fixed array inside the library, so n <= 262144 and nx*ny <= 262143."""
    _call("rubix_spaxel_sort_noalloc", C.byref(p), C.byref(tel), C.c_void_p(perm_out), C.c_void_p(seg_off_out),
          C.c_void_p(stream))


def rubix_serve_create(ssp: rubix_ssp_grid, wavelength_grid: rubix_telescope, hbm_budget_bytes: int,
                       max_slots: int, max_batch: int) -> int:
    h = C.c_void_p()
    _call("rubix_serve_create", C.byref(ssp), C.byref(wavelength_grid), C.c_size_t(hbm_budget_bytes),
          C.c_int32(max_slots), C.c_int32(max_batch), C.byref(h))
    return h.value


def rubix_serve_submit(srv: int, tel: rubix_telescope, p: rubix_particles, noise_seed: int, noise_s2n: float,
                       cube_out: int, cube_on_device: int) -> int:
    t = C.c_uint64()
    _call("rubix_serve_submit", C.c_void_p(srv), C.byref(tel), C.byref(p), C.c_uint64(noise_seed),
          C.c_float(noise_s2n), C.c_void_p(cube_out), C.c_int32(cube_on_device), C.byref(t))
    return t.value


def rubix_serve_footprint(srv: int, tel: rubix_telescope, p: rubix_particles, cube_on_device: int) -> int:
    b = C.c_size_t()
    _call("rubix_serve_footprint", C.c_void_p(srv), C.byref(tel), C.byref(p), C.c_int32(cube_on_device),
          C.byref(b))
    return int(b.value)


def rubix_serve_poll(srv: int, ticket: int) -> tuple[int, float]:
    """(status, latency_s): status is RUBIX_OK, RUBIX_ERR_NOT_READY or the request's error."""
    lat = C.c_double(0.0)
    st = load().rubix_serve_poll(C.c_void_p(srv), C.c_uint64(ticket), C.byref(lat))
    return int(st), float(lat.value)


def rubix_serve_wait(srv: int, ticket: int, timeout_s: float) -> int:
    """Status after waiting (RUBIX_ERR_TIMEOUT if the time ran out); does not raise."""
    return int(load().rubix_serve_wait(C.c_void_p(srv), C.c_uint64(ticket), C.c_double(timeout_s)))


def rubix_serve_cancel(srv: int, ticket: int) -> int:
    return int(load().rubix_serve_cancel(C.c_void_p(srv), C.c_uint64(ticket)))


def rubix_serve_stats(srv: int) -> list[int]:
    buf = (C.c_int64 * 16)()
    n = C.c_int32(16)
    _call("rubix_serve_stats", C.c_void_p(srv), buf, C.byref(n))
    return [int(buf[i]) for i in range(n.value)]


def rubix_serve_destroy(srv: int) -> None:
    _call("rubix_serve_destroy", C.c_void_p(srv))


def rubix_selftest_bounded_wait(limit_s: float) -> bool:
    """True when a device wait with nothing to complete it gave up after limit_s."""
    t = C.c_int32(0)
    _call("rubix_selftest_bounded_wait", C.c_double(limit_s), C.byref(t))
    return bool(t.value)


def rubix_convolve(tel: rubix_telescope, cube_in: int, cube_out: int, n_rows: int, stream: int) -> None:
    _call("rubix_convolve", C.byref(tel), C.c_void_p(cube_in), C.c_void_p(cube_out), C.c_int32(n_rows),
          C.c_void_p(stream))


def rubix_measure_fp32_peak(packed: bool) -> tuple[float, float, float]:
    """(FLOP/s, FMAs per clock per SM, SM MHz) of an FFMA (packed=False) or
    FFMA2 (packed=True) chain benchmark on the current device."""
    f, r, m = C.c_double(), C.c_double(), C.c_double()
    _call("rubix_measure_fp32_peak", C.c_int32(1 if packed else 0), C.byref(f), C.byref(r), C.byref(m))
    return float(f.value), float(r.value), float(m.value)


def rubix_last_error_message() -> str:
    m = load().rubix_last_error_message()
    return m.decode() if m else ""


last_error_message = rubix_last_error_message


def rubix_version() -> str:
    return load().rubix_version().decode()
