"""PyTorch-facing client of the request server (rubix_serve_* in include/rubix.h).

    srv = Server(ssp, wavelength_grid=tel, hbm_budget_bytes=64 << 30, max_slots=16, max_batch=16)
    t = srv.submit(tel, particles_dict, out=cube_tensor)   # returns at once
    srv.wait(t); lat = srv.latency(t)

All work runs in the library's server thread and CUDA kernels; this module
only marshals arguments and keeps the caller's tensors alive until their
request has finished.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .model import SCALAR_KEYS, CubeModel


class Server:
    def __init__(self, ssp, wavelength_grid, hbm_budget_bytes: int, max_slots: int = 16, max_batch: int = 16,
                 template_dtype: str = "f32", device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        la = np.ascontiguousarray(ssp.log10_age_nodes, dtype=np.float64)
        lz = np.ascontiguousarray(ssp.log10_Z_nodes, dtype=np.float64)
        sp = np.ascontiguousarray(ssp.spectra, dtype=np.float64)
        g = capi.rubix_ssp_grid(sp.shape[0], sp.shape[1], sp.shape[2], la.ctypes.data, lz.ctypes.data,
                                float(ssp.lambda0), float(ssp.dlambda), sp.ctypes.data,
                                capi.DTYPES[template_dtype])
        with torch.cuda.device(self.device):
            self.handle = capi.rubix_serve_create(g, CubeModel.c_telescope(wavelength_grid), int(hbm_budget_bytes),
                                                  int(max_slots), int(max_batch))
        self._keep = {}  # ticket -> objects the request reads or writes

    def submit(self, tel, particles: dict, out: torch.Tensor, noise_seed: int = 0, noise_s2n: float = 0.0) -> int:
        """Queue a forward model of `particles` (dict of float32 tensors on this
        device or on the host, plus the scalars 'preprojected', 'inclination', 'azimuth', 'position_angle') into `out`
        (float32 [ny, nx, n_lambda], device or host)."""
        on_dev = [isinstance(v, torch.Tensor) and v.is_cuda for k, v in particles.items()
                  if k not in SCALAR_KEYS]
        if any(on_dev) != all(on_dev):
            raise ValueError("particle arrays must be all on the device or all on the host")
        cp = CubeModel.c_particles(particles, on_device=all(on_dev))
        t = capi.rubix_serve_submit(self.handle, CubeModel.c_telescope(tel), cp, int(noise_seed), float(noise_s2n),
                                    out.data_ptr(), 1 if out.is_cuda else 0)
        self._keep[t] = (particles, out)
        return t

    def footprint(self, tel, particles: dict, out: torch.Tensor) -> int:
        """Device bytes the request would hold on the GPU (admission counts these)."""
        on_dev = all(isinstance(v, torch.Tensor) and v.is_cuda for k, v in particles.items()
                     if k not in SCALAR_KEYS)
        cp = CubeModel.c_particles(particles, on_device=on_dev)
        return capi.rubix_serve_footprint(self.handle, CubeModel.c_telescope(tel), cp, 1 if out.is_cuda else 0)

    def poll(self, ticket: int):
        st, lat = capi.rubix_serve_poll(self.handle, ticket)
        if st != capi.RUBIX_ERR_NOT_READY:
            self._keep.pop(ticket, None)
        return st, lat

    def wait(self, ticket: int, timeout_s: float = -1.0) -> int:
        st = capi.rubix_serve_wait(self.handle, ticket, timeout_s)
        if st != capi.RUBIX_ERR_TIMEOUT:
            self._keep.pop(ticket, None)
        return st

    def latency(self, ticket: int) -> float:
        return capi.rubix_serve_poll(self.handle, ticket)[1]

    def cancel(self, ticket: int) -> int:
        st = capi.rubix_serve_cancel(self.handle, ticket)
        if st == capi.RUBIX_OK:
            self._keep.pop(ticket, None)
        return st

    STATS = ["submitted", "ok", "rejected", "cancelled", "failed", "deposit_launches", "max_batch",
             "bytes_in_use", "peak_bytes", "active", "queued"]

    def stats(self) -> dict:
        return dict(zip(self.STATS, capi.rubix_serve_stats(self.handle)))

    def close(self):
        if getattr(self, "handle", None):
            capi.rubix_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
