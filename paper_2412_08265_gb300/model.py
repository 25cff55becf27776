"""PyTorch-facing API of the forward model: device memory and streams come from
torch; all computation runs in the CUDA library through the C ABI (capi).

    model = CubeModel(ssp, telescope, template_dtype="f32")
    cube = model.forward(particles)                 # torch.float32 [ny, nx, n_lambda] on cuda
    cube = RubixCube.apply(mass, age, Z, v_los, x, y, model)   # differentiable
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import capi


# keys of a particle dict that hold scalars, not arrays
SCALAR_KEYS = ("preprojected", "inclination", "azimuth", "position_angle")


def _dev_f32(a, device) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.float32).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)


class CubeModel:
    """One SSP grid + one telescope resident on the current CUDA device."""

    def __init__(self, ssp, telescope, template_dtype: str = "f32", max_particles: int = 1 << 16,
                 device: torch.device | str | None = None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.tel = telescope
        self.ssp = ssp
        self.template_dtype = template_dtype
        la = np.ascontiguousarray(ssp.log10_age_nodes, dtype=np.float64)
        lz = np.ascontiguousarray(ssp.log10_Z_nodes, dtype=np.float64)
        sp = np.ascontiguousarray(ssp.spectra, dtype=np.float64)
        g = capi.rubix_ssp_grid(sp.shape[0], sp.shape[1], sp.shape[2], la.ctypes.data, lz.ctypes.data,
                                float(ssp.lambda0), float(ssp.dlambda), sp.ctypes.data,
                                capi.DTYPES[template_dtype])
        t = self.c_telescope(telescope)
        with torch.cuda.device(self.device):
            self.handle = capi.rubix_cube_create(g, t, int(max_particles))
        self._last = None
        self.last_tag = 0

    @staticmethod
    def c_telescope(tel) -> capi.rubix_telescope:
        return capi.rubix_telescope(int(tel.nx), int(tel.ny), float(tel.spaxel_size), int(tel.n_lambda),
                                    float(tel.lambda0), float(tel.dlambda), float(tel.psf_fwhm),
                                    float(tel.lsf_sigma), int(tel.psf_radius), int(tel.lsf_radius),
                                    float(tel.z_cosmo), float(tel.flux_scale),
                                    int(getattr(tel, "resample", 0)), int(getattr(tel, "row_lo", 0)),
                                    int(getattr(tel, "row_hi", 0)))

    @staticmethod
    def rows(tel) -> int:
        """Spaxel rows of the cube: the row window's, else all ny."""
        hi = int(getattr(tel, "row_hi", 0))
        return hi - int(getattr(tel, "row_lo", 0)) if hi > 0 else tel.ny

    @property
    def cube_shape(self):
        return (self.rows(self.tel), self.tel.nx, self.tel.n_lambda)

    def close(self):
        if getattr(self, "handle", None):
            capi.rubix_cube_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def device_particles(self, p):
        """Upload a synth.Particles (or dict of arrays) to device tensors."""
        d = {}
        for name in ("x", "y", "z", "vx", "vy", "vz", "v_los", "mass", "age", "Z"):
            a = getattr(p, name, None) if not isinstance(p, dict) else p.get(name)
            if a is not None:
                d[name] = _dev_f32(a, self.device)
        d["preprojected"] = bool(getattr(p, "preprojected", True) if not isinstance(p, dict)
                                 else p.get("preprojected", True))
        for name in ("inclination", "azimuth", "position_angle"):
            d[name] = float(getattr(p, name, 0.0) if not isinstance(p, dict) else p.get(name, 0.0))
        return d

    @staticmethod
    def c_particles(d, on_device: bool = True) -> capi.rubix_particles:
        def ptr(name):
            a = d.get(name)
            if a is None:
                return None
            return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data
        n = int(d["mass"].shape[0])
        return capi.rubix_particles(n, ptr("x"), ptr("y"), ptr("z"), ptr("vx"), ptr("vy"), ptr("vz"),
                                    ptr("v_los"), ptr("mass"), ptr("age"), ptr("Z"),
                                    1 if on_device else 0, 1 if d.get("preprojected", True) else 0,
                                    float(d.get("inclination", 0.0)), float(d.get("azimuth", 0.0)),
                                    float(d.get("position_angle", 0.0)))

    def forward(self, p, noise_seed: int = 0, noise_s2n: float = 0.0, out: torch.Tensor | None = None,
                stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        d = p if isinstance(p, dict) and all(isinstance(v, torch.Tensor) for k, v in p.items()
                                             if k not in SCALAR_KEYS) \
            else self.device_particles(p)
        if out is None:
            out = torch.empty(self.cube_shape, dtype=torch.float32, device=self.device)
        st = stream or torch.cuda.current_stream(self.device)
        cp = self.c_particles(d)
        capi.rubix_cube_forward(self.handle, cp, int(noise_seed), float(noise_s2n), out.data_ptr(), 1,
                                st.cuda_stream)
        self._last = d  # keep the device arrays alive until the kernels have read them
        self.last_tag = capi.rubix_cube_forward_tag(self.handle)
        return out

    def backward(self, dL_dcube: torch.Tensor, want_global: bool = False,
                 stream: torch.cuda.Stream | None = None, forward_tag: int | None = None):
        """Gradients of the forward with tag `forward_tag` (default: the most
        recent forward); raises RubixError if a later forward has replaced
        that forward's state on the handle."""
        n = int(self._last["mass"].shape[0])
        tag = self.last_tag if forward_tag is None else int(forward_tag)
        g = [torch.empty(n, dtype=torch.float32, device=self.device) for _ in range(4)]
        glob = torch.empty(4, dtype=torch.float64, device=self.device) if want_global else None
        st = stream or torch.cuda.current_stream(self.device)
        dc = dL_dcube.to(torch.float32).contiguous()
        capi.rubix_cube_backward(self.handle, tag, dc.data_ptr(), g[0].data_ptr(), g[1].data_ptr(),
                                 g[2].data_ptr(), g[3].data_ptr(), glob.data_ptr() if glob is not None else 0,
                                 st.cuda_stream)
        return (*g, glob)

    def spaxel_keys(self, p, stream=None) -> torch.Tensor:
        d = self.device_particles(p)
        keys = torch.empty(int(d["mass"].shape[0]), dtype=torch.int32, device=self.device)
        st = stream or torch.cuda.current_stream(self.device)
        capi.rubix_cube_spaxel_keys(self.handle, self.c_particles(d), keys.data_ptr(), st.cuda_stream)
        torch.cuda.current_stream(self.device).synchronize()
        return keys

    def sorted(self, stream=None):
        n = int(self._last["mass"].shape[0])
        perm = torch.empty(n, dtype=torch.int32, device=self.device)
        seg = torch.empty(self.tel.nx * self.rows(self.tel) + 2, dtype=torch.int32, device=self.device)
        st = stream or torch.cuda.current_stream(self.device)
        capi.rubix_cube_sorted(self.handle, perm.data_ptr(), seg.data_ptr(), st.cuda_stream)
        return perm, seg

    def stats(self) -> dict:
        s = capi.rubix_cube_stats(self.handle)
        keys = ["n_in_fov", "deposits", "slow_particle_tiles", "deposit_launches", "kernel_launches",
                "device_error", "tile_w", "slab_w", "n_bands"]
        return dict(zip(keys, s))

    def set_profiling(self, on: bool = True):
        capi.rubix_cube_set_profiling(self.handle, on)

    STAGES = {"assign_sort": 0, "setup_items": 1, "deposit": 2, "combine": 3, "psf_lsf": 4, "forward": 5}

    def profile_history(self, stage: str = "deposit") -> list:
        return capi.rubix_cube_profile_history(self.handle, self.STAGES[stage])

    def stage_times(self) -> dict:
        t = capi.rubix_cube_stage_times(self.handle)
        keys = ["assign_sort", "setup_items", "deposit", "combine", "psf_lsf", "forward"]
        return dict(zip(keys, t))


class RubixCube(torch.autograd.Function):
    """Differentiable forward model: cube = F(mass, age, Z, v_los; x, y).

    Backward calls the hand-written adjoint kernels (rubix_cube_backward). The
    spaxel assignment is piecewise constant in (x, y), so positions get no
    gradient."""

    @staticmethod
    def forward(ctx, mass, age, Z, v_los, x, y, model: CubeModel):
        d = {"x": x.detach().contiguous(), "y": y.detach().contiguous(), "mass": mass.detach().contiguous(),
             "age": age.detach().contiguous(), "Z": Z.detach().contiguous(),
             "v_los": v_los.detach().contiguous(), "preprojected": True, "inclination": 0.0}
        cube = model.forward(d)
        ctx.model = model
        ctx.forward_tag = model.last_tag
        return cube

    @staticmethod
    def backward(ctx, grad_cube):
        # the handle keeps the state of its most recent forward only: a graph
        # holding two applications of one model can differentiate the last
        # one, and the library refuses the earlier one (RubixError)
        dm, da, dz, dv, _ = ctx.model.backward(grad_cube, forward_tag=ctx.forward_tag)
        return dm, da, dz, dv, None, None, None
