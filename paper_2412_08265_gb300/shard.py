"""Spaxel-row sharding of one galaxy's forward model.

The paper runs the datacube calculation over several devices (Sec. 4, the
strong and weak scaling runs). Here a galaxy's field is split by spaxel rows:
shard i models rows [lo_i, hi_i) only (the telescope's row window; spaxel
keys are still computed on the whole field, so every particle lands in the
same spaxel as unsharded, bit for bit). The deposit needs nothing from other
shards. The PSF reaches r_psf rows across a block boundary, so before
convolving, each shard takes the r_psf rows on each side from its
neighbours' deposited (pre-PSF) rows -- one point-to-point exchange step --
and convolves its extended block; its own rows of the result are then
exactly the unsharded cube's rows (the LSF is along wavelength, local). At
the field's top and bottom there is no neighbour: the extended block simply
ends there, which is the unsharded cube's zero padding.

Transport of the halo rows: on one GPU, device copies between the shards'
buffers (`ShardedForward`); across processes, point-to-point sends and
receives of torch.distributed (`exchange_halos`, NCCL for device tensors,
gloo for host tensors).
"""
from __future__ import annotations

import math
from dataclasses import replace

import torch

from . import capi
from .model import CubeModel


def row_blocks(ny: int, k: int) -> list[tuple[int, int]]:
    """Contiguous, near-equal blocks of spaxel rows for k shards."""
    if k < 1 or k > ny:
        raise ValueError("need 1 <= k <= ny shards")
    return [(ny * i // k, ny * (i + 1) // k) for i in range(k)]


def psf_halo(tel) -> int:
    """Rows the PSF reaches across a block boundary: its kernel radius (the
    library's rule: psf_radius if > 0, else ceil(4 sigma)); 0 without a PSF."""
    if not tel.psf_fwhm > 0.0:
        return 0
    if tel.psf_radius > 0:
        return int(tel.psf_radius)
    sigma = tel.psf_fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    return int(math.ceil(4.0 * sigma))


def halo_plan(blocks: list[tuple[int, int]], h: int) -> list[tuple[int, int]]:
    """Per shard, the halo rows it takes from below and from above: at most h
    each, fewer at the field's edges. A block must hold at least h rows, so
    that a halo comes from the neighbouring shard alone."""
    if any(hi - lo < h for lo, hi in blocks):
        raise ValueError(f"every block needs at least {h} rows (the PSF radius)")
    k = len(blocks)
    return [(h if i > 0 else 0, h if i < k - 1 else 0) for i in range(k)]


def exchange_halos(own: torch.Tensor, h: int, rank: int, world: int, group=None) -> torch.Tensor:
    """Extended block of this rank's rows `own` ([rows, ...]): the last h rows
    of rank - 1, then its own rows, then the first h rows of rank + 1 (no
    halo at the field's edges: rank 0 has none before, the last rank none
    after). Point-to-point over torch.distributed; every rank calls it with
    the same h and at least h rows of its own."""
    import torch.distributed as dist
    below = h if rank > 0 else 0
    above = h if rank < world - 1 else 0
    ext = own.new_empty((below + own.shape[0] + above, *own.shape[1:]))
    ext[below:below + own.shape[0]].copy_(own)
    ops = []
    if below:
        ops.append(dist.P2POp(dist.isend, own[:h].contiguous(), rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, ext[:below], rank - 1, group))
    if above:
        ops.append(dist.P2POp(dist.isend, own[own.shape[0] - h:].contiguous(), rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, ext[below + own.shape[0]:], rank + 1, group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    return ext


class ShardedForward:
    """k row shards of one galaxy on the current GPU (the logical form of a
    k-GPU run): each shard deposits its rows into the middle of its extended
    buffer, takes its halo rows from the neighbours' buffers by device copies,
    and convolves with the telescope's PSF and LSF (rubix_convolve). No
    noise: the sharded cube is the noiseless one."""

    def __init__(self, ssp, telescope, k: int, template_dtype: str = "f32", max_particles: int = 1 << 16,
                 device=None):
        self.tel = telescope
        self.blocks = row_blocks(telescope.ny, k)
        self.h = psf_halo(telescope)
        self.halos = halo_plan(self.blocks, self.h)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        # the shards deposit only (no PSF/LSF); the convolution follows the exchange
        self.models = [CubeModel(ssp, replace(telescope, row_lo=lo, row_hi=hi, psf_fwhm=0.0, lsf_sigma=0.0),
                                 template_dtype, max_particles=max_particles, device=self.device)
                       for lo, hi in self.blocks]
        self.ext = [torch.empty((b + (hi - lo) + a, telescope.nx, telescope.n_lambda), dtype=torch.float32,
                                device=self.device)
                    for (lo, hi), (b, a) in zip(self.blocks, self.halos)]

    def forward(self, particles, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        tel = self.tel
        if out is None:
            out = torch.empty((tel.ny, tel.nx, tel.n_lambda), dtype=torch.float32, device=self.device)
        st = stream or torch.cuda.current_stream(self.device)
        d = self.models[0].device_particles(particles) if not isinstance(particles, dict) else particles
        # deposit: every shard its own rows, into the middle of its extended buffer
        for m, (lo, hi), (b, _), ext in zip(self.models, self.blocks, self.halos, self.ext):
            m.forward(d, out=ext[b:b + hi - lo], stream=st)
        # exchange: halo rows from the neighbours' deposited rows (device copies)
        with torch.cuda.stream(st):
            for i, ((lo, hi), (b, a), ext) in enumerate(zip(self.blocks, self.halos, self.ext)):
                if b:
                    plo, phi = self.blocks[i - 1]
                    pb = self.halos[i - 1][0]
                    ext[:b].copy_(self.ext[i - 1][pb + (phi - plo) - b:pb + (phi - plo)])
                if a:
                    nb = self.halos[i + 1][0]
                    ext[b + hi - lo:].copy_(self.ext[i + 1][nb:nb + a])
        # convolve each extended block; keep its own rows
        ct = CubeModel.c_telescope(replace(tel, row_lo=0, row_hi=0))
        with torch.cuda.stream(st):
            for (lo, hi), (b, _), ext in zip(self.blocks, self.halos, self.ext):
                conv = torch.empty_like(ext)
                capi.rubix_convolve(ct, ext.data_ptr(), conv.data_ptr(), ext.shape[0], st.cuda_stream)
                out[lo:hi].copy_(conv[b:b + hi - lo])
        return out

    def close(self):
        for m in self.models:
            m.close()
        self.models = []
