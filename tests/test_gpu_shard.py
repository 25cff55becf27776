"""Spaxel-row sharding (Sec. 4's multi-device runs), logically on one GPU:
k shards each deposit their own rows (row window), take the PSF's halo rows
from their neighbours by device copies, convolve (rubix_convolve) and keep
their rows. The assembled cube must equal the unsharded forward bit for bit
(the deposit of a spaxel never depends on other spaxels, and the convolution
of a row reads exactly the rows the halo supplies)."""
import numpy as np
import pytest

import oracle
from paper_2412_08265_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from __graft_entry__ import build
    build()
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("k", [2, 3, 5])
def test_row_shards_equal_unsharded_bitwise(torch_cuda, k):
    torch = torch_cuda
    from paper_2412_08265_gb300.model import CubeModel
    from paper_2412_08265_gb300.shard import ShardedForward
    wl = synth.mid_galaxy(n=120_000, seed=6)
    tel = synth.Telescope(nx=64, ny=61, spaxel_size=0.3, n_lambda=3721, lambda0=4750.0, dlambda=1.25)
    full = CubeModel(wl.ssp, tel, "f32", max_particles=wl.particles.n)
    d = full.device_particles(wl.particles)
    ref = full.forward(d)
    sh = ShardedForward(wl.ssp, tel, k, "f32", max_particles=wl.particles.n)
    got = sh.forward(d)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    # and the unsharded cube is the oracle's (rows around a block boundary)
    rows = [lo for lo, _ in sh.blocks[1:]]
    centres = np.array([r * tel.nx + c for r in rows for c in (5, 31, 50)], dtype=np.int64)
    xp, yp, v = oracle.orient(wl.particles)
    cube0 = oracle.deposit(oracle.spaxel_keys(xp, yp, tel), v, wl.particles, wl.ssp, tel)
    want = oracle.psf_lsf_at(cube0, tel, centres)
    g = got.reshape(-1, tel.n_lambda)[torch.from_numpy(centres).cuda()].cpu().numpy().astype(np.float64)
    assert float(np.abs(g - want).max() / np.abs(want).max()) <= 1e-5
    sh.close()
    full.close()


def test_row_window_keys_and_inclined_shards(torch_cuda):
    """A 3-D disk turned by all three angles, 4 shards: the window's keys are
    the whole field's keys less the window's first row (bit-exact against the
    oracle), and the sharded cube is the unsharded one."""
    torch = torch_cuda
    from dataclasses import replace
    from paper_2412_08265_gb300.model import CubeModel
    from paper_2412_08265_gb300.shard import ShardedForward
    wl = synth.small_galaxy()
    tel = synth.serving_telescope(57)
    p = synth.disk_3d(60_000, 12, inclination=0.9, azimuth=0.3, position_angle=1.2)
    xp, yp, _ = oracle.orient(p)
    key = oracle.spaxel_keys(xp, yp, tel)
    n_s = tel.nx * tel.ny
    for lo, hi in ((0, 20), (20, 41), (41, 57)):
        m = CubeModel(wl.ssp, replace(tel, row_lo=lo, row_hi=hi), "f32", max_particles=p.n)
        got = m.spaxel_keys(p).cpu().numpy()
        iy = key // tel.nx
        inside = (key < n_s) & (iy >= lo) & (iy < hi)
        want = np.where(inside, key - lo * tel.nx, tel.nx * (hi - lo))
        assert np.array_equal(got, want), (lo, hi)
        m.close()
    full = CubeModel(wl.ssp, tel, "f32", max_particles=p.n)
    d = full.device_particles(p)
    ref = full.forward(d)
    sh = ShardedForward(wl.ssp, tel, 4, "f32", max_particles=p.n)
    got = sh.forward(d)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    sh.close()
    full.close()


def test_convolve_matches_the_forward_psf_lsf(torch_cuda):
    """rubix_convolve of the deposit-only cube is the forward's cube, bit for
    bit, for the instrument radii (fused kernels) and for radii with no fused
    kernel (two passes)."""
    torch = torch_cuda
    from dataclasses import replace
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.model import CubeModel
    wl = synth.small_galaxy(n=20_000, seed=2)
    for tel in (wl.telescope, replace(wl.telescope, psf_fwhm=3.0, lsf_sigma=4.0)):
        full = CubeModel(wl.ssp, tel, "f32", max_particles=wl.particles.n)
        raw = CubeModel(wl.ssp, replace(tel, psf_fwhm=0.0, lsf_sigma=0.0), "f32", max_particles=wl.particles.n)
        d = full.device_particles(wl.particles)
        ref = full.forward(d)
        c0 = raw.forward(d)
        out = torch.empty_like(c0)
        capi.rubix_convolve(CubeModel.c_telescope(tel), c0.data_ptr(), out.data_ptr(), tel.ny,
                            torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        full.close()
        raw.close()
