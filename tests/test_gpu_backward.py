"""GPU adjoint (hand-written backward kernels) against the FP64 oracle's analytic
gradient, which the CPU tests pin to central finite differences of the FP64
forward. Tolerance: max|GPU - oracle| <= 1e-4 * max|oracle| per parameter."""
import os

import numpy as np
import pytest

import oracle
from paper_2412_08265_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4
NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from __graft_entry__ import build
    build()
    torch.cuda.set_device(0)
    return torch


def _grad_check(torch, wl, G, dtype="f32", spectra=None, sample=None):
    from paper_2412_08265_gb300.model import CubeModel
    model = CubeModel(wl.ssp, wl.telescope, dtype, max_particles=wl.particles.n)
    model.forward(wl.particles)
    dm, dage, dZ, dv, glob = model.backward(torch.from_numpy(G.astype(np.float32)).cuda(), want_global=True)
    torch.cuda.synchronize()
    p = wl.particles
    idx = np.arange(p.n) if sample is None else sample
    ps = p.subset(idx)
    xp, yp, v = oracle.orient(ps)
    key = oracle.spaxel_keys(xp, yp, wl.telescope)
    tel = wl.telescope
    G0 = oracle.psf(oracle.lsf(G.astype(np.float64), tel, NT), tel, NT) if tel.psf_fwhm > 0 or tel.lsf_sigma > 0 \
        else G.astype(np.float64)
    ref = oracle.gradient(key, v, ps, wl.ssp, tel, G0, n_threads=NT, spectra=spectra)
    got = [a.cpu().numpy()[idx] for a in (dm, dage, dZ, dv)]
    for name, g, o in zip(("mass", "age", "Z", "v_los"), got, ref):
        scale = max(float(np.abs(o).max()), 1e-300)
        assert float(np.abs(g - o).max()) <= TOL * scale, (name, float(np.abs(g - o).max()) / scale)
    model_glob = glob.cpu().numpy()
    model.close()
    return got, ref, model_glob, key


def test_backward_small_random_cotangent(torch_cuda):
    wl = synth.small_galaxy(n=5000, seed=1)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((wl.telescope.ny, wl.telescope.nx, wl.telescope.n_lambda))
    got, ref, glob, key = _grad_check(torch_cuda, wl, G)
    # shared parameters: FP64 sums in a fixed order
    odv, odm = ref[3], ref[0]
    exp0 = float(odv.sum())
    exp1 = float((wl.particles.mass.astype(np.float64) * odm).sum())
    assert abs(glob[0] - exp0) <= 1e-4 * np.abs(odv).sum()
    assert abs(glob[1] - exp1) <= 1e-4 * np.abs(wl.particles.mass * odm).sum()
    # out-of-field particles get exactly zero
    out = key >= wl.telescope.nx * wl.telescope.ny
    assert out.any() and all((g[out] == 0).all() for g in got)


def test_backward_quadratic_loss_small(torch_cuda):
    """L = 1/2 |cube - target|^2 with the target made from perturbed ages,
    metallicities (10%) and velocities (+20 km/s); dL/dcube = cube - target,
    both from the oracle."""
    wl = synth.small_galaxy(n=4000, seed=5)
    tgt = synth.perturbed_target(wl.particles)
    cube = oracle.forward(wl.particles, wl.ssp, wl.telescope, n_threads=NT)
    target = oracle.forward(tgt, wl.ssp, wl.telescope, n_threads=NT)
    _grad_check(torch_cuda, wl, cube - target)


def test_backward_mid_size_sampled(torch_cuda):
    """Differentiable workload shape: 1e6 particles, 150x150x3721; gradients of
    100 sampled particles against the oracle."""
    wl = synth.mid_galaxy()
    rng = np.random.default_rng(11)
    G = rng.standard_normal((wl.telescope.ny, wl.telescope.nx, wl.telescope.n_lambda)).astype(np.float32)
    sample = np.sort(rng.choice(wl.particles.n, 100, replace=False))
    _grad_check(torch_cuda, wl, G, sample=sample)


def test_backward_quadratic_loss_mid_size(torch_cuda):
    """The differentiable workload itself: 1e6 particles, 150x150x3721, loss
    1/2 |cube - target|^2 with the target from ages and metallicities x (1 +
    N(0, 0.1)) and velocities + 20 km/s; dL/dcube = cube - target from the
    oracle; gradients of 100 sampled particles against the oracle's."""
    wl = synth.mid_galaxy()
    tgt = synth.perturbed_target(wl.particles)
    cube = oracle.forward(wl.particles, wl.ssp, wl.telescope, n_threads=NT)
    target = oracle.forward(tgt, wl.ssp, wl.telescope, n_threads=NT)
    rng = np.random.default_rng(12)
    sample = np.sort(rng.choice(wl.particles.n, 100, replace=False))
    _grad_check(torch_cuda, wl, cube - target, sample=sample)


def test_backward_bf16_templates(torch_cuda):
    wl = synth.small_galaxy(n=3000, seed=7)
    rng = np.random.default_rng(8)
    G = rng.standard_normal((wl.telescope.ny, wl.telescope.nx, wl.telescope.n_lambda))
    f = np.ascontiguousarray(wl.ssp.spectra, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    q = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    _grad_check(torch_cuda, wl, G, dtype="bf16", spectra=q)


def test_autograd_function(torch_cuda):
    """RubixCube.apply + loss.backward() reproduces the oracle gradient of
    L = 1/2 |cube - target|^2 (target fixed)."""
    torch = torch_cuda
    from paper_2412_08265_gb300.model import CubeModel, RubixCube
    wl = synth.small_galaxy(n=3000, seed=9)
    p = wl.particles
    model = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=p.n)
    tgt = synth.perturbed_target(p)
    target = torch.from_numpy(oracle.forward(tgt, wl.ssp, wl.telescope, n_threads=NT).astype(np.float32)).cuda()
    t = lambda a, g=False: torch.tensor(a, device="cuda", requires_grad=g)
    mass, age, Z, v = t(p.mass, True), t(p.age, True), t(p.Z, True), t(p.v_los, True)
    cube = RubixCube.apply(mass, age, Z, v, t(p.x), t(p.y), model)
    loss = 0.5 * ((cube - target) ** 2).sum()
    loss.backward()
    G = oracle.forward(p, wl.ssp, wl.telescope, n_threads=NT) - target.cpu().numpy().astype(np.float64)
    tel = wl.telescope
    G0 = oracle.psf(oracle.lsf(G, tel, NT), tel, NT)
    xp, yp, vv = oracle.orient(p)
    key = oracle.spaxel_keys(xp, yp, tel)
    ref = oracle.gradient(key, vv, p, wl.ssp, tel, G0, n_threads=NT)
    for g, o in zip((mass.grad, age.grad, Z.grad, v.grad), ref):
        assert float(np.abs(g.cpu().numpy() - o).max()) <= 2 * TOL * float(np.abs(o).max())
    model.close()


def test_backward_refuses_a_replaced_forward(torch_cuda):
    """A handle keeps the state of its most recent forward only. Two
    RubixCube.apply calls on one model in one graph: loss.backward() reaches
    the later application first (its gradient is right), then the earlier
    one, whose forward state has been replaced -- the library refuses it
    (forward tag mismatch) instead of returning the later galaxy's gradients."""
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.model import CubeModel, RubixCube
    wl = synth.small_galaxy(n=2000, seed=3)
    p = wl.particles
    model = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=p.n)
    t = lambda a, g=False: torch.tensor(a, device="cuda", requires_grad=g)
    mass, age, Z, v = t(p.mass, True), t(p.age, True), t(p.Z, True), t(p.v_los, True)
    c1 = RubixCube.apply(mass, age, Z, v, t(p.x), t(p.y), model)
    assert model.last_tag == 1
    c2 = RubixCube.apply(mass * 2.0, age, Z, v, t(p.x), t(p.y), model)
    assert model.last_tag == 2
    loss = c1.sum() + c2.sum()
    with pytest.raises(capi.RubixError, match="later forward replaced it"):
        loss.backward()
    # through the ABI: the earlier tag is refused, the current one accepted
    g = torch.ones(model.cube_shape, device="cuda")
    with pytest.raises(capi.RubixError):
        model.backward(g, forward_tag=1)
    dm, _, _, _, _ = model.backward(g, forward_tag=2)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(dm).all())
    model.close()


@pytest.mark.parametrize("z", [0.005, 0.02])
def test_backward_redshifted_and_scaled(torch_cuda, z):
    """Galaxy at redshift z with a flux scale: z = 0.005 keeps the deposit's
    fast path (dt/dj > 30/31), z = 0.02 takes the general path."""
    base = synth.mid_galaxy(n=40_000, seed=8)
    tel = synth.Telescope(nx=24, ny=24, spaxel_size=0.5, n_lambda=3721, lambda0=4750.0, dlambda=1.25,
                          z_cosmo=z, flux_scale=3e-3)
    wl = synth.Workload("mid-redshifted", base.particles, base.ssp, tel)
    rng = np.random.default_rng(11)
    G = rng.standard_normal((tel.ny, tel.nx, tel.n_lambda))
    _grad_check(torch_cuda, wl, G)


@pytest.mark.parametrize("case", ["fast", "redshift_general", "coarse_bins", "high_velocity"])
def test_backward_bin_means(torch_cuda, case):
    """Adjoint of the bin means (resample = 1) against the oracle's gradient,
    which differentiates the bin edges too; the cases take the 30-bin-round
    fast path, the per-bin path (dt/dj < 30/31 or ~2.3) and the global path."""
    base = synth.mid_galaxy(n=30_000, seed=12)
    p = base.particles
    kw = dict(nx=20, ny=20, spaxel_size=0.5, n_lambda=3721, lambda0=4750.0, dlambda=1.25,
              flux_scale=4e-3, resample=1)
    if case == "redshift_general":
        kw.update(z_cosmo=0.02)
    elif case == "coarse_bins":
        kw.update(n_lambda=1583, dlambda=2.9, lambda0=4760.0)
    elif case == "high_velocity":
        p.v_los = p.v_los.copy()
        p.v_los[::9] = np.float32(4000.0)
        p.v_los[4::9] = np.float32(-3500.0)
    tel = synth.Telescope(**kw)
    wl = synth.Workload("mid-bin-means", p, base.ssp, tel)
    rng = np.random.default_rng(13)
    G = rng.standard_normal((tel.ny, tel.nx, tel.n_lambda))
    _grad_check(torch_cuda, wl, G)


@pytest.mark.parametrize("resample", [0, 1])
def test_backward_oriented_3d_and_angle_gradients(torch_cuda, resample):
    """3-D disk oriented by (inclination, azimuth, position angle): per-particle
    gradients against the oracle, and the shared-angle gradients d_global[2:4]
    = sum_p dL/dv_p dv_p/d(angle) against the oracle's sums in FP64."""
    from paper_2412_08265_gb300.model import CubeModel
    base = synth.small_galaxy()
    p = synth.disk_3d(20_000, 33, inclination=1.1, azimuth=0.7, position_angle=-0.4)
    tel = synth.Telescope(nx=40, ny=36, spaxel_size=0.35, n_lambda=900, lambda0=4050.0, dlambda=2.4,
                          resample=resample)
    wl = synth.Workload("oriented-3d", p, base.ssp, tel)
    rng = np.random.default_rng(19)
    G = rng.standard_normal((tel.ny, tel.nx, tel.n_lambda))
    got, ref, glob, key = _grad_check(torch_cuda, wl, G)
    _, _, _, di, da = oracle.orient(p, derivatives=True)
    odv = ref[3]
    for c, d in ((2, di), (3, da)):
        exp = float((odv * d).sum())
        assert abs(glob[c] - exp) <= 1e-4 * float(np.abs(odv * d).sum()), (c, glob[c], exp)
        assert abs(exp) > 0.0


@pytest.mark.parametrize("seed", range(4))
def test_backward_random_configurations(torch_cuda, seed):
    """Seeded random grids, telescopes (bin width, redshift, flux scale,
    resampling mode, PSF/LSF) and projected or oriented 3-D galaxies: the
    adjoint against the oracle's gradient for a random cotangent."""
    rng = np.random.default_rng(700 + seed)
    n_ls = int(rng.integers(300, 2000))
    ls_lo = float(rng.uniform(3800.0, 4200.0))
    ssp = synth.ssp_grid(int(rng.integers(2, 20)), int(rng.integers(1, 6)), n_ls, ls_lo,
                         ls_lo + float(rng.uniform(0.8, 2.5)) * n_ls, seed=seed)
    dls = ssp.dlambda
    dl = float(dls * rng.choice([rng.uniform(0.5, 0.97), rng.uniform(0.975, 1.0), rng.uniform(1.0, 2.5)]))
    n_l = int(rng.integers(50, min(1500, int(0.8 * n_ls * dls / dl))))
    tel = synth.Telescope(nx=int(rng.integers(3, 24)), ny=int(rng.integers(3, 24)),
                          spaxel_size=float(rng.uniform(0.3, 1.0)), n_lambda=n_l,
                          lambda0=float(ls_lo + 0.1 * n_ls * dls), dlambda=dl,
                          psf_fwhm=float(rng.choice([0.0, 1.5])), lsf_sigma=float(rng.choice([0.0, 1.2 * dl])),
                          z_cosmo=float(rng.choice([0.0, 0.003])), flux_scale=float(rng.uniform(0.5, 2.0)),
                          resample=int(rng.integers(0, 2)))
    n = int(rng.integers(2_000, 12_000))
    if seed % 2:
        p = synth.disk_3d(n, 800 + seed, inclination=float(rng.uniform(0, np.pi)),
                          azimuth=float(rng.uniform(-np.pi, np.pi)), position_angle=float(rng.uniform(-np.pi, np.pi)))
    else:
        p = synth.disk_projected(n, 800 + seed)
    wl = synth.Workload("random", p, ssp, tel)
    G = rng.standard_normal((tel.ny, tel.nx, tel.n_lambda))
    _grad_check(torch_cuda, wl, G)
