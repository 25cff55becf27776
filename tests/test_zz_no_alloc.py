"""rubix_spaxel_sort_noalloc, the sort entry point for callers that may not
allocate device memory (their memory belongs to another allocator, or a
cudaMalloc's device synchronisation is not acceptable where they call it).

Checked through the C ABI against the FP64 oracle's spaxel keys and stable
sort on consecutive calls; integer results must be identical.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
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


def _oracle_sort(p, tel):
    xp, yp, _ = oracle.orient(p)
    key = oracle.spaxel_keys(xp, yp, tel)
    return oracle.stable_sort(key, tel.nx * tel.ny + 1)


def test_noalloc_sort_matches_oracle_twice(torch_cuda):
    """Pre-projected mid-size galaxy: perm and segment offsets equal the
    oracle's stable sort bit for bit, on consecutive calls, and the calls
    after the first take no device memory."""
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.model import CubeModel

    wl = synth.mid_galaxy(n=200_000, seed=5)
    tel = wl.telescope
    operm, oseg = _oracle_sort(wl.particles, tel)
    d = {k: torch.tensor(getattr(wl.particles, k), dtype=torch.float32, device="cuda")
         for k in ("x", "y", "v_los", "mass", "age", "Z")}
    d.update(preprojected=True, inclination=0.0)
    cp = CubeModel.c_particles(d)
    ct = CubeModel.c_telescope(tel)
    stream = torch.cuda.current_stream().cuda_stream
    n_s = tel.nx * tel.ny
    free_after = []
    perm = torch.empty((wl.particles.n,), dtype=torch.int32, device="cuda")
    seg = torch.empty((n_s + 2,), dtype=torch.int32, device="cuda")
    for call in range(3):
        perm.fill_(-7)
        seg.fill_(-7)
        torch.cuda.synchronize()
        capi.rubix_spaxel_sort_noalloc(cp, ct, perm.data_ptr(), seg.data_ptr(), stream)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        assert np.array_equal(seg.cpu().numpy().astype(np.int64), oseg), call
        assert np.array_equal(perm.cpu().numpy(), operm), call
    # after the first call (which may load the module holding the array), the
    # entry point takes no device memory
    assert free_after[1] == free_after[2]


def test_noalloc_sort_rotated_and_empty(torch_cuda):
    """A 3-D disk turned by inclination, azimuth and position angle (the
    orientation path of the key) against the oracle, then n = 0, whose
    segment offsets are all zero."""
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.model import CubeModel

    tel = synth.serving_telescope(97)
    p = synth.disk_3d(150_000, 31, inclination=1.1, azimuth=0.7, position_angle=-0.4)
    operm, oseg = _oracle_sort(p, tel)
    d = {k: torch.tensor(getattr(p, k), dtype=torch.float32, device="cuda")
         for k in ("x", "y", "z", "vx", "vy", "vz", "mass", "age", "Z")}
    d.update(preprojected=False, inclination=p.inclination, azimuth=p.azimuth, position_angle=p.position_angle)
    ct = CubeModel.c_telescope(tel)
    stream = torch.cuda.current_stream().cuda_stream
    n_s = tel.nx * tel.ny
    perm = torch.empty((p.n,), dtype=torch.int32, device="cuda")
    seg = torch.full((n_s + 2,), -7, dtype=torch.int32, device="cuda")
    for call in range(2):
        capi.rubix_spaxel_sort_noalloc(CubeModel.c_particles(d), ct, perm.data_ptr(), seg.data_ptr(), stream)
        torch.cuda.synchronize()
        assert np.array_equal(seg.cpu().numpy().astype(np.int64), oseg), call
        assert np.array_equal(perm.cpu().numpy(), operm), call
    d0 = {k: (v[:0] if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    seg.fill_(-7)
    capi.rubix_spaxel_sort_noalloc(CubeModel.c_particles(d0), ct, perm.data_ptr(), seg.data_ptr(), stream)
    torch.cuda.synchronize()
    assert not seg.cpu().numpy().any()


def test_noalloc_sort_limits_are_reported(torch_cuda):
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.model import CubeModel

    n = 262145
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    d = {"x": x, "y": x, "mass": x, "age": x, "Z": x, "v_los": x, "preprojected": True, "inclination": 0.0}
    cp = CubeModel.c_particles(d)
    ct = CubeModel.c_telescope(synth.Telescope(nx=10, ny=10, spaxel_size=1.0, n_lambda=1, lambda0=5000.0,
                                               dlambda=1.0))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.RubixError) as e:
        capi.rubix_spaxel_sort_noalloc(cp, ct, out.data_ptr(), out.data_ptr(), 0)
    assert e.value.status == capi.RUBIX_ERR_INVALID_ARG and "262144" in str(e.value)
    big = CubeModel.c_telescope(synth.Telescope(nx=600, ny=600, spaxel_size=1.0, n_lambda=1, lambda0=5000.0,
                                                dlambda=1.0))
    d_small = {k: (v[:10] if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    with pytest.raises(capi.RubixError) as e:
        capi.rubix_spaxel_sort_noalloc(CubeModel.c_particles(d_small), big, out.data_ptr(), out.data_ptr(), 0)
    assert e.value.status == capi.RUBIX_ERR_INVALID_ARG and "262143" in str(e.value)
