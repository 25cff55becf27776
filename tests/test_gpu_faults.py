"""Failure detection on the GPU without a GPU fault: an allocation failure
injected on the host (RUBIX_FAULT_ALLOC_AT) comes back as RUBIX_ERR_OOM with
no device memory leaked, from the single-galaxy handle and from the server
(which keeps serving), and a device wait that nothing completes gives up at
its limit and leaves the context usable."""
import os

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


@pytest.fixture
def fault_env():
    yield os.environ
    os.environ.pop("RUBIX_FAULT_ALLOC_AT", None)


def _free(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failure_handle(torch_cuda, fault_env):
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.model import CubeModel
    wl = synth.small_galaxy(n=3000, seed=4)
    m = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=wl.particles.n)  # warm the context
    m.close()
    free0 = _free(torch)
    for k in (1, 5, 17):
        fault_env["RUBIX_FAULT_ALLOC_AT"] = str(k)
        with pytest.raises(capi.RubixError) as ei:
            CubeModel(wl.ssp, wl.telescope, "f32", max_particles=wl.particles.n)
        assert ei.value.status == capi.RUBIX_ERR_OOM
    fault_env.pop("RUBIX_FAULT_ALLOC_AT")
    assert abs(_free(torch) - free0) <= (2 << 20)
    m = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=wl.particles.n)
    got = m.forward(wl.particles).cpu().numpy()
    ref = oracle.forward(wl.particles, wl.ssp, wl.telescope)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-5
    m.close()


def test_injected_allocation_failure_server(torch_cuda, fault_env):
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.serve import Server
    ssp = synth.mid_galaxy(n=1).ssp
    tel = synth.serving_telescope(24)
    srv = Server(ssp, tel, hbm_budget_bytes=8 << 30, max_slots=4, max_batch=4)
    p = synth.disk_3d(20_000, 5, inclination=0.4)
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float32)).cuda()
         for k in ("x", "y", "z", "vx", "vy", "vz", "mass", "age", "Z")}
    d["preprojected"] = False
    d["inclination"] = p.inclination
    outs = [torch.full((24, 24, 3721), -1.0, device="cuda") for _ in range(3)]
    t0 = srv.submit(tel, d, outs[0])
    assert srv.wait(t0, 60.0) == capi.RUBIX_OK
    fault_env["RUBIX_FAULT_ALLOC_AT"] = "3"
    t1 = srv.submit(tel, d, outs[1])
    assert srv.wait(t1, 60.0) == capi.RUBIX_ERR_OOM
    fault_env.pop("RUBIX_FAULT_ALLOC_AT")
    t2 = srv.submit(tel, d, outs[2])
    assert srv.wait(t2, 60.0) == capi.RUBIX_OK
    st = srv.stats()
    assert st["ok"] == 2 and st["failed"] == 1 and st["bytes_in_use"] == 0 and st["active"] == 0
    assert bool((outs[1] == -1.0).all())  # the failed request never wrote its cube
    assert torch.equal(outs[0], outs[2])
    srv.close()


def test_bounded_device_wait_gives_up(torch_cuda):
    torch = torch_cuda
    from paper_2412_08265_gb300 import capi
    assert capi.rubix_selftest_bounded_wait(0.05) is True
    # the context is still usable: a forward runs and matches the oracle
    from paper_2412_08265_gb300.model import CubeModel
    wl = synth.small_galaxy(n=2000, seed=8)
    m = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=wl.particles.n)
    got = m.forward(wl.particles).cpu().numpy()
    ref = oracle.forward(wl.particles, wl.ssp, wl.telescope)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-5
    assert m.stats()["device_error"] == 0
    m.close()
