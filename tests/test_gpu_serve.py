"""GPU tests of the request server (rubix_serve_*): continuous batching of
galaxies of different particle counts and cube sizes through one resident SSP
grid, admission by device footprint, cancellation and waits with a limit.

The central property: a request's cube is bitwise the same served alone, in a
mix with other requests, and from the single-galaxy handle, because its work
decomposition never depends on the other requests in a deposit launch. One
served request is also checked against the FP64 oracle.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2412_08265_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
NT = os.cpu_count() or 1


@pytest.fixture(scope="module")
def env():
    import torch
    from __graft_entry__ import build
    build()
    torch.cuda.set_device(0)
    ssp = synth.mid_galaxy(n=1).ssp
    return torch, ssp


def requests(n_req, seed=5, n_lo=2e3, n_hi=3e5, side_lo=12, side_hi=64):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        side = int(rng.integers(side_lo, side_hi + 1))
        incl = float(rng.uniform(0, 0.5 * np.pi))
        out.append((synth.disk_3d(n, 100 + i, inclination=incl), synth.serving_telescope(side)))
    return out


def dev(torch, p):
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float32)).cuda()
         for k in ("x", "y", "z", "vx", "vy", "vz", "mass", "age", "Z")}
    d["preprojected"] = False
    d["inclination"] = p.inclination
    return d


def server(ssp, budget=8 << 30, slots=8, batch=16):
    from paper_2412_08265_gb300.serve import Server
    return Server(ssp, synth.serving_telescope(16), hbm_budget_bytes=budget, max_slots=slots, max_batch=batch)


def run_all(torch, srv, reqs, noise=None):
    """Submit every request back to back (inputs uploaded first), wait for all."""
    ins = [dev(torch, p) for p, _ in reqs]
    outs = [torch.full((tel.ny, tel.nx, tel.n_lambda), float("nan"), device="cuda") for _, tel in reqs]
    torch.cuda.synchronize()
    tickets = []
    for i, (_, tel) in enumerate(reqs):
        seed, s2n = (noise[i] if noise else (0, 0.0))
        tickets.append(srv.submit(tel, ins[i], outs[i], noise_seed=seed, noise_s2n=s2n))
    for t in tickets:
        assert srv.wait(t, 120.0) == 0
    return [o.cpu().numpy() for o in outs], tickets


def test_serve_alone_vs_mix_bitwise_and_vs_handle(env):
    torch, ssp = env
    reqs = requests(50)
    noise = [(7 + i, 30.0) if i % 4 == 3 else (0, 0.0) for i in range(len(reqs))]
    # alone: one slot, one galaxy per deposit launch, one request at a time
    srv = server(ssp, slots=1, batch=1)
    alone = []
    for i, r in enumerate(reqs):
        o, _ = run_all(torch, srv, [r], noise=[noise[i]])
        alone.append(o[0])
    st = srv.stats()
    assert st["ok"] == len(reqs) and st["deposit_launches"] == len(reqs) and st["max_batch"] == 1
    srv.close()
    # mix: everything submitted at once, shared deposit launches
    srv = server(ssp, budget=24 << 30, slots=16, batch=16)
    mix, _ = run_all(torch, srv, reqs, noise=noise)
    st = srv.stats()
    assert st["ok"] == len(reqs) and st["failed"] == 0
    assert st["max_batch"] > 1 and st["deposit_launches"] < len(reqs)
    srv.close()
    for i in range(len(reqs)):
        assert np.isfinite(mix[i]).all()
        assert np.array_equal(alone[i].view(np.uint32), mix[i].view(np.uint32)), i
    # the single-galaxy handle gives the same bits
    from paper_2412_08265_gb300.model import CubeModel
    for i in (0, 5, 11):
        p, tel = reqs[i]
        m = CubeModel(ssp, tel, "f32", max_particles=p.n)
        got = m.forward(p, noise_seed=noise[i][0], noise_s2n=noise[i][1]).cpu().numpy()
        m.close()
        assert np.array_equal(got.view(np.uint32), mix[i].view(np.uint32)), i


def test_served_requests_match_oracle(env):
    """20 served requests against the oracle: 19 of 1e3-1e5 particles and
    10-48 spaxels a side on the whole cube (the smallest request included),
    and a 2e6-particle 300x300 request at sampled spaxels (neighbourhoods of
    the densest spaxels, random ones and the field corners)."""
    torch, ssp = env
    reqs = requests(19, seed=9, n_lo=1e3, n_hi=1e5, side_lo=10, side_hi=48)
    big_tel = synth.serving_telescope(300)
    big = synth.disk_3d(2_000_000, 77, inclination=0.9)
    reqs.append((big, big_tel))
    srv = server(ssp, budget=16 << 30)
    outs, _ = run_all(torch, srv, reqs)
    srv.close()
    assert min(p.n for p, _ in reqs[:19]) < 2e3
    for (p, tel), got in zip(reqs[:19], outs[:19]):
        ref = oracle.forward(p, ssp, tel, n_threads=NT)
        err = float(np.abs(got.astype(np.float64) - ref).max() / np.abs(ref).max())
        assert err <= TOL_F32
    # the large request at sampled spaxels
    xp, yp, v = oracle.orient(big)
    key = oracle.spaxel_keys(xp, yp, big_tel)
    ns = big_tel.nx * big_tel.ny
    counts = np.bincount(key, minlength=ns + 1)[:ns]
    rng = np.random.default_rng(3)
    sel = np.unique(np.concatenate([np.argsort(counts)[-3:], rng.choice(np.flatnonzero(counts > 0), 5, replace=False),
                                    [0, big_tel.nx - 1, ns - 1]])).astype(np.int32)
    mask = np.zeros(ns, np.uint8)
    for s_ in sel:
        y, x = divmod(int(s_), big_tel.nx)
        for yy in range(max(0, y - 3), min(big_tel.ny, y + 4)):
            mask[yy * big_tel.nx + max(0, x - 3): yy * big_tel.nx + min(big_tel.nx, x + 4)] = 1
    cube0 = oracle.deposit(key, v, big, ssp, big_tel, mask=mask, n_threads=NT)
    ref = oracle.psf_lsf_at(cube0, big_tel, sel)
    got = outs[19].reshape(-1, big_tel.n_lambda)[sel].astype(np.float64)
    assert float(np.abs(got - ref).max()) / float(np.abs(ref).max()) <= TOL_F32


def test_host_inputs_and_outputs(env):
    """Host particle arrays, pinned and pageable host cubes: same bits as device I/O."""
    torch, ssp = env
    reqs = requests(4, seed=13, n_hi=5e4, side_hi=32)
    srv = server(ssp)
    ref, _ = run_all(torch, srv, reqs)
    tickets, outs = [], []
    for i, (p, tel) in enumerate(reqs):
        d = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float32))
             for k in ("x", "y", "z", "vx", "vy", "vz", "mass", "age", "Z")}
        d["preprojected"] = False
        d["inclination"] = p.inclination
        o = torch.empty((tel.ny, tel.nx, tel.n_lambda), dtype=torch.float32, pin_memory=(i % 2 == 0))
        tickets.append(srv.submit(tel, d, o))
        outs.append(o)
    for t in tickets:
        assert srv.wait(t, 120.0) == 0
    srv.close()
    for a, b in zip(ref, outs):
        assert np.array_equal(a.view(np.uint32), b.numpy().view(np.uint32))


def test_admission_by_footprint(env):
    torch, ssp = env
    from paper_2412_08265_gb300 import capi
    reqs = requests(8, seed=17, n_lo=1e5, n_hi=2e5, side_lo=48, side_hi=64)
    probe = server(ssp, budget=1 << 40)
    outs, _ = run_all(torch, probe, reqs)
    fp = [probe.footprint(tel, dev(torch, p), torch.empty(1, device="cuda")) for p, tel in reqs]
    probe.close()
    # a budget that holds two or three of these requests at a time
    budget = int(2.5 * max(fp))
    srv = server(ssp, budget=budget, slots=8, batch=8)
    got, _ = run_all(torch, srv, reqs)
    st = srv.stats()
    assert st["ok"] == len(reqs) and 0 < st["peak_bytes"] <= budget
    assert st["bytes_in_use"] == 0 and st["active"] == 0 and st["queued"] == 0
    for a, b in zip(outs, got):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # a request whose footprint alone exceeds the budget is rejected at submit
    p, tel = synth.disk_3d(2_000_000, 3, inclination=0.3), synth.serving_telescope(300)
    o = torch.empty((tel.ny, tel.nx, tel.n_lambda), device="cuda")
    with pytest.raises(capi.RubixError) as ei:
        srv.submit(tel, dev(torch, p), o)
    assert ei.value.status == capi.RUBIX_ERR_REJECTED
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_cancel_wait_timeout_and_bad_requests(env):
    torch, ssp = env
    from paper_2412_08265_gb300 import capi
    srv = server(ssp, slots=1, batch=1)
    big = synth.disk_3d(6_000_000, 21, inclination=0.5)
    tel_big = synth.serving_telescope(300)
    o_big = torch.empty((300, 300, 3721), device="cuda")
    d_big = dev(torch, big)
    small = requests(3, seed=23, n_hi=1e4, side_hi=20)
    d_small = [dev(torch, p) for p, _ in small]
    outs = [torch.full((t.ny, t.nx, t.n_lambda), -1.0, device="cuda") for _, t in small]
    torch.cuda.synchronize()
    # every input is ready: the submits below are microseconds apart, and the
    # big request keeps the only slot for tens of milliseconds
    t_big = srv.submit(tel_big, d_big, o_big)
    ts = [srv.submit(t, d, o) for (_, t), d, o in zip(small, d_small, outs)]
    # the big request needs tens of milliseconds on the GPU: a zero wait times out
    assert srv.wait(t_big, 0.0) == capi.RUBIX_ERR_TIMEOUT
    # the last small request is still queued behind it (one slot): cancel it
    assert srv.cancel(ts[2]) == capi.RUBIX_OK
    assert srv.poll(ts[2])[0] == capi.RUBIX_ERR_CANCELLED
    assert srv.wait(t_big, 120.0) == capi.RUBIX_OK
    for t in ts[:2]:
        assert srv.wait(t, 120.0) == capi.RUBIX_OK
    # a cancelled request never touches its cube
    assert bool((outs[2] == -1.0).all())
    # cancelling a finished request returns its final status
    assert srv.cancel(t_big) == capi.RUBIX_OK
    st, lat = srv.poll(t_big)
    assert st == capi.RUBIX_OK and lat > 0.0
    # a wavelength grid other than the server's, and unknown tickets
    bad = synth.Telescope(nx=16, ny=16, spaxel_size=0.2, n_lambda=1000, lambda0=4750.0, dlambda=1.25)
    with pytest.raises(capi.RubixError) as ei:
        srv.submit(bad, dev(torch, small[0][0]), torch.empty((16, 16, 1000), device="cuda"))
    assert ei.value.status == capi.RUBIX_ERR_INVALID_ARG
    assert srv.poll(987654321)[0] == capi.RUBIX_ERR_INVALID_ARG
    s = srv.stats()
    assert s["cancelled"] == 1 and s["ok"] == 3
    srv.close()


def test_empty_request_and_destroy_with_pending(env):
    torch, ssp = env
    srv = server(ssp)
    tel = synth.serving_telescope(16)
    z = np.zeros(0, dtype=np.float32)
    d = {k: torch.from_numpy(z).cuda() for k in ("x", "y", "z", "vx", "vy", "vz", "mass", "age", "Z")}
    d["preprojected"] = False
    d["inclination"] = 0.0
    o = torch.full((16, 16, 3721), 5.0, device="cuda")
    t = srv.submit(tel, d, o)
    assert srv.wait(t, 60.0) == 0
    assert bool((o == 0).all())
    # destroy returns with requests queued and on the GPU
    for p, tl in requests(6, seed=29):
        srv.submit(tl, dev(torch, p), torch.empty((tl.ny, tl.nx, tl.n_lambda), device="cuda"))
    srv.close()
    torch.cuda.synchronize()


def test_concurrent_client_threads(env):
    """Four client threads submit and wait at once: every cube equals the
    cube of the same request run alone, bitwise."""
    import threading
    torch, ssp = env
    reqs = requests(12, seed=31, n_hi=1e5, side_hi=48)
    srv = server(ssp, slots=1, batch=1)
    alone = [run_all(torch, srv, [r])[0][0] for r in reqs]
    srv.close()
    srv = server(ssp, slots=8, batch=8)
    ins = [dev(torch, p) for p, _ in reqs]
    outs = [torch.full((t.ny, t.nx, t.n_lambda), float("nan"), device="cuda") for _, t in reqs]
    torch.cuda.synchronize()
    status = [None] * len(reqs)

    def client(k):
        for i in range(k, len(reqs), 4):
            t = srv.submit(reqs[i][1], ins[i], outs[i])
            status[i] = srv.wait(t, 120.0)

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert all(s == 0 for s in status)
    assert srv.stats()["ok"] == len(reqs)
    srv.close()
    for a, o in zip(alone, outs):
        assert np.array_equal(a.view(np.uint32), o.cpu().numpy().view(np.uint32))


def test_bin_means_share_launches_with_centre_samples(env):
    """Requests with resample = 1 (bin means) and 0 (centre samples) in shared
    deposit launches: every cube equals the same request served alone,
    bitwise, and a served bin-mean request matches the oracle."""
    torch, ssp = env
    reqs = [(p, synth.Telescope(**{**tel.__dict__, "resample": i % 2}))
            for i, (p, tel) in enumerate(requests(10, seed=41, n_hi=8e4, side_hi=40))]
    srv = server(ssp, slots=1, batch=1)
    alone = [run_all(torch, srv, [r])[0][0] for r in reqs]
    srv.close()
    srv = server(ssp, slots=10, batch=10)
    mix, _ = run_all(torch, srv, reqs)
    st = srv.stats()
    assert st["ok"] == len(reqs) and st["max_batch"] > 1
    srv.close()
    for i, (a, b) in enumerate(zip(alone, mix)):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), i
    for i in (1, 3):
        p, tel = reqs[i]
        ref = oracle.forward(p, ssp, tel, n_threads=NT)
        assert float(np.abs(mix[i].astype(np.float64) - ref).max() / np.abs(ref).max()) <= TOL_F32
