"""Multi-process host logic on CPU (gloo, world size 2): the benchmark's
whole-job aggregate over ranks, a rank that fails before the collective ends
the other rank's wait with an error instead of a hang, and the halo exchange
of spaxel-row sharding.
One process per rank, as under torchrun; no GPU is used."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, port, timeout_s=60):
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2, timeout=datetime.timedelta(seconds=timeout_s))


def _aggregate(rank, port, q):
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, port)
    # rank r processed 10 (r + 1) units in 1 + r seconds
    rate, units, secs = bench.whole_job(10.0 * (rank + 1), 1.0 + rank)
    q.put((rank, rate, units, secs))
    dist.barrier()
    dist.destroy_process_group()


def _one_rank_fails(rank, port, q):
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, port, timeout_s=5)
    dist.barrier()  # both ranks are up; rank 1 then leaves between steps
    if rank == 1:
        q.put((rank, "exit"))
        q.close()
        q.join_thread()  # the message is out before the process ends
        os._exit(3)  # the failing rank leaves before the collective, with nothing in flight
    try:
        bench.whole_job(1.0, 1.0)
        q.put((rank, "returned"))
    except Exception as e:  # the surviving rank's collective ends with an error
        q.put((rank, "error:" + type(e).__name__))


def _halo_exchange(rank, port, q):
    sys.path.insert(0, ROOT)
    from paper_2412_08265_gb300.shard import exchange_halos, halo_plan, row_blocks
    _init(rank, port)
    ny, nx, nl, h = 11, 3, 4, 3
    blocks = row_blocks(ny, 2)
    lo, hi = blocks[rank]
    value = lambda r: torch.arange(nx * nl, dtype=torch.float32).reshape(nx, nl) + 1000.0 * r
    own = torch.stack([value(r) for r in range(lo, hi)])
    ext = exchange_halos(own, h, rank, 2)
    b, a = halo_plan(blocks, h)[rank]
    want = torch.stack([value(r) for r in range(lo - b, hi + a)])
    q.put((rank, (lo, hi), (b, a), bool(torch.equal(ext, want))))
    dist.barrier()
    dist.destroy_process_group()


def _run(fn):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=fn, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=60) for _ in range(2)]
    for p in ps:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
    return sorted(out), [p.exitcode for p in ps]


def test_whole_job_aggregate_two_ranks():
    out, codes = _run(_aggregate)
    assert codes == [0, 0]
    for rank, rate, units, secs in out:
        assert units == 30.0 and secs == 2.0 and rate == 15.0


def test_failed_rank_ends_the_collective_with_an_error():
    out, codes = _run(_one_rank_fails)
    assert out[1] == (1, "exit") and codes[1] == 3
    assert out[0][0] == 0 and out[0][1].startswith("error:")


def test_row_shard_halo_exchange_two_ranks():
    """Row sharding's exchange step: each rank ends with its own rows plus the
    PSF-radius rows of its neighbour (none beyond the field's edges), and the
    two blocks cover the field once."""
    out, codes = _run(_halo_exchange)
    assert codes == [0, 0]
    (r0, blk0, halo0, ok0), (r1, blk1, halo1, ok1) = out
    assert blk0 == (0, 5) and blk1 == (5, 11)
    assert halo0 == (0, 3) and halo1 == (3, 0)
    assert ok0 and ok1
