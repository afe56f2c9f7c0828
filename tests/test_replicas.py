"""The N > 1 path of bench.py on CPU: two gloo ranks deal the serving stream's requests as replicas and
time the job by its slowest rank (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reqs = bench.serving_requests(11, seed=3)
    mine = bench.replica_share(reqs, rank, world)
    local_ms = 100.0 * (rank + 1) + len(mine)          # a stand-in for the rank's measured time
    out.put((rank, [r["geom_seed"] for r in mine], bench.max_over_ranks(local_ms, dist, device="cpu"), local_ms))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_deal_requests_and_take_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [r["geom_seed"] for r in bench.serving_requests(11, seed=3)]
    dealt = [s for _, mine, _, _ in res for s in mine]
    assert sorted(dealt) == sorted(seeds)                        # every request once, on one rank
    assert all(len(mine) in (5, 6) for _, mine, _, _ in res)     # balanced deal
    slowest = max(local for *_, local in res)
    assert all(m == slowest for _, _, m, _ in res)               # every rank sees the job's time
