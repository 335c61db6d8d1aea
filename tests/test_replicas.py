"""bench.py with N > 1: independent replicas, one process per GPU.

The ranks exchange nothing on the data path; the only collectives are the
barrier around the timed region and the maximum of the ranks' times, from
which rank 0 reports the whole-job value.  Tested here with two gloo ranks
on the CPU (no GPU): the maximum reaches every rank and the whole-job value
counts every rank's paths over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, local = bench.dist_env()
    bench.barrier(w)
    slowest = bench.max_over_ranks(100.0 + 25.0 * r, w)  # this rank's time of K steps, ms
    bench.barrier(w)
    q.put((r, w, local, slowest, bench.replica_value(w, 45360, 5, slowest)))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_report_the_slowest_rank_and_every_rank_s_paths():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    assert all(o[3] == 125.0 for o in out)
    assert all(abs(o[4] - 2 * 45360 * 5 / 0.125) < 1e-6 for o in out)
