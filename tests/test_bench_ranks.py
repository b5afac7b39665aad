"""The multi-rank logic of bench.py on CPU: two gloo ranks run independent
replicas, barrier around the timed region, reduce the maximum of their times
and report the whole-job throughput (units of all ranks over the slowest
rank's time).  No GPU: the collectives run on CPU tensors."""
import os
import socket
import sys
from pathlib import Path

import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import torch
    import bench
    r = bench.Ranks("gloo", device=torch.device("cpu"))
    r.barrier()
    t_max = r.max(times[rank])
    value = r.aggregate(1000.0, t_max)
    r.barrier()
    out.put((rank, r.world, t_max, value))
    r.close()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_max_time_and_aggregate(world):
    times = [0.5 + 0.25 * k for k in range(world)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, world, port, times, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, t_max, value in got:
        assert w == world
        assert t_max == max(times)
        assert value == pytest.approx(world * 1000.0 / max(times))


def test_single_rank_needs_no_process_group(monkeypatch):
    import torch
    sys.path.insert(0, str(ROOT))
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = bench.Ranks("gloo", device=torch.device("cpu"))
    assert (r.world, r.rank) == (1, 0)
    assert r.max(3.5) == 3.5
    assert r.aggregate(100.0, 2.0) == 50.0
    r.barrier()
    r.close()
