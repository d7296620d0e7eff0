"""The multi-GPU path of bench.py runs independent replicas (one system per
rank, no data-path collective); its only cross-rank step is the reduction of
the figures it reports: the slowest rank's time and the sum of the work.
Checked here with two gloo ranks on the CPU (no GPU needed)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [10.0 + rank, 2.0 * (rank + 1)]          # rank 1 is the slower one
    counts = [1000.0 * (rank + 1), 7.0, 3.0]
    t, c = bench.reduce_over_ranks(dist, times, counts, torch.device("cpu"))
    out.put((rank, t, c))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_figures_reduce_max_time_and_sum_work():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, c in results:
        assert t == [11.0, 4.0]                      # MAX over ranks
        assert c == [3000.0, 14.0, 6.0]              # SUM over ranks


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:  # noqa: N801 - argparse stand-in
        gpus, steps, warmup, ref_rounds = 2, 1, 0, 1
    assert bench.run_reference(A()) == 0             # rank 1 exits without work
