"""bench.py at N > 1 runs independent replicas (no data-path collective):
every rank times its own solves, the job's time is the slowest rank's, and
the value counts the DOFs of every rank.  Checked with two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RANK_MS = [12.5, 30.0]


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if ROOT not in sys.path:
            sys.path.insert(0, ROOT)
        import bench
        got = bench.max_over_ranks(RANK_MS[rank], world, "cpu")
        with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as f:
            f.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [float((tmp_path / f"rank{r}.txt").read_text()) for r in range(world)]
    assert got == [max(RANK_MS)] * world


def test_single_rank_and_job_value():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1, "cpu") == 7.0
    # 2 ranks x 3 steps x 1,000 DOFs in 0.5 s
    assert bench.job_value(2, 3, 1000, 500.0) == pytest.approx(12000.0)
