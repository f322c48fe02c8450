"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): replicas only,
no data-path collective, so what the ranks share is the timing rule (the max
over ranks) and distinct replica inputs.  A rank that never joins is detected
on the host by the collective's timeout, with no GPU involved."""
import datetime
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, scenario):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    try:
        if scenario == "max":
            dist.barrier()
            got = bench.max_over_ranks(10.0 + 3.0 * rank, "cpu")
            seed = bench.replica_seed(rank)
            with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
                f.write(f"{got} {seed}\n")
        elif scenario == "missing":
            if rank == 1:
                return  # leaves before the timed region's collective
            try:
                bench.max_over_ranks(1.0, "cpu")
                msg = "joined"
            except RuntimeError as e:  # the peer never joined: the collective times out
                msg = "timeout " + type(e).__name__
            with open(os.path.join(out_dir, "r0.txt"), "w") as f:
                f.write(msg + "\n")
    finally:
        if scenario == "max":
            dist.destroy_process_group()


def test_max_over_ranks_and_replica_seeds(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path), "max"), nprocs=2, join=True, start_method="spawn")
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(2)]
    assert [float(r[0]) for r in rows] == [13.0, 13.0]
    assert rows[0][1] != rows[1][1]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, "cpu") == 7.5


def test_missing_rank_is_detected_by_timeout(tmp_path):
    port = _free_port()
    ctx = mp.start_processes(_worker, args=(2, port, str(tmp_path), "missing"), nprocs=2, join=False,
                             start_method="spawn")
    while not ctx.join(timeout=60):
        pass
    assert open(tmp_path / "r0.txt").read().startswith("timeout")


def test_cpulist_parsing():
    # the host memory node's CPU list the e2e measurement binds its pinned
    # buffers to (sysfs format)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_cpulist("0-15\n") == set(range(16))
    assert bench.parse_cpulist("0-3,8,10-11") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("") == set()
