"""The multi-rank path of bench.py on CPU (gloo, world size 2).

With N GPUs the benchmark runs one independent cavity per rank (weak
scaling, no data-path collective); the only collectives are the barrier
around the timed region and the maximum of the per-rank times.  These tests
run that plumbing as two gloo ranks on the host.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    dist = bench.init_dist("gloo")
    assert dist is not None and dist.get_world_size() == world
    bench.barrier(dist)
    # each rank "timed" its own cavity; the report takes the slowest rank
    my_seconds = 1.5 + rank  # rank 1 is slower
    mx = bench.reduce_max(dist, my_seconds)
    value = bench.aggregate(cells_per_rank=64 ** 3, steps=10, world=world, max_seconds=mx)
    bench.barrier(dist)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{mx} {value}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_aggregate(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    vals = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for mx, value in vals:
        assert float(mx) == 2.5  # the slower rank's time, on every rank
        assert abs(float(value) - 64 ** 3 * 10 * 2 / 2.5) < 1e-6


def _reference_rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    if rank == 0:
        return  # rank 0 would run the oracle arm (minutes); only the other rank's exit is checked
    rc = bench.main_reference(bench.parse_args(["--impl", "reference", "--gpus", str(world)]))
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(str(rc))


def test_reference_arm_other_ranks_exit_without_work(tmp_path):
    world = 2
    mp.start_processes(_reference_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    assert open(tmp_path / "ref1.txt").read() == "0"


def test_single_rank_needs_no_process_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench.init_dist("gloo") is None
    assert bench.reduce_max(None, 3.25) == 3.25
    bench.barrier(None)
