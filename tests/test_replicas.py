"""The multi-GPU mode of the bench, on CPU.

The iteration does not shard into independent units, so N GPUs run N independent
replicas (one per rank, each with its own seeded problem) and the whole-job figures are
the iterations of all ranks over the slowest rank's time.  Two gloo ranks on the host
check that reduction and that the replicas get different inputs; no GPU is involved.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # rank r took 1.5 + r seconds for 10 (r + 1) iterations
        seconds, iters = bench.reduce_over_ranks(1.5 + rank, 10 * (rank + 1), "cpu")
        wl = bench.make_workload("lowrank500", seed_offset=rank)
        np.save(os.path.join(out_dir, f"vals{rank}.npy"), wl.vals)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{seconds} {iters}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_to_whole_job_figures(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for rank in range(world):
        seconds, iters = map(float, (tmp_path / f"r{rank}.txt").read_text().split())
        assert seconds == 2.5          # the slowest rank's time
        assert iters == 30.0           # 10 + 20 iterations
    v0 = np.load(tmp_path / "vals0.npy")
    v1 = np.load(tmp_path / "vals1.npy")
    assert v0.shape == v1.shape and not np.array_equal(v0, v1)  # each replica its own problem
