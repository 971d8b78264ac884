"""The multi-rank benchmark path on CPU: two gloo ranks (one process each) exercise the rank setup,
the per-rank inputs (independent images, no data exchange), the whole-job aggregation (matches
summed over ranks, time = the slowest rank's) and the reference arm (rank 0 alone runs it)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), FIC_DIST_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    # rank r: matches_per_step 100 (r + 1), steps of (r + 1) ms each
    value, total_s = bench.aggregate(100.0 * (r + 1), [float(r + 1)] * 4, world)
    # per-rank images: the same workload, distinct seeds
    wl = dict(bench.WORKLOADS["encode-256"], seed=2000, H=64, W=64)
    img = bench._image(wl, r)
    np.save(os.path.join(out_dir, f"img{r}.npy"), img)
    # the reference arm: ranks other than 0 return at once without work or output
    if r != 0:
        assert bench.run_reference(None, wl, world, r) == 0
    with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
        f.write(f"{value!r} {total_s!r}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    vals = [tuple(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(world)]
    # total matches 4 * (100 + 200) = 1200 over the slowest rank's 4 * 2 ms = 8 ms
    for value, total_s in vals:
        assert total_s == pytest.approx(0.008)
        assert value == pytest.approx(1200 / 0.008)
    a, b = (np.load(tmp_path / f"img{r}.npy") for r in range(world))
    assert a.shape == b.shape == (64, 64) and not np.array_equal(a, b)
