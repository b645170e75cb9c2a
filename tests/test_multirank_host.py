"""Host logic of the multi-GPU benchmark on CPU: two gloo ranks shard the
events (each rank its own event, no collective on the data path) and the step
time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    ms = bench.reduce_max(10.0 + 5.0 * rank, dist)
    g, fm, ev = bench.make_workload(rank)
    np.save(os.path.join(out_dir, f"wires{rank}.npy"), ev.wire_id)
    with open(os.path.join(out_dir, f"ms{rank}.txt"), "w") as f:
        f.write(f"{ms} {bench.job_value(ws, 1000.0, ms)}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    vals = [open(tmp_path / f"ms{r}.txt").read().split() for r in range(world)]
    for ms, v in vals:
        assert float(ms) == pytest.approx(15.0)                 # the slower rank's time on every rank
        assert float(v) == pytest.approx(2 * 1000.0 / 15e-3)    # both ranks' units over that time
    w0, w1 = (np.load(tmp_path / f"wires{r}.npy") for r in range(world))
    assert not (w0.shape == w1.shape and np.array_equal(w0, w1))  # each rank has its own event
