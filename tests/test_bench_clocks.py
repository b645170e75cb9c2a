"""The benchmark's clock rule on CPU, with a fake clock sampler: a timed region
whose clock record shows a hardware or thermal slowdown, or SM clocks held far
below their maximum with no reason, is run once more and the second run kept;
a power cap is kept as measured; under two gloo ranks one rank's rejection
makes both ranks run again."""
import os
import socket

import bench


class FakeSampler:
    def __init__(self, records):
        self.records = list(records)
        self.started = 0

    def start(self):
        self.started += 1

    def stop(self):
        return dict(self.records.pop(0))


OK = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}


def _runner():
    calls = []

    def run():
        calls.append(len(calls))
        return 10.0 + len(calls)
    return run, calls


def test_rejection_rules():
    assert bench.clock_rejection(OK) is None
    assert bench.clock_rejection(dict(OK, reasons=["sw_power_cap"], sm_mhz=1700.0)) is None
    assert "hw_thermal_slowdown" in bench.clock_rejection(dict(OK, reasons=["hw_thermal_slowdown"]))
    assert "sw_thermal_slowdown" in bench.clock_rejection(dict(OK, reasons=["sw_thermal_slowdown", "sw_power_cap"]))
    assert "no reason" in bench.clock_rejection(dict(OK, sm_mhz=1200.0))
    assert bench.clock_rejection({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}) is None


def test_clean_run_is_kept():
    run, calls = _runner()
    s = FakeSampler([OK])
    out, clocks = bench.timed_region(run, s, lambda: None)
    assert out == 11.0 and len(calls) == 1 and "first_run_rejected" not in clocks


def test_throttled_run_is_measured_again():
    run, calls = _runner()
    s = FakeSampler([dict(OK, reasons=["hw_slowdown"]), OK])
    out, clocks = bench.timed_region(run, s, lambda: None)
    assert out == 12.0 and len(calls) == 2 and s.started == 2
    assert clocks["reasons"] == [] and "hw_slowdown" in clocks["first_run_rejected"]


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first = dict(OK, sm_mhz=900.0) if rank == 1 else OK             # only rank 1 sees a held clock
    run, calls = _runner()
    out, clocks = bench.timed_region(run, FakeSampler([first, OK]), lambda: None, dist)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{len(calls)} {out} {clocks.get('first_run_rejected', '')}")
    dist.barrier()
    dist.destroy_process_group()


def test_one_rank_rejection_reruns_every_rank(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    r0 = open(tmp_path / "r0.txt").read().split(maxsplit=2)
    r1 = open(tmp_path / "r1.txt").read().split(maxsplit=2)
    assert r0[:2] == ["2", "12.0"] and r1[:2] == ["2", "12.0"]
    assert "another rank" in r0[2] and "no reason" in r1[2]
