"""The multi-GPU form of the benchmark is replicas only (faces are
independent, no data-path collective): each rank times its own face and the
job's value is the units of all ranks over the slowest rank's time.  The
cross-rank totals run here as two gloo processes on the CPU, and the reference
arm's non-zero ranks leave without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms, units = bench.job_totals(10.0 * (rank + 1), 1000 * (rank + 1), world, "cpu")
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"ms": ms, "units": units}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_take_the_slowest_rank_and_all_units(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        got = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert got == {"ms": 20.0, "units": 3000.0}      # max(10, 20) ms, 1000 + 2000 units
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(7.5, 42, 1) == (7.5, 42.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29999")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
