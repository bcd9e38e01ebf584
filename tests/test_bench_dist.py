"""The N>1 path of bench.py on CPU: two gloo ranks (127.0.0.1) reduce their
times to the job maximum, the whole-job rate counts every rank's replica, and
the reference arm runs on rank 0 only."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    got = bench.max_over_ranks(local_ms)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write(repr(got))


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    got = [float(open(tmp_path / ("rank%d.txt" % r)).read()) for r in range(world)]
    assert got == [15.0, 15.0]


def test_job_throughput_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench

    # 2 ranks, each 3e9 units, slowest rank 1.5 s -> 4 G units/s for the job
    assert bench.job_throughput(3e9, 1.5, 2) == pytest.approx(4.0)
    assert bench.max_over_ranks(7.25) == 7.25  # no process group: identity


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
