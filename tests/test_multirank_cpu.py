"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1)
exercise the barrier and the max over ranks of the timed region, the
whole-job throughput of replicas, and the reference arm under torchrun,
where ranks other than 0 exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # rank r "took" r + 1 seconds: the job's time is the slowest rank's
        dt_max = bench.allmax(world, float(rank + 1))
        value = bench.replica_throughput(world, 10 ** 9, 4, dt_max)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{dt_max} {value}\n")
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_allmax_and_replica_throughput_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        dt_max, value = map(float, open(tmp_path / f"rank{r}.txt").read().split())
        assert dt_max == 2.0                       # max over ranks, seen by every rank
        assert value == pytest.approx(2 * 1e9 * 4 / 2.0 / 1e9)  # both replicas' bytes over the slowest time


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(1, 7247757312, 500, 0.547) == pytest.approx(7247757312 * 500 / 0.547 / 1e9)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
