"""Several GPUs run independent replicas of the domain (the single-domain
solve is not sharded): bench.py's whole-job figures are the summed work of
all ranks over the slowest rank's time, and the reference arm runs on rank 0
only.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 1.5 + r seconds for (r + 1) * 1e9 unknown-cycles
        t, w = bench.job_totals(dist, 1.5 + rank, (rank + 1) * 1e9, torch.device("cpu"))
        q.put((rank, t, w))
    finally:
        dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, w in got:
        assert t == 2.5 and w == 3e9, (rank, t, w)


def test_job_totals_one_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(None, 2.0, 5.0, None) == (2.0, 5.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and r.stdout.strip() == "", r.stdout + r.stderr
