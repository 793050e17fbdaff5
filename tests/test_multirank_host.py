"""The bench's multi-rank host logic on CPU (gloo, world size 2): registrations
are independent replicas, so the only cross-rank steps are the barrier, the
maximum of the ranks' timed regions and the sum of their work; the reference
arm runs on rank 0 alone."""
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


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench._dist() == (ws, rank, rank)
    bench._barrier(ws)
    mx = bench._barrier_max(10.0 + rank, ws)
    tot = bench._sum_over_ranks(1000.0 * (rank + 1), ws)
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}"), "w") as f:
        f.write(f"{mx} {tot}")


def test_barrier_max_and_sum_over_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        mx, tot = map(float, open(tmp_path / f"r{r}").read().split())
        assert mx == 11.0 and tot == 3000.0


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._barrier_max(3.5, 1) == 3.5 and bench._sum_over_ranks(7.0, 1) == 7.0
    bench._barrier(1)


@pytest.mark.timeout(600)
def test_reference_arm_prints_on_rank_zero_only():
    """torchrun with two CPU ranks: rank 0 prints the reference line, rank 1
    exits 0 without work."""
    env = dict(os.environ)
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and '"impl": "reference"' in lines[0]
