"""The benchmark's N>1 host path, run as two gloo ranks on the CPU.

Multi-GPU runs are replicas: every rank builds its own input; the only
cross-rank steps are the barriers around the timed region and the max of
the per-rank step times.  These run here on world_size 2 over gloo.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, _ = bench.dist_env()
    bench.barrier(got_ws)
    mx = bench.max_over_ranks(10.0 * (rank + 1), got_ws)
    bench.barrier(got_ws)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ws": got_ws, "rank": got_rank, "max": mx}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [r["rank"] for r in res] == [0, 1]
    assert all(r["ws"] == 2 for r in res)
    assert all(r["max"] == 20.0 for r in res)  # every rank sees the slowest rank's time


def test_single_process_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)


@pytest.mark.slow
def test_reference_arm_under_two_ranks(tmp_path):
    """Under torchrun with two ranks the reference arm prints one line from
    rank 0 and the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
