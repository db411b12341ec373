"""The multi-GPU form is replicas only (each rank runs its own instance; no
collective on the data path). Its host logic runs here on CPU ranks with
the gloo backend: the job time is the slowest rank's, the value counts
every rank's units, and the reference arm prints one line from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(times[rank], "cpu")
    v = bench.replica_value(1000.0, ws, t)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "v": v}, f)
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    times = [0.75, 1.25]
    mp.start_processes(_rank_main, args=(2, free_port(), times, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["t"] == 1.25 and got["v"] == pytest.approx(2000.0 / 1.25)


def test_max_over_ranks_without_a_group_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, "cpu") == 0.5
    assert bench.replica_value(10.0, 1, 2.0) == 5.0


def test_reference_arm_under_two_ranks_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--workload", "plain_64", "--ref-cols", "8"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
