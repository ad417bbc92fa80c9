"""bench.py's multi-rank logic on CPU (gloo, world size 2): max-over-ranks
timing, whole-job aggregation of replica throughput, and the reference arm
running on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 1 + r seconds for 1000 units
    t = bench.reduce_max(1.0 + rank, world)
    bench.barrier(world)
    agg = bench.aggregate(1000.0, t, world)
    with open(f"{out_path}.{rank}", "w") as f:
        json.dump({"t": t, "agg": agg}, f)
    dist.destroy_process_group()


def test_reduce_max_and_aggregate_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "res")
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(f"{out}.{r}"))
        assert d["t"] == 2.0                 # the slower rank's time
        assert d["agg"] == pytest.approx(1000.0)  # 2 ranks x 1000 units / 2 s


def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3",
           "--workload", "straight_rod_64"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_on_the_default_workload():
    """The reference arm on the default (headline) workload, as the driver
    runs it: the oracle's sampled force pass, one JSON line with the
    workload's config."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["config"]["workload"] == bench.DEFAULT_WORKLOAD
    assert d["value"] > 0 and d["unit"] == "particle-steps/s" and d["higher_is_better"] is True
    assert "sampled" in d["cpu_baseline"]["sample"]
