"""Replica path on two CPU ranks (gloo): the timing collectives, the sharding
of independent scenes, and bench.py's reference arm under torchrun (rank 0
alone measures and prints; the other rank exits cleanly)."""
import json
import os
import socket
import subprocess
import sys
import tempfile

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2603_16103_gb300 import replicas
    got_ws, got_rank = replicas.init()
    secs = [2.0, 2.5][rank]
    units = [100.0, 300.0][rank]
    res = {
        "env": [got_ws, got_rank],
        "max": replicas.max_over_ranks(secs),
        "sum": replicas.sum_over_ranks(units),
        "rate": replicas.whole_job_rate(units, secs),
        "shard": replicas.shard(range(7), rank, ws),
    }
    replicas.barrier()
    replicas.finish()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_agree_on_timing_and_shards():
    ws = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(ws, _free_port(), d), nprocs=ws, join=True,
                           start_method="spawn")
        res = [json.load(open(os.path.join(d, f"r{r}.json"))) for r in range(ws)]
    for r, x in enumerate(res):
        assert x["env"] == [ws, r]
        assert x["max"] == 2.5 and x["sum"] == 400.0
        assert abs(x["rate"] - 400.0 / 2.5) < 1e-9
    assert res[0]["shard"] == [0, 2, 4, 6] and res[1]["shard"] == [1, 3, 5]
    assert sorted(res[0]["shard"] + res[1]["shard"]) == list(range(7))


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2603_16103_gb300 import replicas
    assert replicas.init() == (1, 0)
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.whole_job_rate(10.0, 2.0) == 5.0
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--workload", "unit20k"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"
