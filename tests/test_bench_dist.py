"""The benchmark's multi-rank host logic on CPU, world size 2 over gloo.

The guide pass shards by image stream: each rank runs its own 1080p stream
with its own seed and nothing crosses ranks on the data path; the only
collectives are the timing barrier and the max over ranks of the timed
seconds. These tests run that aggregation on two gloo ranks, and the
reference arm under torchrun with two ranks (rank 0 alone prints its line)."""
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


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        seconds = [0.50, 0.80][rank]              # rank 1 is the slow one
        rate, slowest = bench.job_rate(ws, seconds, 1000.0)
        res = {"rate": rate, "slowest": slowest, "max": bench.allmax(ws, float(rank + 3))}
        with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_job_rate_is_all_units_over_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(ws)]
    for r in res:
        assert r["slowest"] == 0.80
        assert abs(r["rate"] - 2 * 1000.0 / 0.80) < 1e-9
        assert r["max"] == 4.0


def test_job_rate_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, slowest = bench.job_rate(1, 0.25, 500.0)
    assert slowest == 0.25 and rate == 2000.0


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` with two ranks: rank 0 times the oracle and
    prints exactly one JSON line; rank 1 exits 0 without work."""
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
