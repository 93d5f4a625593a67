"""The benchmark's N > 1 logic, on CPU: gloo ranks agree on the slowest rank's
step time, whole-job throughput adds every rank's units, each rank decodes its
own queries (replicas, no data-path exchange), and under torchrun the
reference arm runs and prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    got = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_value(1 << 20, world, got)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": got, "value": value}, f)
    dist.destroy_process_group()


def test_ranks_agree_on_the_slowest_step(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert all(r["ms"] == 15.0 for r in res)
    assert all(r["value"] == pytest.approx(2 * (1 << 20) / 15e-3 / 1e9) for r in res)


def test_single_rank_and_job_value():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(1 << 24, 4, 2.0) == pytest.approx(4 * (1 << 24) / 2e-3 / 1e9)


def test_ranks_decode_their_own_queries():
    a = synth.random_queries(bench.rank_query_seed(0), 256)
    b = synth.random_queries(bench.rank_query_seed(1), 256)
    assert a.shape == b.shape and not np.array_equal(a, b)


def test_reference_arm_under_torchrun_prints_on_rank_0_only():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--ref-seconds", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env={**os.environ, "OMP_NUM_THREADS": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
