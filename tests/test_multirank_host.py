"""Host side of the bench's N > 1 path on CPU, with world_size-2 gloo ranks.

The path shards into independent replicas (one program per GPU, no data-path
collective): the only exchanges are the barriers around the timed region and
the max over ranks of the timed region's length.  These tests run that logic
with the gloo backend, and the reference arm under torchrun (rank 0 alone runs
the oracle and prints; the other rank exits 0 without work)."""
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


def _rank_main(rank, ws, port, outdir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench._dist()
    dist = bench._dist_init(w, local, False)
    bench._barrier(dist)
    # rank r "took" 10 * (r + 1) ms for its 5 steps
    m = bench._max_over_ranks(dist, 10.0 * (r + 1), False)
    bench._barrier(dist)
    with open(os.path.join(outdir, f"rank{r}.json"), "w") as f:
        json.dump({"ws": w, "rank": r, "max_ms": m, "value": bench._weak_value(w, 5, m)}, f)
    dist.destroy_process_group()


def test_gloo_two_ranks_barrier_and_max(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r, g in enumerate(got):
        assert g["ws"] == ws and g["rank"] == r
        assert g["max_ms"] == 20.0          # the slowest rank's time, on every rank
        assert g["value"] == pytest.approx(2 * 5 / 0.020)  # all ranks' steps / max time


def test_weak_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._weak_value(1, 50, 40.0) == pytest.approx(1250.0)


def test_reference_arm_under_torchrun_prints_once():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3",
           "--matrix-n", "64", "--k", "4"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
