"""Multi-GPU is replicas only (independent grids per rank, no data-path
collective). The benchmark's N > 1 logic — the slowest rank's time, all ranks'
cells over it — runs here as two gloo ranks on the CPU, launched the way the
benchmark is (torch.distributed.run on 127.0.0.1)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_agree_on_the_slowest_time(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "tests", "replica_worker.py")]
    env = dict(os.environ, OMP_NUM_THREADS="1", REPLICA_OUT=str(tmp_path))
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=240, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    rows = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["world"] == 2
        assert r["t"] == 13.0                      # the slower rank's
        assert abs(r["rate"] - 2000.0 / 13.0) < 1e-12
