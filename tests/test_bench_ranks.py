"""bench.py's multi-rank path on the CPU: two gloo ranks launched by torchrun.

Each rank reconstructs its own batch (distinct phantom seeds), the timed region is the slowest
rank's, and the whole-job value counts the units of every rank.  The reference arm runs on
rank 0 only and prints one line; the other ranks leave without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), *args]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_two_ranks_time_the_slowest_and_count_every_rank(tmp_path):
    r = _torchrun([os.path.join(ROOT, "tests", "ranks_worker.py"), str(tmp_path)], 300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    for d in lines:
        assert d["world"] == 2
        assert d["max_ms"] == 15.0
        assert len(set(d["seeds"])) == 2
        assert abs(d["rate"] - 2 * 1000 * 2 / 15e-3) < 1e-6 * d["rate"]


def test_reference_arm_prints_once_under_two_ranks():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--workload", "single-1x128sq-90ang-50it",
                   "--steps", "1", "--warmup", "0"], 600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
