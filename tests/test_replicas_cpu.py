"""The replica path (one process per GPU, no data-path collective) on CPU:
two gloo ranks under torchrun exercise bench.py's rendezvous, max-over-ranks
timing and whole-job aggregation, and the reference arm prints one line from
rank 0 only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _objects(text):
    """Every JSON object in the ranks' combined stdout (their lines may interleave)."""
    dec = json.JSONDecoder()
    out, i = [], 0
    while True:
        i = text.find("{", i)
        if i < 0:
            return out
        obj, i = dec.raw_decode(text, i)
        out.append(obj)


def _torchrun(script_args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port())] + script_args
    env = dict(os.environ, OMP_NUM_THREADS="2")
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def test_two_ranks_aggregate_whole_job_throughput():
    r = _torchrun(["tests/replica_worker.py", "--gpus", "2"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _objects(r.stdout)
    assert sorted(d["rank"] for d in lines) == [0, 1]
    for d in lines:
        assert d["world"] == 2
        assert d["max"] == 1.5                      # max over ranks of rank + 0.5
        assert abs(d["rate"] - 2e9 / 2.0) < 1e-3    # 2 x 1e9 units / slowest rank's 2 s


def test_reference_arm_prints_one_line_from_rank_zero():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                  timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _objects(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the same workload description, metric and direction as the CUDA arm's line
    assert "Barabasi-Albert n=65,536" in d["config"]["workload"]
    assert d["config"]["iterations_per_step"] == 10 and d["config"]["batch"] == 256
    assert d["unit"] == "pair-interactions/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["cores"] >= 1
