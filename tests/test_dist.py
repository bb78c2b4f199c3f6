"""The N > 1 launch path on CPU (gloo, world size 2, 127.0.0.1): replicas only,
so the one collective is the timing (barrier + max over ranks); the reference
arm runs on rank 0 alone and prints one JSON line, the other rank exits 0."""
import json
import os
import re
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def torchrun(args, timeout=300):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_dist_max_and_barrier_two_ranks():
    r = torchrun([os.path.join("tests", "dist_check.py")])
    assert r.returncode == 0, r.stderr[-2000:]
    # the ranks share one stdout: their lines may interleave without newlines
    found = sorted(re.findall(r"rank (\d) world (\d) max ([0-9.]+)", r.stdout))
    assert found == [("0", "2", "2.5"), ("1", "2", "2.5")]


def test_reference_arm_two_ranks_prints_once():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                  "--workload", "lj_fcc10_4000"])
    assert r.returncode == 0, r.stderr[-2000:]
    js = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(js) == 1
    line = js[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
