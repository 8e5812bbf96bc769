"""The N > 1 path of bench.py on CPU: replicas over gloo, world size 2.

bench.py runs one process per GPU and has no collective on the data path
(replicas); the ranks meet only at the barriers around the timed region and
in the max over ranks of the elapsed time, which sets the whole-job rate.
These tests run that logic on host processes: the Dist helper with the gloo
backend, and the reference arm under torchrun, where rank 0 alone works and
prints."""
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


_RANK_SCRIPT = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import bench
d = bench.Dist()
d.init("gloo")
d.barrier()
elapsed = 100.0 * (d.rank + 1)          # a slower rank 1
m = d.max(elapsed)
steps = 10
rate = d.world * steps / (m / 1000.0)   # the whole-job rate bench.py reports
d.barrier()
print(json.dumps({{"rank": d.rank, "world": d.world, "max": m, "rate": rate}}))
d.close()
"""


def test_dist_barrier_and_max_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT.format(root=ROOT)],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2
        assert o["max"] == 200.0            # every rank sees the slowest rank's time
        assert abs(o["rate"] - 2 * 10 / 0.2) < 1e-9


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--gaussians", "20000", "--width", "96", "--height", "64"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    for key in ("metric", "unit", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line
    assert line["e2e"]["h2d_bytes_per_step"] == 0
