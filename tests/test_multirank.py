"""The N > 1 launch path of bench.py on CPU: replicas under torch.distributed.run with the gloo
backend (world size 2).  The data path has no collective; only the timing is reduced (max over
ranks) and rank 0 alone prints."""
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
    port = s.getsockname()[1]
    s.close()
    return port


def _torchrun(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONPATH=ROOT)
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def test_rank_aggregation_gloo(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(
        "import json, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import torch.distributed as dist\n"
        "dist.init_process_group('gloo')\n"
        "import bench\n"
        "r, w = dist.get_rank(), dist.get_world_size()\n"
        "t = bench.max_over_ranks(1.0 + r, 'cpu')\n"
        f"out = {str(tmp_path)!r} + f'/rank{{r}}.json'\n"
        "open(out, 'w').write(json.dumps({'rank': r, 't': t, 'rate': bench.job_rate(350, 3, w, t)}))\n"
        "bench.barrier()\n"
        "dist.destroy_process_group()\n")
    res = _torchrun([str(script)], timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    # one file per rank: two ranks printing to one pipe may interleave their lines
    rows = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in (0, 1)]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["t"] == 2.0                       # the slowest rank's time on every rank
        assert r["rate"] == 350 * 3 * 2 / 2.0      # units of both ranks over that time


def test_max_over_ranks_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_rate(10, 2, 1, 4.0) == 5.0


def test_reference_arm_two_ranks_prints_once():
    """`bench.py --impl reference` under torchrun: rank 0 times the oracle and prints one line,
    rank 1 exits 0 without work."""
    res = _torchrun(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"], timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(l) for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
