"""The benchmark's multi-process host logic on CPU (gloo, world size 2): the
job's time is the slowest rank's, the whole-job rate counts every rank's
units, and under torchrun the reference arm prints one line from rank 0."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    b = _bench()
    # rank r took (r + 1) * 1.5 seconds: the job took the slowest rank's time
    t = b.max_over_ranks(dist, (rank + 1) * 1.5, torch.device("cpu"))
    dist.barrier()
    rate = b.whole_job_rate(ws, 3e9, t)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    mp.start_processes(_rank, args=(ws, port, str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["t"] == 3.0                   # the slowest rank's 2 x 1.5 s
        assert r["rate"] == pytest.approx(2.0)  # 2 ranks x 3e9 units / 3 s = 2 G units/s


def test_one_process_is_its_own_maximum():
    b = _bench()
    assert b.max_over_ranks(None, 1.25, None) == 1.25
    assert b.whole_job_rate(1, 5e9, 2.0) == pytest.approx(2.5)


def test_reference_arm_under_torchrun_prints_one_line():
    """Two ranks of `bench.py --impl reference`: rank 0 times the oracle and
    prints the line, rank 1 exits without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--time-steps", "100"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
