"""Replica path with two CPU ranks over gloo (no GPU)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_2301_12191_gb300 import replicas
    r, w = replicas.init("gloo")
    replicas.barrier()
    # each rank "times" a different duration; every rank must see the max
    t = replicas.max_over_ranks(0.5 + r)
    out[r] = (r, w, replicas.seed_base(r), t, replicas.job_rate(10, w, t))
    replicas.barrier()
    replicas.finish()


def test_two_ranks_max_and_shards():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    seeds = {res[r][2] for r in res}
    assert len(seeds) == 2                        # no shared content
    for r in res:
        assert res[r][1] == 2
        assert res[r][3] == pytest.approx(1.5)    # max over ranks
        assert res[r][4] == pytest.approx(20 / 1.5)


def test_single_rank_needs_no_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2301_12191_gb300 import replicas
    assert replicas.env() == (0, 1, 0)
    assert replicas.init("gloo") == (0, 1)
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.job_rate(5, 1, 0.5) == 10


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _env():
    env = dict(os.environ, PYTHONPATH=ROOT, CUDA_VISIBLE_DEVICES="")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    return env


def test_launcher_runs_two_ranks_of_a_replica_job():
    """replicas.spawn (what bench.py --gpus N uses) starts two ranks; they
    meet over gloo on 127.0.0.1 and rank 0 alone reports the whole job."""
    from paper_2301_12191_gb300 import replicas
    res = replicas.spawn(os.path.join(ROOT, "tests", "replica_job.py"), [], 2, capture_output=True, text=True,
                         env=_env(), timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(ln) for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["n_gpus"] == 2
    assert line["seed_rank0"] == replicas.seed_base(0)
    # both ranks analysed a full 128x64 frame: 2 x (2 + 8 + 32 + 128) CUs evaluated
    assert line["evaluated_cus"] == 2 * (2 + 8 + 32 + 128)


def test_bench_gpus2_starts_its_own_ranks():
    """bench.py --gpus 2 without a launcher's environment starts two ranks
    itself; the oracle arm then runs on rank 0 only and prints one line."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--impl", "reference", "--config",
           "frame416", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, capture_output=True, text=True, env=_env(), timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(ln) for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference"
    assert lines[0]["config"]["workload"] == "frame416"


def test_launch_command_is_torchrun_on_localhost():
    from paper_2301_12191_gb300 import replicas
    cmd = replicas.launch_command("x.py", ["--a", "1"], 4, port=12345)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--master-port=12345" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[-3:] == ["x.py", "--a", "1"]
