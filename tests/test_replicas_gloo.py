"""Replica path with two CPU ranks over gloo (no GPU)."""
import os
import socket

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
